"""Host logic of the learned alpha/m choice (CPU): the label rule and the problem features.

Label rule: each alpha of the sweep is scored by its iteration count plus a quarter of each
neighbour's (an edge repeats its own count); the best score wins, the larger alpha on ties;
m is the smallest of {5, 10, 20, 30, 40} not below the count there (40 if none). The expected
labels below are worked out by hand from that rule.
"""
import math

import numpy as np

from paper_2401_16113_gb300 import alpha_mlp as AM
from paper_2401_16113_gb300 import workloads as W

INF = np.inf


def test_label_rule_hand_worked_rows():
    its = np.array([
        # scores 14.5 12 9.25 7.75 7.75 9.25 ...: tie at 3e-3 / 1e-3 -> the larger alpha, 3e-3
        [10, 8, 6, 5, 5, 6, 8, 10, 12],
        # failed solves (inf) score as 1e6; 3e-3: 4 + (7+4)/4 = 6.75, 1e-3: 4 + (4+4)/4 = 6,
        # 3e-4: 4 + (4+9)/4 = 7.25 -> 1e-3
        [INF, INF, 7, 4, 4, 4, 9, INF, INF],
        # 3e-3: 21 + (22+21)/4 = 31.75 < 1e-3: 21 + (21+23)/4 = 32 -> 3e-3, count 21 -> m = 30
        [30, 25, 22, 21, 21, 23, 26, 29, 33],
        # flat: every score equal -> the largest alpha; 45 iterations exceed every m -> 40
        [45] * 9,
        # edge: the first column repeats itself: 1e-1: 3 + (3+9)/4 = 6 is the best
        [3, 9, 9, 9, 9, 9, 9, 9, 9],
    ], dtype=np.float64)
    a, m, n = AM.labels_from_iterations(its)
    assert list(a) == [3e-3, 1e-3, 3e-3, 1e-1, 1e-1]
    assert list(n) == [5, 4, 21, 45, 3]
    assert list(m) == [5, 5, 30, 40, 5]


def test_features_of_constant_and_local_volatility():
    bs = W.bs_put_255x256()
    assert AM.features(bs) == (0.2, 0.05, 1.0, 255, 256, 0.0)
    # local volatility without its bump is constant: sigma_eff = sigma, no time variation (cv at
    # rounding level: the time mean of equal values)
    flat = W.with_(W.localvol_2047x2048("mixed"), lv_bump=0.0)
    s, r, T, nx, nt, cv = AM.features(flat)
    assert math.isclose(s, 0.15, rel_tol=1e-14) and cv <= 1e-14 and (nx, nt) == (2047, 2048)
    # a bump without a time slope: the RMS over the S window rises above sigma, still no time
    # variation
    bump = W.with_(flat, lv_bump=0.1, lv_tslope=0.0)
    s, *_, cv = AM.features(bump)
    assert s > 0.15 and cv <= 1e-14
    # the time slope makes sigma^2 vary in time: at the money sigma(t) = 0.15 + 0.1 (1 + 0.2 t),
    # whose square deviates from its time mean by at most (0.25 + 0.02 T)^2 / mean - 1 at t -> T
    lv = W.localvol_2047x2048("mixed")
    *_, cv = AM.features(lv)
    t = (np.arange(64) + 0.5) / 64
    s2 = (0.15 + 0.1 * (1 + 0.2 * t)) ** 2
    assert cv >= np.max(np.abs(s2 - s2.mean()) / s2.mean()) - 1e-12
    assert 0.0 < cv < 0.2
