"""The learned choice of alpha and the restart length m.

The paper fixes alpha by hand (Sec. 4: alpha = 0.1 or 0.01 suffices; too small an alpha
amplifies roundoff in steps (a)/(c)). Here a small MLP (6 -> 64 -> 64 -> 2, trained and run by
the library's CUDA kernels) predicts (log10 alpha, m) from problem features, trained on labels
that the solver itself generates: every training instance is solved by the batched
mixed-precision FGMRES for each alpha of a sweep. The alpha label is the centre of the
valley of iteration counts: each alpha is scored by its count plus a quarter of each
neighbour's count on the sweep's log grid (the best-scoring alpha, the larger on ties), so a
label never sits on the edge where a slightly different instance needs more iterations. The
m label is the smallest restart length in {5, 10, 20, 30, 40} not below that count, i.e. the
smallest Krylov workspace (O(m Nt Nx) storage, Sec. 4) that needs no restart. A prediction
whose solve does not converge falls back to alpha = 1e-3.

This module is host orchestration only: feature extraction, the label rule, batching of
the sweep and argument marshalling. Solves, training and inference run in libaao's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import aao, workloads as W

ALPHAS = (1e-1, 3e-2, 1e-2, 3e-3, 1e-3, 3e-4, 1e-4, 3e-5, 1e-5)
M_CHOICES = (5, 10, 20, 30, 40)
DEFAULT_ALPHA, DEFAULT_M = 1e-3, 20


def features(p):
    """(sigma_eff, r, T, nx, nt, cv): sigma_eff = RMS volatility over S in [K/2, 3K/2] and the time
    midpoints, cv = largest relative deviation of sigma^2 from its time mean there (0 for
    constant coefficients)."""
    if p["op"] != "localvol":
        return (float(p["sigma"]), float(p["r"]), float(p["T"]), int(p["nx"]), int(p["nt"]), 0.0)
    S = np.linspace(0.5 * p["K"], 1.5 * p["K"], 41)
    t = (np.arange(64) + 0.5) * p["T"] / 64
    sig = p["sigma"] + p["lv_bump"] * np.exp(-np.log(S / p["K"])[:, None] ** 2) * (1 + p["lv_tslope"] * t[None, :])
    s2 = sig ** 2
    mean_t = s2.mean(axis=1, keepdims=True)
    cv = float(np.max(np.abs(s2 - mean_t) / mean_t))
    return (float(math.sqrt(s2.mean())), float(p["r"]), float(p["T"]), int(p["nx"]), int(p["nt"]), cv)


def normalized_features(feats):
    fm, fs, _, _ = aao.aao_mlp_normalization()
    f = np.array(feats, dtype=np.float64).reshape(-1, 6).copy()
    f[:, 3] = np.log2(f[:, 3])
    f[:, 4] = np.log2(f[:, 4])
    return ((f - fm) / fs).astype(np.float32)


def normalized_targets(alpha, m):
    _, _, ym, ys = aao.aao_mlp_normalization()
    y = np.stack([np.log10(np.asarray(alpha, np.float64)), np.asarray(m, np.float64)], axis=1)
    return ((y - ym) / ys).astype(np.float32)


def sweep_iterations(problems, tol=1e-8, maxit=200, chunk=512, m=40, alphas=ALPHAS):
    """Iteration count of every problem for every alpha (inf where the solve fails); the
    batched solver runs one chunk at a time, sweeping alpha in place."""
    import torch
    its = np.full((len(problems), len(alphas)), np.inf)
    for c0 in range(0, len(problems), chunk):
        ps = [W.with_(p, precision="mixed") for p in problems[c0:c0 + chunk]]
        bt = aao.aao_batch_create(ps, m)
        bs = [torch.empty(n, dtype=torch.float64, device="cuda") for n in bt.sizes]
        xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in bt.sizes]
        aao.aao_batch_rhs(bt, bs)
        for a_i, a in enumerate(alphas):
            aao.aao_batch_set_alpha(bt, [a] * len(ps))
            for x in xs:
                x.zero_()
            st = aao.batch_submit(bt, bs, xs, tol, maxit)
            for i, s in enumerate(st):
                if s["status"] == 0:
                    its[c0 + i, a_i] = s["iterations"]
        bt.close()
    return its


def labels_from_iterations(its, alphas=ALPHAS):
    """alpha* = argmin of its_k + (its_{k-1} + its_{k+1})/4 (edge rows repeat their neighbour;
    the larger alpha on ties); m* = the smallest choice not below the count at alpha*."""
    big = np.where(np.isfinite(its), its, 1e6)
    left = np.concatenate([big[:, :1], big[:, :-1]], axis=1)
    right = np.concatenate([big[:, 1:], big[:, -1:]], axis=1)
    best = np.argmin(big + 0.25 * (left + right), axis=1)
    a = np.array([alphas[k] for k in best])
    n = its[np.arange(len(its)), best]
    m = np.array([next((c for c in M_CHOICES if c >= k), M_CHOICES[-1]) for k in n])
    return a, m, n


def train(problems, its=None, epochs=300, minibatch=256, lr=3e-3, seed=0, init=None, **sweep_kw):
    """Label the problems by the alpha sweep (unless its is given) and train a fresh network
    on the GPU. Returns (mlp handle, final loss, labels)."""
    import torch
    if its is None:
        its = sweep_iterations(problems, **sweep_kw)
    ok = np.isfinite(its).any(axis=1)
    a, m, n = labels_from_iterations(its[ok])
    X = torch.from_numpy(normalized_features([features(p) for p, k in zip(problems, ok) if k])).cuda()
    Y = torch.from_numpy(normalized_targets(a, m)).cuda()
    if init is None:
        rng = np.random.default_rng(seed)
        init = []
        for fan_out, fan_in in ((64, 6), (64, 64), (2, 64)):
            lim = math.sqrt(6.0 / (fan_in + fan_out))
            init.append(rng.uniform(-lim, lim, fan_out * fan_in))
            init.append(np.zeros(fan_out))
        init = np.concatenate(init).astype(np.float32)
    h = aao.aao_mlp_create(init)
    loss = aao.aao_mlp_train(h, X, Y, epochs, minibatch, lr, seed)
    return h, loss, (a, m, n, its)


def predict(h, p):
    """(alpha, m) for problem p from the BF16 forward pass."""
    return aao.alpha_mlp_predict(h, features(p))
