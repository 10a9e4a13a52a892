"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the oracle.

This module holds problem *parameters* and seeded random arrays only. It
contains none of the method's arithmetic (no operator, no FFT, no solve), so
that the oracle and the CUDA path stay independent: both receive the same
plain dictionaries and numpy arrays from here.

A problem is a dict with the keys

  op        'bs' (constant-coefficient Black-Scholes in S), 'localvol'
            (Black-Scholes with sigma(S, t)), 'riesz' (Riesz fractional
            operator in log-price x), 'heston' (the two-dimensional Heston
            operator in (s, v), Sec. 5.1) or 'sabr' (the two-dimensional SABR operator of
            Sec. 5.2, on the same (s, v) grid)
  payoff    'put' or 'call'
  nx, nt    interior spatial nodes, number of Crank-Nicolson steps
  T, r, K   maturity, rate, strike
  sigma     volatility (constant part for 'localvol'; kappa = sigma^2/2 for 'riesz')
  s_max     S-domain [0, s_max] ('bs', 'localvol'); x-domain [-s_max, s_max] ('riesz')
  lv_bump, lv_tslope
            'localvol' only: sigma(S,t) = sigma + lv_bump*exp(-ln(S/K)^2)*(1 + lv_tslope*t)
  lv_shape  optional, 'gauss' (the bump above, the default) or 'flat' (bump shape 1: a
            volatility that depends on time only; the oracle's pins use it, the library
            rejects it)
  beta      'riesz': fractional order in (1, 2]; 'sabr': the CEV exponent of s
  nv, kappa, eta, rho, v_max
            'heston' and 'sabr': nx = Ns nodes in s, nv = Nv nodes in v, mean reversion
            and long-run variance (Heston only), correlation, v-domain [0, v_max]; sigma
            is the volatility of the variance (of the volatility for SABR) and s_max the
            s-domain [0, s_max]
  alpha     the free parameter of the alpha-circulant preconditioner (Sec. 3.1)
  precision 'fp64' or 'mixed' (FP32-complex preconditioner inside FP64 FGMRES)
  m, tol    restart length and relative-residual tolerance of FGMRES(m)

Time t is time-to-maturity throughout (u(., 0) = payoff, Eq. 1.1).
"""
from __future__ import annotations

import copy

import numpy as np

SEED = 2401_16113


def _base(**kw):
    p = dict(op="bs", payoff="put", nx=255, nt=256, T=1.0, r=0.05, K=100.0, sigma=0.2,
             s_max=300.0, lv_bump=0.0, lv_tslope=0.0, beta=2.0, alpha=1e-2,
             precision="fp64", m=20, tol=1e-10)
    p.update(kw)
    return p


def bs_put_255x256():
    """European put, sigma 0.2, r 0.05, K 100, T 1, S in [0, 300], 255 x 256, FP64, alpha 1e-2."""
    return _base()


def localvol_2047x2048(precision="mixed"):
    """Local volatility sigma(S,t) = 0.15 + 0.1 exp(-ln^2(S/K)) (1 + 0.2 t), r 0.03, K 100,
    T 1, S in [0, 300], 2047 x 2048 (4,192,256 unknowns), alpha 1e-3, FGMRES(30), tol 1e-8."""
    return _base(op="localvol", nx=2047, nt=2048, r=0.03, sigma=0.15, lv_bump=0.1,
                 lv_tslope=0.2, alpha=1e-3, precision=precision, m=30, tol=1e-8)


def localvol_8191x8192(precision="mixed"):
    """The same local-volatility problem at 8191 x 8192 (67,100,672 unknowns)."""
    p = localvol_2047x2048(precision)
    p.update(nx=8191, nt=8192, m=40)
    return p


def riesz_1023x512():
    """Riesz fractional (beta 1.5, kappa = sigma^2/2, sigma 0.25) put in log-price x in [-3, 3],
    r 0.05, K 1, 1023 x 512, alpha 1e-3, FGMRES(30)."""
    return _base(op="riesz", nx=1023, nt=512, r=0.05, K=1.0, sigma=0.25, s_max=3.0,
                 beta=1.5, alpha=1e-3, precision="mixed", m=30, tol=1e-8)


def riesz_sym_1023x512():
    """The Riesz workload without drift: r = sigma^2/2 = 0.03125 cancels the (r - sigma^2/2) u_x
    term, so the spatial matrix is symmetric and step (b) runs on its eigendecomposition."""
    return with_(riesz_1023x512(), r=0.03125)


def heston_set1(nt=48, precision="mixed"):
    """Heston parameter Set I of Sec. 5.1 (European call, S in [0, 800], v in [0, 4]): T 1, K 100,
    kappa 1.5, eta 0.04, sigma 0.3, r 0.025, rho -0.9, evaluated at S0 100, V0 0.5; the paper's mesh
    family Nt = Ns = 2 Nv, alpha 1e-3, GMRES(40), tol 1e-9."""
    return _base(op="heston", payoff="call", nx=nt, nv=nt // 2, nt=nt, T=1.0, K=100.0, r=0.025,
                 sigma=0.3, kappa=1.5, eta=0.04, rho=-0.9, s_max=800.0, v_max=4.0, S0=100.0, V0=0.5,
                 alpha=1e-3, precision=precision, m=40, tol=1e-9)


def heston_set2(nt=48, precision="mixed"):
    """Heston parameter Set II of Sec. 5.1: T 3, K 100, kappa 0.6067, eta 0.0707, sigma 0.2928,
    r 0.03, rho -0.7571, S0 100, V0 0.2; same domain and mesh family as Set I."""
    return with_(heston_set1(nt, precision), T=3.0, kappa=0.6067, eta=0.0707, sigma=0.2928, r=0.03,
                 rho=-0.7571, V0=0.2)


def sabr_set3(nt=48, precision="mixed"):
    """SABR parameter Set III of Sec. 5.2 (European call, s in [0, 24], v in [0, 3]): T 2, beta 0.5,
    sigma 0.4, r 0, rho 0, K = S0 = 0.5, V0 0.5; the mesh family Nt = Ns = 2 Nv of Table 3, alpha
    1e-3, GMRES(40), tol 1e-9."""
    return _base(op="sabr", payoff="call", nx=nt, nv=nt // 2, nt=nt, T=2.0, K=0.5, r=0.0, sigma=0.4,
                 beta=0.5, rho=0.0, kappa=0.0, eta=0.0, s_max=24.0, v_max=3.0, S0=0.5, V0=0.5,
                 alpha=1e-3, precision=precision, m=40, tol=1e-9)


def sabr_set4(nt=48, precision="mixed"):
    """SABR parameter Set IV of Sec. 5.2: s in [0, 4], v in [0, 2], T 10, beta 0.5, sigma 0.8, r 0,
    rho -0.6, K = S0 = 0.07, V0 0.4; the same mesh family."""
    return with_(sabr_set3(nt, precision), s_max=4.0, v_max=2.0, T=10.0, sigma=0.8, rho=-0.6, K=0.07,
                 S0=0.07, V0=0.4)


def sabr_set5(nt=48, precision="mixed"):
    """SABR parameter Set V of Sec. 5.2 (Table 4), with a nonzero rate, so that the operator of
    Eq. 5.7 depends on time through D(t) = e^{-rt}: s in [0, 23], v in [0, 3], T 2, beta 0.45,
    sigma 0.4, r 0.03, rho -0.65, K = S0 = 0.5, V0 0.2; the same mesh family and solver."""
    return with_(sabr_set3(nt, precision), s_max=23.0, v_max=3.0, T=2.0, beta=0.45, sigma=0.4, r=0.03,
                 rho=-0.65, K=0.5, S0=0.5, V0=0.2)


def batch_instances(n=512, seed=SEED, nx_choices=(127, 255, 511, 1023),
                    nt_choices=(64, 128, 256, 512, 1024), precision="mixed", alpha=1e-3, m=20,
                    tol=1e-8):
    """Independent European put/call instances: sigma ~ U[0.1, 0.6], r ~ U[0, 0.08],
    K ~ U[50, 150], T ~ U[0.25, 2], put/call ~ Bernoulli(1/2), S in [0, 3K],
    Nx and Nt drawn uniformly from the given sets."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        K = float(rng.uniform(50.0, 150.0))
        out.append(_base(
            op="bs", payoff="put" if rng.random() < 0.5 else "call",
            sigma=float(rng.uniform(0.1, 0.6)), r=float(rng.uniform(0.0, 0.08)), K=K,
            T=float(rng.uniform(0.25, 2.0)), s_max=3.0 * K,
            nx=int(rng.choice(nx_choices)), nt=int(rng.choice(nt_choices)),
            alpha=alpha, precision=precision, m=m, tol=tol))
    return out


def random_vector(n, seed=SEED, dtype=np.float64):
    """Standard-normal test vector of length n."""
    return np.random.default_rng(seed).standard_normal(n).astype(dtype)


def with_(p, **kw):
    q = copy.deepcopy(p)
    q.update(kw)
    return q


def unknowns(p):
    return int(p["nx"]) * int(p.get("nv", 1)) * int(p["nt"])
