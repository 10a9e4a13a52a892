"""Pins for the oracle's time-dependent operator (local volatility), CPU only.

Row k of the all-at-once system uses A(t_{k+1/2}) for both time levels (the form of Eq. 5.8,
where the separable case puts d(t_{k+1/2}) in block row k), and t is time to maturity
(u(., 0) = payoff, Eq. 1.1). Each pin below rests on a fact outside the oracle's own
time stepping, and each comes with the plausible mistake it catches, planted in the oracle:

  * a volatility that depends on time only has the Black-Scholes closed form with the
    integrated variance (1/T) int_0^T sigma(t)^2 dt: evaluating A at t_k instead of t_{k+1/2}
    shifts the integrated variance by O(tau) and fails it;
  * Crank-Nicolson with A at the midpoint is second order in time: against the semi-discrete
    solution (the same spatial operator integrated by a stiff ODE solver to 1e-11) the error
    falls by 4 per halving of tau; with A(t_k) it falls by 2;
  * the time-to-maturity convention: the PDE value equals the risk-neutral expectation of the
    discounted payoff under dS = r S ds + sigma(S, T - s) S dW (Feynman-Kac), estimated by a
    seeded Monte Carlo run; reading sigma's t as calendar time moves the far out-of-the-money
    put by 7% and fails it.
"""
import math

import numpy as np
import scipy.integrate as si

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W


def _lv(**kw):
    return W.with_(W.localvol_2047x2048("fp64"), **kw)


def _at_tk(p, k):
    """Planted mistake: A evaluated at the start of the step, t_k."""
    t, _ = O.time_grid(p)
    return O.operator_at(p, t[k])


def _calendar(p, k):
    """Planted mistake: sigma's t read as calendar time, A(T - t_{k+1/2})."""
    t, tau = O.time_grid(p)
    return O.operator_at(p, p["T"] - t[k] - 0.5 * tau)


def _cn_maturity(p, monkeypatch=None, planted=None):
    if planted is not None:
        monkeypatch.setattr(O, "step_operator", planted)
    try:
        return O.sequential_cn(p)[-1]
    finally:
        if planted is not None:
            monkeypatch.undo()


# ---------------------------------------------------------------- closed form, sigma(t) only

def _time_only_case(nx=255, nt=64):
    # sigma(t) = 0.2 + 0.3 t on t in [0, 1] (time to maturity): a strong slope, so that an O(tau)
    # error in the integrated variance is far above the O(tau^2 + h^2) discretisation error
    return _lv(nx=nx, nt=nt, sigma=0.1, lv_bump=0.1, lv_tslope=3.0, r=0.05, lv_shape="flat")


def _integrated_variance_price(p, S):
    a = p["sigma"] + p["lv_bump"]
    c = p["lv_bump"] * p["lv_tslope"]
    T = p["T"]
    # int_0^T (a + c t)^2 dt
    var = a * a * T + a * c * T * T + c * c * T ** 3 / 3.0
    return O.bs_price(S, p["K"], p["r"], math.sqrt(var / T), T, "put")


def test_time_only_volatility_matches_integrated_variance_closed_form(monkeypatch):
    p = _time_only_case()
    S, _ = O.spatial_grid(p)
    sel = (S >= 0.5 * p["K"]) & (S <= 1.5 * p["K"])
    ref = _integrated_variance_price(p, S)
    err = np.abs(_cn_maturity(p)[sel] - ref[sel]).max()
    assert err < 2e-3, err  # measured 3.0e-4 (h = 300/256, tau = 1/64)
    bad = np.abs(_cn_maturity(p, monkeypatch, _at_tk)[sel] - ref[sel]).max()
    assert bad > 2e-2, bad  # measured 8.6e-2


# ---------------------------------------------------------------- second order in time

def _semi_discrete(p):
    """u' = A(t) u + f(t), u(0) = payoff, on the oracle's spatial grid (method of lines), by an
    implicit Runge-Kutta method (Radau IIA) to 1e-11: the limit of every consistent time stepping
    of the same spatial operator."""
    def rhs(t, u):
        A, cl, cr = O.operator_at(p, t)
        gl, gr = O.boundary_values(p, t)
        return A @ u + cl * gl + cr * gr

    sol = si.solve_ivp(rhs, (0.0, p["T"]), O.payoff(p), method="Radau",
                       jac=lambda t, u: O.operator_at(p, t)[0], rtol=1e-11, atol=1e-11)
    assert sol.success
    return sol.y[:, -1]


def test_localvol_crank_nicolson_is_second_order_in_time(monkeypatch):
    base = _lv(nx=63, nt=16, lv_tslope=2.0)
    ref = _semi_discrete(base)
    nts = [32, 64, 128]
    errs = [np.abs(_cn_maturity(W.with_(base, nt=nt)) - ref).max() for nt in nts]
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.8 < q < 4.2 for q in ratios), (errs, ratios)  # measured 3.999, 4.000
    bad = [np.abs(_cn_maturity(W.with_(base, nt=nt), monkeypatch, _at_tk) - ref).max() for nt in nts]
    bad_ratios = [bad[i] / bad[i + 1] for i in range(len(bad) - 1)]
    assert all(1.8 < q < 2.2 for q in bad_ratios), (bad, bad_ratios)  # first order: 1.997, 1.998


# ---------------------------------------------------------------- time-to-maturity convention

def _monte_carlo_put(p, S0, npaths, nsteps, seed):
    """e^{-rT} E[(K - S_T)^+] for dS = r S ds + sigma(S, T - s) S dW, s calendar time: log-Euler
    steps with sigma taken at the step's time to maturity, antithetic pairs."""
    rng = np.random.default_rng(seed)
    T, r, K = p["T"], p["r"], p["K"]
    ds = T / nsteps
    half = npaths // 2
    x = np.full(2 * half, math.log(S0))
    for n in range(nsteps):
        sig = O.local_sigma(p, np.exp(x), T - (n + 0.5) * ds)
        z = rng.standard_normal(half)
        z = np.concatenate([z, -z])
        x = x + (r - 0.5 * sig * sig) * ds + sig * math.sqrt(ds) * z
    pay = np.maximum(K - np.exp(x), 0.0) * math.exp(-r * T)
    pairs = 0.5 * (pay[:half] + pay[half:])
    return pairs.mean(), pairs.std() / math.sqrt(half)


def test_localvol_time_to_maturity_convention_against_monte_carlo(monkeypatch):
    # a steep slope (sigma up to 0.75 at the strike) makes the convention matter far from it
    p = _lv(nx=299, nt=256, lv_tslope=5.0)
    S, _ = O.spatial_grid(p)
    i = int(np.argmin(np.abs(S - 196.0)))  # a grid node (h = 1), deep out of the money
    mc, se = _monte_carlo_put(p, float(S[i]), 300_000, 256, seed=W.SEED)
    assert se < 0.015, se
    good = _cn_maturity(p)[i]
    bad = _cn_maturity(p, monkeypatch, _calendar)[i]
    # measured: CN 1.6054, calendar-time CN 1.7231, Monte Carlo within 2 standard errors of CN
    assert abs(mc - good) < 0.05, (mc, se, good)
    assert abs(mc - bad) > 0.08, (mc, se, bad)
