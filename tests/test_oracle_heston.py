"""Pins for the oracle's two-dimensional Heston operator (Sec. 5.1, Eq. 5.1-5.5), CPU only.

  * the Heston reference price (Fourier formula) is pinned to the martingale and normalisation
    identities of its characteristic function and to the Black-Scholes closed form in the
    zero-vol-of-vol limit (deterministic variance);
  * the finite-difference discretisation read from Sec. 5.1 reproduces the relative errors the
    paper prints in Tables 1 and 2 for both parameter sets (golden file, cited), which fixes the
    stencils, the boundary treatment and the reference price at once;
  * Lemma 3.1 holds for any spatial matrix: (Nt - 1) N unit eigenvalues of P_alpha^{-1} M, the other
    N equal to 1 / (1 - alpha q(lambda)^Nt), q(l) = (1 + l/2) / (1 - l/2) the Crank-Nicolson
    amplification of an eigenvalue l of tau A. This central-difference Heston matrix has
    eigenvalues with small positive real parts on these grids, outside the hypothesis of
    Theorem 3.1, so its annulus is checked in the widened form 1/(1 + alpha r) <= |z| <=
    1/(1 - alpha r), r = max |q|^Nt (r <= 1 gives the theorem's annulus);
  * right-preconditioned FGMRES(40) to 1e-9: P_alpha takes the same few iterations on every mesh
    (the paper: 4), P_1 many more (the paper: 25-29), and the AaO solution equals sequential CN.
"""
import math
import os

import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "heston_table12.txt")


def price_at(p, U_last):
    """Bilinear interpolation of the maturity values at (S0, V0) (Sec. 5.1)."""
    S, V, hs, hv = O.heston_grid(p)
    Z = U_last.reshape(int(p["nv"]), int(p["nx"]))
    x, y = p["S0"] / hs - 1.0, p["V0"] / hv
    i0, j0 = int(math.floor(x)), int(math.floor(y))
    fx, fy = x - i0, y - j0
    return ((1 - fx) * (1 - fy) * Z[j0, i0] + fx * (1 - fy) * Z[j0, i0 + 1] + (1 - fx) * fy * Z[j0 + 1, i0]
            + fx * fy * Z[j0 + 1, i0 + 1])


def reference(p):
    return O.heston_call(p["S0"], p["V0"], p["K"], p["T"], p["r"], p["kappa"], p["eta"], p["sigma"], p["rho"])


def test_heston_characteristic_function_identities():
    for args in [(1.0, 0.5, 1.5, 0.04, 0.3, -0.9), (3.0, 0.2, 0.6067, 0.0707, 0.2928, -0.7571)]:
        assert abs(O.heston_char(0.0, *args) - 1.0) < 1e-14  # normalisation
        assert abs(O.heston_char(-1j, *args) - 1.0) < 1e-12  # E[S_T] = S_0 e^{rT} (martingale)


def test_heston_zero_vol_of_vol_is_black_scholes_with_integrated_variance():
    T, v0, kap, eta = 1.0, 0.5, 1.5, 0.04
    vbar = eta + (v0 - eta) * (1.0 - math.exp(-kap * T)) / (kap * T)  # (1/T) int_0^T v(t) dt
    for S0 in (80.0, 100.0, 130.0):
        h = O.heston_call(S0, v0, 100.0, T, 0.025, kap, eta, 1e-4, 0.0)
        assert abs(h - O.bs_price(S0, 100.0, 0.025, math.sqrt(vbar), T, "call")) < 1e-5


@pytest.mark.slow
def test_heston_discretisation_reproduces_the_papers_errors():
    rows = np.loadtxt(GOLDEN, ndmin=2)
    for set_, nt, err in rows:
        p = (W.heston_set1 if int(set_) == 1 else W.heston_set2)(int(nt))
        ref = reference(p)
        got = abs(price_at(p, O.sequential_cn(p)[-1]) - ref) / ref
        # printed to four digits
        assert abs(got - err) <= 1.5e-3 * err, (set_, nt, got, err)


@pytest.mark.parametrize("alpha", [1e-1, 1e-3])
@pytest.mark.parametrize("shape", [(6, 4, 6), (8, 4, 8), (12, 6, 7)])
def test_heston_lemma31_eigenvalues(alpha, shape):
    ns, nv, nt = shape
    p = W.with_(W.heston_set1(8), nx=ns, nv=nv, nt=nt, alpha=alpha)
    N = ns * nv
    A, _ = O.heston_matrix(p)
    _, tau = O.time_grid(p)
    lam = np.linalg.eigvals(tau * A.toarray())
    q = (1 + lam / 2) / (1 - lam / 2)
    zf = 1.0 / (1.0 - alpha * q ** nt)
    z = O.preconditioned_eigs(p)
    order = np.argsort(np.abs(z - 1))
    unit, rest = z[order[:(nt - 1) * N]], z[order[(nt - 1) * N:]]
    assert np.abs(unit - 1).max() < 1e-8
    for w in zf:  # the other N, as a multiset
        k = int(np.argmin(np.abs(rest - w)))
        assert abs(rest[k] - w) < 1e-8
        rest = np.delete(rest, k)
    r = np.abs(q).max() ** nt
    assert np.all(np.abs(zf) >= 1 / (1 + alpha * r) - 1e-12) and np.all(np.abs(zf) <= 1 / (1 - alpha * r) + 1e-12)
    assert np.all(zf.real > 0)


def test_heston_fft_apply_equals_dense_inverse():
    p = W.with_(W.heston_set1(8), nx=6, nv=4, nt=6)
    v = W.random_vector(6 * 4 * 6, seed=4)
    assert np.linalg.norm(O.precond_fft(p, v) - O.precond_dense(p, v)) <= 1e-12 * np.linalg.norm(v) * 1e3


@pytest.mark.slow
def test_heston_iterations_are_mesh_independent_and_solution_is_cn():
    its_a, its_1 = [], []
    for nt in (16, 32):
        p = W.heston_set1(nt)
        x, info = O.solve(p, tol=1e-9, m=40, maxit=200)
        _, info1 = O.solve(W.with_(p, alpha=1.0), tol=1e-9, m=40, maxit=200)
        assert info["converged"] and info1["converged"]
        U = O.sequential_cn(p)
        assert np.abs(x - U.ravel()).max() <= 1e-8 * np.abs(U).max()
        its_a.append(info["its"])
        its_1.append(info1["its"])
    assert max(its_a) <= 4 and max(its_a) - min(its_a) <= 1, its_a  # the paper: 4 on every mesh
    assert min(its_1) >= 5 * max(its_a), (its_1, its_a)            # the paper: 25-29
