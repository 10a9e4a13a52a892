"""Pins for the oracle's two-dimensional SABR operator (Sec. 5.2, Eq. 5.7 with r = 0), CPU only.

  * The paper prints the relative error of the price at (S0, V0) against one reference price per
    parameter set (Table 3), but not that price (it comes from an external package). Two meshes
    of one set then fix it twice: Price_k = R (1 -+ Err_k) for the same unknown R. The oracle's
    prices on the Nt = 48 and 96 meshes give the same R to the printed digits, for Set III
    (rho = 0, (S0, V0) a grid node) and Set IV (rho = -0.6, bilinear interpolation between the
    nodes, the s = 0 and v = V_max boundary values included). That fixes the stencils, the mixed
    derivative and the boundary rows at once; a sign error in the mixed term fails it.
  * Remark (singular P_1, the entries marked in Table 3): with r = 0 the v = 0 rows of A are
    zero (u_t = 0 there), so A is singular, and with alpha = 1 the zero-frequency shifted block
    (lambda_1,0 = 0) is singular: P_1 is singular while P_alpha (alpha < 1) is not.
  * Right-preconditioned FGMRES(40) to 1e-9 with P_alpha: the same few iterations on every mesh
    (the paper: 4) and the AaO solution equal to sequential CN.
  * Set V (r = 0.03, Table 4): the operator of Eq. 5.7 depends on time, each term through its own
    power of D(t) = e^{-rt}. With it the Nt = 48 and 96 rows of Table 4 imply one reference price
    (to 5e-5). The form L(t) = d(t) L, which Sec. 5.2 uses to derive the preconditioner, spreads it
    35-fold and is caught. P_alpha built on the time mean of A takes the same few iterations on every
    mesh (the paper: 6), P_1 many more (the paper: 100 and up).
"""
import math
import os

import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sabr_table3.txt")
GOLDEN4 = os.path.join(os.path.dirname(__file__), "golden", "sabr_table4.txt")
SETS = {3: W.sabr_set3, 4: W.sabr_set4, 5: W.sabr_set5}


def price_at(p, U_last):
    """Bilinear interpolation of the maturity values at (S0, V0) on the grid extended by the
    boundary values u(0, v) = 0 and u(s, V_max) = s."""
    ns, nv = int(p["nx"]), int(p["nv"])
    _, _, hs, hv = O.heston_grid(p)
    G = np.zeros((nv + 1, ns + 1))
    G[:nv, 1:] = U_last.reshape(nv, ns)
    G[nv, :] = hs * np.arange(ns + 1)
    x, y = p["S0"] / hs, p["V0"] / hv
    i0, j0 = min(int(math.floor(x)), ns - 1), min(int(math.floor(y)), nv - 1)
    fx, fy = x - i0, y - j0
    return ((1 - fx) * (1 - fy) * G[j0, i0] + fx * (1 - fy) * G[j0, i0 + 1] + (1 - fx) * fy * G[j0 + 1, i0]
            + fx * fy * G[j0 + 1, i0 + 1])


def implied_references(rows, make):
    """For each side (price below or above the reference), the reference price that each row's
    printed error implies."""
    prices = [price_at(make(int(nt)), O.sequential_cn(make(int(nt)))[-1]) for _, nt, _ in rows]
    return {side: [pr / (1.0 + side * err) for pr, (_, _, err) in zip(prices, rows)] for side in (-1.0, 1.0)}


def spread(refs):
    return min(abs(r[0] - r[1]) / abs(r[1]) for r in refs.values())


# the printed errors carry four digits: the Nt = 48 row fixes R to about 6e-5
AGREE = 1.2e-4


@pytest.mark.slow
@pytest.mark.parametrize("set_", [3, 4])
def test_sabr_meshes_imply_one_reference_price(set_):
    rows = [r for r in np.loadtxt(GOLDEN, ndmin=2) if int(r[0]) == set_]
    assert spread(implied_references(rows, SETS[set_])) <= AGREE


@pytest.mark.slow
def test_a_sign_error_in_the_mixed_derivative_breaks_the_agreement():
    rows = [r for r in np.loadtxt(GOLDEN, ndmin=2) if int(r[0]) == 4]
    wrong = implied_references(rows, lambda nt: W.with_(W.sabr_set4(nt), rho=0.6))
    assert spread(wrong) > 10 * AGREE  # measured 3.3e-3, against 6e-6 with the right sign


def test_sabr_zero_rows_at_v0_and_singular_P1():
    p = W.with_(W.sabr_set3(8), nx=6, nv=4, nt=6)
    A, f = O.sabr_matrix(p)
    ns = int(p["nx"])
    assert abs(A[:ns]).sum() == 0.0 and not f[:ns].any()  # u_t = 0 on v = 0
    _, d1, d2 = O.circulant_eigs(int(p["nt"]), 1.0)
    assert abs(d1[0]) < 1e-14
    s = np.linalg.svd(O.dense_P(W.with_(p, alpha=1.0)), compute_uv=False)
    assert s.min() < 1e-12 * s.max()
    s = np.linalg.svd(O.dense_P(p), compute_uv=False)  # alpha = 1e-3
    assert s.min() > 1e-3 * s.max()


def test_sabr_reduces_to_the_heston_stencil_form():
    """With beta = 1 the SABR coefficients are those of a Heston-type operator with v^2 in place
    of v: the interior rows agree with the Heston matrix built on v' = v^2 coefficients (checked
    entry by entry on one interior node)."""
    p = W.with_(W.sabr_set4(8), nx=8, nv=4, nt=4, beta=1.0)
    A, _ = O.sabr_matrix(p)
    S, V, hs, hv = O.heston_grid(p)
    i, j = 4, 2
    row = j * 8 + (i - 1)
    s, v, sig, rho = S[i - 1], V[j], p["sigma"], p["rho"]
    assert math.isclose(A[row, row], -v * v * s * s / hs ** 2 - sig * sig * v * v / hv ** 2, rel_tol=1e-14)
    assert math.isclose(A[row, row + 1], 0.5 * v * v * s * s / hs ** 2, rel_tol=1e-14)
    assert math.isclose(A[row, row + 8], 0.5 * sig * sig * v * v / hv ** 2, rel_tol=1e-14)
    assert math.isclose(A[row, row + 8 + 1], rho * sig * s * v * v / (4 * hs * hv), rel_tol=1e-14)
    assert math.isclose(A[row, row - 8 + 1], -rho * sig * s * v * v / (4 * hs * hv), rel_tol=1e-14)


def test_sabr_rows_conserve_constants_in_v_and_reproduce_linear_functions():
    """u = s solves the SABR equation with r = 0 (u_ss = u_sv = u_vv = 0) and meets every boundary
    condition (u(0) = 0, u_s(S_max) = 1, u(V_max) = s): A u + f = 0 exactly."""
    p = W.with_(W.sabr_set4(8), nx=10, nv=6, nt=4)
    A, f = O.sabr_matrix(p)
    S, V, _, _ = O.heston_grid(p)
    u = np.tile(S, int(p["nv"]))
    assert np.abs(A @ u + f).max() <= 1e-12 * np.abs(f).max()


@pytest.mark.slow
def test_sabr_iterations_are_mesh_independent_and_solution_is_cn():
    for make in (W.sabr_set3, W.sabr_set4):
        its = []
        for nt in (16, 32):
            p = make(nt)
            x, info = O.solve(p, tol=1e-9, m=40, maxit=200)
            assert info["converged"]
            U = O.sequential_cn(p)
            assert np.abs(x - U.ravel()).max() <= 1e-8 * np.abs(U).max()
            its.append(info["its"])
        assert max(its) <= 4 and max(its) - min(its) <= 1, its  # the paper: 4 on every mesh


@pytest.mark.slow
def test_sabr_set5_meshes_imply_one_reference_price():
    rows = np.loadtxt(GOLDEN4, ndmin=2)
    assert spread(implied_references(rows, W.sabr_set5)) <= AGREE


@pytest.mark.slow
def test_the_scalar_time_factor_form_does_not_fit_table4(monkeypatch):
    """L(t) = d(t) L with L the operator at t = 0 (the simplification Sec. 5.2 uses to derive the
    preconditioner), planted in place of Eq. 5.7: Table 4's rows then disagree (measured 1.7e-3)."""
    exact = O.sabr_matrix

    def scalar_form(p, t=0.0):
        A0, f0 = exact(p, 0.0)
        d = math.exp(-p["r"] * t)
        return d * A0, d * f0

    monkeypatch.setattr(O, "sabr_matrix", scalar_form)
    rows = np.loadtxt(GOLDEN4, ndmin=2)
    assert spread(implied_references(rows, W.sabr_set5)) > 10 * AGREE


def test_sabr_with_rate_is_time_dependent_and_reduces_at_t0():
    p = W.with_(W.sabr_set5(8), nx=8, nv=4, nt=4)
    assert O.time_dependent(p) and not O.time_dependent(W.sabr_set3(8))
    A0, _ = O.sabr_matrix(p, 0.0)
    A1, _ = O.sabr_matrix(p, 1.0)
    S, V, hs, hv = O.heston_grid(p)
    i, j = 4, 2
    row = j * 8 + (i - 1)
    s, v, b, r = S[i - 1], V[j], p["beta"], p["r"]
    D = math.exp(-r)
    # the u_ss entry scales by D^(2(1-beta)), the u_sv entry by D^(1-beta), the u_vv entry not at all
    ss0 = 0.5 * v * v * s ** (2 * b) / hs ** 2
    assert math.isclose(A0[row, row + 1], ss0 + r * s / (2 * hs), rel_tol=1e-13)
    assert math.isclose(A1[row, row + 1], ss0 * D ** (2 * (1 - b)) + r * s / (2 * hs), rel_tol=1e-13)
    assert math.isclose(A1[row, row + 9] / A0[row, row + 9], D ** (1 - b), rel_tol=1e-13)
    assert math.isclose(A1[row, row + 8], A0[row, row + 8], rel_tol=1e-15)
    # the v = 0 row: u_t = r s u_s - r u
    assert math.isclose(A1[0, 0], -r, rel_tol=1e-15) and math.isclose(A1[1, 2], r * S[1] / (2 * hs), rel_tol=1e-13)


@pytest.mark.slow
def test_sabr_set5_iterations_and_solution():
    its = []
    for nt in (16, 32):
        p = W.sabr_set5(nt)
        x, info = O.solve(p, tol=1e-9, m=40, maxit=300)
        assert info["converged"]
        U = O.sequential_cn(p)
        assert np.abs(x - U.ravel()).max() <= 1e-8 * np.abs(U).max()
        its.append(info["its"])
    assert max(its) <= 6 and max(its) - min(its) <= 1, its  # the paper: 6 on every mesh
    _, info1 = O.solve(W.with_(W.sabr_set5(16), alpha=1.0), tol=1e-9, m=40, maxit=300)
    assert info1["converged"] and info1["its"] >= 5 * max(its), (info1["its"], its)


@pytest.mark.parametrize("alpha", [1e-1, 1e-3])
@pytest.mark.parametrize("make", [W.sabr_set3, W.sabr_set4], ids=["set3", "set4"])
def test_sabr_lemma31_eigenvalues(alpha, make):
    """Lemma 3.1 on the SABR matrix (r = 0): (Nt - 1) N eigenvalues of P_alpha^{-1} M equal 1, the
    other N are 1 / (1 - alpha q(l)^Nt) with q(l) = (1 + l/2) / (1 - l/2) for the eigenvalues l of
    tau A. The zero eigenvalues of A (the v = 0 rows) give q = 1 and the value 1 / (1 - alpha)."""
    p = W.with_(make(8), nx=6, nv=4, nt=6, alpha=alpha)
    N, nt = 24, 6
    A, _ = O.sabr_matrix(p)
    _, tau = O.time_grid(p)
    lam = np.linalg.eigvals(tau * A.toarray())
    q = (1 + lam / 2) / (1 - lam / 2)
    zf = 1.0 / (1.0 - alpha * q ** nt)
    assert np.sum(np.abs(lam) < 1e-12) >= 6  # one zero row per s node on v = 0
    z = O.preconditioned_eigs(p)
    order = np.argsort(np.abs(z - 1))
    unit, rest = z[order[:(nt - 1) * N]], z[order[(nt - 1) * N:]]
    assert np.abs(unit - 1).max() < 1e-8
    for w in zf:
        k = int(np.argmin(np.abs(rest - w)))
        assert abs(rest[k] - w) < 1e-8
        rest = np.delete(rest, k)
    assert np.sum(np.abs(zf - 1 / (1 - alpha)) < 1e-10) >= 6


@pytest.mark.slow
def test_sabr_set5_P_1_iterations_match_table4():
    """Table 4 prints 100 GMRES(40) iterations for P_1 on Set V at Nt = 48 (and 6 for P_alpha); the
    oracle's FGMRES(40) with the same preconditioners takes 99 and 5. The P_1 count grows with the
    mesh (31 and 79 at Nt = 16 and 32); within 10% of the printed one here."""
    p = W.sabr_set5(48)
    _, info1 = O.solve(W.with_(p, alpha=1.0), tol=1e-9, m=40, maxit=300)
    assert info1["converged"] and abs(info1["its"] - 100) <= 10, info1["its"]
