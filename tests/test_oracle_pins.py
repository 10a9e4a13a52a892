"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, brute force, special cases). CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def same_set(a, b, atol):
    """Multiset equality of complex numbers by greedy nearest matching."""
    b = list(b)
    for z in a:
        i = int(np.argmin(np.abs(np.asarray(b) - z)))
        if abs(b[i] - z) > atol:
            return False
        b.pop(i)
    return not b


def small(base, **kw):
    return W.with_(base, **kw)


BS = small(W.bs_put_255x256(), nx=15, nt=16)
BS_CALL = small(BS, payoff="call")
LV = small(W.localvol_2047x2048("fp64"), nx=15, nt=16)
RZ = small(W.riesz_1023x512(), nx=15, nt=16)
ALL = [BS, BS_CALL, LV, RZ]
IDS = ["bs-put", "bs-call", "localvol", "riesz"]


# ---------------------------------------------------------------- closed form (textbook)

def test_bs_closed_form_textbook_example():
    rows = np.loadtxt(os.path.join(GOLDEN, "bs_textbook.txt"), ndmin=2)
    for S, K, r, sig, T, call, put, tol in rows:
        assert abs(O.bs_price(S, K, r, sig, T, "call") - call) < tol
        assert abs(O.bs_price(S, K, r, sig, T, "put") - put) < tol


def test_bs_put_call_parity():
    S = np.linspace(10, 300, 37)
    c = O.bs_price(S, 100.0, 0.05, 0.2, 1.0, "call")
    p = O.bs_price(S, 100.0, 0.05, 0.2, 1.0, "put")
    assert np.allclose(c - p, S - 100.0 * math.exp(-0.05), atol=1e-10)


# ---------------------------------------------------------------- alpha-circulant algebra

@pytest.mark.parametrize("nt", [1, 2, 3, 8, 16])
@pytest.mark.parametrize("alpha", [1e-1, 1e-3])
def test_circulant_diagonalisation(nt, alpha):
    """C_l = V_alpha D_l V_alpha^{-1} with V_alpha = Lambda^{-1} F^* (Sec. 3.1), and the
    eigenvalue sets match eq. (eigCx) up to the orientation of the frequency index."""
    lam, d1, d2 = O.circulant_eigs(nt, alpha)
    C1, C2 = O.alpha_circulants(nt, alpha)
    F = np.fft.fft(np.eye(nt)) / math.sqrt(nt)
    V = np.diag(1.0 / lam) @ F.conj().T
    Vinv = F @ np.diag(lam)
    assert np.allclose(V @ np.diag(d1) @ Vinv, C1, atol=1e-12)
    assert np.allclose(V @ np.diag(d2) @ Vinv, C2, atol=1e-12)
    k = np.arange(nt)
    printed1 = 1 - alpha ** (1 / nt) * np.exp(2j * math.pi * k / nt)
    printed2 = 0.5 + 0.5 * alpha ** (1 / nt) * np.exp(2j * math.pi * k / nt)
    # the printed formula lists the same eigenvalues with the bins in reverse orientation
    assert same_set(d1, printed1, 1e-12)
    assert np.allclose(d1, printed1.conj(), atol=1e-12)
    assert np.allclose(d2, printed2.conj(), atol=1e-12)
    assert np.all(d1.real > 0) and np.all(d2.real > 0)


@pytest.mark.parametrize("p", ALL, ids=IDS)
def test_P_is_M_minus_alpha_R(p):
    """P_alpha = M - alpha R (Sec. 4) where R holds Q2 in block (1, Nt); pins the Kronecker
    assembly of eq. (3.1) against the block form of Sec. 3.2 (constant operators only)."""
    if p["op"] == "localvol":
        pytest.skip("identity holds for the constant-coefficient operator")
    P = O.dense_P(p)
    assert np.allclose(P, O.dense_M(p) - p["alpha"] * O.R_matrix(p), atol=1e-12)


@pytest.mark.parametrize("p", ALL, ids=IDS)
def test_P_block_form(p):
    """Block form of P_alpha in Sec. 3.2: Q1 on the diagonal, -Q2 below, -alpha Q2 corner."""
    nt, nx = p["nt"], p["nx"]
    _, tau = O.time_grid(p)
    Abar = O._dense(O.mean_operator(p))
    Q1 = np.eye(nx) - 0.5 * tau * Abar
    Q2 = np.eye(nx) + 0.5 * tau * Abar
    P = O.dense_P(p)
    blk = lambda i, j: P[i * nx:(i + 1) * nx, j * nx:(j + 1) * nx]
    for i in range(nt):
        assert np.allclose(blk(i, i), Q1, atol=1e-13)
        if i > 0:
            assert np.allclose(blk(i, i - 1), -Q2, atol=1e-13)
    assert np.allclose(blk(0, nt - 1), -p["alpha"] * Q2, atol=1e-13)


# ---------------------------------------------------------------- the three-step apply

@pytest.mark.parametrize("p", ALL, ids=IDS)
@pytest.mark.parametrize("nt,nx", [(1, 7), (2, 5), (3, 6), (8, 7), (16, 15), (12, 9), (15, 7), (35, 5)])
def test_precond_fft_equals_dense_inverse(p, nt, nx):
    """Eq. (3.2) steps (a)-(c) reproduce the brute-force dense P_alpha^{-1} (eq. 3.1)."""
    q = W.with_(p, nt=nt, nx=nx)
    v = W.random_vector(nt * nx, seed=nt * 100 + nx)
    z = O.precond_fft(q, v)
    zd = O.precond_dense(q, v)
    assert np.linalg.norm(z - zd) <= 1e-11 * np.linalg.norm(zd)


def test_precond_single_step_textbook():
    """Nt = 1: P_alpha = (1-alpha) I - (1+alpha)/2 A~, one real tridiagonal solve."""
    q = W.with_(BS, nt=1)
    _, tau = O.time_grid(q)
    A = O._dense(O.mean_operator(q))
    v = W.random_vector(q["nx"], seed=5)
    a = q["alpha"]
    ref = np.linalg.solve((1 - a) * np.eye(q["nx"]) - 0.5 * (1 + a) * tau * A, v)
    assert np.allclose(O.precond_fft(q, v), ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("nt", [8, 9, 16])
def test_precond_conjugate_pairs(nt):
    """Remark 1: for real v and A the spectra come in conjugate pairs, so bins
    Nt-k are the conjugates of bins k."""
    q = W.with_(LV, nt=nt)
    v = W.random_vector(nt * q["nx"], seed=3)
    z, z1, z2 = O.precond_fft(q, v, return_spectrum=True)
    for k in range(1, nt):
        assert np.allclose(z1[nt - k], z1[k].conj(), atol=1e-12)
        assert np.allclose(z2[nt - k], z2[k].conj(), atol=1e-12)
    assert np.abs(z.imag).max() < 1e-12 * np.abs(z.real).max()


# ---------------------------------------------------------------- M, b and sequential CN

@pytest.mark.parametrize("p", ALL, ids=IDS)
def test_aao_solution_equals_sequential_cn(p):
    """The AaO system (eq. 2.2 / 5.8) is block forward substitution of the CN scheme (2.1)."""
    q = W.with_(p, nx=31, nt=24)
    U = O.sequential_cn(q)
    u = spl.spsolve(O.assemble_M(q).tocsc(), O.assemble_b(q))
    assert np.abs(u - U.ravel()).max() <= 1e-12 * np.abs(U).max()


def test_M_kron_equals_blocks():
    """Kronecker form of eq. (2.2) equals the block-bidiagonal form with Q1, -Q2."""
    q = W.with_(BS, nx=9, nt=7)
    _, tau = O.time_grid(q)
    A = O._dense(O.step_operator(q, 0)[0])
    M = O.dense_M(q)
    nx = q["nx"]
    Q1 = np.eye(nx) - 0.5 * tau * A
    Q2 = np.eye(nx) + 0.5 * tau * A
    for i in range(q["nt"]):
        assert np.allclose(M[i * nx:(i + 1) * nx, i * nx:(i + 1) * nx], Q1)
        if i:
            assert np.allclose(M[i * nx:(i + 1) * nx, (i - 1) * nx:i * nx], -Q2)


def test_localvol_without_bump_is_bs():
    q = W.with_(LV, nx=31, nt=16, lv_bump=0.0)
    b = W.with_(BS, nx=31, nt=16, sigma=q["sigma"], r=q["r"])
    assert np.allclose(O.dense_M(q), O.dense_M(b), atol=1e-14)
    assert np.allclose(O.assemble_b(q), O.assemble_b(b), atol=1e-12)


def test_cn_matches_bs_closed_form_under_refinement():
    """CN + central differences converge to the Black-Scholes price; errors on
    [0.5K, 1.5K] fall monotonically under joint refinement and are < 1e-2 at 255 x 256."""
    errs = []
    for k in (5, 6, 7, 8):
        q = W.with_(W.bs_put_255x256(), nx=2 ** k - 1, nt=2 ** k)
        S, _ = O.spatial_grid(q)
        U = O.sequential_cn(q)
        sel = (S >= 50) & (S <= 150)
        ref = O.bs_price(S[sel], q["K"], q["r"], q["sigma"], q["T"], "put")
        errs.append(np.abs(U[-1][sel] - ref).max())
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-2, errs
    assert errs[-2] / errs[-1] > 2.5, errs  # roughly second order


def test_call_closed_form():
    q = W.with_(W.bs_put_255x256(), payoff="call")
    S, _ = O.spatial_grid(q)
    U = O.sequential_cn(q)
    sel = (S >= 50) & (S <= 150)
    ref = O.bs_price(S[sel], q["K"], q["r"], q["sigma"], q["T"], "call")
    assert np.abs(U[-1][sel] - ref).max() < 1e-2


def test_riesz_weights_beta2_is_three_point_laplacian():
    g = O.riesz_weights(2.0, 6)
    assert np.allclose(g, [2, -1, 0, 0, 0, 0], atol=1e-14)
    g15 = O.riesz_weights(1.5, 400)
    assert g15[0] > 0 and np.all(g15[1:] < 0)
    # sum over all integers is zero: g_0 + 2 sum_{k>=1} g_k -> 0 (slow tail ~ k^-(1+beta))
    assert abs(g15[0] + 2 * g15[1:].sum()) < 2e-3


@pytest.mark.parametrize("beta", [1.2, 1.5, 1.8])
def test_riesz_weights_converge_to_the_closed_form_riesz_derivative(beta):
    """The fractional centred difference -h^-beta sum_k g_k f(x - k h) (the weights and scaling of
    the Riesz operator, Eq. 1.2) converges at second order to the Riesz derivative
    -(-d^2/dx^2)^(beta/2) f. For the Lorentzian f = 1/(1 + x^2), whose Fourier transform is
    pi exp(-|xi|), the derivative has the closed form -Gamma(beta + 1) Re[(1 - i x)^-(beta + 1)]
    (f'' at beta = 2). A wrong sign, scale or exponent in the weights fails this at any beta."""
    f = lambda x: 1.0 / (1.0 + x * x)
    for x0 in (0.0, 0.7):
        exact = -math.gamma(beta + 1.0) * ((1.0 - 1j * x0) ** (-(beta + 1.0))).real
        errs = []
        for h in (0.1, 0.05):
            M = int(round(400.0 / h))  # the sum's tail beyond M h is below 1e-7
            g = O.riesz_weights(beta, M + 1)
            k = np.arange(-M, M + 1)
            approx = -h ** (-beta) * np.sum(g[np.abs(k)] * f(x0 - k * h))
            errs.append(abs(approx - exact))
        assert errs[1] <= 4e-3 * math.gamma(beta + 1.0), (beta, x0, errs, exact)  # the derivative's scale
        assert 3.8 <= errs[0] / errs[1] <= 4.2, (beta, x0, errs)


def test_riesz_beta2_is_log_price_bs():
    """At beta = 2 the Riesz problem is Black-Scholes in x = ln S; compare with the closed form."""
    q = W.with_(W.riesz_1023x512(), beta=2.0, nx=255, nt=128)
    x, _ = O.spatial_grid(q)
    U = O.sequential_cn(q)
    sel = np.abs(x) < 0.5
    ref = O.bs_price(np.exp(x[sel]), q["K"], q["r"], q["sigma"], q["T"], "put")
    assert np.abs(U[-1][sel] - ref).max() < 2e-4


def test_cn_non_growth_symmetric_nsd():
    """Theorem 2.1: for negative semi-definite A, ||R(tau A)||_2 <= 1."""
    q = W.with_(RZ, r=0.5 * RZ["sigma"] ** 2 * 0 + 0.0, sigma=0.25)
    q = W.with_(q, r=0.5 * q["sigma"] ** 2)  # r = kappa removes the drift
    A = O._dense(O.mean_operator(q))
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).max() <= 0
    _, tau = O.time_grid(q)
    I = np.eye(A.shape[0])
    R = np.linalg.solve(I - 0.5 * tau * A, I + 0.5 * tau * A)
    assert np.linalg.norm(R, 2) <= 1 + 1e-12


# ---------------------------------------------------------------- spectral results

@pytest.mark.parametrize("p", [BS, LV, RZ], ids=["bs", "localvol-mean", "riesz"])
@pytest.mark.parametrize("alpha", [0.5, 1e-1, 1e-2])
@pytest.mark.parametrize("nt", [8, 9, 10])
def test_lemma31_theorem31(p, alpha, nt):
    """(Nt-1) Nx eigenvalues of P^{-1} M equal 1; the other Nx lie in the annulus
    1/(1+alpha) <= |z| <= 1/(1-alpha) with Re z > 0 (constant operator); for even and odd Nt."""
    q = W.with_(p, nx=9, nt=nt, alpha=alpha)
    if q["op"] == "localvol":
        q = W.with_(q, op="matrix", A=O._dense(O.mean_operator(q)))
    A = O._dense(O.mean_operator(q))
    assert np.linalg.eigvals(A).real.max() <= 1e-12  # hypothesis Re lambda(A) <= 0
    ev = O.preconditioned_eigs(q)
    ones = np.abs(ev - 1) < 1e-7
    assert ones.sum() == (q["nt"] - 1) * q["nx"]
    rest = ev[~ones]
    assert np.all(np.abs(rest) >= 1 / (1 + alpha) - 1e-10)
    assert np.all(np.abs(rest) <= 1 / (1 - alpha) + 1e-10)
    assert np.all(rest.real > 0)
    # Lemma 3.1: the remaining ones are the eigenvalues of (I - alpha J_Nt)^{-1}
    _, tau = O.time_grid(q)
    I = np.eye(q["nx"])
    J = np.linalg.matrix_power(np.linalg.solve(I - 0.5 * tau * A, I + 0.5 * tau * A), q["nt"])
    ref = np.linalg.eigvals(np.linalg.inv(I - alpha * J))
    assert same_set(rest, ref, 1e-7)


def test_corollary_symmetric_real_interval():
    q = W.with_(RZ, nx=9, nt=8, alpha=0.2)
    q = W.with_(q, r=0.5 * q["sigma"] ** 2)
    ev = O.preconditioned_eigs(q)
    assert np.abs(ev.imag).max() < 1e-8
    assert ev.real.min() >= 1 / 1.2 - 1e-10 and ev.real.max() <= 1 / 0.8 + 1e-10


def test_remark_upper_bound_attained_with_zero_eigenvalue():
    """With a zero eigenvalue of A, 1/(1-alpha) is an eigenvalue of P^{-1} M."""
    A = np.diag([0.0, -1.0, -4.0, -9.0]) * 30
    q = dict(op="matrix", A=A, nx=4, nt=6, T=1.0, alpha=0.3, K=1.0, r=0.0)
    ev = O.preconditioned_eigs(q)
    assert np.min(np.abs(ev - 1 / 0.7)) < 1e-10


def test_remark_P1_singular_with_singular_A():
    A = np.diag([0.0, -1.0, -4.0]) * 10
    q = dict(op="matrix", A=A, nx=3, nt=4, T=1.0, alpha=1.0, K=1.0, r=0.0)
    _, d1, d2 = O.circulant_eigs(4, 1.0)
    assert abs(d1[0]) < 1e-15 and abs(d2[0] - 1) < 1e-15
    s = np.linalg.svd(O.dense_P(q), compute_uv=False)
    assert s.min() < 1e-12 * s.max()
    q["alpha"] = 1e-2
    s = np.linalg.svd(O.dense_P(q), compute_uv=False)
    assert s.min() > 1e-3


@pytest.mark.parametrize("p", [BS, RZ], ids=["bs", "riesz"])
def test_theorem22_condition_bounds(p):
    q = W.with_(p, nx=9, nt=12)
    A = O._dense(O.mean_operator(q))
    s = np.linalg.svd(O.dense_M(q), compute_uv=False)
    _, tau = O.time_grid(q)
    assert s.max() <= 2 + tau * np.linalg.norm(A, 2) + 1e-12
    assert s.min() >= 1 / q["nt"] - 1e-12
    assert s.max() / s.min() <= 2 * q["nt"] + q["T"] * np.linalg.norm(A, 2) + 1e-9


def test_lemma41_normal_A():
    q = W.with_(RZ, nx=9, nt=10)
    q = W.with_(q, r=0.5 * q["sigma"] ** 2)
    MR = np.linalg.solve(O.dense_M(q), O.R_matrix(q))
    assert np.linalg.norm(MR, 2) <= math.sqrt(q["nt"]) + 1e-12


# ---------------------------------------------------------------- FGMRES

@pytest.mark.parametrize("p", ALL, ids=IDS)
def test_fgmres_reaches_tolerance_and_cn(p):
    q = W.with_(p, nx=63, nt=64, tol=1e-10, m=20)
    x, info = O.solve(q)
    assert info["converged"] and info["rel_res"] <= 1e-10
    M, b = O.assemble_M(q), O.assemble_b(q)
    assert np.linalg.norm(b - M @ x) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-9)
    U = O.sequential_cn(q)
    assert np.abs(x - U.ravel()).max() <= 1e-7 * np.abs(U).max()
    assert info["its"] <= 10


def test_fgmres_dense_and_fft_preconditioners_agree():
    q = W.with_(BS, nx=15, nt=16, tol=1e-12)
    x1, i1 = O.solve(q, precond="fft")
    x2, i2 = O.solve(q, precond="dense")
    assert i1["its"] == i2["its"]
    assert np.allclose(x1, x2, rtol=1e-10, atol=1e-10)


def test_P_alpha_beats_P_1_and_is_mesh_independent():
    its = []
    for k in (5, 6, 7):
        q = W.with_(W.bs_put_255x256(), nx=2 ** k - 1, nt=2 ** k, alpha=1e-3, tol=1e-9, m=40)
        _, info = O.solve(q)
        _, info1 = O.solve(W.with_(q, alpha=1.0), maxit=400)
        assert info["its"] < info1["its"]
        its.append(info["its"])
    assert max(its) - min(its) <= 1, its


def test_fgmres_restart_and_history():
    q = W.with_(BS, nx=31, nt=32, tol=1e-12)
    x, info = O.solve(q, m=2, maxit=200)
    assert info["converged"] and info["restarts"] >= 2
    x2, info2 = O.solve(q, m=30)
    assert np.allclose(x, x2, rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------- planted mistakes

def test_planted_conjugated_eigenvalues_are_caught(monkeypatch):
    """Pairing each bin with the conjugate eigenvalue (the sign ambiguity of eq. eigCx)
    must break the dense-inverse pin."""
    real = O.circulant_eigs

    def wrong(nt, alpha):
        lam, d1, d2 = real(nt, alpha)
        return lam, d1.conj(), d2.conj()

    monkeypatch.setattr(O, "circulant_eigs", wrong)
    q = W.with_(BS, nx=7, nt=8)
    v = W.random_vector(56)
    assert np.linalg.norm(O.precond_fft(q, v) - O.precond_dense(q, v)) > 1e-6 * np.linalg.norm(v)


def test_planted_dropped_forcing_is_caught(monkeypatch):
    """Dropping the Dirichlet forcing breaks the closed-form pin (call: far boundary;
    put: near S = 0)."""
    monkeypatch.setattr(O, "forcing", lambda p, k: np.zeros(int(p["nx"])))
    for kind, lo, hi in (("call", 50, 150), ("put", 1, 40)):
        q = W.with_(W.bs_put_255x256(), nx=63, nt=64, payoff=kind)
        S, _ = O.spatial_grid(q)
        U = O.sequential_cn(q)
        sel = (S >= lo) & (S <= hi)
        ref = O.bs_price(S[sel], q["K"], q["r"], q["sigma"], q["T"], kind)
        assert np.abs(U[-1][sel] - ref).max() > 1e-1, kind


def test_block_matvec_equals_assembled_M():
    for p in (W.with_(RZ, nx=17, nt=12), W.with_(BS, nx=13, nt=9)):
        x = W.random_vector(p["nx"] * p["nt"], seed=2)
        assert np.allclose(O.matvec_blocks(p, x), O.matvec(p, x), rtol=1e-13, atol=1e-13)


def test_apply_P_equals_dense_P():
    """The blockwise P_alpha product equals the dense Kronecker form of Eq. 3.1, including the
    alpha corner and Nt = 1, 2."""
    rng = np.random.default_rng(3)
    for nx, nt in [(5, 1), (6, 2), (7, 8), (4, 12)]:
        for p in (W.with_(W.bs_put_255x256(), nx=nx, nt=nt), W.with_(W.localvol_2047x2048("fp64"), nx=nx, nt=nt)):
            z = rng.standard_normal(nx * nt)
            assert np.allclose(O.apply_P(p, z), O.dense_P(p) @ z, rtol=1e-13, atol=1e-13)


def test_apply_P_inverts_precond_fft():
    """P_alpha (P_alpha^{-1} v) = v for the FFT apply of Eq. 3.2 at a size the dense form cannot
    reach."""
    p = W.with_(W.localvol_2047x2048("fp64"), nx=200, nt=64)
    v = W.random_vector(200 * 64, seed=4)
    r = O.apply_P(p, O.precond_fft(p, v)) - v
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(v)
