"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances. FP64 entry points that are pure stencils (rhs, matvec) differ from the oracle
only in rounding order: 1e-13 relative. The preconditioner apply multiplies rounding errors
of the time-axis FFT (~u log2 nt) by up to 1/alpha through Lambda_alpha^{-1}; the bound used
is ||z - z_ref|| <= C u log2(2 nt) / alpha ||z_ref|| with u the unit roundoff of the apply
(2^-53 FP64, 2^-24 mixed) and C = 20.
"""
import math

import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module")
def aao():
    from paper_2401_16113_gb300 import aao as A, build
    build.build()
    A.load()
    assert torch.cuda.is_available()
    return A


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


BS = W.bs_put_255x256()
LV = W.localvol_2047x2048("fp64")

SHAPES = [(2, 1), (3, 2), (15, 16), (37, 8), (64, 64), (65, 32), (127, 128), (300, 256), (511, 64)]


def problems(nx, nt):
    return [W.with_(BS, nx=nx, nt=nt), W.with_(BS, nx=nx, nt=nt, payoff="call"),
            W.with_(LV, nx=nx, nt=nt)]


@pytest.mark.parametrize("nx,nt", SHAPES)
def test_rhs_matches_oracle(aao, nx, nt):
    for p in problems(nx, nt):
        h = aao.aao_create(p)
        b = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
        aao.aao_rhs(h, b)
        ref = O.assemble_b(p)
        assert relmax(host(b), ref) <= 1e-13, p
        h.close()


@pytest.mark.parametrize("nx,nt", SHAPES)
def test_matvec_matches_oracle(aao, nx, nt):
    for p in problems(nx, nt):
        h = aao.aao_create(p)
        x = W.random_vector(nx * nt, seed=nx + 7 * nt)
        y = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
        aao.aao_matvec(h, dev(x), y)
        ref = O.matvec(p, x)
        assert relmax(host(y), ref) <= 1e-13, p
        h.close()


@pytest.mark.parametrize("scale", [1.0, 1e-310])
def test_matvec_zeros_and_subnormals(aao, scale):
    # the kernel forms 2 x_t by bit operations: exact zeros (both signs) mixed into the input, and
    # an input entirely in the FP64 subnormal range (scale 1e-310), where 2 x is a shift of the
    # magnitude bits, must give the oracle's product
    nx, nt = 67, 32
    for p in problems(nx, nt):
        h = aao.aao_create(p)
        x = W.random_vector(nx * nt, seed=11) * scale
        x[::3] = 0.0
        x[1::7] = -0.0
        x[5 * nx:7 * nx] = 0.0
        y = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
        aao.aao_matvec(h, dev(x), y)
        ref = O.matvec(p, x)
        assert relmax(host(y), ref) <= 1e-13, p
        h.close()


def precond_bound(p):
    u = U32 if p["precision"] == "mixed" else U64
    return 20.0 * u * math.log2(2 * p["nt"]) / p["alpha"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("alpha", [1e-2, 1e-3])
@pytest.mark.parametrize("nx,nt", SHAPES)
def test_precond_matches_oracle(aao, nx, nt, precision, alpha):
    for p in problems(nx, nt):
        p = W.with_(p, precision=precision, alpha=alpha)
        h = aao.aao_create(p)
        v = W.random_vector(nx * nt, seed=3 * nx + nt)
        z = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
        aao.precond_apply(h, dev(v), z)
        ref = O.precond_fft(p, v)
        assert rel(host(z), ref) <= precond_bound(p), (p["op"], p["payoff"], rel(host(z), ref))
        h.close()


def test_precond_small_matches_dense_inverse(aao):
    """Brute force: the dense P_alpha^{-1} of eq. (3.1), independent of any FFT."""
    for nx, nt in [(5, 4), (7, 8), (9, 16)]:
        for p in problems(nx, nt):
            h = aao.aao_create(p)
            v = W.random_vector(nx * nt, seed=nx * nt)
            z = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
            aao.precond_apply(h, dev(v), z)
            assert rel(host(z), O.precond_dense(p, v)) <= precond_bound(p)
            h.close()


def test_precond_in_place(aao):
    p = W.with_(BS, nx=63, nt=32)
    h = aao.aao_create(p)
    v = W.random_vector(63 * 32, seed=1)
    t = dev(v)
    aao.precond_apply(h, t, t)
    assert rel(host(t), O.precond_fft(p, v)) <= precond_bound(p)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_precond_full_size_localvol(aao, precision):
    """2047 x 2048 local volatility, the launch configuration of the benchmark."""
    p = W.with_(LV, precision=precision)
    h = aao.aao_create(p)
    v = W.random_vector(W.unknowns(p), seed=11)
    z = torch.empty(W.unknowns(p), dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z)
    ref = O.precond_fft(p, v)
    assert rel(host(z), ref) <= precond_bound(p)


# Every radix plan of the register FFT (nt = 2^7 .. 2^13: 16|8, 16|2|8, 16|4|8, 16|8|8, 16|16|8,
# 16|16|2|8, 16|16|4|8) and every configuration of the partitioned tridiagonal solve (32 .. 512
# threads per bin, coefficients staged in shared memory or read from global memory).
# The check is the backward error ||v - P_alpha z|| / ||v|| (P_alpha applied by the oracle in
# FP64), bounded like the forward error above: an FP32 solve's backward error does not depend on
# the conditioning of the shifted systems. Their forward error does (mu_0 I - tau A-bar reaches a
# condition number ~1e5 for Nx = 8191, Nt = 128), so it is checked only where Nx <= 2047.
PLAN_SHAPES = [(1023, 512, "fp64"), (1023, 512, "mixed"), (1500, 1024, "mixed"), (700, 4096, "fp64"),
               (700, 4096, "mixed"), (300, 8192, "mixed"), (4095, 256, "fp64"), (4095, 256, "mixed"),
               (5000, 128, "mixed"), (8191, 128, "mixed")]


@pytest.mark.parametrize("nx,nt,precision", PLAN_SHAPES)
def test_precond_fft_plans_and_solver_sizes(aao, nx, nt, precision):
    p = W.with_(LV, nx=nx, nt=nt, precision=precision)
    h = aao.aao_create(p)
    v = W.random_vector(nx * nt, seed=5 * nx + nt)
    z = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z)
    zh = host(z)
    back = rel(O.apply_P(p, zh), v)
    assert back <= precond_bound(p), back
    if nx <= 2047:
        assert rel(zh, O.precond_fft(p, v)) <= precond_bound(p)
    h.close()


def test_fgmres_fp64_bs_put(aao):
    """Plain FP64 solve of the 255 x 256 put to 1e-10: equals sequential CN and the
    closed form within the discretisation error."""
    p = BS
    h = aao.aao_create(p)
    n = W.unknowns(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = aao.fgmres_solve(h, b, x, 1e-10, 20, 200)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10
    xs = host(x)
    M, bref = O.assemble_M(p), O.assemble_b(p)
    assert np.linalg.norm(bref - M @ xs) <= 1.01e-10 * np.linalg.norm(bref)
    U = O.sequential_cn(p)
    assert relmax(xs, U.ravel()) <= 1e-8
    S, _ = O.spatial_grid(p)
    sel = (S >= 50) & (S <= 150)
    assert np.abs(xs.reshape(p["nt"], p["nx"])[-1][sel]
                  - O.bs_price(S[sel], p["K"], p["r"], p["sigma"], p["T"], "put")).max() < 1e-2
    assert st["iterations"] <= 10


def test_fgmres_mixed_localvol_full_size(aao):
    """Mixed precision 2047 x 2048 local volatility to relative residual 1e-8 (FP64 check); the
    option values at maturity within 1e-8 of sequential CN."""
    p = W.localvol_2047x2048("mixed")
    h = aao.aao_create(p)
    n = W.unknowns(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = aao.fgmres_solve(h, b, x, 1e-8, 30, 300)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8, st
    xs = host(x)
    M, bref = O.assemble_M(p), O.assemble_b(p)
    assert np.linalg.norm(bref - M @ xs) <= 1.01e-8 * np.linalg.norm(bref)
    U = O.sequential_cn(p)
    err = np.abs(xs.reshape(p["nt"], p["nx"])[-1] - U[-1]).max() / np.abs(U[-1]).max()
    print("mixed localvol: its", st["iterations"], "maturity error", err)
    assert err <= 1e-8


def test_fgmres_host_variant_matches_device(aao):
    p = W.with_(BS, nx=127, nt=128, precision="mixed", alpha=1e-3)
    h = aao.aao_create(p)
    n = W.unknowns(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    st = aao.fgmres_solve_zero(h, b, x, 1e-9, 20, 100)
    bh = host(b).copy()
    xh = np.zeros(n)
    st2 = aao.fgmres_solve_host(h, bh, xh, 1e-9, 20, 100)
    assert st2["iterations"] == st["iterations"]
    assert np.array_equal(xh, host(x))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fgmres_zero_guess_entry_point(aao, precision):
    """fgmres_solve_zero ignores what x holds on entry (NaN here) and reaches the solution of
    fgmres_solve from x = 0 in the same number of iterations; the first residual is b itself, so the
    two differ only in the rounding order of ||b||."""
    cases = [W.with_(BS, nx=127, nt=128, precision=precision, alpha=1e-3),
             W.with_(LV, nx=255, nt=256, precision=precision, alpha=1e-3)]
    if precision == "mixed":
        cases += [W.with_(W.riesz_1023x512(), nx=127, nt=64), W.heston_set1(16)]
    for p in cases:
        h = aao.aao_create(p)
        n = W.unknowns(p)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        aao.aao_rhs(h, b)
        x0 = torch.zeros_like(b)
        st0 = aao.fgmres_solve(h, b, x0, 1e-9, 30, 200)
        xz = torch.full_like(b, float("nan"))
        stz = aao.fgmres_solve_zero(h, b, xz, 1e-9, 30, 200)
        assert stz["status"] == 0 and st0["status"] == 0, (stz, st0)
        assert stz["iterations"] == st0["iterations"], (p["op"], stz, st0)
        assert rel(host(xz), host(x0)) <= 1e-9, p["op"]
        h.close()


def test_fgmres_restart_small_m(aao):
    p = W.with_(BS, nx=63, nt=64)
    h = aao.aao_create(p)
    n = W.unknowns(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = aao.fgmres_solve(h, b, x, 1e-12, 1, 400)
    assert st["status"] == 0 and st["restarts"] >= 2
    ref, _ = O.solve(W.with_(p, tol=1e-12))
    assert relmax(host(x), ref) <= 1e-9


@pytest.mark.parametrize("precision,m,k", [("fp64", 1, 3), ("fp64", 2, 1), ("mixed", 2, 1)])
def test_fgmres_checkpoint_resume(aao, precision, m, k):
    """A restart boundary is a checkpoint: FGMRES(m) restarts from x alone, so a solve stopped
    after k whole cycles (maxit = k m) and resumed from its x takes the same total number of
    inner iterations and reaches the same x as the uninterrupted solve."""
    p = W.with_(BS, nx=63, nt=64, precision=precision)
    h = aao.aao_create(p)
    n = W.unknowns(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    tol = 1e-12 if precision == "fp64" else 1e-10
    x_full = torch.zeros(n, dtype=torch.float64, device="cuda")
    st_full = aao.fgmres_solve(h, b, x_full, tol, m, 400)
    assert st_full["status"] == 0 and st_full["iterations"] > k * m
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st1 = aao.fgmres_solve(h, b, x, tol, m, k * m)
    assert st1["status"] == aao.AAO_NOT_CONVERGED and st1["iterations"] == k * m
    saved = host(x).copy()                      # the checkpoint: x and the iteration count
    x2 = dev(saved)
    st2 = aao.fgmres_solve(h, b, x2, tol, m, 400)
    assert st2["status"] == 0
    assert st1["iterations"] + st2["iterations"] == st_full["iterations"]
    assert relmax(host(x2), host(x_full)) <= 1e-13
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fgmres_exhausted_krylov_space(aao, precision):
    """A 3 x 2 system (6 unknowns) with FGMRES(10) and alpha = 1: the Krylov space fills up, the
    last raw vector cancels almost entirely (the second Gram-Schmidt pass and the steps queued
    behind it are exercised) and the solve still ends at the tolerance."""
    p = W.with_(BS, nx=3, nt=2, alpha=1.0, precision=precision)
    h = aao.aao_create(p)
    b = torch.empty(6, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.zeros(6, dtype=torch.float64, device="cuda")
    st = aao.fgmres_solve(h, b, x, 1e-13, 10, 50)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-13, st
    ref, _ = O.solve(W.with_(p, tol=1e-13))
    assert relmax(host(x), ref) <= 1e-10


def test_fgmres_maxit_reports_not_converged(aao):
    p = W.with_(BS, nx=63, nt=64, alpha=1.0)
    h = aao.aao_create(p)
    n = W.unknowns(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = aao.fgmres_solve(h, b, x, 1e-14, 5, 3)
    assert st["status"] == aao.AAO_NOT_CONVERGED and st["iterations"] == 3


def test_fgmres_zero_rhs(aao):
    p = W.with_(BS, nx=31, nt=16)
    h = aao.aao_create(p)
    b = torch.zeros(31 * 16, dtype=torch.float64, device="cuda")
    x = torch.ones(31 * 16, dtype=torch.float64, device="cuda")
    st = aao.fgmres_solve(h, b, x, 1e-10, 10, 10)
    assert st["status"] == 0 and float(x.abs().max()) == 0.0


def test_fgmres_nan_rhs_reports_breakdown(aao):
    p = W.with_(BS, nx=31, nt=16)
    h = aao.aao_create(p)
    b = torch.ones(31 * 16, dtype=torch.float64, device="cuda")
    b[17] = float("nan")
    x = torch.zeros(31 * 16, dtype=torch.float64, device="cuda")
    st = aao.fgmres_solve(h, b, x, 1e-10, 10, 10)
    assert st["status"] == aao.AAO_BREAKDOWN


# ---------------------------------------------------------------- Riesz (dense Toeplitz) operator

RZ = W.riesz_1023x512()
RZ_SHAPES = [(15, 16), (31, 8), (63, 32), (127, 64), (100, 2)]


@pytest.mark.parametrize("beta", [1.5, 2.0])
@pytest.mark.parametrize("nx,nt", RZ_SHAPES)
def test_riesz_rhs_matvec_match_oracle(aao, nx, nt, beta):
    p = W.with_(RZ, nx=nx, nt=nt, beta=beta)
    h = aao.aao_create(p)
    n = nx * nt
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    ref = O.assemble_b(p)
    assert relmax(host(b), ref) <= 1e-12
    x = W.random_vector(n, seed=nx + nt)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_matvec(h, dev(x), y)
    assert relmax(host(y), O.matvec(p, x)) <= 1e-12


@pytest.mark.parametrize("alpha", [1e-2, 1e-3])
@pytest.mark.parametrize("nx,nt", RZ_SHAPES)
def test_riesz_precond_matches_oracle(aao, nx, nt, alpha):
    p = W.with_(RZ, nx=nx, nt=nt, alpha=alpha)
    h = aao.aao_create(p)
    v = W.random_vector(nx * nt, seed=5 * nx + nt)
    z = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z)
    ref = O.precond_fft(p, v)
    assert rel(host(z), ref) <= precond_bound(p), rel(host(z), ref)


@pytest.mark.parametrize("nx", [1800, 2047])
def test_riesz_precond_wide_grids(aao, nx):
    """The Riesz operator with drift at nx above 1784, where the create-time inverse runs with 8
    identity columns per CTA (16 do not fit in shared memory); its matvec and right-hand side at
    the same widths."""
    p = W.with_(RZ, nx=nx, nt=4, alpha=1e-2)
    h = aao.aao_create(p)
    v = W.random_vector(nx * 4, seed=nx)
    z = torch.empty(nx * 4, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z)
    assert rel(host(z), O.precond_fft(p, v)) <= precond_bound(p)
    # the FP64 matvec and right-hand side at the widest circulant embedding (N2 = 4096)
    b = torch.empty(nx * 4, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    assert relmax(host(b), O.assemble_b(p)) <= 1e-12
    y = torch.empty(nx * 4, dtype=torch.float64, device="cuda")
    aao.aao_matvec(h, dev(v), y)
    assert relmax(host(y), O.matvec(p, v)) <= 1e-12
    h.close()


def test_riesz_precond_small_matches_dense_inverse(aao):
    for nx, nt in [(7, 4), (9, 8)]:
        p = W.with_(RZ, nx=nx, nt=nt, alpha=1e-2)
        h = aao.aao_create(p)
        v = W.random_vector(nx * nt, seed=nx)
        z = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
        aao.precond_apply(h, dev(v), z)
        assert rel(host(z), O.precond_dense(p, v)) <= precond_bound(p)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_P_alpha_beats_P_1_on_the_gpu_and_matches_oracle_counts(aao, precision):
    """Sec. 3-4: P_alpha (alpha = 1e-3) needs fewer FGMRES iterations than the block-circulant
    P_1 (alpha = 1), and its count does not grow with the mesh (nx = 2^k - 1, nt = 2^k). In FP64
    the GPU counts equal the oracle's on the smallest mesh."""
    its_a, its_1 = [], []
    for k in (6, 7, 8):
        q = W.with_(BS, nx=2 ** k - 1, nt=2 ** k, precision=precision)
        res = {}
        for alpha in (1e-3, 1.0):
            p = W.with_(q, alpha=alpha)
            h = aao.aao_create(p)
            n = W.unknowns(p)
            b = torch.empty(n, dtype=torch.float64, device="cuda")
            aao.aao_rhs(h, b)
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            st = aao.fgmres_solve(h, b, x, 1e-9, 40, 400)
            assert st["status"] == 0, (k, alpha, st)
            res[alpha] = st["iterations"]
            h.close()
        its_a.append(res[1e-3])
        its_1.append(res[1.0])
        assert res[1e-3] < res[1.0], (k, res)
        if precision == "fp64" and k == 6:
            for alpha in (1e-3, 1.0):
                _, info = O.solve(W.with_(q, alpha=alpha, tol=1e-9, m=40), maxit=400)
                assert abs(info["its"] - res[alpha]) <= 1, (alpha, info["its"], res[alpha])
    assert max(its_a) - min(its_a) <= 1, its_a
    print(precision, "P_alpha its", its_a, "P_1 its", its_1)


RZS = W.riesz_sym_1023x512()


@pytest.mark.parametrize("alpha", [1e-2, 1e-3])
@pytest.mark.parametrize("nx,nt", RZ_SHAPES + [(200, 4), (64, 1)])
def test_riesz_symmetric_precond_matches_oracle(aao, nx, nt, alpha):
    """No drift (r = sigma^2/2): step (b) by the eigendecomposition and two complex x real
    products per apply, against the oracle's dense shifted solves."""
    p = W.with_(RZS, nx=nx, nt=nt, alpha=alpha)
    assert p["r"] == 0.5 * p["sigma"] ** 2
    h = aao.aao_create(p)
    v = W.random_vector(nx * nt, seed=7 * nx + nt)
    z = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z)
    ref = O.precond_fft(p, v)
    assert rel(host(z), ref) <= precond_bound(p), rel(host(z), ref)
    # a second apply (the padding of the half spectrum must still be zero) gives the same bits
    z2 = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z2)
    assert np.array_equal(host(z), host(z2))


def test_riesz_symmetric_precond_small_matches_dense_inverse(aao):
    for nx, nt in [(7, 4), (9, 8), (2, 2)]:
        p = W.with_(RZS, nx=nx, nt=nt, alpha=1e-2)
        h = aao.aao_create(p)
        v = W.random_vector(nx * nt, seed=nx)
        z = torch.empty(nx * nt, dtype=torch.float64, device="cuda")
        aao.precond_apply(h, dev(v), z)
        assert rel(host(z), O.precond_dense(p, v)) <= precond_bound(p)


def test_riesz_symmetric_full_size_solve():
    """1023 x 512 Riesz without drift, mixed precision, spectral step (b): true residual <= 1e-8
    and the solution against sequential CN."""
    from paper_2401_16113_gb300 import aao as A
    p = RZS
    h = A.aao_create(p)
    n = W.unknowns(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A.aao_rhs(h, b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = A.fgmres_solve(h, b, x, 1e-8, 30, 300)
    assert st["status"] == 0, st
    xs, bs = host(x), host(b)
    assert np.linalg.norm(bs - O.matvec_blocks(p, xs)) <= 1.01e-8 * np.linalg.norm(bs)
    U = O.sequential_cn(p)
    err = np.abs(xs.reshape(p["nt"], p["nx"])[-1] - U[-1]).max() / np.abs(U[-1]).max()
    print("riesz symmetric full size: its", st["iterations"], "maturity error", err)
    assert err <= 1e-8


def test_riesz_full_size_solve():
    """1023 x 512 Riesz (beta 1.5) put, mixed precision: the true residual (FP64, by the
    oracle's block-row product with the dense A) <= 1e-8 and the solution against sequential CN."""
    from paper_2401_16113_gb300 import aao as A
    p = RZ
    h = A.aao_create(p)
    n = W.unknowns(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A.aao_rhs(h, b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = A.fgmres_solve(h, b, x, 1e-8, 30, 300)
    assert st["status"] == 0, st
    xs, bs = host(x), host(b)
    assert np.linalg.norm(bs - O.matvec_blocks(p, xs)) <= 1.01e-8 * np.linalg.norm(bs)
    U = O.sequential_cn(p)
    err = np.abs(xs.reshape(p["nt"], p["nx"])[-1] - U[-1]).max() / np.abs(U[-1]).max()
    print("riesz full size: its", st["iterations"], "maturity error", err)
    assert err <= 1e-8
