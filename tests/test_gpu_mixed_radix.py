"""Parity of the mixed-radix FFT path (nt with prime factors 2, 3, 5, 7 but not a power of two)
with the FP64 oracle, through the C ABI.

The oracle's apply takes the DFT along t for any nt (steps (a)-(c) of Eq. 3.2); it is pinned
against the dense P_alpha^{-1} for nt = 3, 9, 12, 15 and 35 in the CPU tests. The error bound
is the one of the power-of-two path: ||z - z_ref|| <= 20 u log2(2 nt) / alpha ||z_ref||.
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


def bound(p):
    u = U32 if p["precision"] == "mixed" else U64
    return 20.0 * u * math.log2(2 * p["nt"]) / p["alpha"]


BS = W.bs_put_255x256()
LV = W.localvol_2047x2048("fp64")

# every radix alone (3, 5, 7, 2 x 3), mixed plans with radix-4 stages, ragged nx that leaves
# partial tiles, odd nt (no Nyquist bin) and even nt
SHAPES = [(5, 3), (7, 5), (15, 6), (33, 7), (37, 12), (64, 15), (65, 35), (127, 96), (300, 105), (511, 210)]


def problems(nx, nt):
    return [W.with_(BS, nx=nx, nt=nt), W.with_(BS, nx=nx, nt=nt, payoff="call"),
            W.with_(LV, nx=nx, nt=nt)]


def apply(aao, p, v):
    h = aao.aao_create(p)
    z = torch.empty(v.size, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z)
    out = host(z)
    h.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("alpha", [1e-2, 1e-3])
@pytest.mark.parametrize("nx,nt", SHAPES)
def test_mixed_radix_precond_matches_oracle(aao, nx, nt, precision, alpha):
    for p in problems(nx, nt):
        p = W.with_(p, precision=precision, alpha=alpha)
        v = W.random_vector(nx * nt, seed=7 * nx + nt)
        z = apply(aao, p, v)
        ref = O.precond_fft(p, v)
        assert rel(z, ref) <= bound(p), (p["op"], p["payoff"], rel(z, ref))


def test_mixed_radix_precond_matches_dense_inverse(aao):
    """Brute force: the dense P_alpha^{-1} of Eq. 3.1, independent of any FFT."""
    for nx, nt in [(5, 3), (7, 6), (6, 10), (4, 21)]:
        for p in problems(nx, nt):
            v = W.random_vector(nx * nt, seed=nx * nt)
            assert rel(apply(aao, p, v), O.precond_dense(p, v)) <= bound(p)


# larger plans up to the shared-memory limits (FP64 nt <= 4096, mixed nt <= 8192): 3 x 2^9,
# 2^4 x 3 x 5^3 (FP64), 3 x 2^10 (FP64), 7 x 2^10, 3^8, 3^2 x 5 x 7^2; the backward error
# ||v - P_alpha z|| / ||v|| and, for nx <= 2047, the forward error
LARGE = [(1023, 1536, "mixed"), (1023, 1536, "fp64"), (700, 2000, "fp64"), (500, 3072, "fp64"),
         (300, 7168, "mixed"), (257, 6561, "mixed"), (1000, 2205, "mixed")]


@pytest.mark.parametrize("nx,nt,precision", LARGE)
def test_mixed_radix_large_plans(aao, nx, nt, precision):
    p = W.with_(LV, nx=nx, nt=nt, precision=precision)
    v = W.random_vector(nx * nt, seed=3 * nx + nt)
    z = apply(aao, p, v)
    assert rel(O.apply_P(p, z), v) <= bound(p)
    assert rel(z, O.precond_fft(p, v)) <= bound(p)


def test_mixed_radix_in_place(aao):
    p = W.with_(BS, nx=63, nt=24)
    h = aao.aao_create(p)
    v = W.random_vector(63 * 24, seed=2)
    t = dev(v)
    aao.precond_apply(h, t, t)
    assert rel(host(t), O.precond_fft(p, v)) <= bound(p)
    h.close()


@pytest.mark.parametrize("sym", [False, True])
def test_mixed_radix_riesz_precond(aao, sym):
    """The dense step (b) of the Riesz operator (inverse or spectral) on an odd number of bins."""
    base = W.riesz_sym_1023x512() if sym else W.riesz_1023x512()
    for nx, nt, alpha in [(31, 6, 1e-2), (63, 15, 1e-3), (100, 24, 1e-2)]:
        p = W.with_(base, nx=nx, nt=nt, alpha=alpha)
        v = W.random_vector(nx * nt, seed=nx + nt)
        z = apply(aao, p, v)
        assert rel(z, O.precond_fft(p, v)) <= bound(p)


def test_mixed_radix_solve_localvol(aao):
    """Mixed-precision 2047 x 1536 local volatility (nt = 3 x 2^9) to relative residual 1e-8;
    option values at maturity within 1e-8 of sequential CN."""
    p = W.with_(W.localvol_2047x2048("mixed"), nt=1536)
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
    print("mixed radix localvol 2047x1536: its", st["iterations"], "maturity error", err)
    assert err <= 1e-8
    h.close()
