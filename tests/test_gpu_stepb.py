"""Step (b) of Eq. 3.2 for the tridiagonal operators: the factored partition method (per-bin
pivot tables made at create) and the recomputing one (no tables; pivots recomputed from the
three shared diagonals in every apply), each selected with the problem's step_b flag and checked
against the FP64 oracle through the C ABI. Sizes span one to sixteen rows per thread, ragged
last chunks, 32 to 512 threads per bin and the FP64 path up to nx = 8191 (the recomputing solver
is the only one that fits there)."""
import math

import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24
LV = W.localvol_2047x2048("fp64")
BS = W.bs_put_255x256()


@pytest.fixture(scope="module")
def aao():
    from paper_2401_16113_gb300 import aao as A, build
    build.build()
    A.load()
    return A


def bound(p):
    u = U32 if p["precision"] == "mixed" else U64
    return 20.0 * u * math.log2(2 * p["nt"]) / p["alpha"]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def apply(aao, p, v):
    h = aao.aao_create(p)
    z = torch.empty(v.size, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, torch.from_numpy(v).cuda(), z)
    torch.cuda.synchronize()
    h.close()
    return z.cpu().numpy()


SHAPES = [(2, 4), (3, 2), (31, 8), (33, 16), (100, 64), (255, 256), (257, 32), (1000, 128), (2047, 256)]


@pytest.mark.parametrize("step_b", ["factored", "recompute"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,nt", SHAPES)
def test_step_b_variants_match_oracle(aao, nx, nt, precision, step_b):
    for base in (LV, W.with_(BS, payoff="call")):
        p = W.with_(base, nx=nx, nt=nt, precision=precision, alpha=1e-3, step_b=step_b)
        v = W.random_vector(nx * nt, seed=7 * nx + nt)
        z = apply(aao, p, v)
        ref = O.precond_fft(p, v)
        assert rel(z, ref) <= bound(p), (base["op"], rel(z, ref), bound(p))


LARGE = [(4095, 64, "fp64"), (5000, 32, "fp64"), (8191, 16, "fp64"), (8191, 64, "mixed")]


def norm_P_inf(p):
    """||P_alpha||_inf <= ||C1||_inf + ||C2||_inf ||tau Abar||_inf = 2 + ||tau Abar||_inf (Eq. 3.1;
    rows of C1 hold 1 and -1 or -alpha, rows of C2 two halves)."""
    _, tau = O.time_grid(p)
    A = O.mean_operator(p)
    return 2.0 + tau * float(np.abs(A).sum(axis=1).max())


@pytest.mark.parametrize("nx,nt,precision", LARGE)
def test_step_b_recompute_large_nx(aao, nx, nt, precision):
    """Normwise backward error eta = ||v - P_alpha z|| / (||P_alpha|| ||z|| + ||v||) in the max norm
    (P_alpha applied blockwise by the oracle): the shifted systems of the largest nx are too
    ill-conditioned for a forward-error check in FP32, and with ||P_alpha|| ~ 1e5 the plain
    ||v - P z|| / ||v|| of an FP64 solve sits at the rounding of the product P z itself."""
    p = W.with_(LV, nx=nx, nt=nt, precision=precision, step_b="recompute")
    v = W.random_vector(nx * nt, seed=nx + 3 * nt)
    z = apply(aao, p, v)
    r = O.apply_P(p, z) - v
    eta = np.abs(r).max() / (norm_P_inf(p) * np.abs(z).max() + np.abs(v).max())
    assert eta <= bound(p), eta
    if precision == "fp64":
        assert rel(z, O.precond_fft(p, v)) <= 1e3 * bound(p)


def test_step_b_factored_refused_where_it_does_not_fit(aao):
    p = W.with_(LV, nx=8191, nt=16, precision="fp64", step_b="factored")
    with pytest.raises(aao.AaoError) as e:
        aao.aao_create(p)
    assert e.value.code == aao.AAO_EUNSUPPORTED


def test_step_b_variants_agree_at_the_bench_shape(aao):
    p = W.localvol_2047x2048("mixed")
    v = W.random_vector(W.unknowns(p), seed=12)
    za = apply(aao, W.with_(p, step_b="factored"), v)
    zb = apply(aao, W.with_(p, step_b="recompute"), v)
    ref = O.precond_fft(p, v)
    assert rel(za, ref) <= bound(p) and rel(zb, ref) <= bound(p)
    assert rel(za, zb) <= bound(p)
