"""The two-dimensional Heston operator (Sec. 5.1) through the C ABI against the FP64 oracle:
the right-hand side and the matrix-vector product of Eq. 2.2 (rounding-order differences only),
the preconditioner apply of Eq. 3.2 with its block-elimination step (b) (the FP32 bound of the
other parity tests, and the brute-force dense inverse on a tiny grid), and the mixed-precision
FGMRES(40) solve to 1e-9: its iteration count matches the oracle's, P_1 needs many more, the
solution equals sequential Crank-Nicolson, and the price at (S0, V0) reproduces the relative
error the paper prints in Table 1."""
import math

import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def aao():
    from paper_2401_16113_gb300 import aao as A, build
    build.build()
    A.load()
    return A


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bound(p):
    return 20.0 * U32 * math.log2(2 * p["nt"]) / p["alpha"]


SHAPES = [(3, 3, 2), (8, 4, 8), (13, 5, 12), (40, 20, 16), (64, 32, 32), (100, 6, 6), (300, 3, 4)]


@pytest.mark.parametrize("ns,nv,nt", SHAPES)
def test_heston_rhs_and_matvec_match_oracle(aao, ns, nv, nt):
    for base in (W.heston_set1(), W.heston_set2()):
        p = W.with_(base, nx=ns, nv=nv, nt=nt)
        n = W.unknowns(p)
        h = aao.aao_create(p)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        aao.aao_rhs(h, b)
        bref = O.assemble_b(p)
        assert np.abs(host(b) - bref).max() <= 1e-13 * np.abs(bref).max()
        x = W.random_vector(n, seed=ns + nt)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        aao.aao_matvec(h, dev(x), y)
        yref = O.matvec(p, x)
        assert np.abs(host(y) - yref).max() <= 1e-12 * np.abs(yref).max()
        h.close()


@pytest.mark.parametrize("ns,nv,nt", SHAPES)
@pytest.mark.parametrize("alpha", [1e-2, 1e-3])
def test_heston_precond_matches_oracle(aao, ns, nv, nt, alpha):
    p = W.with_(W.heston_set1(), nx=ns, nv=nv, nt=nt, alpha=alpha)
    n = W.unknowns(p)
    h = aao.aao_create(p)
    v = W.random_vector(n, seed=2 * ns + nt)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z)
    assert rel(host(z), O.precond_fft(p, v)) <= bound(p)
    h.close()


def test_heston_precond_tiny_matches_dense_inverse(aao):
    p = W.with_(W.heston_set2(), nx=6, nv=4, nt=6)
    n = W.unknowns(p)
    h = aao.aao_create(p)
    v = W.random_vector(n, seed=5)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, dev(v), z)
    assert rel(host(z), O.precond_dense(p, v)) <= bound(p)
    h.close()


def price_at(p, last):
    S, V, hs, hv = O.heston_grid(p)
    Z = last.reshape(int(p["nv"]), int(p["nx"]))
    x, y = p["S0"] / hs - 1.0, p["V0"] / hv
    i0, j0 = int(math.floor(x)), int(math.floor(y))
    fx, fy = x - i0, y - j0
    return ((1 - fx) * (1 - fy) * Z[j0, i0] + fx * (1 - fy) * Z[j0, i0 + 1] + (1 - fx) * fy * Z[j0 + 1, i0]
            + fx * fy * Z[j0 + 1, i0 + 1])


@pytest.mark.parametrize("nt", [16, 32, 48])
def test_heston_solve_matches_cn_and_oracle_iterations(aao, nt):
    p = W.heston_set1(nt)
    n = W.unknowns(p)
    h = aao.aao_create(p)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.zeros_like(b)
    st = aao.fgmres_solve(h, b, x, 1e-9, 40, 200)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-9, st
    U = O.sequential_cn(p)
    xs = host(x)
    assert np.abs(xs - U.ravel()).max() <= 1e-7 * np.abs(U).max()
    _, info = O.solve(p, tol=1e-9, m=40, maxit=200)
    assert abs(st["iterations"] - info["its"]) <= 1, (st["iterations"], info["its"])
    assert st["iterations"] <= 5  # the paper: 4 on every mesh
    if nt == 48:
        ref = O.heston_call(p["S0"], p["V0"], p["K"], p["T"], p["r"], p["kappa"], p["eta"], p["sigma"], p["rho"])
        err = abs(price_at(p, xs.reshape(nt, -1)[-1]) - ref) / ref
        assert abs(err - 1.348e-2) <= 1.5e-3 * 1.348e-2, err  # Table 1, Set I, Nt = 48
    h.close()


def test_heston_P_alpha_beats_P_1(aao):
    p = W.heston_set2(32)
    n = W.unknowns(p)
    its = {}
    for alpha in (1e-3, 1.0):
        h = aao.aao_create(W.with_(p, alpha=alpha))
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        aao.aao_rhs(h, b)
        x = torch.zeros_like(b)
        st = aao.fgmres_solve(h, b, x, 1e-9, 40, 400)
        assert st["status"] == 0, st
        its[alpha] = st["iterations"]
        h.close()
    assert its[1.0] >= 5 * its[1e-3], its


def test_heston_rejects_what_is_not_built(aao):
    for bad, code in ((dict(precision="fp64"), aao.AAO_EUNSUPPORTED), (dict(payoff="put"), aao.AAO_EUNSUPPORTED),
                      (dict(nv=2), aao.AAO_EUNSUPPORTED), (dict(rho=-1.5), aao.AAO_EINVAL)):
        with pytest.raises(aao.AaoError) as e:
            aao.aao_create(W.with_(W.heston_set1(16), **bad))
        assert e.value.code == code
