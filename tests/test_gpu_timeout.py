"""The bounded device-side wait of the tensor-core step (b) (symmetric Riesz operator), made
to run out without a GPU fault: fault injection makes the TMA producer issue no operator load,
so the first wait for an operator tile gives up with nothing in flight. The kernels return, the
host reads AAO_TIMEOUT, and the context stays usable: the next apply and solve on the same
handle, with injection off, match the oracle."""
import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RZS = W.with_(W.riesz_sym_1023x512(), nx=127, nt=32)


@pytest.fixture(scope="module")
def aao():
    from paper_2401_16113_gb300 import aao as A, build
    build.build()
    A.load()
    return A


def test_tensor_core_wait_runs_out_and_the_handle_recovers(aao):
    p = RZS
    n = W.unknowns(p)
    h = aao.aao_create(p)
    v_np = W.random_vector(n, seed=7)
    v = torch.from_numpy(v_np).cuda()
    z = torch.empty(n, dtype=torch.float64, device="cuda")

    # injected: the apply reports the timeout (each wait bounded at 20 ms)
    aao.aao_fault_inject(h, aao.AAO_INJECT_TC_NO_LOAD, 20.0)
    with pytest.raises(aao.AaoError) as e:
        aao.precond_apply(h, v, z)
    assert e.value.code == aao.AAO_TIMEOUT
    # and so does a solve that uses it
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.zeros_like(b)
    with pytest.raises(aao.AaoError) as e:
        aao.fgmres_solve(h, b, x, 1e-8, 30, 4)
    assert e.value.code == aao.AAO_TIMEOUT

    # injection off: the same handle applies and solves correctly
    aao.aao_fault_inject(h, 0, 0.0)
    aao.precond_apply(h, v, z)
    torch.cuda.synchronize()
    zr = O.precond_fft(p, v_np)
    assert np.linalg.norm(z.cpu().numpy() - zr) <= 1e-3 * np.linalg.norm(zr)
    x.zero_()
    st = aao.fgmres_solve(h, b, x, 1e-8, 30, 100)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8, st
    U = O.sequential_cn(p)
    xs = x.cpu().numpy()
    assert np.abs(xs - U.ravel()).max() <= 1e-6 * np.abs(U).max()
    h.close()
