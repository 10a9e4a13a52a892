"""precond_apply_static: the preconditioner apply for callers that cannot allocate device
memory (a fixed device-memory budget handed out up front, or latency-critical paths that cannot
afford an allocation's synchronisation). On two calls in a row that share its static scratch it
must give what the allocating precond_apply gives and what the FP64 oracle gives, and it must
refuse problems larger than that scratch. This file is named to be collected last."""
import math

import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aao():
    from paper_2401_16113_gb300 import aao as A, build
    build.build()
    A.load()
    return A


def bound(p):
    # same bound as the oracle parity tests: C u log2(2 nt) / alpha
    u = 2.0 ** -24 if p["precision"] == "mixed" else 2.0 ** -53
    return 20.0 * u * math.log2(2 * p["nt"]) / p["alpha"]


CASES = [
    W.localvol_2047x2048("mixed"),
    W.with_(W.bs_put_255x256(), precision="fp64"),
    W.with_(W.bs_put_255x256(), nx=37, nt=16, precision="mixed", payoff="call"),
    W.with_(W.localvol_2047x2048("mixed"), nt=1536),
    W.with_(W.bs_put_255x256(), nx=100, nt=15, precision="fp64"),
    W.with_(W.bs_put_255x256(), nx=63, nt=24, precision="mixed", payoff="call"),
]


@pytest.mark.parametrize("p", CASES, ids=["localvol-2047x2048-mixed", "bs-255x256-fp64", "bs-37x16-mixed",
                                          "localvol-2047x1536-mixed", "bs-100x15-fp64", "bs-63x24-mixed"])
def test_static_matches_allocating_apply_and_oracle_twice(aao, p):
    n = W.unknowns(p)
    h = aao.aao_create(p)
    for call, seed in enumerate((101, 202)):
        v_np = W.random_vector(n, seed=seed)
        v = torch.from_numpy(v_np).cuda()
        z_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        z = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        aao.precond_apply(h, v, z_ref)
        aao.precond_apply_static(p, v, z)
        torch.cuda.synchronize()
        a, b = z.cpu().numpy(), z_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.linalg.norm(a - b) <= bound(p) * np.linalg.norm(b), (call, np.linalg.norm(a - b) / np.linalg.norm(b))
        zo = O.precond_fft(p, v_np)
        assert np.linalg.norm(a - zo) <= bound(p) * np.linalg.norm(zo), (call, np.linalg.norm(a - zo) / np.linalg.norm(zo))
    h.close()


def test_static_rejects_the_riesz_operator(aao):
    p = W.with_(W.riesz_1023x512(), nx=63, nt=16)
    n = W.unknowns(p)
    v = torch.zeros(n, dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(aao.AaoError) as e:
        aao.precond_apply_static(p, v, z)
    assert e.value.code == aao.AAO_EUNSUPPORTED


def test_static_rejects_problems_beyond_its_scratch(aao):
    p = W.localvol_8191x8192("mixed")
    n = W.unknowns(p)
    v = torch.zeros(n, dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(aao.AaoError) as e:
        aao.precond_apply_static(p, v, z)
    assert e.value.code == aao.AAO_EINVAL
    assert "32 MiB" in str(e.value)
