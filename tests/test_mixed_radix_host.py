"""Host-side facts the mixed-radix FFT path relies on (CPU, no GPU needed).

1. Which nt aao_create admits: every nt <= the shared-memory limit whose prime factors are
   2, 3, 5 and 7 passes validation; any other prime factor gives AAO_EUNSUPPORTED. (On a
   machine without a GPU an admitted problem then fails at its first device allocation, with
   AAO_ECUDA; with a GPU the handle is created and destroyed.)
2. The stage kernels divide the butterfly index j by the stride Ns with a multiply-high by
   ceil(2^32 / Ns). That quotient is exact for every Ns in [2, 8192] and every j < 2^14; the
   kernels use j < nt/2 <= 4096 (checked exhaustively here).
"""
import ctypes

import numpy as np
import pytest

from paper_2401_16113_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_2401_16113_gb300 import aao, build
    build.build()
    return aao.load()


def _create(lib, p):
    from paper_2401_16113_gb300 import aao
    h = ctypes.c_void_p()
    rc = lib.aao_create(ctypes.byref(aao.make_problem(p)), ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("nt", [3, 5, 6, 7, 12, 96, 105, 1536, 2205, 6561, 7168])
def test_create_admits_nt_with_prime_factors_up_to_7(lib, nt):
    from paper_2401_16113_gb300 import aao
    rc, h = _create(lib, W.with_(W.bs_put_255x256(), nx=31, nt=nt, precision="mixed"))
    assert rc not in (aao.AAO_EINVAL, aao.AAO_EUNSUPPORTED), lib.aao_last_error().decode()
    if rc == aao.AAO_OK:
        lib.aao_destroy(h)
    else:
        assert rc == aao.AAO_ECUDA and h.value is None


@pytest.mark.parametrize("nt", [11, 13, 22, 51, 88, 4097, 11 * 512])
def test_create_rejects_other_prime_factors(lib, nt):
    from paper_2401_16113_gb300 import aao
    rc, h = _create(lib, W.with_(W.bs_put_255x256(), nx=31, nt=nt, precision="mixed"))
    assert rc == aao.AAO_EUNSUPPORTED and h.value is None
    assert "prime factor" in lib.aao_last_error().decode()


def test_multiply_high_division_is_exact():
    j = np.arange(1 << 14, dtype=np.uint64)
    for d in range(2, 8193):
        m = np.uint64(((1 << 32) + d - 1) // d)
        q = (j * m) >> np.uint64(32)
        assert np.array_equal(q, j // np.uint64(d)), d
