"""The C-ABI library builds, loads and exports every entry point include/aao.h declares;
host-side argument checks reject bad problems before touching a GPU. CPU only."""
import ctypes
import os
import re

import pytest

from paper_2401_16113_gb300 import aao, build, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:int|const char\*|uint64_t|void|unsigned int)\s+\**\s*([A-Za-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return aao.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(aao.EXPORTS) <= set(names)


def test_struct_layout_matches_header():
    # int32 x 6, double x 9, pointer, then the Heston fields: int32 x 2, double x 4
    assert ctypes.sizeof(aao.AaoProblem) == 6 * 4 + 9 * 8 + 8 + 2 * 4 + 4 * 8
    assert aao.AaoProblem.alpha.offset == 24 + 8 * 8
    assert aao.AaoProblem.nv.offset == 24 + 9 * 8 + 8
    assert aao.AaoProblem.v_max.offset == 24 + 9 * 8 + 8 + 8 + 3 * 8
    assert ctypes.sizeof(aao.AaoStats) == 4 * 4 + 3 * 8


def _create(lib, p):
    h = ctypes.c_void_p()
    return lib.aao_create(ctypes.byref(aao.make_problem(p)), ctypes.byref(h)), h


@pytest.mark.parametrize("bad,code", [
    (dict(nx=1), aao.AAO_EINVAL),
    (dict(nt=0), aao.AAO_EINVAL),
    (dict(nt=88), aao.AAO_EUNSUPPORTED),
    (dict(nt=13), aao.AAO_EUNSUPPORTED),
    (dict(alpha=0.0), aao.AAO_EINVAL),
    (dict(alpha=1.5), aao.AAO_EINVAL),
    (dict(sigma=-0.1), aao.AAO_EINVAL),
    (dict(T=0.0), aao.AAO_EINVAL),
    (dict(op="riesz", precision="fp64"), aao.AAO_EUNSUPPORTED),
    (dict(op="riesz", precision="mixed", beta=2.5), aao.AAO_EINVAL),
    (dict(op="riesz", precision="mixed", nx=4095), aao.AAO_EUNSUPPORTED),
    (dict(nt=6144, precision="fp64"), aao.AAO_EUNSUPPORTED),
    (dict(nt=16384, precision="mixed"), aao.AAO_EUNSUPPORTED),
    (dict(nx=8193, precision="fp64"), aao.AAO_EUNSUPPORTED),
])
def test_create_rejects_bad_problems_on_host(lib, bad, code):
    rc, h = _create(lib, W.with_(W.bs_put_255x256(), **bad))
    assert rc == code
    assert h.value is None
    assert lib.aao_last_error().decode()


def test_create_rejects_unknown_flags_on_host(lib):
    s = aao.make_problem(W.bs_put_255x256())
    s.flags = 3
    h = ctypes.c_void_p()
    assert lib.aao_create(ctypes.byref(s), ctypes.byref(h)) == aao.AAO_EINVAL
    assert h.value is None
    with pytest.raises(KeyError):
        aao.make_problem(W.with_(W.bs_put_255x256(), step_b="fastest"))


def test_null_arguments_rejected(lib):
    assert lib.aao_create(None, None) == aao.AAO_EINVAL
    assert lib.aao_matvec(None, None, None) == aao.AAO_EINVAL
    assert lib.precond_apply(None, None, None) == aao.AAO_EINVAL
    assert lib.fgmres_solve(None, None, None, 1e-8, 10, 10, None) == aao.AAO_EINVAL
    assert lib.fgmres_solve_zero(None, None, None, 1e-8, 10, 10, None) == aao.AAO_EINVAL
    assert lib.aao_destroy(None) == aao.AAO_OK


def test_product_code_never_references_the_oracle():
    pkg = os.path.join(ROOT, "paper_2401_16113_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


@pytest.mark.slow
def test_checked_build_compiles_and_exports():
    """The bounds-checked variant (-DAAO_CHECK) builds for sm_103a and exports the same entry points."""
    from paper_2401_16113_gb300 import build
    lib = ctypes.CDLL(build.build(check=True))
    for name in aao.EXPORTS:
        assert hasattr(lib, name), name
    lib.aao_check_failures.restype = ctypes.c_uint
