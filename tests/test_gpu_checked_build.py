"""The bounds-checked build (-DAAO_CHECK, libaao_check.so) on the GPU: a set of preconditioner
applies, matrix-vector products and solves over the operators and ragged sizes runs in a separate
process against the checked library; every guarded store must pass its index test
(aao_check_failures() == 0) and the results must still match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, ROOT_PATH)
import numpy as np, torch
from oracle import aao_oracle as O
from paper_2401_16113_gb300 import aao, build, workloads as W
aao.load(build.build(check=True))
cases = [W.with_(W.localvol_2047x2048("mixed"), nx=301, nt=96), W.with_(W.bs_put_255x256(), nx=37, nt=15),
         W.with_(W.localvol_2047x2048("fp64"), nx=129, nt=64, step_b="recompute"),
         W.with_(W.localvol_2047x2048("mixed"), nx=1000, nt=128, step_b="recompute"),
         W.with_(W.riesz_1023x512(), nx=100, nt=16), W.with_(W.riesz_sym_1023x512(), nx=63, nt=16),
         W.with_(W.heston_set1(), nx=13, nv=5, nt=12)]
worst = 0.0
for p in cases:
    n = W.unknowns(p)
    h = aao.aao_create(p)
    v = W.random_vector(n, seed=n % 97)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.precond_apply(h, torch.from_numpy(v).cuda(), z)
    torch.cuda.synchronize()
    zr = O.precond_fft(p, v)
    worst = max(worst, float(np.linalg.norm(z.cpu().numpy() - zr) / np.linalg.norm(zr)))
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    aao.aao_rhs(h, b)
    x = torch.zeros_like(b)
    st = aao.fgmres_solve(h, b, x, 1e-9, 30, 200)
    assert st["status"] == 0, (p["op"], st)
    h.close()
print("FAILURES", aao.load().aao_check_failures(), "WORST", worst)
""".replace("ROOT_PATH", repr(ROOT))


def test_checked_build_runs_clean():
    out = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stderr[-3000:]
    line = [l for l in out.stdout.splitlines() if l.startswith("FAILURES")][-1].split()
    assert int(line[1]) == 0, out.stdout
    assert float(line[3]) <= 1.5e-2, out.stdout  # the mixed-precision bound of the parity tests
