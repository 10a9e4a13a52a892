"""CPU baseline runner for the benchmark (test infrastructure, like the rest of oracle/): the
oracle's FP64 FGMRES on independent instances, one single-threaded worker process per host core.
The worker lives in this importable module so that spawned worker processes can load it."""
from __future__ import annotations

import multiprocessing as mp
import time


def solve_iterations(p):
    """The oracle's right-preconditioned FGMRES(m) solve of p (FFT apply of Eq. 3.2); returns the
    iteration count."""
    from oracle import aao_oracle as O
    M = O.assemble_M(p)
    b = O.assemble_b(p)
    _, info = O.fgmres(lambda v: M @ v, lambda v: O.precond_fft(p, v), b, p["tol"], p["m"], 300)
    return info["its"]


def run_pool(problems, cores):
    """Wall seconds to solve every problem on a spawned pool of `cores` workers (after one warm-up
    problem per worker), and the mean iteration count."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(solve_iterations, problems[:cores])
        t0 = time.perf_counter()
        its = pool.map(solve_iterations, problems)
        s = time.perf_counter() - t0
    return s, sum(its) / len(its)
