"""The multi-rank logic of bench.py on the CPU: two processes on a gloo process group (the GPU
runs use NCCL, one rank per GPU). Every rank gets the slowest rank's time, and the whole-job
rate counts the units of all ranks in that time. CPU only."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B = load_bench()
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        dist.barrier()
        slowest = B.max_over_ranks(ms, "cpu")
        rate = B.whole_job_rate(world, 1000, slowest / 1e3)
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time_and_the_job_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [15.0, 15.0]
    assert all(abs(g[2] - 2 * 1000 / 0.015) < 1e-6 for g in got)


def test_one_process_without_a_group_keeps_its_own_time():
    B = load_bench()
    assert B.max_over_ranks(12.5, "cpu") == 12.5
    assert B.whole_job_rate(1, 4_192_256, 1.1e-3) == pytest.approx(3.811e9, rel=1e-3)
