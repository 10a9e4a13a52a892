"""Host-side logic of bench.py: the clock-sample window, the default step counts, the
preconditioner roofline arithmetic and the traffic record's source check."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def row(sm, reasons=("Not Active",) * 4):
    return ["0", str(sm), "2070", "900.0", "0x0", *reasons]


def test_clock_summary_keeps_region_rows_and_the_closing_sample():
    b = load_bench()
    c = b.ClockSampler()
    c.t0, c.t1 = 10.0, 11.0
    c.rows = [(9.5, row(345)), (10.2, row(2070)), (10.6, row(1980)), (11.05, row(2055)), (11.2, row(345))]
    s = c.summary()
    assert s["samples"] == 2 and s["samples_after"] == 1
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == []


def test_clock_summary_reports_throttle_reasons_and_unsampled():
    b = load_bench()
    c = b.ClockSampler()
    c.t0, c.t1 = 0.0, 1.0
    c.rows = [(0.5, row(1800, ("Not Active", "Active", "Not Active", "Active")))]
    assert c.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    c.rows = [(2.0, row(2070)), (3.0, row(2070))]
    s = c.summary()
    assert s["samples"] == 0 and s["samples_after"] == 1
    c.rows = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_default_steps_per_arm(monkeypatch):
    b = load_bench()
    seen = {}
    monkeypatch.setattr(b, "run_ours", lambda a: seen.setdefault("ours", a.steps))
    monkeypatch.setattr(b, "run_reference", lambda a: seen.setdefault("reference", a.steps))
    for argv in (["bench.py"], ["bench.py", "--impl", "reference"], ["bench.py", "--steps", "7"]):
        monkeypatch.setattr(sys, "argv", argv)
        b.main()
    assert seen == {"ours": 200, "reference": 3}


def test_precond_roofline_arithmetic():
    """The apply's three kernel classes as one unit: 16 B per unknown (FP64 v in, z out) over the
    time per apply; the argument sizes and the in-solve FP32 ends are reported beside it."""
    B = load_bench()
    # (launches, total ms, argument bytes, flops) per class over 4 applies
    prof = {"fft_fwd": (4, 0.08, 4 * 30e6, 0.0), "tridiag": (4, 0.12, 4 * 60e6, 0.0),
            "fft_inv": (4, 0.08, 4 * 30e6, 0.0), "matvec": (5, 0.5, 1e9, 1e8)}
    n = 4_192_256
    r = B.precond_roofline(prof, 6800.0, n)
    assert r["applies"] == 4
    assert abs(r["ms_per_apply"] - 0.07) < 1e-12
    assert r["algorithmic_bytes_per_apply"] == 16 * n
    assert abs(r["achieved"] - 16 * n / 0.07e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-12
    assert abs(r["in_solve_io_gbs"] - r["achieved"] / 2) < 1e-9
    assert abs(r["argument_bytes_per_apply"] - 120e6) < 1e-3
    assert B.precond_roofline(dict(prof, fft_fwd=(0, 0.0, 0.0, 0.0)), 6800.0, n) is None


def test_traffic_record_is_used_only_on_its_own_sources(monkeypatch):
    """profiles/ncu_traffic.json gives DRAM bytes per launch only while its source hash matches
    the sources; after any change to them the bench reports no traffic."""
    import json
    B = load_bench()
    rec = json.load(open(os.path.join(B.ROOT, "profiles", "ncu_traffic.json")))["matvec"]
    monkeypatch.setattr(B, "source_sha", lambda files=None: rec["source_sha"])
    assert B.ncu_traffic("matvec") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(B, "source_sha", lambda files=None: "0" * 16)
    assert B.ncu_traffic("matvec") is None
    assert B.ncu_traffic("no_such_kernel") is None


def test_source_hash_covers_a_kernels_translation_unit(monkeypatch, tmp_path):
    """The traffic record's hash follows the code of the named sources and of the headers they
    include: a change to another source leaves it alone, a change of code in an included header
    changes it, and an edit of comments or blank lines alone does not."""
    import shutil
    B = load_bench()
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(B.ROOT, "paper_2401_16113_gb300", "csrc"), root / "paper_2401_16113_gb300" / "csrc")
    shutil.copytree(os.path.join(B.ROOT, "include"), root / "include")
    monkeypatch.setattr(B, "ROOT", str(root))
    cs = root / "paper_2401_16113_gb300" / "csrc"
    h0 = B.source_sha(["krylov.cu"])
    assert h0 == B.source_sha(["krylov.cu"])
    (cs / "heston.cu").write_text((cs / "heston.cu").read_text() + "\nint edit_marker;\n")
    assert B.source_sha(["krylov.cu"]) == h0
    (cs / "krylov.cu").write_text((cs / "krylov.cu").read_text() + "\n// a comment\n\n/* and another */\n")
    assert B.source_sha(["krylov.cu"]) == h0
    (cs / "aao_internal.cuh").write_text((cs / "aao_internal.cuh").read_text() + "\nint edit_marker;\n")
    h1 = B.source_sha(["krylov.cu"])
    assert h1 != h0
    (root / "include" / "aao.h").write_text((root / "include" / "aao.h").read_text() + "\n#define AAO_EDIT 1\n")
    assert B.source_sha(["krylov.cu"]) != h1
