"""The oracle arm of bench.py (`--impl reference`) runs end to end on the CPU
and prints its JSON line; a small phantom workload stands in for the full one."""
import argparse
import json

import bench
from paper_2406_02518_gb300 import synthetic as syn


def test_reference_arm_prints_its_line(monkeypatch, capsys):
    small = syn.registration_workload(n_gauss=3000, n_views=2, size=32, grid=64)
    monkeypatch.setattr(bench, "workload", lambda rank, **kw: small)
    monkeypatch.setattr(bench, "_dist_env", lambda: (0, 1, 0))
    args = argparse.Namespace(variant="disentangled", warmup=1, steps=1)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_traffic_is_reported_only_for_the_captured_sources_and_shape(monkeypatch):
    import hashlib
    import os
    src = os.path.join(bench.ROOT, "paper_2406_02518_gb300", "csrc", "raster.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    entry = {"sources_sha256": {"raster.cu": sha}, "tile": 8, "batch_depth": 32, "views": 64,
             "gaussians": 500_000, "bytes_per_launch": 123.0}
    monkeypatch.setattr(bench, "TRAFFIC", {"raster_bwd": entry})
    assert bench.captured_traffic("raster_bwd", 8, 32, 64, 500_000) == 123.0
    assert bench.captured_traffic("raster_bwd", 16, 32, 64, 500_000) is None   # other shape
    assert bench.captured_traffic("raster_bwd", 8, 32, 16, 500_000) is None    # other workload
    assert bench.captured_traffic("raster_fwd", 8, 32, 64, 500_000) is None    # not captured
    monkeypatch.setattr(bench, "TRAFFIC", {"raster_bwd": dict(entry, sources_sha256={"raster.cu": "0" * 64})})
    assert bench.captured_traffic("raster_bwd", 8, 32, 64, 500_000) is None    # source changed


def test_kernel_table_divides_step_bytes_by_step_time():
    """A kernel launched 4 times per step: its bytes per step over the sum of
    its 4 launches, never over one launch's time."""
    shape = {"pairs": 1_000_000, "n": 1000, "views": 2}
    # 2 profiled steps: bin_sort 4 launches per step of 0.25 ms each (2 ms in
    # all), preprocess_fwd 1 launch per step of 0.5 ms
    prof = {"bin_sort": (2.0, 8), "preprocess_fwd": (1.0, 2), "raster_bwd": (5.0, 2)}
    t = bench.kernel_table(prof, 2, shape)
    assert t["bin_sort"]["launches_per_step"] == 4 and t["bin_sort"]["ms_per_launch"] == 0.25
    assert t["bin_sort"]["ms_per_step"] == 1.0
    # 12 B per pair per step over 1 ms per step
    assert t["bin_sort"]["algorithmic_GBps"] == round(12e6 / 1e-3 / 1e9, 1)
    assert t["bin_sort"]["pass_24B_per_pair_GBps"] == round(24e6 / 1e-3 / 1e9, 1)
    pf = 76 * 1000 + 48 * 1000 * 2
    assert t["preprocess_fwd"]["algorithmic_GBps"] == round(pf / 0.5e-3 / 1e9, 1)
    assert "algorithmic_GBps" not in t["raster_bwd"]  # ALU-bound: no byte roofline
    assert abs(sum(e["share"] for e in t.values()) - 1.0) < 1e-3
