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
