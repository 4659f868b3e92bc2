"""Host logic of the autotuner: candidate selection, caching, keys (no GPU)."""
import json

import pytest

from paper_2406_02518_gb300 import autotune as at


def test_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def step(tile, depth):
        calls.append((tile, depth))
        return {8: 3.0, 16: 1.0, 32: 2.0}[tile] + (0.5 if depth in (32, 128) else 0.0)

    r = at.tune(step, "k1", cache_path=path)
    assert (r["tile"], r["batch_depth"], r["cached"]) == (16, 256, False)
    assert len(calls) == len(at.CANDIDATES)
    r2 = at.tune(step, "k1", cache_path=path)
    assert r2["cached"] and r2["tile"] == 16 and len(calls) == len(at.CANDIDATES)
    assert json.load(open(path))["k1"]["batch_depth"] == 256
    r3 = at.tune(step, "k1", cache_path=path, force=True)
    assert not r3["cached"] and len(calls) == 2 * len(at.CANDIDATES)


def test_failing_candidates_are_skipped(tmp_path):
    def step(tile, depth):
        if tile == 16:
            raise RuntimeError("does not fit")
        return float(tile + depth / 1000)

    r = at.tune(step, "k2", cache_path=str(tmp_path / "c.json"))
    assert r["tile"] == 8 and r["batch_depth"] == 32
    assert r["timings"]["16x256"] is None
    with pytest.raises(RuntimeError):
        at.tune(lambda t, d: (_ for _ in ()).throw(ValueError("x")), "k3",
                cache_path=str(tmp_path / "d.json"))


def test_keys_bucket_workloads():
    k = at.workload_key("NVIDIA GB300", 152, 256 * 256, 500_000, 64)
    assert k == at.workload_key("NVIDIA GB300", 152, 250 * 250, 400_000, 40)
    assert k != at.workload_key("NVIDIA GB300", 152, 1024 * 1024, 500_000, 64)
    assert at.bucket(1) == 0 and at.bucket(2) == 1 and at.bucket(1025) == 11
