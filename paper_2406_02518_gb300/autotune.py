"""Autotuner of the rasteriser launch shape: tile edge and staging depth.

For a given workload the tuner times one full step (the caller's function,
which renders and back-propagates with the candidate configuration) for every
(tile, batch_depth) pair and keeps the fastest. Depth 32 selects the
warp-streamed rasterisers; the others are block-staged depths. Results are cached in a JSON
file keyed by the GPU (name, SM count) and coarse buckets of the workload
(largest detector, Gaussians, views), so a workload of the same class reuses
the choice without re-timing.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Callable, Dict, Iterable, Optional, Tuple

TILES = (8, 16, 32)
DEPTHS = (32, 128, 256, 512)  # 32: warp-streamed rasterisers (no block staging)
CANDIDATES = tuple((t, d) for t in TILES for d in DEPTHS)


def default_cache_path() -> str:
    return os.environ.get("DDGS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ddgs", "autotune.json"))


def bucket(x: float) -> int:
    """Power-of-two bucket (0 for x <= 1)."""
    return 0 if x <= 1 else int(math.ceil(math.log2(x)))


def workload_key(device_name: str, sms: int, max_pixels: int, n_gauss: int, n_views: int) -> str:
    return (f"{device_name}|sm{sms}|px2^{bucket(max_pixels)}|n2^{bucket(n_gauss)}"
            f"|v2^{bucket(n_views)}")


def load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: Dict[str, dict]) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(step: Callable[[int, int], float], key: str,
         candidates: Iterable[Tuple[int, int]] = CANDIDATES, cache_path: Optional[str] = None,
         force: bool = False) -> dict:
    """Return {"tile", "batch_depth", "ms", "timings", "cached"} for `key`.

    `step(tile, depth)` runs the workload once (warm-up and timing are the
    caller's) and returns its time in milliseconds; it may raise to reject a
    candidate (for example a workspace that does not fit)."""
    path = cache_path or default_cache_path()
    cache = load_cache(path)
    if not force and key in cache:
        out = dict(cache[key])
        out["cached"] = True
        return out
    timings = {}
    for tile, depth in candidates:
        try:
            timings[f"{tile}x{depth}"] = float(step(tile, depth))
        except Exception as e:  # a candidate that cannot run is skipped
            timings[f"{tile}x{depth}"] = None
            last_err = e
    ok = {k: v for k, v in timings.items() if v is not None}
    if not ok:
        raise RuntimeError(f"no autotune candidate ran for {key}: {last_err}")
    best = min(ok, key=ok.get)
    tile, depth = (int(x) for x in best.split("x"))
    entry = {"tile": tile, "batch_depth": depth, "ms": ok[best], "timings": timings,
             "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    cache[key] = entry
    save_cache(path, cache)
    out = dict(entry)
    out["cached"] = False
    return out
