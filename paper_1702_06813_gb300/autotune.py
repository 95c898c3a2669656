"""Autotuner for the screen-tile size, the number of poses per kernel wave and the bin capacity
(triangle records per screen-tile bin).

For one (map, camera, batch size) it times rm_cost_grad over each (tile, wave) candidate with
CUDA events on the current stream, then, at the fastest of those, each initial bin capacity,
and keeps the fastest, caching the choice in a JSON file keyed by image size, triangle count
and batch size. A capacity that a bin overflows is doubled by the library until every bin
fits (in the untimed warm-up call), so the capacity recorded is the one that ran.
"""
from __future__ import annotations

import json
import os

import torch

from . import rendermap as rm

TILES = ((64, 32), (32, 32), (32, 16), (16, 16))
WAVES = (16, 32, 64, 128)
CAPACITIES = (256, 512, 1024)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rendermap_autotune.json")


def _key(m, intr, n):
    return f"{intr.width}x{intr.height}-model{intr.model}-T{m.n_faces}-N{n}"


def _time(m, scan, poses, params, reps):
    s = torch.cuda.current_stream()
    rm.cost_grad(m, scan, poses, params)  # warm, and grow the bins if needed
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        rm.cost_grad(m, scan, poses, params)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _apply(m, best):
    m.set_tuning(tile=tuple(best["tile"]), wave_poses=best["wave_poses"],
                 bin_capacity=best.get("bin_capacity", 0))


def autotune(m: rm.Map, scan: rm.Scan, poses, params=None, tiles=TILES, waves=WAVES,
             capacities=CAPACITIES, reps=3, cache: str | None = DEFAULT_CACHE,
             force: bool = False) -> dict:
    """Pick and apply the fastest (tile, wave_poses, bin_capacity); returns {"tile",
    "wave_poses", "bin_capacity", "ms"} (plus the timed "candidates" when it searched)."""
    poses = torch.as_tensor(poses, dtype=torch.float64, device="cuda").reshape(-1, 16)
    n = poses.shape[0]
    key = _key(m, scan.intr, n)
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as fh:
                table = json.load(fh)
        except (OSError, ValueError):
            table = {}
    if key in table and not force:
        best = table[key]
        _apply(m, best)
        return best
    results = []
    # every (tile, wave) candidate starts from the same capacity: a capacity that a larger tile
    # grew (panoramic tiles can hold thousands of records) would otherwise carry over to the
    # smaller tiles and their waves, whose scratch it sizes
    cap0 = m.get_tuning()["bin_capacity"]
    for tile in tiles:
        for wave in [w for w in waves if w <= max(n, waves[0])]:
            m.set_tuning(tile=tile, wave_poses=wave, bin_capacity=cap0)
            ms = _time(m, scan, poses, params, reps)
            results.append({"tile": list(tile), "wave_poses": wave,
                            "bin_capacity": m.get_tuning()["bin_capacity"], "ms": ms})
    best = min(results, key=lambda r: r["ms"])
    for cap in capacities:
        m.set_tuning(tile=tuple(best["tile"]), wave_poses=best["wave_poses"], bin_capacity=cap)
        ms = _time(m, scan, poses, params, reps)
        results.append({"tile": best["tile"], "wave_poses": best["wave_poses"],
                        "bin_capacity": m.get_tuning()["bin_capacity"], "ms": ms})
    best = min(results, key=lambda r: r["ms"])
    _apply(m, best)
    if cache:
        table[key] = best
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1)
        os.replace(tmp, cache)
    return dict(best, candidates=results)
