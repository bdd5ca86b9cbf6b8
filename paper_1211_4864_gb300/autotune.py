"""Autotuner of the pair-kernel launch shape.

The paper picks its BG/Q operating point (ranks per node x threads per core)
by measuring the force kernel over neighbour-list sizes (Sec. IV-B, Fig. 5);
the GPU analogue is the launch shape of the persistent pair kernel: warps per
CTA, resident CTAs per SM, staged j-tile length and pipeline depth.  ``tune``
times each candidate on the caller's actual mesh and lists with CUDA events
and records the fastest per workload name and GPU model in a JSON cache that
``cached`` reads back.
"""

from __future__ import annotations

import itertools
import json
import os
import statistics

from .sr import Launch

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")

# the launch shapes the library instantiates (jtile, stages)
TILE_STAGES = [(32, 2), (32, 4), (64, 2), (64, 3), (64, 4), (128, 2), (128, 3), (128, 4), (256, 2)]


def candidates(quick: bool = False):
    warps = [4, 8, 16]
    per_sm = [1, 2, 3, 4]
    ts = TILE_STAGES
    if quick:
        warps, per_sm, ts = [4, 8], [2, 3], [(32, 4), (64, 4), (128, 2), (128, 4)]
    out = []
    for w, c, (jt, st) in itertools.product(warps, per_sm, ts):
        if w * c > 48:  # more resident warps than an SM holds
            continue
        out.append(Launch(w, c, jt, st))
    return out


def _key(config: str) -> str:
    try:
        import torch
        name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    except Exception:  # pragma: no cover - no device
        name = "unknown"
    return f"{config}|{name}"


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cached(config: str, mode: str = "force", path: str = CACHE) -> Launch | None:
    ent = load_cache(path).get(_key(config), {}).get(mode)
    if not ent:
        return None
    return Launch(**ent["launch"])


def tune(run, config: str, mode: str = "force", quick: bool = False, reps: int = 3, path: str = CACHE,
         write: bool = True):
    """Time ``run(launch)`` for every candidate; returns (best Launch, table)."""
    import torch
    table = []
    for L in candidates(quick):
        try:
            run(L)
            torch.cuda.synchronize()
        except Exception as ex:  # a shape the device cannot host
            table.append((L, None, str(ex)))
            continue
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run(L)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        table.append((L, statistics.median(ts), None))
    ok = [t for t in table if t[1] is not None]
    best = min(ok, key=lambda t: t[1])
    if write:
        cache = load_cache(path)
        ent = cache.setdefault(_key(config), {})
        ent[mode] = {"launch": best[0].__dict__, "ms": best[1], "candidates": len(ok)}
        with open(path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return best[0], table
