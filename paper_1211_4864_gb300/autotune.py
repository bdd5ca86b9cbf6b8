"""Autotuner of the pair-kernel launch shape.

The paper picks its BG/Q operating point (ranks per node x threads per core)
by measuring the force kernel over neighbour-list sizes (Sec. III, Fig. 5);
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
    warps = [4, 8]
    per_sm = [1, 2, 3, 4, 6]
    ts = TILE_STAGES
    if quick:
        warps, per_sm, ts = [4, 8], [2, 3], [(32, 4), (64, 4), (128, 2), (128, 4)]
    out = []
    for w, c, (jt, st) in itertools.product(warps, per_sm, ts):
        if w * c > 32:  # more warps than the kernel's 80 registers let an SM hold
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


def cached_split(config: str, default: int = 64, path: str = CACHE) -> int:
    """The split threshold (particles per task) chosen for a workload."""
    ent = load_cache(path).get(_key(config), {}).get("force")
    return int(ent.get("split_T", default)) if ent else default


def tune(run, config: str, mode: str = "force", quick: bool = False, reps: int = 3, path: str = CACHE,
         write: bool = True, extra: dict | None = None, cands=None):
    """Time ``run(launch)`` for every candidate; returns (best Launch, table)."""
    import torch
    table = []
    for L in (cands if cands is not None else candidates(quick)):
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
        ent[mode] = {"launch": best[0].__dict__, "ms": best[1], "candidates": len(ok), **(extra or {})}
        with open(path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return best[0], table


def tune_workload(config: str, splits=(32, 64, 128), quick: bool = False, path: str = CACHE) -> dict:
    """Tune one of the standard workloads (synth.make_config names): the split
    threshold by the symmetric force kernel (the step's force), then, on those
    lists, the launch shapes of the symmetric and gather force kernels and of
    both adjoints."""
    import numpy as np
    import torch

    from synth import default_coeffs, make_config

    from .sr import ShortRange, SRParams

    w = make_config(config)
    prm = SRParams(w.eps, w.rcut, default_coeffs(w.rcut, w.eps))
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    out = torch.empty((3, w.N), device="cuda")
    best = None
    report = {}
    for T in splits:
        sr = ShortRange(w.L, w.vol_off, w.rcut, cell_min=w.cell_min, split_T=T)
        sr.prepare(pos, m)
        _, table = tune(lambda L: sr.force_symmetric(prm, out, launch=L), config, quick=True, write=False)
        ms = min(t[1] for t in table if t[1] is not None)
        report[T] = [(t[0].__dict__, t[1]) for t in table]
        if best is None or ms < best[1]:
            best = (T, ms)
        del sr
        torch.cuda.empty_cache()
    T = best[0]
    sr = ShortRange(w.L, w.vol_off, w.rcut, cell_min=w.cell_min, split_T=T)
    sr.prepare(pos, m)
    cache = load_cache(path)
    ent = cache.setdefault(_key(config), {})
    Ls, tab_s = tune(lambda L: sr.force_symmetric(prm, out, launch=L), config, quick=quick, write=False)
    ent["symmetric"] = {"launch": Ls.__dict__, "ms": min(t[1] for t in tab_s if t[1] is not None)}
    L, tab = tune(lambda L: sr.force(prm, out, launch=L), config, quick=quick, write=False)
    ent["force"] = {"launch": L.__dict__, "ms": min(t[1] for t in tab if t[1] is not None), "split_T": T}
    lam = torch.randn((3, w.N), device="cuda")
    La, _ = tune(lambda L: sr.adjoint(prm, lam, want_gm=False, launch=L), config, mode="adjoint", quick=True,
                 write=False)
    ent["adjoint"] = {"launch": La.__dict__}
    # 128 registers per thread: at most 16 warps per SM
    cands = [c for c in candidates(quick) if c.warps_per_cta * c.ctas_per_sm <= 16]
    Lsa, tab_sa = tune(lambda L: sr.adjoint_symmetric(prm, lam, want_gm=False, launch=L), config,
                       mode="adjoint_symmetric", write=False, cands=cands)
    ent["adjoint_symmetric"] = {"launch": Lsa.__dict__, "ms": min(t[1] for t in tab_sa if t[1] is not None)}
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return {"best": ent, "table": report}


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="tune split threshold and launch shape per workload")
    ap.add_argument("configs", nargs="*", default=["clustered256"])
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--out", default=CACHE, help="cache file to update")
    args = ap.parse_args()
    for name in args.configs:
        res = tune_workload(name, quick=args.quick, path=args.out)
        print(name, json.dumps(res["best"]))
        for T, rows in res["table"].items():
            for L, ms in sorted(rows, key=lambda r: (r[1] is None, r[1] or 0))[:8]:
                print(f"  T={T} {L} {ms}")
