"""Tile-size and launch-shape autotuner for the tiled paths.

The tile size (nodes per tile) sets the partition of the grid: larger tiles
recompute fewer halo elements but need more shared memory per block, so fewer
blocks are resident per SM (the launch then switches to 512-thread CTAs).
`tune()` builds a plan for each candidate size, times the requested pass with
CUDA events and keeps the fastest; results are cached in a JSON file keyed by
the grid, the pass, the arithmetic form and the GPU, so later runs reuse the
choice.  `tune_batch()` does the same for a batch of grids, over tile sizes
and the batched launch shapes.
"""
from __future__ import annotations

import json
import os

import torch

from . import api
from ._lib import EMError

CANDIDATES = (64, 96, 128, 160, 192, 256)


def _cache_path():
    return os.environ.get("EM_AUTOTUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "edgemetrics",
                                                               "autotune.json")


def _key(topo, what, precision, paths):
    dev = torch.cuda.get_device_name()
    return f"{dev}|dim{topo.dim}|v{topo.n_nodes}|e{topo.n_elems}|{what}|{precision}|{','.join(paths)}"


def _load():
    p = _cache_path()
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return {}


def _store(d):
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".{os.getpid()}"
        json.dump(d, open(tmp, "w"), indent=1)
        os.replace(tmp, p)
    except OSError:
        pass


def _time(fn, reps=5):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune(topo, x, w=None, c=None, what="fused", precision="dw", candidates=CANDIDATES, reps=5, use_cache=True,
         paths=("gather", "tiled")):
    """Pick (path, tile_nodes) for `what` in {"fwd", "adj", "fused"} among
    the tiled paths `paths`; builds the winning plan into topo and returns
    (path, tile_nodes, {"path/tile": ms or error})."""
    cache = _load() if use_cache else {}
    key = _key(topo, what, precision, paths)
    if use_cache and key in cache:
        t = int(cache[key]["tile_nodes"])
        api.plan_build(topo, t)
        return cache[key]["path"], t, cache[key].get("sweep", {})
    sweep = {}
    best = None
    for t in candidates:
        try:
            api.plan_build(topo, t)
        except EMError as ex:
            sweep[f"*/{t}"] = f"unusable: {str(ex)[:80]}"
            continue
        for p in paths:
            try:
                if what == "fwd":
                    fn = lambda: api.edge_metrics(topo, x, precision, p)  # noqa: E731
                elif what == "adj":
                    fn = lambda: api.edge_metrics_adjoint(topo, x, w, c, precision, p)  # noqa: E731
                else:
                    fn = lambda: api.edge_metrics_fused(topo, x, w, c, precision, path=p)  # noqa: E731
                ms = _time(fn, reps)
                sweep[f"{p}/{t}"] = round(ms, 4)
                if best is None or ms < best[2]:
                    best = (p, t, ms)
            except EMError as ex:
                sweep[f"{p}/{t}"] = f"unusable: {str(ex)[:80]}"
    if best is None:
        raise EMError(-1, f"no usable tile size among {candidates}")
    api.plan_build(topo, best[1])
    cache[key] = {"path": best[0], "tile_nodes": best[1], "ms": best[2], "sweep": sweep}
    if use_cache:
        _store(cache)
    return best[0], best[1], sweep


def tune_batch(topos, xs, ws, cs, precision="dw", candidates=(96, 192, 256), shapes=(0, -1), reps=5):
    """Pick (tile_nodes, launch shape) for the batched forward + adjoint of
    the grids `topos`: every grid is re-planned at each candidate tile size
    and each launch shape of api.Batch (0: one CTA per work item, -1:
    persistent) is timed as a CUDA-graph replay.  Leaves every grid planned
    at the winning size and returns (tile_nodes, blocks, {"tile/shape": ms})."""
    sweep = {}
    best = None
    for t in candidates:
        try:
            for topo in topos:
                api.plan_build(topo, t)
        except EMError as ex:
            sweep[f"{t}/*"] = f"unusable: {str(ex)[:80]}"
            continue
        for b in shapes:
            try:
                bt = api.Batch(topos, xs, ws, cs, precision, blocks=b)
                g = bt.capture()
                ms = _time(g.replay, reps)
                bt.check_status()
                sweep[f"{t}/{b}"] = round(ms, 4)
                if best is None or ms < best[2]:
                    best = (t, b, ms)
            except EMError as ex:
                sweep[f"{t}/{b}"] = f"unusable: {str(ex)[:80]}"
    if best is None:
        raise EMError(-1, f"no usable tile size among {candidates}")
    for topo in topos:
        api.plan_build(topo, best[0])
    return best[0], best[1], sweep
