"""Autotuner for the batched, graph-captured hot path.

The tunables are the frontier kernel's tile shape -- threads per block and
paths per thread (a tile is block x items consecutive paths; one path per
1/items of a thread, i.e. 1/(32*items) warps per path) -- its work split
(parts per chunk of a level, for balance between warps) -- and the path-arena
segment policy (exact sizing from a counting run, or a margin over a
prediction, which the sizer supplies).  Results never depend on them.

The tuner measures every supported shape on a tuning batch drawn from seeds
disjoint from the benchmark's (cfggen.TUNER_SEED0 + i), with the whole hot
path captured in a CUDA graph and replayed, and caches the fastest shape per
bitset width W (vertex-count class) in a JSON file.
"""
from __future__ import annotations

import json
import os
import time

from . import cfggen
from . import tpg

SHAPES_NARROW = [(256, 1), (256, 2), (256, 4), (512, 1), (512, 2), (1024, 1)]
SHAPES_WIDE = [(256, 1)]
SPLITS = (1, 2)  # work units per chunk tried with the best shapes
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuned_shapes.json")


def bitset_words(maxn: int) -> int:
    w = (maxn + 31) // 32
    for s in (1, 2, 3, 4, 5, 6, 8, 16, 32, 64, 128):
        if w <= s:
            return s
    raise ValueError("graph too large")


def load_cache(path: str = CACHE) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(table: dict, path: str = CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuning_batch(count: int = 1024, seed0: int = cfggen.TUNER_SEED0):
    return [cfggen.random_cfg(seed0 + i) for i in range(count)]


def measure_shapes(cfgs, shapes=None, reps: int = 3):
    """Median replay time (ms) of the captured hot path for each tile:
    every shape with split 1, then the two fastest shapes with the other
    splits.  Keys are (block, items, split)."""
    import torch

    ns, rp, col, ent, ext = cfggen.concat_batch(cfgs)
    W = bitset_words(int(max(ns)))
    shapes = shapes or (SHAPES_NARROW if W <= 8 else SHAPES_WIDE)
    out = {}
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE) as h:
        def measure(tile):
            tpg.set_tile(h, tile)
            tpg.tpg_graph_capture(h)
            times = []
            for _ in range(reps + 1):
                pp, tp = tpg.tpg_graph_launch(h)
                pp.free()
                tp.free()
                times.append(tpg.tpg_get_stats(h)["t_graph_ms"])
            torch.cuda.synchronize()
            times = sorted(times[1:])
            out[tile] = times[len(times) // 2]

        for sh in shapes:
            measure((sh[0], sh[1], 1))
        for tile in sorted(out, key=out.get)[:2]:
            for sp in SPLITS[1:]:
                measure((tile[0], tile[1], sp))
    return W, out


def tune(cfgs=None, reps: int = 3, path: str = CACHE, force: bool = False):
    """Best (block, items, split) for the batch's bitset width, from the cache or by measuring."""
    cfgs = cfgs if cfgs is not None else tuning_batch()
    W = bitset_words(max(c.n for c in cfgs))
    table = load_cache(path)
    key = f"W{W}"
    if not force and key in table and len(table[key].get("shape", ())) == 3:
        e = table[key]
        return tuple(e["shape"]), e
    t0 = time.perf_counter()
    W, res = measure_shapes(cfgs, reps=reps)
    best = min(res, key=res.get)
    entry = {"shape": list(best), "ms": res[best],
             "all": {f"{b}x{i}/{sp}": ms for (b, i, sp), ms in res.items()},
             "graphs": len(cfgs), "seconds": time.perf_counter() - t0}
    table[key] = entry
    save_cache(table, path)
    return best, entry
