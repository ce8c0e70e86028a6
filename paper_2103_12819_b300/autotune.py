"""Tuning for batches: time candidate launch shapes on a scratch copy of the
batch and cache the winner as JSON.

Two knobs, both run-time properties of a batch:
  * planes (``Batch.set_planes``; 0 = a whole grid): the z planes each fused
    CTA marches.  Short chunks give more CTAs and better balance across
    instances of uneven size; long chunks recompute fewer chunk-boundary
    planes.
  * box blocks per SM (``Batch.set_box_blocks``; 0 = as many as are
    resident): the size of the cooperative H/M launch.  Fewer blocks mean
    fewer arrivals at each grid-wide vote of the iteration and more faces
    per thread.
The tile shape of the fused pass (a 32 V-column strip by 7 rows, V = 16
bytes / element size) and the H/M block shape (256 threads) are compile-time
properties of the kernels, chosen by measurement and not tuned here; the
iteration count per half step is set by the scheme's stopping rule, not by
the launch.

Tuning runs on solvers built by the caller's factory (fresh instances of the
same workload), so the batch being tuned for is not advanced.  Results are
cached per size class: the multiset of instance sizes and the precision.

    cfg = tune(lambda: [mmx.from_workload(w, prec=mmx.FP32) for w in ws])
    batch.set_planes(cfg["planes"])
    batch.set_box_blocks(cfg["box_blocks"])
"""
import json
import os
import time

import paper_2103_12819_b300 as mmx

CANDIDATES = (0, 64, 32, 16, 8)
BOX_CANDIDATES = (0, 4, 3, 2)
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune.json")


def _signature(solvers):
    sizes = sorted(tuple(s.n) for s in solvers)
    counts = {}
    for n in sizes:
        counts["x".join(map(str, n))] = counts.get("x".join(map(str, n)), 0) + 1
    return "prec%d:" % solvers[0].prec + ",".join("%s*%d" % kv for kv in sorted(counts.items()))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _time(batch, steps, warmup):
    batch.step(warmup)
    batch.sync()
    t0 = time.perf_counter()
    batch.step(steps)
    batch.sync()
    return (time.perf_counter() - t0) / steps


def tune(make_solvers, candidates=CANDIDATES, box_candidates=BOX_CANDIDATES, steps=10, warmup=2, cache=CACHE,
         force=False):
    """The fastest (planes, box blocks per SM) for the batch the factory
    builds, as {"planes": p, "box_blocks": b}.  Planes are timed first with
    the default H/M launch, then the box-block candidates with the best
    planes (the two launches of a step are independent, so the knobs
    separate); each candidate over `steps` batch steps after `warmup`."""
    solvers = make_solvers()
    key = _signature(solvers)
    table = _load(cache) if cache else {}
    hit = table.get(key) if not force else None
    if hit and "box_blocks" in hit and set(box_candidates) <= set(hit.get("box_candidates", [0])):
        for s in solvers:
            s.close()
        return {"planes": int(hit["planes"]), "box_blocks": int(hit["box_blocks"])}
    batch = mmx.Batch(solvers)
    t_planes = {}
    for planes in candidates:
        batch.set_planes(planes)
        t_planes[planes] = _time(batch, steps, warmup)
    best_planes = min(t_planes, key=t_planes.get)
    batch.set_planes(best_planes)
    t_box = {}
    for nb in box_candidates:
        batch.set_box_blocks(nb)
        t_box[nb] = _time(batch, steps, warmup)
    best_box = min(t_box, key=t_box.get)
    batch.close()
    for s in solvers:
        s.close()
    if cache:
        table = _load(cache)
        table[key] = {"planes": int(best_planes), "box_blocks": int(best_box),
                      "box_candidates": sorted(int(x) for x in box_candidates),
                      "ms_per_step": {"planes": {str(k): round(1e3 * v, 4) for k, v in t_planes.items()},
                                      "box_blocks": {str(k): round(1e3 * v, 4) for k, v in t_box.items()}}}
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return {"planes": int(best_planes), "box_blocks": int(best_box)}


def tune_planes(make_solvers, candidates=CANDIDATES, steps=10, warmup=2, cache=CACHE, force=False):
    """The fastest chunk length (planes) for the batch the factory builds,
    with the default H/M launch (``tune`` with one box-block candidate)."""
    return tune(make_solvers, candidates, (0,), steps, warmup, cache, force)["planes"]
