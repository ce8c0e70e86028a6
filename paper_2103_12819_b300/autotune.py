"""Tile tuning for batches: time the candidate z-chunk lengths of the fused
launch on a scratch copy of the batch and cache the winner as JSON.

The knob is the number of z planes each fused CTA marches
(``Batch.set_planes``; 0 = a whole grid): short chunks give more CTAs and
better balance across instances of uneven size, long chunks recompute fewer
chunk-boundary planes.  Tuning runs on solvers built by the caller's
factory (fresh instances of the same workload), so the batch being tuned
for is not advanced.  Results are cached per size class: the multiset of
instance sizes and the precision.

    planes = tune_planes(lambda: [mmx.from_workload(w, prec=mmx.FP32) for w in ws])
    batch.set_planes(planes)
"""
import json
import os
import time

import paper_2103_12819_b300 as mmx

CANDIDATES = (0, 64, 32, 16, 8)
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


def tune_planes(make_solvers, candidates=CANDIDATES, steps=10, warmup=2, cache=CACHE, force=False):
    """The fastest chunk length (planes) for the batch the factory builds;
    each candidate is timed over `steps` batch steps after `warmup` steps."""
    solvers = make_solvers()
    key = _signature(solvers)
    table = _load(cache) if cache else {}
    if not force and key in table:
        for s in solvers:
            s.close()
        return int(table[key]["planes"])
    batch = mmx.Batch(solvers)
    timings = {}
    for planes in candidates:
        batch.set_planes(planes)
        batch.step(warmup)
        batch.sync()
        t0 = time.perf_counter()
        batch.step(steps)
        batch.sync()
        timings[planes] = (time.perf_counter() - t0) / steps
    batch.close()
    for s in solvers:
        s.close()
    best = min(timings, key=timings.get)
    if cache:
        table = _load(cache)
        table[key] = {"planes": int(best), "ms_per_step": {str(k): round(1e3 * v, 4) for k, v in timings.items()}}
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return int(best)
