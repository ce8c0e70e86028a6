"""Run one synthetic workload for a number of steps and report the time.

    python -m paper_2103_12819_b300.run_case --workload waveguide --prec fp32 \
        --path fused --steps 20 --warmup 3

Workloads: waveguide (128x128x512, z-PML, YIG slab, TE10 source), yig_slab
(32^3), stress (512^3, centred random magnetic block), sweep (the batched
bias sweep's first --count instances, advanced together as one batch).  Used
for timing single configurations and as the small, single-kernel target of
profiler captures."""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import paper_2103_12819_b300 as mmx
    import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="waveguide", choices=["waveguide", "yig_slab", "stress", "sweep"])
    ap.add_argument("--n", type=int, default=0, help="stress: cube edge (default 512)")
    ap.add_argument("--count", type=int, default=256, help="sweep: instances")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "fp16"])
    ap.add_argument("--path", default="fused", choices=["fused", "plain"])
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--box", default="auto", choices=["auto", "list"],
                    help="H/M kernel: records in shared memory where they fit (auto) or list-driven")
    a = ap.parse_args()
    prec = {"fp32": mmx.FP32, "fp64": mmx.FP64, "fp16": mmx.FP16}[a.prec]
    if a.workload == "sweep":
        return run_sweep(mmx, workloads, a, prec)
    if a.workload == "waveguide":
        w = workloads.waveguide()
    elif a.workload == "yig_slab":
        w = workloads.yig_slab_32()
    else:
        w = workloads.stress(n=a.n or 512)
    path = mmx.PATH_FUSED if a.path == "fused" else mmx.PATH_PLAIN
    s = mmx.from_workload(w, prec=prec, path=path)
    s.set_box_kernel(0 if a.box == "list" else 1)
    s.step(a.warmup)
    rc = s.sync(check=False)
    t0 = time.perf_counter()
    s.step(a.steps)
    rc = rc or s.sync(check=False)
    dt = time.perf_counter() - t0
    st = s.get_stats()
    info = s.get_info()
    print(json.dumps({"workload": w.name, "prec": a.prec, "path": a.path, "steps": a.steps,
                      "fused_kernel": info["fused_kernel_name"], "box_kernel": info["box_kernel_name"],
                      "ms_per_step": 1e3 * dt / max(a.steps, 1),
                      "cell_updates_per_s": w.ncells * a.steps / dt, "status": rc,
                      "iters": [st["iters_min"], st["iters_max"]]}))
    return 0 if rc == 0 else 1


def run_sweep(mmx, workloads, a, prec):
    sols, cells = [], 0
    for n, h0, seed in workloads.bias_sweep(256)[:a.count]:
        w = workloads.tunable_filter(n, h0, steps=2000, seed=seed)
        sols.append(mmx.from_workload(w, prec=prec))
        cells += w.ncells
    b = mmx.Batch(sols)
    b.step(a.warmup)
    rc = b.sync(check=False)
    t0 = time.perf_counter()
    b.step(a.steps)
    rc = rc or b.sync(check=False)
    dt = time.perf_counter() - t0
    print(json.dumps({"workload": "bias_sweep_%d" % len(sols), "prec": a.prec, "instances": len(sols),
                      "cells": cells, "steps": a.steps, "ms_per_step": 1e3 * dt / max(a.steps, 1),
                      "cell_updates_per_s": cells * a.steps / dt, "status": rc,
                      "iters_max": max(s.get_stats()["iters_max"] for s in sols)}))
    b.close()
    for s in sols:
        s.close()
    return 0 if rc == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
