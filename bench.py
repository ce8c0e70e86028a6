#!/usr/bin/env python
"""Throughput of the coupled E/H/M step on the 128x128x512 waveguide.

One "step" is one full time step of the scheme (H/M half step, E update,
H/M half step, Sec. 3.2 of arXiv 2103.12819) on the 128x128x512 PEC
waveguide with 10-cell z-PML ends, a YIG-like slab and a TE10 soft source,
from seeded synthetic inputs already resident in HBM.  The headline runs in
FP32; the FP64 path and the plain one-kernel-per-update path are measured
beside it.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank advances its own
replica: the method has no exchange step at one GPU per instance, so the
scaling is weak and `value` is the sum over ranks.  `--impl reference` times
the FP64 CPU oracle on the host cores instead (rank 0 only).
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled E/H/M cell-updates/s and % of HBM roofline; FP32 vs FP64 path at stated error"
UNIT = "cell-updates/s"
WORKLOAD = "waveguide_128x128x512"
L2_BYTES = 126 * 2 ** 20
ACCURACY_STEPS = (1000, 5000)   # the waveguide's stated checkpoints


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def config_block(w, prec_name, path_name):
    state_bytes = 6 * w.ncells * (4 if prec_name == "fp32" else 8)
    return {
        "workload": WORKLOAD,
        "cells": w.ncells,
        "grid": list(w.n),
        "cell_size_m": w.d[0],
        "dt_s": w.dt,
        "boundaries": "PEC x/y, 10-cell z-PML",
        "magnetic_fraction": float(np.count_nonzero(w.Ms > 0)) / w.ncells,
        "precision": prec_name,
        "path": path_name,
        "tol": w.tol,
        "l2_policy": "inputs larger than L2 (E+H state %.0f MB > %d MB L2)" % (state_bytes / 1e6, L2_BYTES >> 20),
    }


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- helpers

def alg_bytes_per_cell(kernel, w, esz, ssz=None):
    """Algorithmic DRAM bytes per cell for one launch of each kernel (what the
    method must move, single pass): E update reads E, H, eps_r and writes E
    (10 words); a non-magnetic H half step reads E, H and writes H (9 words);
    a fused E+H+H pass reads E, H, eps_r and writes E, H (13 words); the H/M
    box kernel reads E, H, M, Ms, alpha, gamma and writes H, M on its faces
    (per magnetic cell 6 + 9 + 3 read, 3 + 9 written).  E and H words are
    ssz bytes (the stored type), eps_r esz bytes (the arithmetic type)."""
    ssz = esz if ssz is None else ssz
    fields = {"e_update": 9, "h_update": 9, "fused_eh": 12, "fused_eh_vec": 12, "fused_eh_vec_tma": 12}.get(kernel)
    coef = {"e_update": 1, "h_update": 0, "fused_eh": 1, "fused_eh_vec": 1, "fused_eh_vec_tma": 1}.get(kernel)
    if fields is not None:
        return fields * ssz + coef * esz
    return None


def effective_fraction(w, value_per_gpu, word, peak_gbs):
    """Step-level HBM fraction: B_alg x cell-updates/s / peak, with
    B_alg = (13 + 21 f) words per cell-update (E, H, eps_r in and E, H out
    everywhere; M, Ms, alpha, gamma in and M out on the magnetic fraction f)."""
    f = float(np.count_nonzero(w.Ms > 0)) / w.ncells if w.Ms is not None else 0.0
    return round((13 + 21 * f) * word * value_per_gpu / (peak_gbs * 1e9), 4), f


def replica_layout(env=None):
    """(world, rank, local_rank) from the torchrun environment; 1 GPU if unset."""
    env = os.environ if env is None else env
    return (int(env.get("WORLD_SIZE", "1")), int(env.get("RANK", "0")), int(env.get("LOCAL_RANK", "0")))


def max_over_ranks(torch, ms, dist, device):
    """The slowest rank's time: every replica must finish before the job has."""
    if dist is None:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, world, K, ms):
    """Cell-updates per second of the whole job: all ranks' cells x K steps
    over the slowest rank's time (weak scaling, one replica per GPU)."""
    return cells_per_rank * world * K / (ms * 1e-3)


def time_steps(torch, sim, stream, K, dist=None):
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    return max_over_ranks(torch, e0.elapsed_time(e1), dist, "cuda")


def run_path(torch, mmx, w, prec, path, K, W, stream, dist=None, profile=True):
    sim = mmx.from_workload(w, prec=prec, stream=stream.cuda_stream, path=path)
    sim.step(W)
    rc = sim.sync(check=False)
    if rc:
        raise RuntimeError("warm-up failed: %s" % sim.last_error())
    ms = time_steps(torch, sim, stream, K, dist)
    rc = sim.sync(check=False)
    if rc:
        raise RuntimeError("timed run failed: %s" % sim.last_error())
    prof = None
    if profile:
        sim.set_profiling(True)
        sim.get_profile(reset=True)
        sim.step(K)
        prof = sim.get_profile(reset=True)
        sim.set_profiling(False)
    stats = sim.get_stats()
    return sim, ms, prof, stats


# The files that define the fused kernel, its device helpers and its tile
# configuration: a captured DRAM traffic figure is reported only while they
# are unchanged.
KERNEL_SOURCES = ("mmx_device.cuh", "mmx_kernels.cuh", "mmx_fused.cuh")


def kernel_source_sha256():
    """sha256 over KERNEL_SOURCES (in that order)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_12819_b300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def captured_traffic(kernel, prec_name):
    """DRAM bytes (read + write) per launch of `kernel` on this workload from
    the committed ncu summary, or None if there is none for these sources."""
    path = os.path.join(ROOT, "profiles", "%s_%s_%s.md" % (kernel, WORKLOAD, prec_name))
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    fields = dict(re.findall(r"^- (source_sha256|traffic_bytes_per_launch): `?([0-9a-f]+)`?$", text, re.M))
    if fields.get("source_sha256") != kernel_source_sha256() or "traffic_bytes_per_launch" not in fields:
        return None
    return int(fields["traffic_bytes_per_launch"])


def roofline_of(prof, K, w, esz, peak_gbs, peak_kind, ssz=None, prec_name=None):
    if not prof:
        return None, None
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (launches, total_ms) = dom
    avg_ms = total_ms / launches
    bpc = alg_bytes_per_cell(name, w, esz, ssz)
    launches_per_step = sum(v[0] for v in prof.values()) / K
    if bpc is None:
        return {"bound": "hbm", "kernel": name, "achieved": None, "peak": peak_gbs, "unit": "GB/s",
                "frac": None, "traffic": None, "peak_kind": peak_kind}, launches_per_step
    achieved = bpc * w.ncells / (avg_ms * 1e-3) / 1e9
    shares = {k: round(v[1] / sum(x[1] for x in prof.values()), 4) for k, v in prof.items()}
    traffic = captured_traffic(name, prec_name or ("fp32" if esz == 4 else "fp64"))
    return {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak_gbs,
            "unit": "GB/s", "frac": round(achieved / peak_gbs, 4), "traffic": traffic,
            "alg_bytes_per_launch": bpc * w.ncells,
            "peak_kind": peak_kind, "alg_bytes_per_cell": bpc, "avg_launch_us": round(avg_ms * 1e3, 2),
            "kernel_shares": shares}, launches_per_step


def accuracy_leg(mmx, w, stream, checkpoints=ACCURACY_STEPS, prec=None):
    """The FP32 (or `prec`) path against the FP64 path (which matches the FP64
    oracle to 1e-12, see the parity tests) after each of `checkpoints` steps
    from the same initial state: relative L2 per field (E 0-2, H 3-5, M 6-14,
    PML split parts 15-18, a split part against the norm of its component)."""
    low = mmx.FP32 if prec is None else prec
    sims = {p: mmx.from_workload(w, prec=p, stream=stream.cuda_stream, path=mmx.PATH_FUSED)
            for p in (low, mmx.FP64)}
    parent = {15: 0, 16: 1, 17: 3, 18: 4}
    out, done = {}, 0
    for n in checkpoints:
        for x in sims.values():
            x.step(n - done)
            x.sync()
        done = n
        a_s, b_s = sims[low], sims[mmx.FP64]
        errs = {}
        for fid in range(19):
            a, b = a_s.get_field(fid), b_s.get_field(fid)
            nb = np.linalg.norm(b_s.get_field(parent[fid]) if fid in parent else b)
            errs[fid] = float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.abs(a - b).max())
        # the E, H and M vector fields as a whole (components near zero, such
        # as Ex and Ez of a TE10 guide, are measured against their vector)
        vec = {}
        for grp, fids in (("E", range(0, 3)), ("H", range(3, 6)), ("M", range(6, 15))):
            e2 = sum(float(np.sum((a_s.get_field(f) - b_s.get_field(f)) ** 2)) for f in fids)
            n2 = sum(float(np.sum(b_s.get_field(f) ** 2)) for f in fids)
            vec[grp] = float("%.3e" % ((e2 / n2) ** 0.5)) if n2 > 0 else 0.0
        out[str(n)] = {"max": max(errs.values()), "vector_fields": vec,
                       "per_field": {str(k): float("%.3e" % v) for k, v in errs.items()}}
    for x in sims.values():
        x.close()
    return out


def m_upload_elems(w):
    """Elements an M-component upload moves: M lives on the magnetic box (the
    magnetic cells' bounding box grown by one face, clipped to the field), so
    set_field transfers that region only.  Per family (x, y, z faces)."""
    import workloads
    if w.Ms is None or not np.any(w.Ms > 0):
        return [0, 0, 0]
    kk, jj, ii = np.nonzero(w.Ms > 0)
    c0 = (int(ii.min()), int(jj.min()), int(kk.min()))
    c1 = (int(ii.max()), int(jj.max()), int(kk.max()))
    lo, hi = [], []
    for a in range(3):
        if w.bc[a] == workloads.PERIODIC and (c0[a] == 0 or c1[a] == w.n[a] - 1):
            lo.append(0)
            hi.append(w.n[a] + 1)
        else:
            lo.append(max(c0[a] - 1, 0))
            hi.append(min(c1[a] + 2, w.n[a] + 1))
    out = []
    for d in range(3):
        e = workloads.field_extent(6 + 3 * d, w.n)
        out.append(int(np.prod([max(0, min(hi[a], e[a]) - lo[a]) for a in range(3)])))
    return out


def e2e_leg(torch, mmx, w, prec, path, K, stream):
    """Through the public API with host buffers: upload the state from pinned
    host memory, K steps, read the whole state back, all inside the timed
    region (host wall clock around synchronising calls)."""
    sim = mmx.from_workload(w, prec=prec, stream=stream.cuda_stream, path=path)
    sim.step(2)
    sim.sync()
    fids = list(range(15))
    host = {}
    for fid in fids:
        t = torch.empty(sim.field_size(fid), dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = sim.get_field(fid)
        host[fid] = t
    out = {fid: torch.empty(sim.field_size(fid), dtype=torch.float64, pin_memory=True) for fid in fids}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for fid in fids:
        sim.set_field(fid, host[fid].numpy())
    sim.step(K)
    for fid in fids:
        sim.get_field(fid, out=out[fid].numpy())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nbytes = sum(8 * sim.field_size(f) for f in fids)
    mreg = m_upload_elems(w)
    nbytes_up = sum(8 * sim.field_size(f) for f in fids if f < 6) + sum(8 * 3 * m for m in mreg)
    sim.close()
    return {"value": w.ncells * K / dt, "unit": UNIT, "h2d_bytes_per_step": nbytes_up // K,
            "d2h_bytes_per_step": nbytes // K, "what": "set all 15 state fields from pinned host "
            "float64 (M components move their magnetic-box region only), %d steps, read all 15 "
            "back" % K}


def _oracle_rate(w, variant, budget_s, max_steps=50):
    import oracle
    s = oracle.from_workload(w, variant=variant)
    s.step(1)
    n, t0 = 0, time.perf_counter()
    while True:
        s.step(1)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= max_steps:
            break
    s.close()
    return w.ncells * n / el, n, el


def oracle_stress_timing(single_steps=1, omp_steps=3):
    """The FP64 oracle on the 512^3 configuration (bounded samples: set-up
    excluded, `single_steps` steps on one thread, `omp_steps` steps of the
    OpenMP build on all host cores).  Opt-in (--oracle-512): the oracle's
    arrays take about 44 GB of host memory and its set-up minutes."""
    import workloads
    w = workloads.stress()
    out = {"workload": "stress_512^3", "cells": w.ncells}
    for variant, steps, key in (("", single_steps, "single_thread"), ("omp", omp_steps, "all_cores")):
        import oracle
        t0 = time.perf_counter()
        s = oracle.from_workload(w, variant=variant)
        setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        s.step(steps)
        el = time.perf_counter() - t0
        s.close()
        out[key] = {"value": w.ncells * steps / el, "unit": UNIT, "steps": steps, "seconds": round(el, 1),
                    "setup_s": round(setup, 1), "cores": 1 if not variant else (os.cpu_count() or 1)}
    return out


def cpu_baseline(w, budget_s=15.0, all_cores=True):
    """The FP64 oracle as it stands, single thread, on a bounded sample of
    the same workload (first steps of the run); beside it the oracle's
    OpenMP build (bit-identical, loops over z planes and magnetic faces in
    parallel) on all host cores, timed the same way."""
    rate, n, el = _oracle_rate(w, "", budget_s)
    out = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%s, %d oracle steps after 1 warm-up step, single thread, %.1f s" % (w.name, n, el)}
    if all_cores:
        cores = os.cpu_count() or 1
        r2, n2, el2 = _oracle_rate(w, "omp", budget_s / 2)
        out["all_cores"] = {"value": r2, "unit": UNIT, "cores": cores, "kind": "oracle (OpenMP build)",
                            "sample": "%s, %d steps after 1 warm-up step, %d threads, %.1f s"
                                      % (w.name, n2, cores, el2)}
    return out


# ---------------------------------------------------------------- arms

def reference_arm(args):
    import workloads
    _, rank, _ = replica_layout()
    if rank != 0:
        return 0
    w = workloads.waveguide()
    base = cpu_baseline(w, budget_s=min(120.0, 5.0 + 2.5 * args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * w.ncells / base["value"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(w, "fp64", "oracle"), "cpu_baseline": base,
        "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def stress_leg(torch, mmx, stream, peak, K=10, W=3, prec=None):
    """The 512^3 throughput configuration (PEC box, centred random 256^3
    magnetic block, no source, FP32 or FP16 storage with FP32 arithmetic,
    tol 1e-6): cell-updates/s, the step-level HBM fraction and the
    per-kernel shares (CUDA events).  With FP16 storage B_alg counts E and H
    as 2-byte words: (12 x 2 + 4) + 21 f x 4 bytes."""
    import workloads
    prec = mmx.FP32 if prec is None else prec
    w = workloads.stress()
    sim = mmx.from_workload(w, prec=prec, stream=stream.cuda_stream, path=mmx.PATH_FUSED)
    sim.step(W)
    if sim.sync(check=False):
        raise RuntimeError("stress warm-up failed: %s" % sim.last_error())
    ms = time_steps(torch, sim, stream, K)
    sim.sync()
    sim.set_profiling(True)
    sim.get_profile(reset=True)
    sim.step(K)
    prof = sim.get_profile(reset=True)
    st = sim.get_stats()
    info = sim.get_info()
    sim.close()
    value = w.ncells * K / (ms * 1e-3)
    tot = sum(v[1] for v in prof.values())
    eff, f = effective_fraction(w, value, 4, peak)
    if prec == mmx.FP16:
        eff = round((28 + 84 * f) * value / (peak * 1e9), 4)
    return {"workload": "stress_512^3 (PEC, centred random 256^3 magnetic block, no source, tol 1e-6)",
            "cells": w.ncells, "steps": K, "warmup": W, "value": value, "unit": UNIT,
            "ms_per_step": ms / K, "dtype": "f32" if prec != mmx.FP16 else "f16 storage, f32 arithmetic",
            "magnetic_fraction": round(f, 4),
            "effective_hbm_fraction": eff, "fused_kernel": info["fused_kernel_name"],
            "box_faces_magnetic": info["box_faces_magnetic"],
            "kernel_shares": {k: round(v[1] / tot, 4) for k, v in prof.items()},
            "kernel_avg_us": {k: round(1e3 * v[1] / v[0], 1) for k, v in prof.items()},
            "iters": [st["iters_min"], st["iters_max"]]}


def sweep_leg(torch, mmx, stream, peak, K=200, W=10):
    """The batched bias sweep: 256 independent instances with sizes from
    {32, 48, 64, 96}^3, bias U[5e4, 2e5] A/m, FP32, advanced together by the
    batched launches (one CUDA graph per call)."""
    import workloads
    specs = workloads.bias_sweep(256)
    sols, cells, magcells = [], 0, 0
    for n, h0, seed in specs:
        w = workloads.tunable_filter(n, h0, steps=2000, seed=seed)
        sols.append(mmx.from_workload(w, prec=mmx.FP32, stream=stream.cuda_stream))
        cells += w.ncells
        magcells += int(np.count_nonzero(w.Ms > 0))
    b = mmx.Batch(sols, stream=stream.cuda_stream)
    b.step(W)
    if b.sync(check=False):
        raise RuntimeError("sweep warm-up failed")
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ok = b.sync(check=False) == 0
    iters = [s.get_stats()["iters_max"] for s in sols]
    b.close()
    for s in sols:
        s.close()
    value = cells * K / (ms * 1e-3)
    f = magcells / cells
    return {"workload": "bias_sweep_256 (sizes {32,48,64,96}^3, centred slab, point source, tol 1e-6)",
            "instances": len(specs), "cells": cells, "steps": K, "warmup": W, "value": value, "unit": UNIT,
            "ms_per_step": ms / K, "dtype": "f32", "magnetic_fraction": round(f, 4),
            "effective_hbm_fraction": round((13 + 21 * f) * 4 * value / (peak * 1e9), 4),
            "status_ok": ok, "iters_max": max(iters)}


def ours_arm(args):
    import torch
    import paper_2103_12819_b300 as mmx
    import workloads
    world, rank, local = replica_layout()
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    else:
        torch.cuda.set_device(0)
    peak, peak_kind = peaks()
    K, W = args.steps, max(3, args.warmup)
    w = workloads.waveguide()
    stream = torch.cuda.Stream()
    path = mmx.PATH_FUSED
    with torch.cuda.stream(stream):
        with ClockSampler(local) as clk:
            sim32, ms32, prof32, stats32 = run_path(torch, mmx, w, mmx.FP32, path, K, W, stream, dist)
        clocks = clk.summary()
        info32 = sim32.get_info()
        roof, lps = roofline_of(prof32, K, w, 4, peak, peak_kind)
        sim64, ms64, prof64, stats64 = run_path(torch, mmx, w, mmx.FP64, path, K, W, stream, dist)
        roof64, _ = roofline_of(prof64, K, w, 8, peak, peak_kind)
        sim16, ms16, prof16, stats16 = run_path(torch, mmx, w, mmx.FP16, path, K, W, stream, dist)
        roof16, _ = roofline_of(prof16, K, w, 4, peak, peak_kind, ssz=2, prec_name="fp16")
        sim16.close()
        simp, msp, profp, _ = run_path(torch, mmx, w, mmx.FP64, mmx.PATH_PLAIN, K, W, stream, dist,
                                       profile=False)
        simp.close()
        sim32.close()
        sim64.close()
        acc = accuracy_leg(mmx, w, stream)
        acc16 = accuracy_leg(mmx, w, stream, checkpoints=(1000,), prec=mmx.FP16)
        e2e = e2e_leg(torch, mmx, w, mmx.FP32, path, K, stream)
        stress = None if args.no_stress else stress_leg(torch, mmx, stream, peak)
        stress16 = None if args.no_stress else stress_leg(torch, mmx, stream, peak, prec=mmx.FP16)
        sweep = None if args.no_sweep else sweep_leg(torch, mmx, stream, peak)
    value = whole_job_rate(w.ncells, world, K, ms32)
    eff, mag_frac = effective_fraction(w, value / world, 4, peak)
    if roof:
        # the whole step against the same peak, beside the dominant kernel's
        # own fraction: B_alg = (13 + 21 f) words per cell-update
        roof["step_frac"] = eff
        roof["step_alg_bytes_per_cell"] = round((13 + 21 * mag_frac) * 4, 2)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms32 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded workload generator; no dataset)",
        "config": config_block(w, "fp32", "fused" if path == mmx.PATH_FUSED else "plain"),
        # the step-level fraction first: the whole coupled step's algorithmic
        # bytes over its time; roofline.frac is the dominant kernel's own
        "effective_hbm_fraction": eff,
        "roofline": roof,
        "fused_kernel": info32["fused_kernel_name"], "tma_fallback": info32["tma_fallback"],
        "clocks": clocks,
        "gpu_launches": int(round(lps * K)) if lps else None,
        "e2e": e2e,
        "fp64": {"value": whole_job_rate(w.ncells, world, K, ms64), "ms_per_step": ms64 / K, "roofline": roof64,
                 "iters_min": stats64["iters_min"], "iters_max": stats64["iters_max"]},
        "plain_fp64": {"value": whole_job_rate(w.ncells, world, K, msp), "ms_per_step": msp / K},
        "fp16_storage": {"value": whole_job_rate(w.ncells, world, K, ms16), "ms_per_step": ms16 / K,
                         "roofline": roof16, "iters_min": stats16["iters_min"], "iters_max": stats16["iters_max"],
                         "vs_fp64_rel_l2_after_steps": acc16},
        "fp32_vs_fp64_rel_l2_after_steps": acc,
        "iters": {"min": stats32["iters_min"], "max": stats32["iters_max"]},
        "stress_512": stress,
        "stress_512_fp16": stress16,
        "bias_sweep_256": sweep,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0 and args.oracle_512:
        line["oracle_stress_512"] = oracle_stress_timing()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stress", action="store_true", help="skip the 512^3 sub-record")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 256-instance sweep sub-record")
    ap.add_argument("--oracle-512", action="store_true",
                    help="also time the FP64 oracle on the 512^3 configuration (about 44 GB of host memory)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
