#!/usr/bin/env python
"""Throughput of the MP-PIC parcel-grid coupling step on GB300.

A "step" is one pass of the whole hot path over the bed: deposit of the solids volume,
node fields, interpolation, Wen-Yu drag, stress gradient, drag-sum deposit, push with wall
reflection, re-binning, objectives, and the sort by cell every --sort-every steps (default
every 2 steps, the fastest schedule over the run). The default workload is the dense bed: 128x128x512 cells of 1 cm, 32M parcels
filling the bottom quarter at solids fraction 0.5 (lognormal d, median 100 um, sigma 0.4),
inflow 0.8 m/s, FP32 state with exact fixed-point deposits, run for 500 steps.

The bed fluidises over the run and a step gets slower as it does, so the timed window is
centred in the run: with the default 500 timed steps it is the whole run (after the
warm-up); a shorter --steps is preceded by untimed settling steps. config.timed_steps
states the window.

Prints one JSON line. `value` is whole-job parcel-updates/s with inputs resident in HBM
(CUDA events on the library's stream around exactly --steps steps). `e2e` is the same
metric through the C ABI with a parcel state copied in from pinned host memory and the new
state copied back out every step (pipelined over three device buffer sets: one step's
kernels overlap the next uploads and the previous downloads). `roofline` is the fused step kernel's algorithmic bytes per launch
over its event-timed duration against the measured HBM copy bandwidth. `cpu_baseline` is
the FP64 CPU oracle on a bounded sample of the same bed. `alt_schedule` times the same bed
over the same window sorted every 1 and every 10 steps (the schedules this workload
compares, each on a fresh handle); `fp64_form` the FP64 form;
`adjoint` the forward (with checkpoints) and reverse sweeps on the 500k-parcel
differentiation bed.

--impl reference times the oracle itself (the slow program this build is checked
against) on a bounded sample per step, with the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "parcel-updates/s and % HBM roofline, FP32 vs FP64 form on one GB300, at stated err"
UNIT = "parcel-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's whole run)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--run-steps", type=int, default=None,
                    help="length of the workload's run (default: its own); the timed window is "
                         "centred in it")
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--workload", choices=("dense", "fourier", "settle", "grad", "batched",
                                           "paper_sec3", "paper_sec4"),
                    default="dense")
    ap.add_argument("--nbeds", type=int, default=256, help="beds of the batched workload")
    ap.add_argument("--np", type=int, default=None, help="override the parcel count")
    ap.add_argument("--grid", type=str, default=None, help="override the grid, e.g. 64,64,256")
    ap.add_argument("--sort-every", type=int, default=2)
    ap.add_argument("--alt-sort-every", type=str, default="1,10",
                    help="other sort schedules, each timed over the same window on a fresh "
                         "handle (comma list; 0 = none)")
    ap.add_argument("--precision", type=int, choices=(32, 64), default=32)
    ap.add_argument("--fp64-steps", type=int, default=5, help="steps of the FP64-form comparison (0 = skip)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--forms-steps", type=int, default=50,
                    help="timed steps of each other closure / implicit coupling (0 = skip)")
    ap.add_argument("--paper-steps", type=int, default=50,
                    help="timed steps on each of the paper's two bed shapes (0 = skip)")
    ap.add_argument("--batched-steps", type=int, default=200,
                    help="steps of the 256-bed batched leg in the default line (0 = skip)")
    ap.add_argument("--adjoint-steps", type=int, default=200,
                    help="steps of the reverse-mode timing on the differentiation bed (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="timed seconds of each CPU-oracle leg (single thread, all cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="budget of the reference arm's timed oracle steps")
    args = ap.parse_args()
    if args.run_steps is None:
        args.run_steps = RUN_STEPS[args.workload]
    if args.steps is None:
        args.steps = args.run_steps
    return args


# length of each workload's run (the configurations' step counts)
RUN_STEPS = {"dense": 500, "fourier": 1000, "settle": 100, "grad": 200, "batched": 200,
             "paper_sec3": 500, "paper_sec4": 500}


def make_workload(name, np_override=None, seed_offset=0, grid=None):
    from paper_2211_15605_gb300 import synth
    kw = {}
    if np_override:
        kw["n"] = np_override
    if grid:
        kw["nx"], kw["ny"], kw["nz"] = (int(t) for t in grid.split(","))
    if name == "dense":
        bed = synth.dense_bed(seed=synth.SEED_BASE + 3 + 1000 * seed_offset, **kw)
    elif name == "fourier":
        bed = synth.fourier_bed(seed=synth.SEED_BASE + 2 + 1000 * seed_offset, **kw)
    elif name == "settle":
        bed = synth.settle_bed(seed=synth.SEED_BASE + 1 + 1000 * seed_offset, **kw)
    elif name == "paper_sec3":
        bed = synth.paper_verification_bed(seed=synth.SEED_BASE + 6 + 1000 * seed_offset)
    elif name == "paper_sec4":
        bed = synth.paper_scaling_bed(seed=synth.SEED_BASE + 7 + 1000 * seed_offset)
    else:
        bed = synth.grad_bed(seed=synth.SEED_BASE + 5 + 1000 * seed_offset, **kw)
    return bed


def settle_steps(args):
    """Untimed steps before the warm-up that centre the timed window in the run."""
    return max(0, (args.run_steps - args.steps) // 2 - args.warmup)


def settle_steps_for(args, steps):
    """Untimed steps (warm-up included) before a window of `steps` centred in the run."""
    return max(args.warmup, (args.run_steps - steps) // 2)


def workload_config(bed, args):
    p = bed.params
    t0 = settle_steps(args) + args.warmup
    return {"workload": bed.meta["workload"], "parcels": bed.np,
            "grid": [p["nx"], p["ny"], p["nz"]], "cell_m": p["dx"], "sort_every": args.sort_every,
            "run_steps": args.run_steps, "timed_steps": [t0, t0 + args.steps],
            "state": "fp32" if args.precision == 32 else "fp64",
            "deposit": "exact fixed point (int64)" if args.precision == 32 else "exact fixed point (int128)",
            "l2": "inputs larger than L2 (parcel state %.2f GB)" % (bed.np * (36 if args.precision == 32 else 68) / 1e9)}


# ------------------------------------------------------------------ clocks --

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------- GPU arm --

# FP64 operations per parcel of the FP64 step kernel (k_cells<double,1>): DADD + DMUL + 2 DFMA
# thread instructions per parcel from the instruction counters of one ncu capture on the
# 8M-parcel dense case: the work of the FP64 pipe, divisions and powers included.
FP64_FLOPS_PER_PARCEL = 602
FP64_FLOPS_SOURCE = "ncu counters: (DADD + DMUL + 2 DFMA) / parcels of one launch, 8M-parcel dense bed"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the FP32 step kernel per
# parcel, from ncu captures on the 128x128x128 / 8M-parcel dense bed sorted every 2 steps,
# in proportion to the parcels. Reported only while the kernel source is the one captured.
STEP_TRAFFIC = {"workload": "dense", "precision": 32,
                # DRAM bytes per parcel of one launch of each step-kernel instance, ncu on the
                # 8M-parcel dense bed at step 150: a step that updates the values in place, and
                # a step after a sort that reads them through the sort's permutation
                "in_place_bytes_per_parcel": 61.9, "perm_bytes_per_parcel": 70.8,
                "source_sha256": "6a46ab409e1b245d058fe8ad935e3c46650bde69f439a3f8ffdd2ac5cb2579a5"}


def step_traffic(args, np_, start):
    """Measured DRAM bytes per step launch over the timed window, from the per-instance
    captures, or None if the kernel source has changed since the captures."""
    import hashlib
    src = os.path.join(ROOT, "paper_2211_15605_gb300", "csrc", "mppic_device.cuh")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    t = STEP_TRAFFIC
    if args.workload != t["workload"] or args.precision != t["precision"] or sha != t["source_sha256"]:
        return None
    due = lambda k: args.sort_every > 0 and k % args.sort_every == 0
    per = [t["perm_bytes_per_parcel"] if due(start + it) else t["in_place_bytes_per_parcel"]
           for it in range(args.steps)]
    return int(round(sum(per) / len(per) * np_))


def state_bytes_per_parcel(precision, sort_every, start, nsteps, perm_sorts=True):
    """Parcel-state bytes per parcel of the step launches of one mppic_step call of nsteps
    steps starting at step `start`, averaged over the launches, as the library schedules
    them (the call follows an earlier call on the same handle): a step updates the values
    where they are (8 values read, x,y,z,u,v,w written: 14 values); the step after a sort
    reads the values through the sort's permutation (a 4-byte index) and writes all 8 to the
    other buffer (16 values + 4 B), unless perm_sorts is off (a pid or checkpoint travels
    with the parcels: the sort moved the values, the step reads the copy, 16 values)."""
    t = 4 if precision == 32 else 8
    due = lambda k: sort_every > 0 and k % sort_every == 0
    per = []
    for it in range(nsteps):
        if due(start + it):
            per.append(16 * t + 4 if perm_sorts else 16 * t)
        else:
            per.append(14 * t)
    return sum(per) / max(len(per), 1)


def bytes_per_launch(np_, active_bricks, precision, per_parcel=None):
    """Algorithmic DRAM bytes of one fused step launch: every parcel's state read once and
    written once (per_parcel bytes; default the in-place step: x,y,z,u,v,w,d,w read, 8
    values, and x,y,z,u,v,w written, 6 values), plus per occupied brick its node-field tile
    read once (5 fields x 405 nodes) and its five accumulator planes written once (405
    nodes)."""
    t = 4 if precision == 32 else 8
    words = 1 if precision == 32 else 2
    if per_parcel is None:
        per_parcel = 14 * t
    per_brick = 405 * (5 * t + 5 * 8 * words)
    return np_ * per_parcel + active_bricks * per_brick


def fp64_peak(stream, dev):
    """Measured FP64 fused multiply-add rate of this GPU in TFLOP/s: the probe library's
    independent DFMA chains (8 per thread, 8 blocks of 256 threads per SM), best of three
    launches timed with CUDA events on the given stream after one warm-up launch."""
    import ctypes
    import torch
    from paper_2211_15605_gb300 import build
    L = ctypes.CDLL(build.PROBE_LIB)
    L.mppic_probe_dfma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_double)]
    L.mppic_probe_dfma.restype = ctypes.c_int
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    best = 0.0
    for rep in range(4):
        flops = ctypes.c_double()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = L.mppic_probe_dfma(20000, 8, ctypes.c_void_p(stream.cuda_stream),
                                ctypes.c_void_p(out.data_ptr()), ctypes.byref(flops))
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            return None
        if rep > 0:
            best = max(best, flops.value / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def time_bed(bed, precision, sort_every, steps, pre, stream, dev, barrier, params=None):
    """One bed on a fresh handle: `pre` untimed steps, then `steps` steps in one mppic_step call
    timed with CUDA events on the library's stream, with the library's per-phase events.
    Returns the throughput, the per-phase split and the step kernel's HBM roofline fraction."""
    import torch
    from paper_2211_15605_gb300 import mppic
    prm = bed.params if params is None else params
    b = mppic.Bed(prm, precision=precision, sort_every=sort_every, stream=stream)
    p = mppic.parcels_to_device(bed.parcels, precision, device=dev)
    g = mppic.gas_to_device(bed.U, None, precision, device=dev)
    obj = torch.zeros((max(pre, steps, 1), 2), dtype=torch.float64, device=dev)
    if pre:
        b.step(p, g, pre, obj[:pre])
    b.check()
    barrier()
    b.profile(True)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    b.step(p, g, steps, obj[:steps])
    h1.record(stream)
    barrier()
    pr = b.profile_read()
    b.profile(False)
    b.check()
    ms = h0.elapsed_time(h1)
    peak, _ = measured_peak()
    n_step = max(pr["launches"]["step"], 1)
    step_ms = pr["ms"]["step"] / n_step
    bpl = bytes_per_launch(bed.np, pr["active_bricks"], precision,
                           state_bytes_per_parcel(precision, sort_every, pre, steps))
    out = {"value": bed.np * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
           "steps": steps, "timed_steps": [pre, pre + steps], "sort_every": sort_every,
           "phase_ms_per_step": {k: round(v / steps, 4) for k, v in pr["ms"].items() if v > 0},
           "step_kernel_ms": round(step_ms, 5),
           "step_kernel_roofline_frac": round(bpl / (step_ms / 1e3) / 1e9 / peak, 4),
           "gpu_launches": pr["total_launches"]}
    b.close()
    del p
    torch.cuda.empty_cache()
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2211_15605_gb300 import mppic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    bed = make_workload(args.workload, args.np, seed_offset=rank, grid=args.grid)
    # a stream of its own: the legacy default stream would order the end-to-end leg's copies
    # behind the library's kernels
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    b = mppic.Bed(bed.params, precision=args.precision, sort_every=args.sort_every, stream=stream)
    parcels = mppic.parcels_to_device(bed.parcels, args.precision, device=dev)
    gas = mppic.gas_to_device(bed.U, None, args.precision, device=dev)
    pre = settle_steps(args) + args.warmup
    obj = torch.zeros((max(pre, args.steps, 2), 2), dtype=torch.float64, device=dev)

    # settling and warm-up steps, then exactly --steps timed steps in one call
    if pre:
        b.step(parcels, gas, pre, obj[:pre])
    b.check()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    b.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(parcels, gas, args.steps, obj[: args.steps])
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = b.profile_read()
    b.profile(False)
    b.check()
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * bed.np * args.steps / (ms_max / 1e3)

    # roofline of the dominant kernel (the fused step kernel)
    peak, peak_kind = measured_peak()
    n_step = max(prof["launches"]["step"], 1)
    step_ms = prof["ms"]["step"] / n_step
    bpl = bytes_per_launch(bed.np, prof["active_bricks"], args.precision,
                           state_bytes_per_parcel(args.precision, args.sort_every, pre, args.steps))
    achieved = bpl / (step_ms / 1e3) / 1e9
    shares = {k: round(v / max(sum(prof["ms"].values()), 1e-9), 4) for k, v in prof["ms"].items()}
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": step_traffic(args, bed.np, pre),
                "kernel": "k_cells<float,1> (fused interp/drag/push/deposit)" if args.precision == 32
                else "k_cells<double,1>", "peak_kind": peak_kind + " (hbm_gbs copy burst)",
                "bytes_per_launch": bpl, "ms_per_launch": round(step_ms, 5), "phase_ms": prof["ms"],
                "phase_share": shares}

    # the same bed and window under the other sort schedules, each on a fresh handle
    alt = []
    for se in (int(t) for t in args.alt_sort_every.split(",") if t.strip()):
        if se <= 0 or se == args.sort_every:
            continue
        r = time_bed(bed, args.precision, se, args.steps, pre, stream, dev, barrier)
        alt.append({"sort_every": se, "value": world * r["value"], "unit": UNIT,
                    "ms_per_step": r["ms_per_step"], "phase_ms_per_step": r["phase_ms_per_step"],
                    "step_kernel_roofline_frac": r["step_kernel_roofline_frac"]})

    # end to end through the C ABI with host buffers: every step copies a parcel state in from
    # pinned host memory (all 8 arrays) and its new state and objectives back out (6 arrays +
    # 2 doubles). The host state is the device state sorted into the handle's layout (a host
    # code that mirrors the device state sends it back in that order); sorting it again gives
    # the same order, so every step, with or without a sort, finds the parcels in the ranges
    # the handle holds, and the leg runs the headline's sort schedule. Steps are pipelined
    # over three device buffer sets: the uploads of the next steps and the downloads of the
    # previous ones run on the copy engines (both directions at once) while step k's kernels
    # run. Every copy and every step is bracketed by events on its own stream, so the time of
    # each leg and their overlap are measured.
    e2e = None
    if args.e2e_steps > 0:
        fields = mppic.PARCEL_FIELDS
        outs = ("x", "y", "z", "u", "v", "w")
        b.bin(parcels, do_sort=True)                # the state in the handle's layout
        b.tune(0, args.sort_every)
        torch.cuda.synchronize()
        host = {k: parcels[k].cpu().pin_memory() for k in fields}
        NB = 3
        bufs = [parcels] + [{k: torch.empty_like(v) for k, v in parcels.items()} for _ in range(NB - 1)]
        out_host = [{k: torch.empty_like(host[k]).pin_memory() for k in outs} for _ in range(NB)]
        obj_host = [torch.empty((1, 2), dtype=torch.float64).pin_memory() for _ in range(NB)]
        obj2 = [torch.zeros((1, 2), dtype=torch.float64, device=dev) for _ in range(NB)]
        up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        up_done, step_done, down_done = ([torch.cuda.Event() for _ in range(NB)] for _ in range(3))
        ev = lambda: torch.cuda.Event(enable_timing=True)
        legs = {"h2d": [], "step": [], "d2h": []}
        barrier()
        f0, f1 = ev(), ev()
        f0.record(stream)
        up.wait_stream(stream)
        down.wait_stream(stream)
        for k in range(args.e2e_steps):
            s_ = k % NB
            X = bufs[s_]
            if k >= NB:
                up.wait_event(down_done[s_])          # the buffer's previous state is out
            with torch.cuda.stream(up):
                a0, a1 = ev(), ev()
                a0.record(up)
                for f in fields:
                    X[f].copy_(host[f], non_blocking=True)
                a1.record(up)
                up_done[s_].record(up)
                legs["h2d"].append((a0, a1))
            stream.wait_event(up_done[s_])
            c0, c1 = ev(), ev()
            c0.record(stream)
            b.step(X, gas, 1, obj2[s_])
            c1.record(stream)
            legs["step"].append((c0, c1))
            step_done[s_].record(stream)
            down.wait_event(step_done[s_])
            with torch.cuda.stream(down):
                g0, g1 = ev(), ev()
                g0.record(down)
                for f in outs:
                    out_host[s_][f].copy_(X[f], non_blocking=True)
                obj_host[s_].copy_(obj2[s_], non_blocking=True)
                g1.record(down)
                down_done[s_].record(down)
                legs["d2h"].append((g0, g1))
        stream.wait_stream(up)
        stream.wait_stream(down)
        f1.record(stream)
        barrier()
        ems = f0.elapsed_time(f1)
        t2 = torch.tensor([ems], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t2, op=dist.ReduceOp.MAX)
        tsz = 4 if args.precision == 32 else 8
        leg_ms = {k: sum(a.elapsed_time(c) for a, c in v) / args.e2e_steps for k, v in legs.items()}
        wall = float(t2.item()) / args.e2e_steps
        e2e = {"value": world * bed.np * args.e2e_steps / (float(t2.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": bed.np * 8 * tsz, "d2h_bytes_per_step": bed.np * 6 * tsz + 16,
               "steps": args.e2e_steps, "sort_every": args.sort_every, "ms_per_step": wall,
               "leg_ms_per_step": {k: round(v, 4) for k, v in leg_ms.items()},
               "overlap": round(sum(leg_ms.values()) / wall, 3),
               "h2d_gbs": round(bed.np * 8 * tsz / (leg_ms["h2d"] / 1e3) / 1e9, 1),
               "d2h_gbs": round((bed.np * 6 * tsz + 16) / (leg_ms["d2h"] / 1e3) / 1e9, 1),
               "pipelined": "3 device buffer sets; uploads, kernels and downloads on three streams"}
        b.check()
        del bufs

    # FP64 form on the same bed, for the FP32-vs-FP64 comparison
    fp64 = None
    if args.fp64_steps > 0 and args.precision == 32 and world == 1:
        del parcels
        torch.cuda.empty_cache()
        b64 = mppic.Bed(bed.params, precision=64, sort_every=args.sort_every, stream=stream)
        p64 = mppic.parcels_to_device(bed.parcels, 64, device=dev)
        g64 = mppic.gas_to_device(bed.U, None, 64, device=dev)
        b64.step(p64, g64, 1)
        b64.check()
        barrier()
        b64.profile(True)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        b64.step(p64, g64, args.fp64_steps)
        g1.record(stream)
        barrier()
        pr64 = b64.profile_read()
        b64.check()
        fms = g0.elapsed_time(g1)
        k_ms = pr64["ms"]["step"] / max(pr64["launches"]["step"], 1)
        fp64 = {"value": bed.np * args.fp64_steps / (fms / 1e3), "unit": UNIT,
                "ms_per_step": fms / args.fp64_steps, "steps": args.fp64_steps,
                "step_kernel_ms": k_ms, "bound": "fp64 alu (GB300 FP64 rate)"}
        b64.close()
        del p64
        torch.cuda.empty_cache()
        peak64 = fp64_peak(stream, dev)
        if peak64:
            flops = FP64_FLOPS_PER_PARCEL * bed.np
            fp64["roofline"] = {"bound": "fp64", "achieved": round(flops / (k_ms / 1e3) / 1e12, 4),
                                "peak": round(peak64, 4), "unit": "TFLOP/s",
                                "frac": round(flops / (k_ms / 1e3) / 1e12 / peak64, 4),
                                "peak_kind": "measured here (DFMA-chain probe, best of 3)",
                                "flops_per_parcel": FP64_FLOPS_PER_PARCEL,
                                "flops_source": FP64_FLOPS_SOURCE}

    # the paper's other closures and implicit coupling on the same bed and window, each on a
    # fresh handle (the FP32 form): Syamlal-O'Brien, the Gidaspow blend, and implicit coupling
    # with 3 gas iterations per step (Wen-Yu)
    forms = None
    if args.forms_steps > 0 and world == 1:
        forms = {}
        fpre = settle_steps_for(args, args.forms_steps)
        for name, over in (("syamlal_obrien", dict(drag_model=1)),
                           ("gidaspow_blend", dict(drag_model=3)),
                           ("implicit_3_iterations", dict(coupling_iters=3))):
            r = time_bed(bed, args.precision, args.sort_every, args.forms_steps, fpre, stream, dev,
                         barrier, params=dict(bed.params, **over))
            forms[name] = {k: r[k] for k in ("value", "unit", "ms_per_step", "timed_steps",
                                             "phase_ms_per_step", "step_kernel_roofline_frac")}

    # the paper's own bed shapes (Sec. 3 verification bed, 3.0M parcels; Sec. 4.1 scaling bed,
    # 47.9M parcels) as throughput cases, FP32 form, after 50 settling steps
    paper = None
    if args.paper_steps > 0 and world == 1:
        from paper_2211_15605_gb300 import synth
        paper = {}
        for maker in (synth.paper_verification_bed, synth.paper_scaling_bed):
            pb = maker()
            r = time_bed(pb, args.precision, args.sort_every, args.paper_steps, 50, stream, dev,
                         barrier)
            paper[pb.meta["workload"]] = dict(
                parcels=pb.np, grid=[pb.params["nx"], pb.params["ny"], pb.params["nz"]],
                cell_m=pb.params["dx"], **{k: r[k] for k in ("value", "unit", "ms_per_step",
                                                             "timed_steps", "phase_ms_per_step",
                                                             "step_kernel_roofline_frac")})
            del pb

    # 256 uneven beds in one handle (autotuned, graph-captured), the batched configuration
    batched = None
    if args.batched_steps > 0 and world == 1:
        batched = batched_leg(args, args.batched_steps, with_cpu=False)

    # reverse mode on the differentiation bed (500k parcels, 32x32x128 cells): the forward
    # steps with checkpoints every 20, then the gradient of a weighted sum of the two
    # time-averaged objectives with respect to (C, s_d, u_in)
    adj = None
    if args.adjoint_steps > 0 and world == 1:
        from paper_2211_15605_gb300 import synth
        gb = synth.grad_bed()
        adj = {"workload": "grad_32x32x128", "parcels": gb.np, "steps": args.adjoint_steps,
               "checkpoint_every": 20}
        for prec in (64, 32):
            ba = mppic.Bed(gb.params, precision=prec, sort_every=10, stream=stream)
            ba.checkpoint(20)
            pa = mppic.parcels_to_device(gb.parcels, prec, device=dev)
            ba.step(pa, None, 20)                # first use of the handle's scratch
            ba.backward(1.0, 0.5)
            pa = mppic.parcels_to_device(gb.parcels, prec, device=dev)
            barrier()
            a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a0.record(stream)
            ba.step(pa, None, args.adjoint_steps)
            a1.record(stream)
            ba.backward(1.0, 0.5)                # synchronous
            a2.record(stream)
            barrier()
            ba.check()
            fw, bw = a0.elapsed_time(a1), a1.elapsed_time(a2)
            adj[f"fp{prec}"] = {"forward_ms": round(fw, 3), "backward_ms": round(bw, 3),
                                "backward_over_forward": round(bw / fw, 2)}
            ba.close()
            del pa

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(bed, seconds=args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
                "config": workload_config(bed, args), "roofline": roofline, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": prof["total_launches"], "clocks": clk,
                "fp64_form": fp64, "alt_schedule": alt, "adjoint": adj, "forms": forms,
                "paper_beds": paper, "batched": batched,
                "parallelism": "replicas" if world > 1 else "single"}
        print(json.dumps(line))
    b.close()
    if world > 1:
        dist.destroy_process_group()


def batched_leg(args, steps, with_cpu=True):
    """256 uneven independent beds in one handle: autotuned launch settings, then the timed
    steps replayed as captured CUDA graphs (one host call per sort period). Returns the leg's
    measurements (value, timing, roofline, e2e, CPU baseline)."""
    import torch

    from paper_2211_15605_gb300 import mppic, synth, tune

    beds = synth.batched_beds(nbeds=args.nbeds)
    total = sum(b.np for b in beds)
    stream = torch.cuda.current_stream()
    batch = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=args.precision,
                        sort_every=args.sort_every, stream=stream)
    parcels, gas = mppic.concat_beds(beds, args.precision)
    tuned = tune.autotune(batch, parcels, gas, steps=10, grids=(0, 2, 3), sorts=(1, 2, 5, 10, 20))
    period = tuned["best"][1]
    rounds = max(1, steps // period)
    steps = rounds * period
    obj = torch.empty((period, len(beds), 2), dtype=torch.float64, device="cuda")
    for _ in range(max(1, args.warmup // period)):
        batch.step_graph(parcels, gas, period, obj)
    batch.check()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(rounds):
        batch.step_graph(parcels, gas, period, obj)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    batch.check()
    ms = e0.elapsed_time(e1)
    value = total * steps / (ms / 1e3)
    # eager, event-profiled pass for the kernel roofline and the launch count of a step
    batch.profile(True)
    batch.step(parcels, gas, period)
    prof = batch.profile_read()
    batch.profile(False)
    batch.check()
    peak, peak_kind = measured_peak()
    n_step = max(prof["launches"]["step"], 1)
    step_ms = prof["ms"]["step"] / n_step
    bpl = bytes_per_launch(total, prof["active_bricks"], args.precision,
                           state_bytes_per_parcel(args.precision, period, 0, period))
    achieved = bpl / (step_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "k_cells<%s,1> (persistent, all beds)" % ("float" if args.precision == 32 else "double"),
                "peak_kind": peak_kind + " (hbm_gbs copy burst)", "bytes_per_launch": bpl,
                "ms_per_launch": round(step_ms, 5), "phase_ms": prof["ms"]}
    # end to end with host buffers: H2D of the parcel state, one graph replay, D2H
    fields = mppic.PARCEL_FIELDS
    host = {k: parcels[k].cpu().pin_memory() for k in fields}
    out_host = {k: torch.empty_like(host[k]).pin_memory() for k in ("x", "y", "z", "u", "v", "w")}
    obj_host = torch.empty_like(obj, device="cpu").pin_memory()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for k in fields:
        parcels[k].copy_(host[k], non_blocking=True)
    batch.step_graph(parcels, gas, period, obj)
    for k in out_host:
        out_host[k].copy_(parcels[k], non_blocking=True)
    obj_host.copy_(obj, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    tsz = 4 if args.precision == 32 else 8
    e2e = {"value": total * period / (f0.elapsed_time(f1) / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": total * 8 * tsz // period, "d2h_bytes_per_step": (total * 6 * tsz + obj.numel() * 8) // period,
           "steps": period}
    cpu = None
    if with_cpu and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        info = host_cpu()
        try:
            threads = oracle.max_threads()
        except Exception:
            threads = 1
        run = _oracle_stepper(threads)
        t0 = time.perf_counter()
        n_done, nb = 0, 0
        for b in beds:                              # whole beds, until the time budget is spent
            if time.perf_counter() - t0 >= args.cpu_seconds:
                break
            st = b.parcels
            for _ in range(2):
                st, _ = run(b, st)
            n_done += b.np
            nb += 1
        dt = time.perf_counter() - t0
        cpu = {"value": n_done * 2 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"the first {nb} of {len(beds)} beds ({n_done} of {total} parcels), 2 steps each",
               "seconds": dt, **info}
    out = {"value": value, "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
           "workload": f"batched_{len(beds)}_beds", "parcels": total, "beds": len(beds),
           "grids": "8..32 x 8..32 x 16..64", "sort_every": period,
           "tuned": {"grid_per_sm": tuned["best"][0], "sort_every": tuned["best"][1],
                     "ms_per_step": {f"{g},{s_}": round(v, 4) for (g, s_), v in tuned["ms_per_step"].items()}},
           "launch": "captured CUDA graph per sort period, persistent kernels",
           "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
           "gpu_launches": prof["total_launches"]}
    batch.close()
    del parcels
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    """The batched workload as the headline line."""
    import torch
    torch.cuda.set_device(0)
    r = batched_leg(args, args.steps)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["steps"],
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == 32 else "f64",
            "data": "synthetic",
            "config": {"workload": r["workload"], "parcels": r["parcels"], "beds": r["beds"],
                       "grids": r["grids"], "sort_every": r["sort_every"], "tuned": r["tuned"],
                       "launch": r["launch"],
                       "l2": "inputs larger than L2 (parcel state %.2f GB)" % (r["parcels"] * 36 / 1e9)},
            "roofline": r["roofline"], "cpu_baseline": r["cpu_baseline"], "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "parallelism": "single"}
    print(json.dumps(line))


# --------------------------------------------------------------- CPU side --

def _sample(bed, m):
    import numpy as np
    m = min(m, bed.np)
    return {k: np.ascontiguousarray(v[:m]) for k, v in bed.parcels.items()}, m


def host_cpu():
    """The host's CPU model and core count (what the CPU legs ran on): lscpu's model name, else
    /proc/cpuinfo's (x86 "model name"; Arm implementer and part numbers)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        fields = {}
        try:
            for line in open("/proc/cpuinfo"):
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
        except OSError:
            pass
        model = fields.get("model name")
        if not model and "cpu part" in fields:
            model = f"implementer {fields.get('cpu implementer', '?')} part {fields['cpu part']}"
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count()}


def _oracle_stepper(threads):
    """One oracle step of a column (single thread: the oracle as it stands; threads > 1: its
    OpenMP driver over the same functions)."""
    import oracle

    def run(col, state):
        if threads == 1:
            out, _, st = oracle.step(col.params, state, 1, U=col.U, outputs=False)
        else:
            out, _, st = oracle.step_mt(col.params, state, 1, U=col.U, nthreads=threads)
        return out, st
    return run


def column_for_budget(bed, seconds_per_step, stepper):
    """The side s of the s x s x nz column of cells at the bed's origin corner whose oracle
    step takes about seconds_per_step: a two-point cost calibration, then one timed step of
    the chosen column that shrinks it while it overshoots by more than 1.5x."""
    p = bed.params
    costs = []
    for side in (4, 8):
        col = sub_column(bed, side)
        t0 = time.perf_counter()
        stepper(col, col.parcels)
        costs.append((col.params["nx"] * col.params["ny"] * p["nz"], time.perf_counter() - t0))
    (ca, ta), (cb, tb) = costs
    per_cell = max((tb - ta) / max(cb - ca, 1), 1e-12)      # cells and parcels grow together
    side = 4
    for s_try in range(4, max(p["nx"], p["ny"]) + 1):
        if per_cell * s_try * s_try * p["nz"] > seconds_per_step:
            break
        side = s_try
    for _ in range(3):
        col = sub_column(bed, side)
        t0 = time.perf_counter()
        stepper(col, col.parcels)
        dt = time.perf_counter() - t0
        if dt <= 1.5 * seconds_per_step or side <= 4:
            break
        side = max(4, int(side * math.sqrt(seconds_per_step / dt)))
    return sub_column(bed, side)


def time_column(col, steps, warmup, stepper):
    state = col.parcels
    for _ in range(warmup):
        state, _ = stepper(col, state)
    t0 = time.perf_counter()
    st = 0
    for _ in range(steps):
        state, st = stepper(col, state)
    return col.np * steps / (time.perf_counter() - t0), time.perf_counter() - t0, st


def cpu_baseline(bed, seconds=10.0, steps=3):
    """The FP64 oracle on the machine's host cores, single-threaded (the oracle as it stands) and
    on every core (its OpenMP driver, fixed per-thread parcel ranges reduced in thread order),
    each on a full-height column of the bed sized for about `seconds` of timed steps, so that
    per-parcel cost is not dominated by grid work: parcel-updates/s of the column."""
    import oracle
    oracle.build()
    info = host_cpu()
    legs = {}
    for name, threads in (("single_thread", 1), ("all_cores", 0)):
        try:
            if threads == 0:
                threads = oracle.max_threads()
            run = _oracle_stepper(threads)
            col = column_for_budget(bed, seconds / steps, run)
            value, dt, st = time_column(col, steps, 1, run)
        except Exception as e:                       # the OpenMP driver may not build
            legs[name] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
            continue
        legs[name] = {"value": value, "cores": threads, "seconds": round(dt, 2),
                      "sample": f"the {col.params['nx']}x{col.params['ny']}x{bed.params['nz']}-cell "
                                f"column at the origin corner with its {col.np} of {bed.np} parcels, "
                                f"{steps} steps after 1 warm-up, status {st}"}
    best = legs.get("all_cores") if "value" in legs.get("all_cores", {}) else legs["single_thread"]
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle",
            "sample": best["sample"], **info, "legs": legs}


def sub_column(bed, side):
    """The bed's side x side x nz column of cells at the origin corner, with the parcels in it
    (and the gas fields on its nodes): a bounded sample of the same workload."""
    import numpy as np
    from paper_2211_15605_gb300 import synth
    p = bed.params
    side = max(1, side)
    q = dict(p, nx=min(side, p["nx"]), ny=min(side, p["ny"]))
    keep = (bed.parcels["x"] < q["nx"] * p["dx"]) & (bed.parcels["y"] < q["ny"] * p["dy"])
    parcels = {k: np.ascontiguousarray(v[keep]) for k, v in bed.parcels.items()}
    U = []
    for u in bed.U:
        if u is None:
            U.append(None)
            continue
        g = np.asarray(u).reshape(p["nz"] + 1, p["ny"] + 1, p["nx"] + 1)
        U.append(np.ascontiguousarray(g[:, : q["ny"] + 1, : q["nx"] + 1]).ravel())
    return synth.Bed(q, parcels, U=tuple(U), nsteps=bed.nsteps, meta=dict(bed.meta))


def run_reference(args):
    """Time the FP64 CPU oracle on a bounded sample per step (rank 0 only) on every host core
    (the oracle's OpenMP driver; the single-threaded oracle where that driver does not build):
    a column of the bed (full height) sized from a cost calibration so that the warm-up and
    timed steps fit the budget."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    bed = make_workload(args.workload, args.np, grid=args.grid)
    p = bed.params
    try:
        threads = oracle.max_threads()
    except Exception:
        threads = 1
    run = _oracle_stepper(threads)
    budget = args.ref_seconds / max(args.steps + args.warmup, 1)
    col = column_for_budget(bed, budget, run)
    value, dt, st = time_column(col, args.steps, args.warmup, run)
    dens = bed.np / (p["nx"] * p["ny"] * p["nz"])          # parcels per cell, whole bed
    cfg = workload_config(bed, args)
    info = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"the {col.params['nx']}x{col.params['ny']}x{p['nz']}-cell "
                                       f"column at the origin corner with its {col.np} of {bed.np} "
                                       f"parcels (bed mean {dens:.2f} per cell), sized for "
                                       f"{args.ref_seconds:.0f} s of timed oracle steps, status {st}",
                             **info},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
