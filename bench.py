"""Benchmark: cells/s of one pressure projection at 1024x1024x512 on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--size NXxNYxNZ]

A step is one full projection (divergence, forward transforms, tridiagonal sweeps,
singular mode, inverse transforms, one refinement sweep, velocity correction) of a
1024x1024x512 staggered grid (periodic x,y of length 2 pi, walls at z = 0, 2 with
tanh stretching beta = 2.5), inputs resident in HBM.  The headline is the mixed
path (fp32 transforms and sweeps, float-float residual / correction, one
refinement sweep); the plain fp64 path is timed on the same inputs beside it.
Each field is 4.3 GB, far larger than the 129 MB L2, so no flush is needed
between steps.  One JSON line is printed by rank 0.

--impl reference times the FP64 CPU oracle (the method's plain definition, naive
DFT + Thomas, OpenMP on all host cores) on a bounded sample of the same workload
(the same 1024x1024 planes, fewer z levels) and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cells/s per pressure projection, 1024x1024x512, FP32+refine vs FP64, %HBM peak"
LX = LY = 2 * math.pi
LZ = 2.0
BETA = 2.5
DT = 1e-3
SEED = 4
# Algorithmic HBM bytes per cell of each kernel (fp64 user fields, fp32 spectrum of
# ~4 B per cell, float-float right-hand side): x_forward_div reads u*, v*, w* (24) and
# writes b (8) and the spectrum (4); a y/z pass reads and writes the spectrum and reads
# the fp32 pivot table (4 + 4 + 2); the inverse x-FFT reads the spectrum and writes phi_0
# (4 + 4); the first sweep's residual reads phi_0 and b (4 + 8) and writes the spectrum,
# its accumulation reads the spectrum and writes the low word of phi (4 + 4); a later
# sweep's residual reads the float-float phi and b (8 + 8) and writes the spectrum, its
# accumulation reads the spectrum and phi and writes phi (4 + 8 + 8); the correction reads
# u*, v*, w*, phi (24 + 8) and writes u, v, w, phi (24 + 8).
BYTES_MIXED = {"x_forward_div": 36.0, "yz_forward": 10.0, "yz_backward": 10.0, "x_inverse_store": 8.0,
               "x_forward_residual": 16.0, "x_inverse_accumulate": 8.0, "x_forward_residual2": 20.0,
               "x_inverse_accumulate2": 20.0, "x_inverse_last": 8.0, "correct": 64.0, "mode00": 0.0}
# with two or more sweeps the last correction is kept apart (phi = hi + lo + lo2): the last
# sweep's inverse x-FFT writes lo2 (4 + 4) and the correction also reads it (64 + 4); the
# first sweep's residual is kept per cell (its kernel writes 8 more bytes) and the second
# sweep reads it instead of b, with delta_1 (4 + neighbours), phi_0 at the cell (4) and
# writes the spectrum (4): 20
BYTES_CORRECT_LO2 = 68.0
BYTES_RESID_KEPT = 24.0


def bytes_mixed(refine):
    b = dict(BYTES_MIXED)
    if refine >= 2:
        b["correct"] = BYTES_CORRECT_LO2
        b["x_forward_residual"] = BYTES_RESID_KEPT
    return b
BYTES_FP64 = {"x_forward_div": 32.0, "yz_forward": 20.0, "yz_backward": 20.0, "x_inverse_store": 16.0,
              "correct": 56.0, "mode00": 0.0}
# fp64 path: its transforms and sweeps keep the fp64 pipe busy, so its roofline is that
# pipe's rate (measured by libibf_probe.so) against algorithmic flops per cell: a complex
# FFT of length N counted as 5 N log2 N flops (a real one of N as 2.5 N log2 N), so the
# x transform of a real row costs 2.5 log2(nx) per cell and the y transform of the
# nx/2 + 1 complex columns 5 log2(ny) (nx/2 + 1)/nx per cell; the divergence 8 flops and
# its plane sum 1; a forward Thomas step per complex mode value 6 (r - a d: two FMAs,
# times the pivot: two products), a backward step 4; the correction 12 (three
# differences, three scalings, three FMAs).
def fp64_flops_per_cell(nx, ny):
    lx, ly = math.log2(nx), math.log2(ny)
    cy = (nx // 2 + 1) / nx  # complex y-columns per cell
    return {"x_forward_div": 9.0 + 2.5 * lx, "yz_forward": cy * (5.0 * ly + 6.0),
            "yz_backward": cy * (5.0 * ly + 4.0), "x_inverse_store": 2.5 * lx, "correct": 12.0,
            "mode00": 0.0}


FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense fp64, NVIDIA's figure


def fp64_peak():
    """(TFLOP/s, kind, fp64 add Gop/s or None): the fp64 FMA rate of this device measured by
    libibf_probe.so (two flops per FMA), else the nominal figure."""
    import ctypes
    try:
        from paper_2609_19130_gb300 import build as B
        lib = ctypes.CDLL(B.PROBE_LIB)
        f, a = ctypes.c_double(0.0), ctypes.c_double(0.0)
        lib.ibfprobe_fp64_rates.argtypes = [ctypes.POINTER(ctypes.c_double)] * 2
        if lib.ibfprobe_fp64_rates(ctypes.byref(f), ctypes.byref(a)) == 0 and f.value > 0:
            return 2.0 * f.value / 1e3, "measured (fp64 FMA chains, libibf_probe.so)", a.value
    except OSError:
        pass
    return FP64_NOMINAL_TFLOPS, "nominal", None


# DRAM bytes per cell (dram__bytes_read.sum + dram__bytes_write.sum / cells) of each
# kernel from one ncu capture (512x512x128 mixed, two refinement sweeps, see profiles/),
# valid while the kernel sources hash to NCU_SOURCES_SHA256; otherwise the roofline's
# traffic is null.
NCU_TRAFFIC_B_PER_CELL = {"x_forward_div": 35.57, "x_forward_residual": 22.95, "x_forward_residual2": 19.41,
                          "correct": 69.61, "yz_forward": 8.43, "yz_backward": 8.43, "x_inverse_store": 6.49,
                          "x_inverse_accumulate": 6.51, "x_inverse_last": 6.51}
NCU_SOURCES_SHA256 = "bddd4ec4a7446bfbed8731152b2e999e3e19d7c2400c4567ff40496e7a98425f"
KERNEL_SOURCES = ("ibf_kernels.cu", "ibf_yz.cu", "ibf_viscous.cu", "ibf_common.cuh", "ibf_device.cuh",
                  "ibf_internal.h", "ibf_viscous.h")
# the same for the viscous solve's kernels (mixed path)
NCU_VISC_TRAFFIC_B_PER_CELL = {"viscous_y": 6.22, "viscous_z": 17.31}


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2609_19130_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"ibf_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace('.', '', 1).isdigit()) if rows else None,
                "reasons": sorted(reasons)}


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """Largest value over the ranks (the slowest replica sets the whole-job time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def chunked_copy(dst, src, chunk_bytes):
    """dst.copy_(src) as one asynchronous copy, or as copies of chunk_bytes each."""
    if not chunk_bytes or dst.numel() * dst.element_size() <= chunk_bytes:
        dst.copy_(src, non_blocking=True)
        return
    n = max(1, chunk_bytes // dst.element_size())
    d, s_ = dst.view(-1), src.view(-1)
    for a in range(0, d.numel(), n):
        d[a:a + n].copy_(s_[a:a + n], non_blocking=True)


def host_link_rates(h_in, h_out, d_in, d_out):
    """Pinned host <-> device copy times for one step's traffic, measured in the same
    process right after the end-to-end run: all input fields up alone, all output fields
    down alone, and both directions at once on two streams (CUDA events; three repeats,
    median and best).  The host side of the link is shared, so these rates move from run to
    run; taking them beside the end-to-end number is what makes the two comparable."""
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nb_up = sum(t.numel() * t.element_size() for t in h_in)
    nb_down = sum(t.numel() * t.element_size() for t in h_out)

    def timed(fn):
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s1.wait_event(e0)
            s2.wait_event(e0)
            fn()
            torch.cuda.current_stream().wait_stream(s1)
            torch.cuda.current_stream().wait_stream(s2)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        return ts[1], ts[0]

    def up():
        with torch.cuda.stream(s1):
            for d, h in zip(d_in, h_in):
                d.copy_(h, non_blocking=True)

    def down():
        with torch.cuda.stream(s2):
            for h, d in zip(h_out, d_out):
                h.copy_(d, non_blocking=True)

    def both():
        up()
        down()

    (u_med, u_best), (d_med, d_best), (b_med, b_best) = timed(up), timed(down), timed(both)
    return {"h2d_ms": u_med, "d2h_ms": d_med, "both_ms": b_med,
            "h2d_gbs": nb_up / u_med / 1e6, "d2h_gbs": nb_down / d_med / 1e6,
            "both_gbs": (nb_up + nb_down) / b_med / 1e6,
            "best_ms": {"h2d": u_best, "d2h": d_best, "both": b_best},
            "repeats": 3, "statistic": "median",
            "bytes": [nb_up, nb_down]}


def time_steps(plan, ins, outs, K, W, ws, flush=None):
    """W warm-up then K timed projections; returns ms per step (CUDA events, max over ranks)
    and the per-kernel profile over the timed steps.  With `flush` (a buffer larger than
    L2) every step is timed alone, after the buffer has been rewritten outside its events."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(W):
        plan.project_into([ins], [outs], DT, 1.0)
    plan.profile(True)
    plan.profile_read(reset=True)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(K):
            plan.project_into([ins], [outs], DT, 1.0)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
    else:
        evs = []
        for _ in range(K):
            flush.add_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            plan.project_into([ins], [outs], DT, 1.0)
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / K
    barrier(ws)
    torch.cuda.synchronize()
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    return max_over_ranks(ms, ws), prof


# Factored implicit viscous solve (ibf_viscous_solve): algorithmic bytes per cell and
# component of each launch (mixed path; fp64 path in brackets): x-FFT of the field 8 in +
# 4 spectrum (8 + 8), y transforms with the factors 4 + 4 (8 + 8), inverse x-FFT 4 + 4
# (8 + 8), z Thomas: read and write the forward sweep, read it back, write fp64 out 4+4+4+8
# (8+8+8+8).
VISC_BYTES = {"viscous_x_forward": (12.0, 16.0), "viscous_y": (8.0, 16.0), "viscous_x_inverse": (8.0, 16.0),
              "viscous_z": (20.0, 32.0)}
VISC_BETA = 1e-4  # beta = alpha dt / (2 Re); beta / dx^2 = 2.7 on the 1024^2 planes: strongly coupled lines


def measure_viscous(plan, ins, outs, K, W, ws, mixed, cells, hbm_peak):
    """W warm-up then K timed viscous solves of the three components (CUDA events on the
    current stream); per-kernel profile, and the roofline of the dominant kernel."""
    import torch
    st = torch.cuda.current_stream()
    outs = outs[:3]
    for _ in range(W):
        plan.viscous_solve_into([ins], [outs], VISC_BETA)
    plan.profile(True)
    plan.profile_read(reset=True)
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(K):
        plan.viscous_solve_into([ins], [outs], VISC_BETA)
    e1.record(st)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / K, ws)
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    col = 0 if mixed else 1
    kernels = {k: {"launches": c, "ms_per_launch": t / c,
                   "gbs_algorithmic": VISC_BYTES[k][col] * cells / (t / c * 1e-3) / 1e9 if k in VISC_BYTES else None}
               for k, (c, t) in prof.items()}
    dname, (dc, dt_) = max(((k, v) for k, v in prof.items() if k in VISC_BYTES), key=lambda kv: kv[1][1])
    achieved = VISC_BYTES[dname][col] * cells / (dt_ / dc * 1e-3) / 1e9
    traffic = None
    if mixed and dname in NCU_VISC_TRAFFIC_B_PER_CELL and NCU_SOURCES_SHA256 == kernel_sources_sha256():
        traffic = NCU_VISC_TRAFFIC_B_PER_CELL[dname] * cells
    total_b = 3 * sum(b[col] for b in VISC_BYTES.values())
    return {"ms_per_solve": ms, "value": ws * cells / (ms * 1e-3), "unit": "cells/s (three components)",
            "bytes_per_cell_model": total_b, "hbm_frac": total_b * cells / (ms * 1e-3) / 1e9 / hbm_peak,
            "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic,
                         "bytes_per_cell": VISC_BYTES[dname][col]},
            "kernels": kernels, "gpu_launches": int(sum(c for c, _ in prof.values()))}


def viscous_oracle_sample(nx, ny, nz_sample):
    """The viscous-solve oracle (oracle/viscous.py) timed on the host on nx x ny x nz_sample."""
    import numpy as np
    from oracle import oracle as O
    from oracle import viscous as V
    from paper_2609_19130_gb300 import synth
    zf = O.zfaces_tanh(nz_sample, LZ, BETA)
    u, v, w = synth.uniform_velocity_np(SEED, nx, ny, nz_sample)
    t0 = time.perf_counter()
    V.viscous_solve(nx, ny, nz_sample, LX, LY, zf, u, v, w, VISC_BETA)
    sec = time.perf_counter() - t0
    return {"value": nx * ny * nz_sample / sec, "unit": "cells/s (three components)", "cores": 1, "kind": "oracle",
            "sample": f"fp64 numpy oracle (Thomas + Sherman-Morrison per line) on {nx}x{ny}x{nz_sample}, {sec:.1f} s"}


def workload_config(nx, ny, nz, refine, zbeta=BETA):
    return {"workload": f"{nx}x{ny}x{nz} staggered projection, periodic x,y (2pi), walls z in [0,2], "
                        f"tanh beta {zbeta}{' (uniform z)' if zbeta == 0 else ''}; velocity = k^-5/3 Fourier modes + U[-0.01,0.01] noise (seed {SEED}); "
                        f"mixed precision (fp32 transforms/sweeps, float-float stencils, fp64 I/O), "
                        f"{refine} refinement sweep(s)",
            "grid": [nx, ny, nz], "refine_steps": refine}


def cpu_baseline_child(spec: str, reps: int = 1):
    """Runs in a fresh process: the FP64 oracle on an nx x ny x nz_sample slab of the workload,
    `reps` times on the same inputs; prints the seconds of each run."""
    from oracle import oracle as O
    from paper_2609_19130_gb300 import synth
    nx, ny, nz_sample = (int(x) for x in spec.split("x"))
    g = O.Grid(nx, ny, nz_sample, lx=LX, ly=LY, lz=LZ, beta=BETA)
    u, v, w = synth.uniform_velocity_np(SEED, nx, ny, nz_sample)
    O.lib()
    secs = []
    for _ in range(reps):
        t0 = time.perf_counter()
        O.project(g, u, v, w, dt=DT)
        secs.append(time.perf_counter() - t0)
    print(json.dumps({"seconds": secs[-1], "all_seconds": secs, "cells": nx * ny * nz_sample,
                      "cores": os.cpu_count()}))


def host_sample_nz(requested, nz):
    """z levels of an oracle sample: the oracle's transforms run one plane per thread, so
    the sample is rounded up to a multiple of the host's cores (at most nz)."""
    c = os.cpu_count() or 1
    return min(nz, max(c, ((requested + c - 1) // c) * c))


def run_cpu_baseline(nx: int, ny: int, nz_sample: int, reps: int = 1):
    env = dict(os.environ)
    env["OMP_NUM_THREADS"] = str(os.cpu_count())
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", f"{nx}x{ny}x{nz_sample}",
                        "--cpu-reps", str(reps)],
                       capture_output=True, text=True, env=env, timeout=900 + 120 * reps)
    line = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not line:
        return None, r.stderr[-2000:]
    return json.loads(line[-1]), None


def reference_arm(args):
    """The oracle as it stands, on the host cores, K timed bounded samples after W warm-ups."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    nx, ny, nz = (int(x) for x in args.size.split("x"))
    nz_sample = host_sample_nz(args.ref_nz, nz)
    res, err = run_cpu_baseline(nx, ny, nz_sample, reps=args.warmup + args.steps)
    if res is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + (err or "")[-200:]}))
        return 0
    cores = res["cores"]
    times = res["all_seconds"][args.warmup:]
    cells = nx * ny * nz_sample
    sec = sum(times) / len(times)
    value = cells / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(nx, ny, nz, args.refine), parallelism="host cores"),
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 oracle (naive DFT/DCT + Thomas) on {nx}x{ny}x{nz_sample} cells per step "
                                   f"(the workload's planes, {nz_sample} z levels), U[-1,1] velocity seed {SEED}"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def shard(n, ws, rank):
    """Grid indices of one rank: the batch's independent grids dealt round-robin."""
    return list(range(rank, n, ws))


def measure_batch64(args, ws, rank, dev, autotune=True):
    """The batched workload (config 3): 64 uneven grids (nx, ny in {64,96,128,192}, nz in
    {64,128,256}, tanh beta in U[1,3], splitmix64 seed 1; velocity U[-1,1] of seed 1000+g)
    projected by one plan whose launch shapes are autotuned per grid shape, one ibf_project
    call per step.  Under torchrun the grids are dealt across the ranks (independent
    problems: no collective on the data path).  Returns the measurement as a dict."""
    import torch
    from paper_2609_19130_gb300 import MIXED, Grid, Plan, synth
    draws = synth.batch_grid_draws(1, 64)
    mine = shard(len(draws), ws, rank)
    all_cells = sum(nx * ny * nz for nx, ny, nz, _ in draws)
    grids = [Grid(*draws[i][:3], LX, LY, LZ, beta=draws[i][3]) for i in mine]
    ins, outs = [], []
    for i, g in zip(mine, grids):
        u, v, w = synth.uniform_velocity_torch(1000 + i, g.nx, g.ny, g.nz, dev)
        ins.append((u, v, w))
        outs.append((torch.empty_like(u), torch.empty_like(v), torch.empty_like(w),
                     torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device=dev)))
    cells = sum(g.cells for g in grids)
    t0 = time.perf_counter()
    plan = Plan(grids, precision=MIXED, refine_steps=args.refine, autotune=bool(autotune))
    plan_s = time.perf_counter() - t0
    for _ in range(max(3, args.warmup)):
        plan.project_into(ins, outs, DT, 1.0)
    plan.profile(True)
    plan.profile_read(reset=True)
    torch.cuda.synchronize()
    barrier(ws)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(args.steps, 10)
    with Clocks(dev.index) as ck:
        e0.record(st)
        for _ in range(steps):
            plan.project_into(ins, outs, DT, 1.0)
        e1.record(st)
        torch.cuda.synchronize()
    barrier(ws)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, ws)
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    # the same step replayed from a CUDA graph (one capture of one ibf_project call): the
    # difference to the eager time is what issuing the step's launches one by one costs
    graph = {}
    try:
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            plan.project_into(ins, outs, DT, 1.0)
        for _ in range(3):
            cg.replay()
        torch.cuda.synchronize()
        barrier(ws)
        e0.record(st)
        for _ in range(steps):
            cg.replay()
        e1.record(st)
        torch.cuda.synchronize()
        barrier(ws)
        gms = max_over_ranks(e0.elapsed_time(e1) / steps, ws)
        graph = {"ms_per_step": gms, "value": all_cells / (gms * 1e-3), "eager_minus_graph_ms": ms - gms}
        del cg
    except Exception as exc:  # capture refused by this torch build: report, keep the eager number
        graph = {"unavailable": str(exc)[:200]}
    kinds = {}
    for gi in range(len(grids)):
        t = plan.tuning(gi)
        key = {1: "streaming", 2: "slab", 3: "split", 4: "spectral_z"}[t["yz_kernel"]]
        kinds[key] = kinds.get(key, 0) + 1
    plan.close()
    launches = int(sum(c for c, _ in prof.values()))
    return {
        "metric": "cells/s per batched pressure projection (64 uneven grids)", "value": all_cells / (ms * 1e-3),
        "unit": "cells/s", "ms_per_step": ms, "steps": steps, "scaling": "strong",
        "hbm_frac_180B": 180.0 * all_cells / (ms * 1e-3) / 1e9 / peaks()[0],
        "config": {"workload": "64 grids, nx,ny in {64,96,128,192}, nz in {64,128,256}, beta U[1,3] (seed 1), "
                               "U[-1,1] velocity (seed 1000+g), mixed, "
                               f"{args.refine} refinement sweep(s)", "cells": all_cells,
                   "parallelism": f"grids dealt round-robin over {ws} rank(s)",
                   "autotuned": bool(autotune), "plan_seconds": plan_s, "yz_kernels": kinds,
                   "l2_policy": f"batch fields {cells * 56 / 1e9:.1f} GB > 129 MB L2: no flush"},
        "kernels": {k: {"launches": c, "ms_per_launch": t / c, "share": t / sum(x[1] for x in prof.values())}
                    for k, (c, t) in prof.items()},
        "launches_per_step": launches / steps, "gpu_launches": launches * (2 if "ms_per_step" in graph else 1),
        "graph_replay": graph, "clocks": ck.summary()}


def bench_batch64(args):
    """--batch64: the batched workload alone, as its own JSON line."""
    import torch
    ws, rank, _ = dist_init()
    from paper_2609_19130_gb300 import build as B
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    r = measure_batch64(args, ws, rank, dev, autotune=bool(args.autotune) or not args.no_autotune_batch)
    if rank == 0:
        line = dict(r, n_gpus=ws, warmup=args.warmup, higher_is_better=True, dtype="f32", data="synthetic")
        print(json.dumps(line))
    return 0


PROBE_OPS = ("dfma", "dadd", "ffma", "f64_f32_f64_roundtrip_pair", "u32_to_f32_plus_xor_pair", "iadd_plus_xor_pair")


def probe_rates():
    """Instruction rates of this device (libibf_probe.so, Gop/s device-wide and per SM per
    clock at the SM clock read before and after), as one JSON line."""
    import ctypes
    import torch
    from paper_2609_19130_gb300 import build as B
    B.build()
    lib = ctypes.CDLL(B.PROBE_LIB)
    n = len(PROBE_OPS)
    buf = (ctypes.c_double * n)()
    lib.ibfprobe_op_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    clk0 = sm_clock_mhz()
    rc = lib.ibfprobe_op_rates(buf, n)
    clk1 = sm_clock_mhz()
    props = torch.cuda.get_device_properties(0)
    mhz = max(clk0 or 0, clk1 or 0) or None
    out = {"device": props.name, "sms": props.multi_processor_count, "status": rc, "sm_mhz": [clk0, clk1],
           "gops": {k: buf[i] for i, k in enumerate(PROBE_OPS)}}
    if mhz:
        out["per_sm_per_clk"] = {k: buf[i] * 1e3 / (props.multi_processor_count * mhz) for i, k in enumerate(PROBE_OPS)}
    print(json.dumps(out))
    return rc


def sm_clock_mhz():
    try:
        r = subprocess.run(["nvidia-smi", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits", "-i", "0"],
                           capture_output=True, text=True, timeout=20)
        return float(r.stdout.strip().splitlines()[0])
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", default="1024x1024x512")
    ap.add_argument("--zbeta", type=float, default=BETA, help="tanh clustering of the z faces (0: uniform)")
    ap.add_argument("--refine", type=int, default=2,
                    help="refinement sweeps of the headline mixed run (two reach the fp64 round-off floor of the "
                         "divergence on the benchmark's stretched grid; one meets the bound on phi only)")
    ap.add_argument("--no-one-sweep", action="store_true", help="skip the one-sweep comparison run")
    ap.add_argument("--ref-nz", type=int, default=16,
                    help="z levels of the oracle sample per reference step (rounded up to a multiple of the host's cores)")
    ap.add_argument("--cpu-nz", type=int, default=16,
                    help="z levels of the cpu_baseline sample (rounded up to a multiple of the host's cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunk-mb", type=int, default=0,
                    help="split the end-to-end host copies into chunks of this many MiB (0: one copy per field)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-viscous", action="store_true", help="skip the viscous-solve measurement")
    ap.add_argument("--autotune", type=int, default=0, help="1: plan-time autotuning of the launch shapes")
    ap.add_argument("--tuning", default="", help="JSON dict of ibf_tuning fields forced for the mixed plan")
    ap.add_argument("--batch64", action="store_true", help="time the 64-grid batched workload alone")
    ap.add_argument("--no-batch64", action="store_true", help="skip the 64-grid batched measurement")
    ap.add_argument("--no-autotune-batch", action="store_true", help="default launch shapes for the 64 grids")
    ap.add_argument("--probe-rates", action="store_true",
                    help="print the instruction rates measured by libibf_probe.so as one JSON line and exit")
    ap.add_argument("--cpu-child", default="", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-reps", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_child:
        cpu_baseline_child(args.cpu_child, args.cpu_reps)
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    if args.batch64:
        return bench_batch64(args)
    if args.probe_rates:
        return probe_rates()
    if args.warmup < 3:
        args.warmup = 3

    import torch
    ws, rank, local = dist_init()
    from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth
    from paper_2609_19130_gb300 import build as B
    B.build()

    nx, ny, nz = (int(x) for x in args.size.split("x"))
    cells = nx * ny * nz
    g = Grid(nx, ny, nz, LX, LY, LZ, beta=args.zbeta)
    dev = torch.device("cuda", torch.cuda.current_device())
    us, vs, ws_ = synth.kolmogorov_velocity_torch(SEED, nx, ny, nz, dev)
    ins = (us, vs, ws_)
    outs = (torch.empty_like(us), torch.empty_like(vs), torch.empty_like(ws_),
            torch.empty((nz, ny, nx), dtype=torch.float64, device=dev))
    torch.cuda.synchronize()

    hbm_peak, peak_kind = peaks()
    # inputs + outputs of one step; below twice the 129 MB L2, flush it between timed steps
    step_bytes = 8 * (sum(t.numel() for t in ins) + sum(t.numel() for t in outs))
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev) if step_bytes < (258 << 20) else None
    l2_policy = (f"step fields {step_bytes / 1e9:.2f} GB > 2x the 129 MB L2: no flush between steps" if flush is None
                 else "L2 flushed (256 MB written) before every timed step, outside its events")
    res = {}
    clocks = None
    # the headline (mixed, --refine sweeps), the fp64 path, and one sweep for comparison;
    # outside the timed regions each run's phi and max|D u| are kept for the accuracy notes
    runs = [("mixed", MIXED, args.refine)] + ([] if args.no_fp64 else [("fp64", FP64, 0)])
    if args.refine != 1 and not args.no_one_sweep:
        runs.append(("mixed_1sweep", MIXED, 1))
    phis = {}
    for key, prec, R in runs:
        tun = [json.loads(args.tuning)] if (args.tuning and prec == MIXED) else None
        plan = Plan([g], precision=prec, refine_steps=R, device=dev.index,
                    autotune=bool(args.autotune), tuning=tun)
        if key == "mixed":
            with Clocks(dev.index) as ck:
                ms, prof = time_steps(plan, ins, outs, args.steps, args.warmup, ws, flush)
            clocks = ck.summary()
        else:
            ms, prof = time_steps(plan, ins, outs, args.steps, args.warmup, ws, flush)
        # diagnostics outside the timed region: divergence of the output, phi kept
        (_, st) = plan.project_batch([ins], DT, out=[outs], stats=True)
        torch.cuda.synchronize()
        diag = {"max_div_out": float(st["max_div"][0]), "max_div_in": float(st["max_div_in"][0]),
                "div_rel": float(st["max_div"][0]) / max(float(st["max_div_in"][0]), 1e-300),
                "status": plan.sync_status()}
        phis[key] = outs[3].clone()
        res[key] = {"ms": ms, "prof": prof, "diag": diag, "plan": plan, "tuning": plan.tuning(0), "refine": R}
    if "fp64" in phis:
        ref = phis["fp64"]
        for key in res:
            if key != "fp64":
                res[key]["diag"]["phi_rel_l2_vs_fp64"] = float(torch.linalg.norm(phis[key] - ref) / torch.linalg.norm(ref))
    del phis
    res[MIXED] = res.pop("mixed")
    if "fp64" in res:
        res[FP64] = res.pop("fp64")

    mixed = res[MIXED]
    ms = mixed["ms"]
    value = ws * cells / (ms * 1e-3)
    prof = mixed["prof"]
    launches_per_step = sum(c for c, _ in prof.values()) / args.steps
    # dominant kernel and its roofline
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dname, (dcount, dms) = dom
    per_launch_ms = dms / dcount
    BM = bytes_mixed(args.refine)
    per_launch_bytes = BM.get(dname, 0.0) * cells
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    traffic = None
    if dname in NCU_TRAFFIC_B_PER_CELL and NCU_SOURCES_SHA256 == kernel_sources_sha256():
        traffic = NCU_TRAFFIC_B_PER_CELL[dname] * cells
    bytes_model = sum(BM[k] * c / args.steps for k, (c, _) in prof.items() if k in BM)
    kernels = {k: {"launches": c, "ms_per_launch": t / c, "share": t / sum(x[1] for x in prof.values()),
                   "gbs_algorithmic": (BM.get(k, 0.0) * cells / (t / c * 1e-3) / 1e9)}
               for k, (c, t) in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(nx, ny, nz, args.refine, args.zbeta), **{
                   "parallelism": "replicas" if ws > 1 else "1 GPU",
                   "launch_shape": mixed["tuning"], "autotuned": bool(args.autotune),
                   "l2_policy": l2_policy}),
        "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                     "bytes_per_cell": BM.get(dname, 0.0)},
        "projection_hbm": {"bytes_per_cell_model": bytes_model,
                           "achieved_gbs": bytes_model * cells / (ms * 1e-3) / 1e9,
                           "frac": bytes_model * cells / (ms * 1e-3) / 1e9 / hbm_peak,
                           "compulsory_56B_frac": 56.0 * cells / (ms * 1e-3) / 1e9 / hbm_peak},
        "kernels": kernels,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clocks,
        "diagnostics": mixed["diag"],
    }
    if FP64 in res:
        f = res[FP64]
        flops = fp64_flops_per_cell(nx, ny)
        tf_peak, tf_kind, dadd_gops = fp64_peak()
        fk = {k: {"launches": c, "ms_per_launch": t / c,
                  "tflops_algorithmic": flops.get(k, 0.0) * cells / (t / c * 1e-3) / 1e12}
              for k, (c, t) in f["prof"].items()}
        fd = max(((k, v) for k, v in f["prof"].items() if flops.get(k, 0.0) > 0), key=lambda kv: kv[1][1])
        fdn, (fdc, fdt) = fd
        f_ach = flops[fdn] * cells / (fdt / fdc * 1e-3) / 1e12
        f_step = sum(flops.get(k, 0.0) * c / args.steps for k, (c, _) in f["prof"].items())
        line["fp64"] = {"value": ws * cells / (f["ms"] * 1e-3), "ms_per_step": f["ms"],
                        "kernels": fk, "speedup_mixed_over_fp64": f["ms"] / ms,
                        "roofline": {"bound": "alu", "pipe": "fp64", "kernel": fdn, "achieved": f_ach,
                                     "peak": tf_peak, "unit": "TFLOP/s", "frac": f_ach / tf_peak,
                                     "peak_kind": tf_kind, "flops_per_cell": flops[fdn],
                                     "peak_nominal": FP64_NOMINAL_TFLOPS, "dadd_gops": dadd_gops},
                        "diagnostics": f["diag"],
                        "projection_alu": {"flops_per_cell_model": f_step,
                                           "achieved_tflops": f_step * cells / (f["ms"] * 1e-3) / 1e12,
                                           "frac": f_step * cells / (f["ms"] * 1e-3) / 1e12 / tf_peak}}

    if "mixed_1sweep" in res:
        r1 = res["mixed_1sweep"]
        line["mixed_1sweep"] = {
            "value": ws * cells / (r1["ms"] * 1e-3), "ms_per_step": r1["ms"], "refine_steps": 1,
            "diagnostics": r1["diag"],
            "kernels": {k: {"launches": c, "ms_per_launch": t / c} for k, (c, t) in r1["prof"].items()}}

    # End to end through the public API with host buffers (pinned), copies inside the timed
    # region: every step uploads its own u*, v*, w* and downloads its own u, v, w, phi.  Steps
    # are pipelined the way a caller streaming projections would run them: the upload of
    # step i+1 and the download of step i run on their own streams while step i projects
    # (device fields double-buffered; one pinned host set each way: uploads only read it and
    # downloads are ordered on their stream; ordering by events).
    if not args.no_e2e:
        plan = mixed["plan"]
        # three device buffer sets: the upload of step i+1, the projection of step i and the
        # download of step i-1 each have a set of their own
        nsets = 3
        dev_sets = [(ins, outs)] + [(tuple(torch.empty_like(t) for t in ins), tuple(torch.empty_like(t) for t in outs))
                                    for _ in range(nsets - 1)]
        # pinned host buffers allocated pinned (no pageable staging copy first): the step's
        # inputs copied into them from the device, the outputs' buffers touched once
        h_in = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in ins]
        h_out = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs]
        for h, t in zip(h_in, ins):
            h.copy_(t)
        for h in h_out:
            h.zero_()
        s_comp, s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        s_comp.wait_stream(torch.cuda.current_stream())
        h2d = sum(t.numel() * 8 for t in h_in)
        d2h = sum(t.numel() * 8 for t in h_out)

        def run_steps(n):
            # buffer set b = i % nsets; its inputs may be overwritten once step i-nsets has
            # projected, its outputs once step i-nsets has been downloaded
            projected = [None] * nsets
            downloaded = [None] * nsets
            for i in range(n):
                b_ = i % nsets
                d_in, d_out = dev_sets[b_]
                with torch.cuda.stream(s_up):
                    if projected[b_] is not None:
                        s_up.wait_event(projected[b_])
                    for d, h in zip(d_in, h_in):
                        chunked_copy(d, h, chunk)
                    up = torch.cuda.Event()
                    up.record(s_up)
                s_comp.wait_event(up)
                if downloaded[b_] is not None:
                    s_comp.wait_event(downloaded[b_])
                plan.project_into([d_in], [d_out], DT, 1.0, stream=s_comp)
                done = torch.cuda.Event()
                done.record(s_comp)
                projected[b_] = done
                with torch.cuda.stream(s_down):
                    s_down.wait_event(done)
                    for h, d in zip(h_out, d_out):
                        chunked_copy(h, d, chunk)
                    dn = torch.cuda.Event()
                    dn.record(s_down)
                    downloaded[b_] = dn
            s_comp.wait_stream(s_down)
            s_comp.wait_stream(s_up)

        chunk = args.e2e_chunk_mb << 20
        run_steps(nsets)
        torch.cuda.synchronize()
        barrier(ws)
        ke = max(4, min(args.steps, 10))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s_comp)
        s_up.wait_stream(s_comp)
        s_down.wait_stream(s_comp)
        run_steps(ke)
        e1.record(s_comp)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1) / ke, ws)
        link = host_link_rates(h_in, h_out, dev_sets[1][0], dev_sets[1][1])
        line["e2e"] = {"value": ws * cells / (ems * 1e-3), "unit": "cells/s", "ms_per_step": ems,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ke,
                       "pipelined": "upload of step i+1 and download of step i-1 overlap step i's projection "
                                    "(three device buffer sets, one pinned host set each way)",
                       "copy_chunk_mb": args.e2e_chunk_mb or None, "link": link,
                       # the link alone, in the better of its two schedules: the directions one
                       # after the other, or both at once
                       "link_bound_ms": min(link["h2d_ms"] + link["d2h_ms"], link["both_ms"])}
        line["gpu_launches"] += int(round(launches_per_step * ke))
        del dev_sets, h_in, h_out

    # the batched workload (64 uneven grids, autotuned; separate object: not the headline)
    if not args.no_batch64:
        line["batch64"] = measure_batch64(args, ws, rank, dev, autotune=not args.no_autotune_batch)
        line["gpu_launches"] += line["batch64"]["gpu_launches"]

    # the factored implicit viscous solve on the same workload and plans (separate object:
    # not part of the projection's step)
    if not args.no_viscous:
        visc = {"beta": VISC_BETA,
                "workload": f"{nx}x{ny}x{nz}: (I - beta Lz)^-1 (I - beta Ly)^-1 (I - beta Lx)^-1 of u, v, w "
                            f"(the same fields as right-hand sides)"}
        for prec, r in res.items():
            if prec not in (MIXED, FP64):
                continue
            visc["mixed" if prec == MIXED else "fp64"] = measure_viscous(
                r["plan"], ins, outs, args.steps, args.warmup, ws, prec == MIXED, cells, hbm_peak)
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:
            visc["cpu_oracle"] = viscous_oracle_sample(nx, ny, min(8, nz))
        line["viscous_solve"] = visc

    for r in res.values():
        r["plan"].close()

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        nzs = host_sample_nz(args.cpu_nz, nz)
        cb, err = run_cpu_baseline(nx, ny, nzs)
        if cb is not None:
            line["cpu_baseline"] = {"value": cb["cells"] / cb["seconds"], "unit": "cells/s", "cores": cb["cores"],
                                    "kind": "oracle",
                                    "sample": f"FP64 oracle on {nx}x{ny}x{nzs} (the workload's planes, {nzs} "
                                              f"z levels), {cb['seconds']:.1f} s"}
        else:
            line["cpu_baseline"] = {"value": None, "unit": "cells/s", "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": "failed: " + (err or "")[-200:]}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
