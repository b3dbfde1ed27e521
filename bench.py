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
# Algorithmic HBM bytes per cell of each kernel (fp64 user fields, fp32 spectrum,
# float-float right-hand side); derivation in the design doc.
BYTES_MIXED = {"x_forward_div": 36.0, "yz_forward": 10.0, "yz_backward": 10.0, "x_inverse_store": 8.0,
               "x_forward_residual": 16.0, "x_inverse_accumulate": 16.0, "correct": 64.0, "mode00": 0.0}
BYTES_FP64 = {"x_forward_div": 32.0, "yz_forward": 20.0, "yz_backward": 20.0, "x_inverse_store": 16.0,
              "correct": 56.0, "mode00": 0.0}
# DRAM bytes per cell (dram__bytes_read.sum + dram__bytes_write.sum / cells) of each
# kernel from one ncu capture (512x512x128 mixed, see profiles/), valid while the
# kernel sources hash to SOURCES_SHA256; otherwise the roofline's traffic is null.
NCU_TRAFFIC_B_PER_CELL = {}
NCU_SOURCES_SHA256 = None
KERNEL_SOURCES = ("ibf_kernels.cu", "ibf_yz.cu", "ibf_common.cuh", "ibf_device.cuh", "ibf_internal.h")


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
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(plan, ins, outs, K, W, ws):
    """W warm-up then K timed projections; returns ms per step (CUDA events, max over ranks)
    and the per-kernel profile over the timed steps."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(W):
        plan.project_into([ins], [outs], DT, 1.0)
    plan.profile(True)
    plan.profile_read(reset=True)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(K):
        plan.project_into([ins], [outs], DT, 1.0)
    e1.record(st)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    return max_over_ranks(ms, ws), prof


def cpu_baseline_child(nz_sample: int):
    """Runs in a fresh process: the FP64 oracle on nx=ny=1024 with nz_sample levels."""
    import numpy as np
    from oracle import oracle as O
    from paper_2609_19130_gb300 import synth
    n = 1024
    g = O.Grid(n, n, nz_sample, lx=LX, ly=LY, lz=LZ, beta=BETA)
    u, v, w = synth.uniform_velocity_np(SEED, n, n, nz_sample)
    O.lib()
    t0 = time.perf_counter()
    O.project(g, u, v, w, dt=DT)
    dt = time.perf_counter() - t0
    cells = n * n * nz_sample
    print(json.dumps({"seconds": dt, "cells": cells, "cores": os.cpu_count()}))


def run_cpu_baseline(nz_sample: int):
    env = dict(os.environ)
    env["OMP_NUM_THREADS"] = str(os.cpu_count())
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", str(nz_sample)],
                       capture_output=True, text=True, env=env, timeout=900)
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
    nz_sample = args.ref_nz
    times = []
    cores = None
    for i in range(args.warmup + args.steps):
        res, err = run_cpu_baseline(nz_sample)
        if res is None:
            print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + (err or "")[-200:]}))
            return 0
        cores = res["cores"]
        if i >= args.warmup:
            times.append(res["seconds"])
    cells = 1024 * 1024 * nz_sample
    sec = sum(times) / len(times)
    value = cells / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"FP64 CPU oracle (naive DFT + Thomas), 1024x1024x{nz_sample} sample of the "
                               f"1024x1024x512 stretched-z projection (beta {BETA})"},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "sample": f"1024x1024x{nz_sample} cells per step, U[-1,1] velocity seed {SEED}"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", default="1024x1024x512")
    ap.add_argument("--refine", type=int, default=1)
    ap.add_argument("--ref-nz", type=int, default=4, help="z levels of the oracle sample per reference step")
    ap.add_argument("--cpu-nz", type=int, default=16, help="z levels of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--autotune", type=int, default=0, help="1: plan-time autotuning of the launch shapes")
    ap.add_argument("--tuning", default="", help="JSON dict of ibf_tuning fields forced for the mixed plan")
    ap.add_argument("--cpu-child", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_child:
        cpu_baseline_child(args.cpu_child)
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    if args.warmup < 3:
        args.warmup = 3

    import torch
    ws, rank, local = dist_init()
    from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth
    from paper_2609_19130_gb300 import build as B
    B.build()

    nx, ny, nz = (int(x) for x in args.size.split("x"))
    cells = nx * ny * nz
    g = Grid(nx, ny, nz, LX, LY, LZ, beta=BETA)
    dev = torch.device("cuda", torch.cuda.current_device())
    us, vs, ws_ = synth.kolmogorov_velocity_torch(SEED, nx, ny, nz, dev)
    ins = (us, vs, ws_)
    outs = (torch.empty_like(us), torch.empty_like(vs), torch.empty_like(ws_),
            torch.empty((nz, ny, nx), dtype=torch.float64, device=dev))
    torch.cuda.synchronize()

    hbm_peak, peak_kind = peaks()
    res = {}
    clocks = None
    for prec in ([MIXED] + ([] if args.no_fp64 else [FP64])):
        tun = [json.loads(args.tuning)] if (args.tuning and prec == MIXED) else None
        plan = Plan([g], precision=prec, refine_steps=args.refine if prec == MIXED else 0, device=dev.index,
                    autotune=bool(args.autotune), tuning=tun)
        if prec == MIXED:
            with Clocks(dev.index) as ck:
                ms, prof = time_steps(plan, ins, outs, args.steps, args.warmup, ws)
            clocks = ck.summary()
            # diagnostics outside the timed region: divergence of the output
            (_, st) = plan.project_batch([ins], DT, out=[outs], stats=True)
            torch.cuda.synchronize()
            diag = {"max_div_out": float(st["max_div"][0]), "max_div_in": float(st["max_div_in"][0]),
                    "status": plan.sync_status()}
        else:
            ms, prof = time_steps(plan, ins, outs, args.steps, args.warmup, ws)
            diag = None
        res[prec] = {"ms": ms, "prof": prof, "diag": diag, "plan": plan, "tuning": plan.tuning(0)}

    mixed = res[MIXED]
    ms = mixed["ms"]
    value = ws * cells / (ms * 1e-3)
    prof = mixed["prof"]
    launches_per_step = sum(c for c, _ in prof.values()) / args.steps
    # dominant kernel and its roofline
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dname, (dcount, dms) = dom
    per_launch_ms = dms / dcount
    per_launch_bytes = BYTES_MIXED.get(dname, 0.0) * cells
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    traffic = None
    if dname in NCU_TRAFFIC_B_PER_CELL and NCU_SOURCES_SHA256 == kernel_sources_sha256():
        traffic = NCU_TRAFFIC_B_PER_CELL[dname] * cells
    bytes_model = sum(BYTES_MIXED[k] * c / args.steps for k, (c, _) in prof.items() if k in BYTES_MIXED)
    kernels = {k: {"launches": c, "ms_per_launch": t / c, "share": t / sum(x[1] for x in prof.values()),
                   "gbs_algorithmic": (BYTES_MIXED.get(k, 0.0) * cells / (t / c * 1e-3) / 1e9)}
               for k, (c, t) in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{nx}x{ny}x{nz} staggered projection, periodic x,y (2pi), walls z in [0,2], "
                               f"tanh beta {BETA}; velocity = k^-5/3 Fourier modes + U[-0.01,0.01] noise (seed {SEED}); "
                               f"mixed precision (fp32 transforms/sweeps, float-float stencils, fp64 I/O), "
                               f"{args.refine} refinement sweep(s)",
                   "grid": [nx, ny, nz], "refine_steps": args.refine, "parallelism": "replicas" if ws > 1 else "1 GPU",
                   "launch_shape": mixed["tuning"], "autotuned": bool(args.autotune),
                   "l2_policy": "inputs 4.3 GB per field (> 129 MB L2): no flush between steps"},
        "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                     "bytes_per_cell": BYTES_MIXED.get(dname, 0.0)},
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
        line["fp64"] = {"value": ws * cells / (f["ms"] * 1e-3), "ms_per_step": f["ms"],
                        "kernels": {k: {"launches": c, "ms_per_launch": t / c} for k, (c, t) in f["prof"].items()},
                        "speedup_mixed_over_fp64": f["ms"] / ms}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    if not args.no_e2e:
        plan = mixed["plan"]
        h_in = [t.cpu().pin_memory() for t in ins]
        h_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
        st = torch.cuda.current_stream()
        h2d = sum(t.numel() * 8 for t in h_in)
        d2h = sum(t.numel() * 8 for t in h_out)

        def e2e_step():
            for d, h in zip(ins, h_in):
                d.copy_(h, non_blocking=True)
            plan.project_into([ins], [outs], DT, 1.0)
            for h, d in zip(h_out, outs):
                h.copy_(d, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        ke = max(2, min(args.steps, 5))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(ke):
            e2e_step()
        e1.record(st)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1) / ke, ws)
        line["e2e"] = {"value": ws * cells / (ems * 1e-3), "unit": "cells/s", "ms_per_step": ems,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ke}
        line["gpu_launches"] += int(round(launches_per_step * ke))

    for r in res.values():
        r["plan"].close()

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, err = run_cpu_baseline(args.cpu_nz)
        if cb is not None:
            line["cpu_baseline"] = {"value": cb["cells"] / cb["seconds"], "unit": "cells/s", "cores": cb["cores"],
                                    "kind": "oracle",
                                    "sample": f"FP64 oracle on 1024x1024x{args.cpu_nz} (same planes, {args.cpu_nz} "
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
