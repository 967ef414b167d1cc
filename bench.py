"""Benchmark of the locality-optimised res_calc loop (and its baselines).

Default workload: res_calc on a jittered, randomly renumbered 2400x1200 quad
mesh (2.88M cells, 5.756M interior edges), FP64, through the C ABI.  A step
is one full res_calc pass (every block colour) of the two-layer staged
kernel on the RCM + partitioned plan.  The metric is interior edges per
second (Gedges/s); useful bandwidth follows the paper's formula (Sec. 3.1:
each dataset counted once, twice if read and written; maps as int32).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun each rank runs an
independent replica of the workload (replicas only; no collective on the
data path) and the value is the total edges of all ranks over the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import meshgen  # noqa: E402

METRIC = "res_calc Gedges/s & HBM GB/s % of peak: two-layer vs atomics vs global color"
NX, NY = 2400, 1200
GAM, EPS = 1.4, 0.05


def useful_bytes_res_calc(ncell, nnode, nedge, elt):
    """Sec. 3.1 useful bytes: x (2/node) + q (4/cell) + adt (1/cell) read,
    res (4/cell) read and written (w = 2), two int32 maps of 2 per edge."""
    return (2 * nnode + 4 * ncell + ncell + 2 * 4 * ncell) * elt + 2 * 2 * 4 * nedge


# algorithmic floating-point operations of one interior edge of res_calc as
# the oracle evaluates it: two normal fluxes (20 each: pressure 7, normal
# velocity 4, components 9), the normal 2, mu 3, four flux components 5 each,
# and the two increments of 4 components (8)
FLOPS_PER_EDGE = 73


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 FMA throughput of GB300: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def synthetic_adt(m):
    """A positive per-cell time-step field of the magnitude the free stream
    gives on an h x h cell ((2h(|u|+|v|) + 4h)/0.9, about 5.4 h)."""
    return meshgen.positive_field(m.ncell, 5.0 * m.h, 6.0 * m.h)


def oracle_res_calc_rate(m, q, adt, budget_s):
    """The oracle's sequential res_calc on the host, repeated for ~budget_s."""
    import oracle
    res = np.zeros((m.ncell, 4))
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt, res=res)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    return n * m.nedge / dt / 1e9, n, dt


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    m = meshgen.quad_mesh(args.nx, args.ny)
    q = meshgen.quad_state(m.ncell)
    adt = synthetic_adt(m)
    res = np.zeros((m.ncell, 4))
    for _ in range(args.warmup):
        oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt, res=res)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt, res=res)
    dt = time.perf_counter() - t0
    v = args.steps * m.nedge / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gedges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"res_calc {args.nx}x{args.ny} jittered renumbered quads, FP64", "cells": m.ncell,
                       "edges": m.nedge},
            "cpu_baseline": {"value": v, "unit": "Gedges/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full res_calc passes ({m.nedge} edges each)"},
            "e2e": {"value": v, "unit": "Gedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block-size", type=int, default=480)
    ap.add_argument("--layout", default="aos", choices=["aos", "soa"])
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-variants", action="store_true", help="skip the baseline variants")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--nx", type=int, default=NX, help="quad grid size (profiling runs use smaller meshes)")
    ap.add_argument("--ny", type=int, default=NY)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_1802_03749_gb300 as ml
    from paper_1802_03749_gb300.mesh import AirfoilPlans

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    m = meshgen.quad_mesh(args.nx, args.ny)
    q = meshgen.quad_state(m.ncell)
    adt = synthetic_adt(m)
    tdt = torch.float64 if args.dtype == "f64" else torch.float32
    elt = 8 if args.dtype == "f64" else 4
    useful = useful_bytes_res_calc(m.ncell, m.nnode, m.nedge, elt)
    stream = torch.cuda.current_stream()

    def setup(coloring, reorder, layout):
        P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                         block_size=args.block_size, reorder=reorder, coloring=coloring, layout=layout)
        P.res.upload()
        d = {"x": torch.tensor(P.to_plan(m.x, "node"), dtype=tdt, device="cuda"),
             "q": torch.tensor(P.to_plan(q, "cell"), dtype=tdt, device="cuda"),
             "adt": torch.tensor(P.to_plan(adt, "cell"), dtype=tdt, device="cuda")}
        d["res"] = torch.zeros_like(d["q"])
        return P, d

    def time_steps(P, d, steps, warmup, per_launch=False):
        for _ in range(warmup):
            ml.loop_res_calc(P.res, d["x"], d["q"], d["adt"], d["res"], GAM, EPS)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ml.loop_res_calc(P.res, d["x"], d["q"], d["adt"], d["res"], GAM, EPS)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if dist is not None:
            t = torch.tensor([ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    # ---------------------------------------------------------- headline
    P, d = setup("hier", "partition", args.layout)
    st = P.res.stats()
    clk = ClockSampler(local)
    clk.start()
    ms = time_steps(P, d, args.steps, args.warmup)
    clocks = clk.stop()
    ms_step = ms / args.steps
    value = world * m.nedge / (ms_step * 1e-3) / 1e9
    gbs = useful / (ms_step * 1e-3) / 1e9
    hbm_peak, peak_kind = read_peaks()
    tflops = FLOPS_PER_EDGE * m.nedge / (ms_step * 1e-3) / 1e12

    # ---------------------------------------------------------- e2e (host buffers)
    hx = torch.tensor(P.to_plan(m.x, "node"), dtype=tdt).pin_memory()
    hq = torch.tensor(P.to_plan(q, "cell"), dtype=tdt).pin_memory()
    ha = torch.tensor(P.to_plan(adt, "cell"), dtype=tdt).pin_memory()
    hr = torch.zeros_like(hq).pin_memory()
    hout = torch.empty_like(hq).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))

    def e2e_step():
        d["x"].copy_(hx, non_blocking=True)
        d["q"].copy_(hq, non_blocking=True)
        d["adt"].copy_(ha, non_blocking=True)
        d["res"].copy_(hr, non_blocking=True)
        ml.loop_res_calc(P.res, d["x"], d["q"], d["adt"], d["res"], GAM, EPS)
        hout.copy_(d["res"], non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = (hx.numel() + hq.numel() + ha.numel() + hr.numel()) * elt
    d2h = hout.numel() * elt

    # ---------------------------------------------------------- variants
    variants = {"two_layer_partition": {"gedges_s": value / world, "ms": ms_step, "useful_gbs": gbs,
                                        "block_colors": st["nblock_colors"],
                                        "thread_colors_mean": st["mean_thread_colors"],
                                        "reuse": st["reuse_all"], "plan_seconds": st["seconds_total"]}}
    del d
    if not args.no_variants:
        for name, (coloring, reorder) in {"two_layer_rcm": ("hier", "rcm"), "global_rcm": ("global", "rcm"),
                                          "global_none": ("global", "none"), "atomic_rcm": ("atomic", "rcm"),
                                          "atomic_none": ("atomic", "none")}.items():
            try:
                Pv, dv = setup(coloring, reorder, args.layout)
            except ml.MeshLoopError as e:
                variants[name] = {"error": str(e)}
                continue
            msv = time_steps(Pv, dv, max(5, args.steps // 2), 2) / max(5, args.steps // 2)
            sv = Pv.res.stats()
            variants[name] = {"gedges_s": m.nedge / (msv * 1e-3) / 1e9, "ms": msv,
                              "useful_gbs": useful / (msv * 1e-3) / 1e9, "colors": sv["nblock_colors"]}
            del dv, Pv

    # ---------------------------------------------------------- CPU baseline (oracle)
    cpu = None
    if rank == 0 and args.cpu_seconds > 0:
        r, n, dt = oracle_res_calc_rate(m, q, adt, args.cpu_seconds)
        cpu = {"value": r, "unit": "Gedges/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} full res_calc passes of the same mesh ({m.nedge} edges) in {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gedges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"res_calc {args.nx}x{args.ny} jittered renumbered quads, two-layer colouring, "
                                   f"RCM + partition, block {args.block_size}, {args.layout.upper()}",
                       "cells": m.ncell, "nodes": m.nnode, "edges": m.nedge, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (useful bytes %.0f MB > 129 MB)" % (useful / 1e6)},
            "useful_gbs": gbs, "useful_frac_hbm": gbs / hbm_peak,
            "roofline": {"bound": "alu" if args.dtype == "f64" else "hbm",
                         "achieved": tflops if args.dtype == "f64" else gbs,
                         "peak": FP64_PEAK_TFLOPS if args.dtype == "f64" else hbm_peak,
                         "unit": "TFLOP/s" if args.dtype == "f64" else "GB/s",
                         "frac": (tflops / FP64_PEAK_TFLOPS) if args.dtype == "f64" else gbs / hbm_peak,
                         "traffic": None,
                         "peak_kind": "derived FP64 FMA rate" if args.dtype == "f64" else peak_kind},
            "cpu_baseline": cpu,
            "e2e": {"value": world * m.nedge / e2e_s / 1e9, "unit": "Gedges/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * st["nblock_colors"],
            "clocks": clocks,
            "plan": {"blocks": st["nblocks"], "block_colors": st["nblock_colors"],
                     "thread_colors_max": st["max_thread_colors"], "reuse": st["reuse_all"],
                     "plan_seconds": st["seconds_total"]},
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
