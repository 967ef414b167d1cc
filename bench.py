"""Benchmark of the locality-optimised res_calc loop, its baselines and the
other loops of the library, on synthetic meshes shaped like the paper's.

Headline workload: res_calc on a jittered, randomly renumbered 2400x1200 quad
mesh (2,880,000 cells, 5,756,400 interior edges) with FP64 data, through the
C ABI.  A step is one full res_calc pass (every block colour) of the
two-layer staged kernel (RCM + partition plan).  The metric is interior
edges per second; useful bandwidth follows the paper's formula (Sec. 3.1:
each dataset once, twice if read and written, maps as int32 datasets).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun every rank runs an
independent replica of the workload (no collective on the data path); the
value is the edges of all ranks over the slowest rank's time.
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
L2_BYTES = 129 * 10 ** 6

# algorithmic floating-point operations of one interior edge as the oracle
# evaluates it: two normal fluxes of 20 (pressure 7, normal velocity 4,
# components 9), the normal 2, mu 3, four flux components of 5, two
# increments of 4 components
FLOPS_PER_EDGE = 73
# FP64 FMA throughput of GB300: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Double-word arithmetic: the res_calc flux uses 26 additions of 11 FP32
# operations and 19 products of 8, 9.7 FP32 operations per double-word
# operation, on 152 SMs x 128 FP32 lanes x 2.07 GHz
DW_FP32_OPS_PER_OP = 9.7
DW_PEAK_TFLOPS = 152 * 128 * 2.07e9 / DW_FP32_OPS_PER_OP / 1e12


# DRAM bytes (read + write) of one pass of the headline kernel (all block
# colours: double-word res_calc, gather increments, 2400x1200, block 256,
# partitioned) from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum over the 4 launches of a pass; summary in
# profiles/res_calc_hier_dw_2400x1200.md).  Valid only for the sources it
# was measured on: a change to any of them reports null until re-measured.
HEADLINE_TRAFFIC = {"bytes_per_pass": 416253952, "launches_per_pass": 4,
                    "config": ("dw", "gather", 256, 2400, 1200, "aos"),
                    "sha256": "ffa4749a30bc752f8ae7c794d691a0db127651c7afeace5f3f687deff2564325",
                    "sources": ("loops_res_dw.cu", "dw.cuh", "plan.cpp")}


def headline_traffic(args, head_staged):
    """Measured DRAM bytes per pass when the kernel sources and the launch
    configuration are the ones the capture was taken on, else None."""
    import hashlib
    T = HEADLINE_TRAFFIC
    if (args.compute, head_staged, args.block_size, args.nx, args.ny, args.layout) != T["config"]:
        return None
    h = hashlib.sha256()
    for f in T["sources"]:
        with open(os.path.join(ROOT, "paper_1802_03749_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return T["bytes_per_pass"] if h.hexdigest() == T["sha256"] else None


def useful_bytes_res_calc(ncell, nnode, nedge, elt):
    """x (2/node) + q (4/cell) + adt (1/cell) read, res (4/cell) read and
    written (w = 2), two int32 maps of 2 per edge."""
    return (2 * nnode + 4 * ncell + ncell + 2 * 4 * ncell) * elt + 2 * 2 * 4 * nedge


def useful_bytes_hex(nelem, nnode, elt):
    """x, v (3/node) read, f (3/node) read and written, sig (3/elem) read,
    vol (1/elem) written, map 8 int32 per element."""
    return (3 * nnode + 3 * nnode + 2 * 3 * nnode + 3 * nelem + nelem) * elt + 8 * 4 * nelem


def useful_bytes_adjoint(ncell, nnode, nedge):
    """x, q, adt, res_bar read; q_bar (4/cell) and x_bar (2/node) read and
    written; two int32 maps."""
    return (2 * nnode + 4 * ncell + ncell + 4 * ncell + 2 * 4 * ncell + 2 * 2 * nnode) * 8 + 16 * nedge


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def synthetic_adt(m):
    """A positive per-cell time-step field of the magnitude the free stream
    gives on an h x h cell ((2h(|u|+|v|) + 4h)/0.9, about 5.4 h)."""
    return meshgen.positive_field(m.ncell, 5.0 * m.h, 6.0 * m.h)


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons, each line stamped with the
    host time it arrived, so that samples can be matched to a time window."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self, wait_s=3.0):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()
        t0 = time.time()
        while not self.samples and time.time() - t0 < wait_s:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm, smax = float(f[0]), float(f[1])
            except ValueError:
                continue
            reasons = [n for n, v in zip(self.NAMES, f[3:7]) if v.lower().startswith("active")]
            self.samples.append((time.time(), sm, smax, reasons))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def window(self, t0, t1, pad=0.06):
        s = [x for x in self.samples if t0 - pad <= x[0] <= t1 + pad]
        kind = "timed region"
        if not s:   # a timed region shorter than the sampling period: nearest samples
            s = sorted(self.samples, key=lambda x: min(abs(x[0] - t0), abs(x[0] - t1)))[:2]
            kind = "nearest samples to the timed region"
        if not s:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median([x[1] for x in s])), "sm_max_mhz": max(x[2] for x in s),
                "reasons": sorted({r for x in s for r in x[3]}), "samples": len(s), "window": kind}


def dist_setup():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(ms, dist, device="cpu"):
    """Slowest rank's time (replicas run independently; the job ends with
    the slowest).  ``dist`` is torch.distributed or None for one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_per_step):
    """Whole-job throughput: the units of all ranks over the slowest time."""
    return world * units_per_rank / (ms_per_step * 1e-3)


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
    """Reference arm: the FP64 CPU oracle's res_calc on the host (1 core)."""
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
            "config": {"workload": f"res_calc {args.nx}x{args.ny} jittered renumbered quads, FP64 data",
                       "cells": m.ncell, "nodes": m.nnode, "edges": m.nedge,
                       "implementation": "sequential FP64 CPU oracle (edge loop in mesh order), 1 host core"},
            "cpu_baseline": {"value": v, "unit": "Gedges/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full res_calc passes of {m.nedge} edges, 1 host core"},
            "e2e": {"value": v, "unit": "Gedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Timer:
    """CUDA-event timing of a callable on the current stream, with a
    barrier and synchronisation on both sides and max over ranks."""

    def __init__(self, torch, dist):
        self.torch, self.dist = torch, dist

    def __call__(self, fn, steps, warmup):
        torch, dist = self.torch, self.dist
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.time()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t1 = time.time()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, device="cuda")
        return ms / steps, (t0, t1)


def bench_rows(ml, torch, timer, args):
    """Measurements of the other loops (not the headline): hex assembly,
    the adjoint and the batched graph-captured time step (``--rows``)."""
    rows = {}
    want = set(args.rows.split(",")) if args.rows and args.rows != "none" else set()
    if "hex" in want:
        rows.update(bench_hex(ml, torch, timer, args))
    if "adjoint" in want:
        rows.update(bench_adjoint(ml, torch, timer, args))
    if "batch" in want:
        rows.update(bench_batch(ml, torch, timer, args))
    if "shapes" in want:
        rows.update(bench_shapes(ml, torch, timer, args))
    if "increment" in want:
        rows.update(bench_increment(ml, torch, timer, args))
    if "face" in want:
        rows.update(bench_face(ml, torch, timer, args))
    return rows


def bench_face(ml, torch, timer, args):
    """The miniAero-style face flux on the paper's mesh size (Sec. 3.1.5):
    128^3 hex cells, 6,242,304 interior faces.  FP64 (the paper's
    precision): the staged forms (28 cell values staged or increments only,
    thread colours or gather) on one partitioned plan, RCM two-layer, global
    colours, atomics and the original code's two-step temporary array;
    FP32 staged and atomics.  Useful bytes: face data and map once, cell data
    once, res read and written."""
    from paper_1802_03749_gb300.mesh import ScatterPlan
    hbm, _ = read_peaks()
    hm = meshgen.hex_mesh(128)
    f2c, fd = meshgen.hex_faces(hm)
    cd = meshgen.aero_cells(hm)
    nf, nc = f2c.shape[0], hm.nelem
    rows = {}

    def measure(S, name, dtype):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        elt = 4 if dtype == "f32" else 8
        comp = "dw" if dtype == "f64dw" else None
        fdd = torch.tensor(S.to_plan(fd, "from"), dtype=tdt, device="cuda")
        cdd = torch.tensor(S.to_plan(cd, "to"), dtype=tdt, device="cuda")
        res = torch.zeros((nc, 5), dtype=tdt, device="cuda")
        ms, _ = timer(lambda: ml.loop_face_flux(S.plan, fdd, cdd, res, compute=comp), 10, 2)
        ub = nf * (12 * elt + 8) + nc * (28 * elt + 2 * 5 * elt)
        st = S.plan.stats()
        rows[f"face_{dtype}_{name}"] = {
            "workload": f"miniAero-style face flux, {nc} hex cells, {nf} faces, "
                        + {"f64": "FP64", "f32": "FP32", "f64dw": "FP64 data, double-word arithmetic"}[dtype],
            "ms": ms,
            "gfaces_s": nf / ms / 1e6, "useful_gbs": ub / ms / 1e6, "frac_hbm": ub / ms / 1e6 / hbm,
            "block_colors": st["nblock_colors"], "reuse": st["reuse_all"]}
        del fdd, cdd, res

    S = ScatterPlan(nc, f2c, block_size=128, reorder="partition", coloring="hier")
    S.plan.upload()
    for staged in ("simple", "gather", "inc_only", "inc_only_gather"):
        S.plan.set_staged(staged)
        measure(S, f"hier_partition_{staged}", "f64")
    S.plan.set_staged(None)
    measure(S, "hier_partition_simple", "f64dw")
    measure(S, "hier_partition_simple", "f32")
    del S
    for coloring in ("hier", "global", "atomic", "twostep"):
        S = ScatterPlan(nc, f2c, block_size=128, reorder="rcm", coloring=coloring)
        S.plan.upload()
        measure(S, f"{coloring}_rcm", "f64")
        if coloring == "atomic":
            measure(S, f"{coloring}_rcm", "f32")
        del S
    return rows


def bench_increment(ml, torch, timer, args):
    """The increment-only loops at the paper's mesh sizes (Sec. 3.1.3 and
    3.1.4): the Volna-style edge loop in FP32 on 1100x1100 quads split into
    2.42M triangles (3.63M edges; the paper's mesh has 2.4M triangles and
    3.59M edges), the BookLeaf-style cell loop in FP64 on 2000x2000 quads
    (4M cells).  Useful bytes: each dataset once (twice if incremented),
    maps as int32."""
    from paper_1802_03749_gb300.mesh import ScatterPlan
    hbm, _ = read_peaks()
    rows = {}
    variants = (("hier", "partition", "gather", "aos"), ("hier", "partition", "gather", "soa"),
                ("hier", "partition", "simple", "aos"), ("hier", "rcm", "gather", "aos"),
                ("global", "rcm", None, "aos"), ("atomic", "rcm", None, "aos"), ("atomic", "rcm", None, "soa"),
                ("atomic", "none", None, "aos"), ("twostep", "rcm", None, "aos"), ("twostep", "rcm", None, "soa"))
    tm = meshgen.tri_mesh(1100, 1100)
    ed, ia = meshgen.volna_fields(tm)
    ub = tm.nedge * (7 * 4 + 4 + 2 * 4) + tm.ncell * (4 + 2 * 16)
    for coloring, reorder, staged, layout in variants:
        S = ScatterPlan(tm.ncell, tm.edge2cell, block_size=256, reorder=reorder, coloring=coloring, staged=staged,
                        layout=layout)
        S.plan.upload()
        t = lambda a, w: torch.tensor(S.to_plan(a, w), dtype=torch.float32, device="cuda")
        edd, iad = t(ed, "from"), t(ia, "to")
        fl = torch.tensor(S.to_plan(tm.eflag, "from"), dtype=torch.int32, device="cuda")
        res = torch.zeros((tm.ncell, 4), dtype=torch.float32, device="cuda")
        ms, _ = timer(lambda: ml.loop_space_disc(S.plan, edd, fl, iad, res), 20, 3)
        st = S.plan.stats()
        rows[f"space_disc_f32_{coloring}_{reorder}" + (f"_{staged}" if staged else "") + f"_{layout}"] = {
            "workload": f"Volna-style edge loop, {tm.ncell} triangles, {tm.nedge} edges, FP32", "ms": ms,
            "gedges_s": tm.nedge / ms / 1e6, "useful_gbs": ub / ms / 1e6, "frac_hbm": ub / ms / 1e6 / hbm,
            "block_colors": st["nblock_colors"], "reuse": st["reuse_all"]}
        del edd, iad, fl, res, S
    del tm, ed, ia
    qm = meshgen.quad_mesh(2000, 2000)
    cd = meshgen.bookleaf_fields(qm.ncell)
    ub = qm.ncell * (17 * 8 + 4 * 4) + qm.nnode * 2 * 32
    for coloring, reorder, staged, layout in variants:
        S = ScatterPlan(qm.nnode, qm.cell2node, block_size=256, reorder=reorder, coloring=coloring, staged=staged,
                        layout=layout)
        S.plan.upload()
        cdd = torch.tensor(S.to_plan(cd, "from"), device="cuda")
        nd = torch.zeros((qm.nnode, 4), dtype=torch.float64, device="cuda")
        ms, _ = timer(lambda: ml.loop_getacc(S.plan, cdd, nd), 20, 3)
        st = S.plan.stats()
        rows[f"getacc_f64_{coloring}_{reorder}" + (f"_{staged}" if staged else "") + f"_{layout}"] = {
            "workload": f"BookLeaf-style cell loop, {qm.ncell} quads, FP64", "ms": ms,
            "gcells_s": qm.ncell / ms / 1e6, "useful_gbs": ub / ms / 1e6, "frac_hbm": ub / ms / 1e6 / hbm,
            "block_colors": st["nblock_colors"], "reuse": st["reuse_all"]}
        del cdd, nd, S
    return rows


def bench_hex(ml, torch, timer, args):
    from paper_1802_03749_gb300.mesh import HexPlan
    hbm, _ = read_peaks()
    rows = {}
    # hex assembly, n^3 elements
    hm = meshgen.hex_mesh(args.hex_n)
    sig, v = meshgen.hex_fields(hm)
    for dtype in ("f64", "f32"):
        tdt = torch.float64 if dtype == "f64" else torch.float32
        elt = 8 if dtype == "f64" else 4
        for coloring, reorder, variant in (("hier", "partition", "simple"), ("hier", "partition", "smem_atomic"),
                                           ("hier", "partition", "warp_agg"), ("atomic", "rcm", None),
                                           ("global", "rcm", None), ("twostep", "rcm", None)):
            H = HexPlan(hm.nnode, hm.elem2node, block_size=256, reorder=reorder, coloring=coloring, staged=variant)
            H.plan.upload()
            x = torch.tensor(H.to_plan(hm.x, "node"), dtype=tdt, device="cuda")
            vd = torch.tensor(H.to_plan(v, "node"), dtype=tdt, device="cuda")
            sd = torch.tensor(H.to_plan(sig, "elem"), dtype=tdt, device="cuda")
            f = torch.zeros_like(x)
            vol = torch.zeros(hm.nelem, dtype=tdt, device="cuda")
            ms, _ = timer(lambda: ml.loop_elem_assemble(H.plan, x, vd, sd, f, vol, 0.01), 10, 2)
            ub = useful_bytes_hex(hm.nelem, hm.nnode, elt)
            st = H.plan.stats()
            rows[f"hex_{dtype}_{coloring}_{reorder}" + (f"_{variant}" if variant else "")] = {
                "workload": f"hex assembly {args.hex_n}^3 elements", "ms": ms,
                "gelems_s": hm.nelem / ms / 1e6, "useful_gbs": ub / ms / 1e6, "frac_hbm": ub / ms / 1e6 / hbm,
                "block_colors": st["nblock_colors"], "thread_colors_mean": st["mean_thread_colors"],
                "reuse": st["reuse_all"]}
            del x, vd, sd, f, vol
    # hex assembly with FP64 data in double-word arithmetic (two-layer, S = 128):
    # gather increments (default) and thread colours, partitioned and RCM
    for reorder in ("partition", "rcm"):
        H = HexPlan(hm.nnode, hm.elem2node, block_size=128, reorder=reorder, coloring="hier")
        H.plan.upload()
        x = torch.tensor(H.to_plan(hm.x, "node"), device="cuda")
        vd = torch.tensor(H.to_plan(v, "node"), device="cuda")
        sd = torch.tensor(H.to_plan(sig, "elem"), device="cuda")
        f = torch.zeros_like(x)
        vol = torch.zeros(hm.nelem, dtype=torch.float64, device="cuda")
        ub = useful_bytes_hex(hm.nelem, hm.nnode, 8)
        st = H.plan.stats()
        for staged in ("gather", "simple"):
            H.plan.set_staged(staged)
            ms, _ = timer(lambda: ml.loop_elem_assemble(H.plan, x, vd, sd, f, vol, 0.01, compute="dw"), 10, 2)
            rows[f"hex_f64dw_hier_{reorder}_{staged}"] = {
                "workload": f"hex assembly {args.hex_n}^3 elements, double-word arithmetic", "ms": ms,
                "gelems_s": hm.nelem / ms / 1e6, "useful_gbs": ub / ms / 1e6, "frac_hbm": ub / ms / 1e6 / hbm,
                "block_colors": st["nblock_colors"], "thread_colors_mean": st["mean_thread_colors"],
                "reuse": st["reuse_all"]}
        del x, vd, sd, f, vol
    return rows


def bench_shapes(ml, torch, timer, args):
    """Handcrafted block shapes on a structured hex grid (Sec. 3.1.6): 128
    elements per block as 1D lines, 2D slabs or 3D bricks, against the
    partitioner and RCM chunks, on a 128 x 64 x 64 grid the shapes tile."""
    from paper_1802_03749_gb300.mesh import HexPlan
    dims = (128, 64, 64)
    hm = meshgen.hex_mesh(dims[0], nyz=dims[1:])
    sig, v = meshgen.hex_fields(hm)
    rows = {}
    layouts = {"line_128x1x1": (128, 1, 1), "slab_16x8x1": (16, 8, 1), "brick_8x4x4": (8, 4, 4),
               "partition": None, "rcm": None}
    for name, shape in layouts.items():
        blk = meshgen.hex_bricks(hm, shape, dims) if shape else None
        reorder = "rcm" if name == "rcm" else "partition"
        for comp, staged in ((None, "smem_atomic"), (None, "simple"), ("dw", None)):
            H = HexPlan(hm.nnode, hm.elem2node, block_size=128, reorder=reorder, coloring="hier", staged=staged,
                        block_of=blk)
            H.plan.upload()
            tdt = torch.float32 if comp is None else torch.float64
            x = torch.tensor(H.to_plan(hm.x, "node"), dtype=tdt, device="cuda")
            vd = torch.tensor(H.to_plan(v, "node"), dtype=tdt, device="cuda")
            sd = torch.tensor(H.to_plan(sig, "elem"), dtype=tdt, device="cuda")
            f = torch.zeros_like(x)
            vol = torch.zeros(hm.nelem, dtype=tdt, device="cuda")
            ms, _ = timer(lambda: ml.loop_elem_assemble(H.plan, x, vd, sd, f, vol, 0.01, compute=comp), 10, 2)
            st = H.plan.stats()
            key = f"hex_shape_{name}_" + ("f64dw" if comp else f"f32_{staged}")
            rows[key] = {"workload": "hex assembly 128x64x64, blocks of 128", "ms": ms,
                         "gelems_s": hm.nelem / ms / 1e6, "reuse": st["reuse_all"],
                         "thread_colors_mean": st["mean_thread_colors"], "block_colors": st["nblock_colors"]}
            del x, vd, sd, f, vol
    return rows


def bench_adjoint(ml, torch, timer, args):
    from paper_1802_03749_gb300.mesh import AirfoilPlans
    hbm, _ = read_peaks()
    rows = {}
    # adjoint, 1200x600
    am = meshgen.quad_mesh(1200, 600)
    aq = meshgen.quad_state(am.ncell)
    aadt = synthetic_adt(am)
    rb = meshgen.adjoint_seed(am.ncell)
    for coloring, reorder, comp, staged in (("hier", "partition", None, None), ("hier", "partition", "dw", "gather"),
                                            ("hier", "partition", "dw", "simple"), ("atomic", "rcm", None, None)):
        P = AirfoilPlans(am.ncell, am.nnode, am.edge2node, am.edge2cell, am.bedge2node, am.bedge2cell, am.cell2node,
                         block_size=256 if comp else 384, reorder=reorder, coloring=coloring, adjoint=True,
                         staged=staged)
        P.res.upload()
        t = lambda a, w: torch.tensor(P.to_plan(a, w), device="cuda")
        x, qd, ad, rbd = t(am.x, "node"), t(aq, "cell"), t(aadt, "cell"), t(rb, "cell")
        qb, xb = torch.zeros_like(qd), torch.zeros_like(x)
        ms, _ = timer(lambda: ml.loop_adjoint(P.res, x, qd, ad, rbd, qb, xb, compute=comp), 10, 2)
        ub = useful_bytes_adjoint(am.ncell, am.nnode, am.nedge)
        rows[f"adjoint_{'f64dw' if comp else 'f64'}_{coloring}_{reorder}" + (f"_{staged}" if staged else "")] = {
            "workload": "res_calc adjoint 1200x600", "ms": ms, "gedges_s": am.nedge / ms / 1e6,
            "useful_gbs": ub / ms / 1e6, "frac_hbm": ub / ms / 1e6 / hbm}
    return rows


def bench_batch(ml, torch, timer, args):
    from paper_1802_03749_gb300 import autotune
    from paper_1802_03749_gb300.mesh import AirfoilBatch, AirfoilPlans, AirfoilStep
    rows = {}
    # batched time step: meshes of uneven size, FP32 data, FP64 update and sum
    sizes = meshgen.batch_sizes(args.batch)
    meshes = [meshgen.quad_mesh(nx, ny, seed=meshgen.DEFAULT_SEED + 97 * i) for i, (nx, ny) in enumerate(sizes)]
    states = [meshgen.quad_state(mm.ncell, seed=meshgen.DEFAULT_SEED + 97 * i) for i, mm in enumerate(meshes)]
    adts = [synthetic_adt(mm) for mm in meshes]
    qinf = meshgen.freestream()
    tune_t0 = time.time()
    tuned, choices = autotune.tune(meshes, states, adts, dtype="f32", reps=10)
    tune_s = time.time() - tune_t0
    B = AirfoilBatch(meshes, states, qinf, choices, dtype="f32")
    B.capture(steps_per_graph=1)
    ms_graph, _ = timer(lambda: B.graph.replay(), 20, 3)
    ms_batch_eager, _ = timer(B.step, 20, 3)
    per = [AirfoilStep(AirfoilPlans(mm.ncell, mm.nnode, mm.edge2node, mm.edge2cell, mm.bedge2node, mm.bedge2cell,
                                    mm.cell2node, block_size=480, reorder="partition"), mm.x, s, qinf, dtype="f32")
           for mm, s in zip(meshes, states)]

    def per_mesh():
        for S in per:
            S.step()

    ms_per, _ = timer(per_mesh, 5, 1)
    cells = sum(mm.ncell for mm in meshes)
    edges = sum(mm.nedge for mm in meshes)
    rows["batch_step_f32"] = {
        "workload": f"{args.batch} quad meshes, {cells} cells, {edges} edges, full time step, FP32 data, "
                    "FP64 update and residual sum",
        "ms_graph_batched": ms_graph, "ms_eager_batched": ms_batch_eager, "ms_per_mesh_launches": ms_per,
        "speedup_vs_per_mesh": ms_per / ms_graph, "gedges_s": edges / ms_graph / 1e6,
        "autotune": tuned, "autotune_seconds": tune_s}
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block-size", type=int, default=256)
    ap.add_argument("--layout", default="aos", choices=["aos", "soa"])
    ap.add_argument("--staged", default=None, choices=["simple", "gather", "smem_atomic", "pipelined"],
                    help="increment form of the staged headline kernel (default: the library's)")
    ap.add_argument("--compute", default="dw", choices=["dw", "f64", "f32"],
                    help="dw: FP64 data with double-word arithmetic; f64: native FP64; f32: FP32 data")
    ap.add_argument("--no-variants", action="store_true", help="skip the baseline variants")
    ap.add_argument("--rows", default="hex,adjoint,batch,shapes,increment,face",
                    help="other loops to measure (comma list of hex, adjoint, batch, shapes, increment, face; "
                         "none for none)")
    ap.add_argument("--no-rows", action="store_true", help="skip the hex / adjoint / batch measurements")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--nx", type=int, default=NX, help="quad grid size (profiling runs use smaller meshes)")
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--hex-n", type=int, default=120)
    ap.add_argument("--batch", type=int, default=64)
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
    timer = Timer(torch, dist)

    m = meshgen.quad_mesh(args.nx, args.ny)
    q = meshgen.quad_state(m.ncell)
    adt = synthetic_adt(m)
    f32 = args.compute == "f32"
    tdt = torch.float32 if f32 else torch.float64
    elt = 4 if f32 else 8
    compute = "dw" if args.compute == "dw" else None
    useful = useful_bytes_res_calc(m.ncell, m.nnode, m.nedge, elt)
    hbm_peak, peak_kind = read_peaks()

    def setup(coloring, reorder, layout=args.layout, bs=args.block_size, staged=None, recolor=-1):
        P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                         block_size=bs, reorder=reorder, coloring=coloring, layout=layout, staged=staged,
                         recolor=recolor)
        P.res.upload()
        d = {"x": torch.tensor(P.to_plan(m.x, "node"), dtype=tdt, device="cuda"),
             "q": torch.tensor(P.to_plan(q, "cell"), dtype=tdt, device="cuda"),
             "adt": torch.tensor(P.to_plan(adt, "cell"), dtype=tdt, device="cuda")}
        d["res"] = torch.zeros_like(d["q"])
        return P, d

    # ---------------------------------------------------------- headline
    P, d = setup("hier", "partition", staged=args.staged)
    st = P.res.stats()
    step = lambda: ml.loop_res_calc(P.res, d["x"], d["q"], d["adt"], d["res"], GAM, EPS, compute=compute)
    clk = ClockSampler(local)
    clk.start()
    ms_step, (t0, t1) = timer(step, args.steps, args.warmup)
    clocks = clk.window(t0, t1)
    value = job_rate(m.nedge, world, ms_step) / 1e9
    gbs = useful / (ms_step * 1e-3) / 1e9
    if args.compute == "f64":
        roof = {"bound": "alu", "achieved": FLOPS_PER_EDGE * m.nedge / ms_step / 1e9, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_kind": "derived FP64 FMA rate (152 SMs x 2 DFMA/clk x 2.07 GHz)"}
    elif args.compute == "dw":
        roof = {"bound": "alu", "achieved": FLOPS_PER_EDGE * m.nedge / ms_step / 1e9, "peak": DW_PEAK_TFLOPS,
                "unit": "TFLOP/s",
                "peak_kind": "derived double-word rate: FP32 issue (152 SMs x 128 lanes x 2.07 GHz) / "
                             f"{DW_FP32_OPS_PER_OP} FP32 operations per double-word operation; "
                             f"FP64-equivalent flops (the FP64 pipe's own peak is {FP64_PEAK_TFLOPS:.3f})"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "peak_kind": f"{peak_kind} copy bandwidth (burst)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    head_staged = args.staged or ("simple" if args.compute == "f64" else "gather")
    roof["traffic"] = headline_traffic(args, head_staged)
    roof["traffic_scope"] = "DRAM bytes per pass (all block-colour launches), as achieved; ncu capture"
    roof["useful_bytes"] = useful
    # the data reuse measure of the plan: useful bytes / DRAM bytes per pass
    roof["useful_over_dram"] = useful / roof["traffic"] if roof["traffic"] else None

    # ---------------------------------------------------------- e2e (host buffers)
    # through the C-ABI call with host arrays (loop_res_calc_host): every step
    # copies its inputs from pinned host memory and reads res back; steps
    # alternate two streams and two sets of host arrays, so one step's copies
    # overlap the other's loop
    hsets = []
    for _ in range(2):
        hsets.append([torch.tensor(P.to_plan(m.x, "node"), dtype=tdt).pin_memory(),
                      torch.tensor(P.to_plan(q, "cell"), dtype=tdt).pin_memory(),
                      torch.tensor(P.to_plan(adt, "cell"), dtype=tdt).pin_memory(),
                      torch.zeros((m.ncell, 4), dtype=tdt).pin_memory()])
    e2e_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    e2e_k = [0]

    def e2e_step():
        k = e2e_k[0]
        e2e_k[0] += 1
        ml.loop_res_calc_host(P.res, *hsets[k % 2], GAM, EPS, stream=e2e_streams[k % 2], compute=compute)

    def e2e_timed(n, w):
        for _ in range(w):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            e2e_step()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / n

    e2e_ms = e2e_timed(max(4, min(args.steps, 20)), 3)
    h2d = sum(t.numel() for t in hsets[0]) * elt
    d2h = hsets[0][3].numel() * elt
    launches = args.steps * st["nblock_colors"]
    del d

    # ---------------------------------------------------------- variants
    head_name = "two_layer_partition" + ("_dw" if compute else "") + f"_{head_staged}"
    variants = {head_name: {
        "gedges_s": value / world, "ms": ms_step, "useful_gbs": gbs, "block_colors": st["nblock_colors"],
        "thread_colors_mean": st["mean_thread_colors"], "reuse": st["reuse_all"],
        "plan_seconds": st["seconds_total"]}}
    if not args.no_variants:
        ks = max(5, args.steps // 2)
        other = "gather" if head_staged != "gather" else "simple"
        todo = [("two_layer_partition" + ("_dw" if compute else "") + f"_{other}", "hier", "partition",
                 compute, other),
                ("two_layer_partition" + ("_dw" if compute else "") + "_first_fit_colours", "hier", "partition",
                 compute, args.staged, 0),
                ("two_layer_rcm", "hier", "rcm", compute, args.staged), ("global_rcm", "global", "rcm", None, None),
                ("global_none", "global", "none", None, None), ("atomic_rcm", "atomic", "rcm", None, None),
                ("atomic_none", "atomic", "none", None, None), ("twostep_rcm", "twostep", "rcm", None, None)]
        pre = "two_layer_partition_" + ("native_f64_" if compute else "")
        todo += [(pre + "smem_atomic", "hier", "partition", None, "smem_atomic"),
                 (pre + "warp_agg", "hier", "partition", None, "warp_agg")]
        if compute == "dw":
            todo.insert(1, ("two_layer_partition_native_f64", "hier", "partition", None, None))
            todo.insert(2, ("two_layer_partition_native_f64_gather", "hier", "partition", None, "gather"))
        for name, coloring, reorder, comp, stg, *rc in todo:
            try:
                Pv, dv = setup(coloring, reorder, staged=stg, recolor=rc[0] if rc else -1)
            except ml.MeshLoopError as e:
                variants[name] = {"error": str(e)}
                continue
            fn = lambda: ml.loop_res_calc(Pv.res, dv["x"], dv["q"], dv["adt"], dv["res"], GAM, EPS, compute=comp)
            msv, _ = timer(fn, ks, 2)
            variants[name] = {"gedges_s": m.nedge / msv / 1e6, "ms": msv, "useful_gbs": useful / msv / 1e6,
                              "colors": Pv.res.stats()["nblock_colors"]}
            del dv, Pv

    rows = None if args.no_rows else bench_rows(ml, torch, timer, args)
    clk.stop()

    # ---------------------------------------------------------- CPU baseline (oracle)
    cpu = None
    if rank == 0 and args.cpu_seconds > 0:
        r, n, dt = oracle_res_calc_rate(m, q, adt, args.cpu_seconds)
        cpu = {"value": r, "unit": "Gedges/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} full FP64 res_calc passes of the same mesh ({m.nedge} edges), {dt:.1f} s on 1 core"}

    if rank == 0:
        dtype = {"dw": "f64dw", "f64": "f64", "f32": "f32"}[args.compute]
        line = {
            "metric": METRIC, "value": value, "unit": "Gedges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": f"res_calc {args.nx}x{args.ny} jittered renumbered quads, "
                                   + ("FP32 data" if f32 else "FP64 data"),
                       "cells": m.ncell, "nodes": m.nnode, "edges": m.nedge,
                       "implementation": ("double-word arithmetic, " if compute else "")
                                         + f"two-layer colouring"
                                         + f" ({'thread-coloured' if head_staged == 'simple' else head_staged}"
                                         + f" increments), RCM + partition, block {args.block_size}, "
                                         + args.layout.upper(),
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 (useful bytes {useful / 1e6:.0f} MB > {L2_BYTES / 1e6:.0f} MB)"},
            "useful_gbs": gbs, "useful_frac_hbm": gbs / hbm_peak,
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": world * m.nedge / e2e_ms / 1e6, "unit": "Gedges/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clocks,
            "plan": {"blocks": st["nblocks"], "block_colors": st["nblock_colors"],
                     "thread_colors_max": st["max_thread_colors"], "reuse": st["reuse_all"],
                     "plan_seconds": st["seconds_total"]},
            "variants": variants, "rows": rows,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
