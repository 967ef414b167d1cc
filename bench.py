"""Benchmark of the locality-optimised res_calc loop, its baselines and the
other loops of the library, on synthetic meshes shaped like the paper's.

Headline workload: res_calc on a jittered, randomly renumbered 2400x1200 quad
mesh (2,880,000 cells, 5,756,400 interior edges) with FP64 data and native
FP64 arithmetic (the paper's precision, Table 2), through the C ABI.  A step
is one full res_calc pass (every block colour) of the two-layer staged
kernel on an RCM + partition plan.  The metric is interior edges per second;
useful bandwidth follows the paper's formula (Sec. 3.1: each dataset once,
twice if read and written, maps as int32 datasets).

Timing protocol: after max(W, 10) warm-up calls, 5 repetitions of n calls
(n >= max(K, 100) and long enough for 0.1 s per repetition), each bracketed
by a barrier and a device synchronisation and timed by CUDA events on the
launching stream; the median repetition gives ms per call.  Two regimes:
warm (calls back to back; the inputs exceed L2) and L2-flushed (a write of
twice the L2 size before every call, each call timed by its own events).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--compute f64|dw|f32]

Prints one JSON line on rank 0.  Under torchrun every rank runs an
independent replica of the workload (no collective on the data path); the
value is the edges of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
REPS = 5
MIN_CALLS = 100
MIN_WARMUP = 10
MIN_REP_SECONDS = 0.1
FIELDS = ("rho", "rho_u", "rho_v", "E")
# block size S of the two-layer plans per arithmetic, the fastest measured on
# the 2400x1200 pass (FP64: 0.496 / 0.487 / 0.483 / 0.478 / 0.492 ms at S =
# 192 / 256 / 320 / 384 / 512; double-word and FP32: 256)
BLOCK_DEFAULT = {"f64": 384, "dw": 256, "f32": 256}

# algorithmic floating-point operations of one interior edge as the oracle
# evaluates it: two normal fluxes of 20 (pressure 7, normal velocity 4,
# components 9), the normal 2, mu 3, four flux components of 5, two
# increments of 4 components
FLOPS_PER_EDGE = 73
# FP64 FMA throughput of GB300: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 FMA throughput: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# DRAM traffic records: one text file per configuration under profiles/,
# written by --record-traffic from an ncu CSV of the headline kernel
TRAFFIC_SOURCES = ("loops_res.cu", "loops_res_dw.cu", "rows.cuh", "dw.cuh", "common.cuh", "plan_internal.h",
                   "plan.cpp")
HEAD_KERNEL = {"f64": "res_calc_hier_g", "f32": "res_calc_hier_g", "dw": "res_calc_hier_dw"}


def sources_sha256():
    """Hash of the sources the headline kernels and their plans compile from."""
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1802_03749_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_path(compute, nx, ny):
    return os.path.join(ROOT, "profiles", f"traffic_res_calc_{compute}_{nx}x{ny}.txt")


def read_traffic(compute, staged, args):
    """The recorded DRAM bytes of one headline pass when the record's
    configuration and source hash match the running one, else None (with
    the reason)."""
    p = traffic_path(compute, args.nx, args.ny)
    if not os.path.exists(p):
        return None, "no capture recorded for this configuration"
    rec = {}
    with open(p) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                rec[k.strip()] = v.strip()
    want = {"compute": compute, "staged": staged, "block": str(args.block_size or BLOCK_DEFAULT[compute]),
            "layout": args.layout}
    if any(rec.get(k) != v for k, v in want.items()):
        return None, "recorded for another launch configuration"
    if rec.get("sources_sha256") != sources_sha256():
        return None, "kernel or planner sources changed since the capture"
    return {k: (int(v) if v.isdigit() else v) for k, v in rec.items()}, "ncu capture of the current sources"


def record_traffic(args):
    """Write profiles/traffic_res_calc_<compute>_<nx>x<ny>.txt from an ncu CSV
    (``--csv --print-units base --metrics dram__bytes_read.sum,
    dram__bytes_write.sum,gpu__time_duration.sum``) of consecutive headline
    passes: DRAM bytes per pass = bytes over the captured launches x the
    launches of one pass / captured launches."""
    import csv
    rows = {}
    with open(args.record_traffic) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        if HEAD_KERNEL[args.compute] + "<" not in r.get("Kernel Name", "") and \
                HEAD_KERNEL[args.compute] + "(" not in r.get("Kernel Name", ""):
            continue
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1, "usecond": 1e3,
                 "msecond": 1e6}.get(r["Metric Unit"], 1)
        rows.setdefault(r["ID"], {})[r["Metric Name"]] = float(r["Metric Value"].replace(",", "")) * scale
    if not rows:
        raise SystemExit(f"no {HEAD_KERNEL[args.compute]} launches in {args.record_traffic}")
    n = len(rows)
    lpp = args.launches_per_pass
    rd = sum(v.get("dram__bytes_read.sum", 0) for v in rows.values())
    wr = sum(v.get("dram__bytes_write.sum", 0) for v in rows.values())
    ns = sum(v.get("gpu__time_duration.sum", 0) for v in rows.values())
    staged = args.staged or default_staged(args.compute)
    out = traffic_path(args.compute, args.nx, args.ny)
    with open(out, "w") as f:
        f.write(f"# DRAM traffic of one res_calc pass ({lpp} block-colour launches of {HEAD_KERNEL[args.compute]}),\n"
                f"# {args.nx}x{args.ny} quads, from {n} consecutive launches captured with ncu --cache-control none\n"
                f"# (dirty lines of one launch are written back during the following ones, so writes are counted).\n"
                f"# command: {args.record_command}\n")
        for k, v in (("compute", args.compute), ("staged", staged),
                     ("block", args.block_size or BLOCK_DEFAULT[args.compute]),
                     ("layout", args.layout), ("nx", args.nx), ("ny", args.ny), ("launches_captured", n),
                     ("launches_per_pass", lpp), ("read_bytes_per_pass", int(round(rd * lpp / n))),
                     ("write_bytes_per_pass", int(round(wr * lpp / n))),
                     ("bytes_per_pass", int(round((rd + wr) * lpp / n))),
                     ("ncu_ns_per_pass", int(round(ns * lpp / n))), ("sources_sha256", sources_sha256())):
            f.write(f"{k}={v}\n")
    print(open(out).read())


def default_staged(compute):
    """The library's default increment form of the headline kernel."""
    return "gather"


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


def rel_l2(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / (nb if nb > 0 else 1.0))


def field_errors(got, ref):
    """rel-L2 over all components and per field (rho, rho u, rho v, E)."""
    return {"rel_l2": rel_l2(got, ref), "per_field": {f: rel_l2(got[:, k], ref[:, k]) for k, f in enumerate(FIELDS)}}


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
                pw = float(f[2])
            except ValueError:
                continue
            reasons = [n for n, v in zip(self.NAMES, f[3:7]) if v.lower().startswith("active")]
            self.samples.append((time.time(), sm, smax, reasons, pw))

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
                "sm_mhz_min": min(x[1] for x in s), "power_w_max": max(x[4] for x in s),
                "reasons": sorted({r for x in s for r in x[3]}), "samples": len(s), "window": kind,
                "seconds": round(t1 - t0, 3)}


def dist_setup():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(vals, dist, device="cpu"):
    """Element-wise slowest rank's times (replicas run independently; the
    job ends with the slowest).  ``dist`` is torch.distributed or None."""
    if dist is None:
        return list(vals)
    import torch
    t = torch.tensor(list(vals), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_rate(units_per_rank, world, ms_per_step):
    """Whole-job throughput: the units of all ranks over the slowest time."""
    return world * units_per_rank / (ms_per_step * 1e-3)


class Protocol:
    """CUDA-event timing on the current stream after the measurement
    protocol: warm-up calls, then repetitions of n calls, each bracketed by
    a barrier and a device synchronisation; the median repetition (max over
    ranks) gives ms per call.  ``flushed`` writes a buffer of twice the L2
    size before every call and times each call by its own event pair."""

    def __init__(self, torch, dist):
        self.torch, self.dist = torch, dist
        self.flush_buf = None

    def _fence(self):
        torch = self.torch
        torch.cuda.synchronize()
        if self.dist is not None:
            self.dist.barrier()
        torch.cuda.synchronize()

    def calls_for(self, fn, min_calls, warmup):
        """Warm up, then the calls per repetition: at least ``min_calls`` and
        enough for MIN_REP_SECONDS at the estimated rate."""
        torch = self.torch
        for _ in range(warmup):
            fn()
        self._fence()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        e0.record(s)
        for _ in range(10):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        est = max(e0.elapsed_time(e1) / 10, 1e-4)
        n = max(min_calls, int(math.ceil(MIN_REP_SECONDS * 1e3 / est)))
        return int(max_over_ranks([n], self.dist, "cuda")[0])

    def warm(self, fn, calls, reps):
        torch = self.torch
        s = torch.cuda.current_stream()
        times = []
        t0 = time.time()
        for _ in range(reps):
            self._fence()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(calls):
                fn()
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / calls)
        t1 = time.time()
        times = max_over_ranks(times, self.dist, "cuda")
        return float(np.median(times)), times, (t0, t1)

    def flushed(self, fn, calls, reps):
        torch = self.torch
        if self.flush_buf is None:
            self.flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
        times = []
        t0 = time.time()
        for r in range(reps):
            self._fence()
            for i in range(calls):
                self.flush_buf.fill_(r * calls + i)
                ev[i][0].record(s)
                fn()
                ev[i][1].record(s)
            torch.cuda.synchronize()
            times.append(sum(a.elapsed_time(b) for a, b in ev) / calls)
        t1 = time.time()
        times = max_over_ranks(times, self.dist, "cuda")
        return float(np.median(times)), times, (t0, t1)

    def __call__(self, fn, calls, warmup, reps=3):
        """Warm regime with ``calls`` calls per repetition (the other loops'
        rows): median ms per call and the host time window."""
        for _ in range(warmup):
            fn()
        ms, _, win = self.warm(fn, calls, reps)
        return ms, win


def oracle_leg(m, q, adt, budget_s):
    """CPU baseline: the oracle's sequential FP64 res_calc on the host,
    repeated for about ``budget_s`` seconds.  Its result is kept: it is the
    expected value of the error figures reported beside each GPU variant."""
    import oracle
    res = np.zeros((m.ncell, 4))
    n = 0
    t0 = time.perf_counter()
    while True:
        res[:] = 0.0
        oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt, res=res)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    return n * m.nedge / dt / 1e9, n, dt, res


def oracle_res_f32_inputs(m, q, adt):
    """The oracle's FP64 res_calc on the FP32-rounded inputs: what the FP32
    path computes, up to its own arithmetic."""
    import oracle
    r = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
    return oracle.res_calc(m.edge2node, m.edge2cell, r(m.x), r(q), r(adt))


def precision_rows(ml, torch, steps=(1, 2, 5, 10, 20, 50, 100)):
    """FP32 storage with the FP64 update and residual sum, against the FP64
    oracle, per field and per step count: the 200x100 Airfoil-style time
    step (save_soln, adt_calc, res_calc, bres_calc, update).  Reported: q's
    rel-L2 per field (against the oracle started from the FP32-rounded state
    and from the exact state), the rel-L2 of the accumulated change
    q_k - q_0, and the relative error of the RMS residual."""
    import oracle
    from paper_1802_03749_gb300.mesh import AirfoilPlans, AirfoilStep
    m = meshgen.quad_mesh(200, 100)
    q0 = meshgen.quad_state(m.ncell)
    qinf = meshgen.freestream()
    P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                     block_size=256, reorder="partition", coloring="hier")
    S = AirfoilStep(P, m.x, q0, qinf, dtype="f32")
    q_s = q0.astype(np.float32).astype(np.float64)   # the stored initial state
    q_r = q_s.copy()                                  # the oracle from the stored initial state
    q_e = q0.copy()                                   # the oracle from the exact state
    out = {}
    for k in range(1, max(steps) + 1):
        S.rms.zero_()
        S.step()
        torch.cuda.synchronize()
        rms_ref, _ = oracle.step(m, q_r, qinf)
        oracle.step(m, q_e, qinf)
        if k in steps:
            got = S.q_original()
            rms = float(np.sqrt(S.rms.item() / m.ncell))
            out[str(k)] = {
                "q_per_field": {f: rel_l2(got[:, i], q_r[:, i]) for i, f in enumerate(FIELDS)},
                "q_per_field_vs_exact_start": {f: rel_l2(got[:, i], q_e[:, i]) for i, f in enumerate(FIELDS)},
                "dq_per_field": {f: rel_l2(got[:, i] - q_s[:, i], q_r[:, i] - q_s[:, i]) for i, f in enumerate(FIELDS)},
                "rms_rel_err": abs(rms - rms_ref) / rms_ref}
    return {"workload": "Airfoil-style time step 200x100, FP32 storage and arithmetic, FP64 update and residual sum, "
                        "against the FP64 oracle", "steps": out}


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


def bench_rows(ml, torch, timer, args):
    """Measurements of the other loops (not the headline, ``--rows``): hex
    assembly, the adjoint, the batched graph-captured time step, handcrafted
    block shapes, the increment-only loops, the face flux and the FP32
    error per field and step count.  ``timer(fn, calls, warmup)`` is the
    warm regime of the protocol with 3 repetitions."""
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
    if "precision" in want and dist_setup()[1] == 0:
        rows["precision_f32_steps"] = precision_rows(ml, torch)
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
    """The increment-only loops at the paper's mesh sizes (Sec. 3.1.2 and
    3.1.3): the Volna-style edge loop in FP32 on 1100x1100 quads split into
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
    # hex assembly with FP64 data in double-word arithmetic: two-layer (S =
    # 128; gather increments, the default, and thread colours, partitioned
    # and RCM) and the atomics and global-colour baselines in the same
    # arithmetic
    for coloring, reorder in (("hier", "partition"), ("hier", "rcm"), ("atomic", "rcm"), ("global", "rcm")):
        H = HexPlan(hm.nnode, hm.elem2node, block_size=128, reorder=reorder, coloring=coloring)
        H.plan.upload()
        x = torch.tensor(H.to_plan(hm.x, "node"), device="cuda")
        vd = torch.tensor(H.to_plan(v, "node"), device="cuda")
        sd = torch.tensor(H.to_plan(sig, "elem"), device="cuda")
        f = torch.zeros_like(x)
        vol = torch.zeros(hm.nelem, dtype=torch.float64, device="cuda")
        ub = useful_bytes_hex(hm.nelem, hm.nnode, 8)
        st = H.plan.stats()
        for staged in (("gather", "simple") if coloring == "hier" else (None,)):
            if staged:
                H.plan.set_staged(staged)
            ms, _ = timer(lambda: ml.loop_elem_assemble(H.plan, x, vd, sd, f, vol, 0.01, compute="dw"), 10, 2)
            rows[f"hex_f64dw_{coloring}_{reorder}" + (f"_{staged}" if staged else "")] = {
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


ADJ_BLOCK = 320  # native adjoint, gather form (fastest of 128-512)


def bench_adjoint(ml, torch, timer, args):
    from paper_1802_03749_gb300.mesh import AirfoilPlans
    hbm, _ = read_peaks()
    rows = {}
    # adjoint, 1200x600
    am = meshgen.quad_mesh(1200, 600)
    aq = meshgen.quad_state(am.ncell)
    aadt = synthetic_adt(am)
    rb = meshgen.adjoint_seed(am.ncell)
    for coloring, reorder, comp, staged, bs in (("hier", "partition", None, "gather", ADJ_BLOCK),
                                                ("hier", "partition", None, "simple", 384),
                                                ("hier", "partition", "dw", "gather", 192),
                                                ("hier", "partition", "dw", "simple", 256),
                                                ("atomic", "rcm", None, None, 256), ("global", "rcm", None, None, 256),
                                                ("atomic", "rcm", "dw", None, 256), ("global", "rcm", "dw", None, 256)):
        P = AirfoilPlans(am.ncell, am.nnode, am.edge2node, am.edge2cell, am.bedge2node, am.bedge2cell, am.cell2node,
                         block_size=bs, reorder=reorder, coloring=coloring, adjoint=True, staged=staged)
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
    # the fused res_calc as one persistent launch for all colour phases
    Bp = AirfoilBatch(meshes, states, qinf, choices, dtype="f32", res_staged="persistent")
    Bp.capture(steps_per_graph=1)
    ms_graph_persistent, _ = timer(lambda: Bp.graph.replay(), 20, 3)
    del Bp
    # the same meshes with the same plans (the autotuner's choice per mesh),
    # one step per mesh: eagerly (64 launch sequences) and as 64 graphs
    per = [AirfoilStep(AirfoilPlans(mm.ncell, mm.nnode, mm.edge2node, mm.edge2cell, mm.bedge2node, mm.bedge2cell,
                                    mm.cell2node, block_size=c[0], reorder=c[1], coloring=c[2]), mm.x, s, qinf,
                       dtype="f32")
           for mm, s, c in zip(meshes, states, choices)]

    def per_mesh():
        for S in per:
            S.step()

    ms_per, _ = timer(per_mesh, 5, 1)
    for S in per:
        S.capture(steps_per_graph=1)

    def per_mesh_graphs():
        for S in per:
            S.graph.replay()

    ms_per_graphs, _ = timer(per_mesh_graphs, 10, 2)
    cells = sum(mm.ncell for mm in meshes)
    edges = sum(mm.nedge for mm in meshes)
    rows["batch_step_f32"] = {
        "workload": f"{args.batch} quad meshes, {cells} cells, {edges} edges, full time step, FP32 data, "
                    "FP64 update and residual sum",
        "ms_graph_batched": ms_graph, "ms_graph_batched_persistent_res_calc": ms_graph_persistent,
        "ms_eager_batched": ms_batch_eager, "ms_per_mesh_launches": ms_per,
        "ms_per_mesh_graphs": ms_per_graphs, "speedup_vs_per_mesh": ms_per / ms_graph,
        "speedup_vs_per_mesh_graphs": ms_per_graphs / ms_graph, "gedges_s": edges / ms_graph / 1e6,
        "autotune": tuned, "autotune_seconds": tune_s}
    return rows


def res_variants(compute_head):
    """The comparison matrix of res_calc: (plan key, name, arithmetic,
    staged form).  Plans: (colouring, reordering, layout, first-fit colours)."""
    part, part_ff, rcm = ("hier", "partition", "aos", False), ("hier", "partition", "aos", True), \
        ("hier", "rcm", "aos", False)
    g_rcm, g_none = ("global", "rcm", "aos", False), ("global", "none", "aos", False)
    a_rcm, a_none = ("atomic", "rcm", "aos", False), ("atomic", "none", "aos", False)
    t_rcm = ("twostep", "rcm", "aos", False)
    part_soa, a_rcm_soa = ("hier", "partition", "soa", False), ("atomic", "rcm", "soa", False)
    g_rcm_soa = ("global", "rcm", "soa", False)
    v = [
        # FP64 data, native FP64 arithmetic (the paper's precision)
        (part, "two_layer_partition_f64_simple", "f64", "simple"),
        (part, "two_layer_partition_f64_gather", "f64", "gather"),
        (part, "two_layer_partition_f64_smem_atomic", "f64", "smem_atomic"),
        (part, "two_layer_partition_f64_warp_agg", "f64", "warp_agg"),
        (part, "two_layer_partition_f64_pipelined", "f64", "pipelined"),
        (part, "two_layer_partition_f64_persistent", "f64", "persistent"),
        (part_ff, "two_layer_partition_f64_first_fit_colours", "f64", "simple"),
        (rcm, "two_layer_rcm_f64", "f64", None),
        (g_rcm, "global_rcm_f64", "f64", None), (g_none, "global_none_f64", "f64", None),
        (a_rcm, "atomic_rcm_f64", "f64", None), (a_none, "atomic_none_f64", "f64", None),
        (t_rcm, "twostep_rcm_f64", "f64", None),
        # FP64 data, double-word arithmetic on the FP32 pipes
        (part, "two_layer_partition_dw_gather", "dw", "gather"),
        (part, "two_layer_partition_dw_simple", "dw", "simple"),
        (part_ff, "two_layer_partition_dw_first_fit_colours", "dw", "gather"),
        (rcm, "two_layer_rcm_dw", "dw", None),
        (g_rcm, "global_rcm_dw", "dw", None), (g_none, "global_none_dw", "dw", None),
        (a_rcm, "atomic_rcm_dw", "dw", None), (a_none, "atomic_none_dw", "dw", None),
        # FP32 data and arithmetic
        (part, "two_layer_partition_f32_gather", "f32", "gather"),
        (part, "two_layer_partition_f32_simple", "f32", "simple"),
        (part, "two_layer_partition_f32_smem_atomic", "f32", "smem_atomic"),
        (part, "two_layer_partition_f32_pipelined", "f32", "pipelined"),
        (part, "two_layer_partition_f32_persistent", "f32", "persistent"),
        (rcm, "two_layer_rcm_f32", "f32", None),
        (part_soa, "two_layer_partition_f32_gather_soa", "f32", "gather"),
        (g_rcm, "global_rcm_f32", "f32", None), (g_rcm_soa, "global_rcm_f32_soa", "f32", None),
        (a_rcm, "atomic_rcm_f32", "f32", None), (a_rcm_soa, "atomic_rcm_f32_soa", "f32", None),
        (t_rcm, "twostep_rcm_f32", "f32", None),
    ]
    return v


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=MIN_CALLS,
                    help="least calls per timed repetition (raised to 100 and to 0.1 s per repetition)")
    ap.add_argument("--warmup", type=int, default=MIN_WARMUP, help="warm-up calls (at least 10)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block-size", type=int, default=None,
                    help="block size S of the two-layer plans (default: 384 for FP64, 256 otherwise)")
    ap.add_argument("--layout", default="aos", choices=["aos", "soa"])
    ap.add_argument("--staged", default=None,
                    choices=["simple", "gather", "smem_atomic", "pipelined", "warp_agg", "persistent"],
                    help="increment form of the staged headline kernel (default: the library's)")
    ap.add_argument("--compute", default="f64", choices=["f64", "dw", "f32"],
                    help="f64: FP64 data and arithmetic (the paper's); dw: FP64 data with double-word "
                         "arithmetic; f32: FP32 data")
    ap.add_argument("--no-variants", action="store_true", help="skip the baseline variants")
    ap.add_argument("--variants", default=None,
                    help="comma list of the variants to measure (default: all; e.g. atomic_rcm_f32_soa)")
    ap.add_argument("--rows", default="hex,adjoint,batch,shapes,increment,face,precision",
                    help="other loops to measure (comma list of hex, adjoint, batch, shapes, increment, face, "
                         "precision; none for none)")
    ap.add_argument("--no-rows", action="store_true", help="skip the other loops")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--nx", type=int, default=NX, help="quad grid size (profiling runs use smaller meshes)")
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--hex-n", type=int, default=120)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--record-traffic", default=None, metavar="CSV",
                    help="write the DRAM-traffic record of the headline configuration from an ncu CSV and exit")
    ap.add_argument("--launches-per-pass", type=int, default=4)
    ap.add_argument("--record-command", default="", help="the ncu command line the CSV came from")
    args = ap.parse_args()
    if args.record_traffic:
        return record_traffic(args)
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
    proto = Protocol(torch, dist)
    warmup = max(args.warmup, MIN_WARMUP)

    m = meshgen.quad_mesh(args.nx, args.ny)
    q = meshgen.quad_state(m.ncell)
    adt = synthetic_adt(m)
    hbm_peak, peak_kind = read_peaks()

    # ------------------------------------------------- CPU baseline (oracle)
    # rank 0 only, before any GPU work; the oracle's result is the expected
    # value of every error figure reported below
    cpu, ref, ref32 = None, None, None
    if rank == 0 and args.cpu_seconds > 0:
        r, n, dt, ref = oracle_leg(m, q, adt, args.cpu_seconds)
        cpu = {"value": r, "unit": "Gedges/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} full FP64 res_calc passes of the same mesh ({m.nedge} edges), {dt:.1f} s on 1 core"}
        ref32 = oracle_res_f32_inputs(m, q, adt)

    tdt_of = {"f64": torch.float64, "dw": torch.float64, "f32": torch.float32}
    elt_of = {"f64": 8, "dw": 8, "f32": 4}

    def make_plan(coloring, reorder, layout=args.layout, first_fit=False, staged=None, bs=256):
        P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                         block_size=bs, reorder=reorder, coloring=coloring, layout=layout,
                         staged=staged, recolor=0 if first_fit else -1)
        P.res.upload()
        return P

    def make_data(P, compute):
        tdt = tdt_of[compute]
        d = {"x": torch.tensor(P.to_plan(m.x, "node"), dtype=tdt, device="cuda"),
             "q": torch.tensor(P.to_plan(q, "cell"), dtype=tdt, device="cuda"),
             "adt": torch.tensor(P.to_plan(adt, "cell"), dtype=tdt, device="cuda")}
        d["res"] = torch.zeros_like(d["q"])
        return d

    def caller(P, d, compute):
        comp = "dw" if compute == "dw" else None
        return lambda: ml.loop_res_calc(P.res, d["x"], d["q"], d["adt"], d["res"], GAM, EPS, compute=comp)

    def parity(P, d, fn, compute):
        """One call on a zeroed res, compared with the oracle (FP32: with the
        oracle on the FP32-rounded inputs, and with the exact inputs)."""
        if ref is None:
            return None
        d["res"].zero_()
        fn()
        torch.cuda.synchronize()
        got = P.from_plan(d["res"].double().cpu().numpy(), "cell", 4)
        if compute == "f32":
            e = field_errors(got, ref32)
            e["against"] = "FP64 oracle on the FP32-rounded inputs"
            e["vs_exact_inputs"] = field_errors(got, ref)
        else:
            e = field_errors(got, ref)
            e["against"] = "FP64 oracle, same inputs"
        return e

    def measure(fn):
        calls = proto.calls_for(fn, max(args.steps, MIN_CALLS), warmup)
        ms, reps, win = proto.warm(fn, calls, REPS)
        msf, repsf, winf = proto.flushed(fn, calls, REPS)
        return calls, ms, reps, msf, repsf, (win[0], winf[1])

    # ---------------------------------------------------------- headline
    compute = args.compute
    elt = elt_of[compute]
    useful = useful_bytes_res_calc(m.ncell, m.nnode, m.nedge, elt)
    head_staged = args.staged or default_staged(compute)
    head_bs = args.block_size or BLOCK_DEFAULT[compute]
    P = make_plan("hier", "partition", bs=head_bs)
    P.res.set_staged(head_staged)
    st = P.res.stats()
    d = make_data(P, compute)
    step = caller(P, d, compute)
    clk = ClockSampler(local)
    clk.start()
    calls, ms_step, reps_warm, ms_flushed, reps_flushed, (t0, t1) = measure(step)
    clocks = clk.window(t0, t1)
    head_parity = parity(P, d, step, compute)
    value = job_rate(m.nedge, world, ms_step) / 1e9
    gbs = useful / (ms_step * 1e-3) / 1e9
    if compute == "f64":
        roof = {"bound": "alu", "achieved": FLOPS_PER_EDGE * m.nedge / ms_step / 1e9, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s",
                "peak_kind": "derived FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz (1.2 TFLOP/s measured "
                             "by an FMA probe); achieved = the oracle's 73 flops per edge (each add, multiply "
                             "counted once) / time"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "peak_kind": f"{peak_kind} copy bandwidth (burst)"
                             + ("; the double-word kernel is FP32-issue bound" if compute == "dw" else "")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["useful_bytes"] = useful
    roof["useful_frac_hbm"] = gbs / hbm_peak
    tr, why = read_traffic(compute, head_staged, args)
    roof["traffic"] = tr["bytes_per_pass"] if tr else None
    roof["traffic_source"] = why
    roof["traffic_scope"] = ("DRAM bytes (read + write) per pass of 4 block-colour launches, ncu "
                             "--cache-control none over consecutive passes")
    if tr:
        roof["traffic_read"] = tr["read_bytes_per_pass"]
        roof["traffic_write"] = tr["write_bytes_per_pass"]
        # the data reuse measure of the plan: useful bytes / DRAM bytes per pass
        roof["useful_over_dram"] = useful / tr["bytes_per_pass"]
        roof["achieved_dram_gbs"] = tr["bytes_per_pass"] / (ms_step * 1e-3) / 1e9
        # DRAM reads over the useful reads (x, q, adt, res, maps as int32):
        # above 1 by the plan tables and the re-read halo of shared points
        useful_reads = useful - 4 * m.ncell * elt
        roof["read_amplification"] = tr["read_bytes_per_pass"] / useful_reads

    # ---------------------------------------------------------- e2e (host buffers)
    # through the C-ABI call with host arrays (loop_res_calc_host): every step
    # copies its inputs from pinned host memory and reads res back; steps
    # alternate two streams and two sets of host arrays, so one step's copies
    # overlap the other's loop
    tdt = tdt_of[compute]
    hsets = []
    for _ in range(2):
        hsets.append([torch.tensor(P.to_plan(m.x, "node"), dtype=tdt).pin_memory(),
                      torch.tensor(P.to_plan(q, "cell"), dtype=tdt).pin_memory(),
                      torch.tensor(P.to_plan(adt, "cell"), dtype=tdt).pin_memory(),
                      torch.zeros((m.ncell, 4), dtype=tdt).pin_memory()])
    e2e_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    e2e_k = [0]
    comp = "dw" if compute == "dw" else None

    def e2e_step():
        k = e2e_k[0]
        e2e_k[0] += 1
        ml.loop_res_calc_host(P.res, *hsets[k % 2], GAM, EPS, stream=e2e_streams[k % 2], compute=comp)

    def e2e_rep(n):
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t = time.perf_counter()
        for _ in range(n):
            e2e_step()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3 / n

    for _ in range(3):
        e2e_step()
    e2e_ms = float(np.median(max_over_ranks([e2e_rep(20) for _ in range(3)], dist, "cuda")))
    h2d = sum(t.numel() for t in hsets[0]) * elt
    d2h = hsets[0][3].numel() * elt
    launches = 2 * REPS * calls * st["nblock_colors"]
    del d, hsets

    # ---------------------------------------------------------- variants
    head_name = f"two_layer_partition_{compute}_{head_staged}"
    variants = {head_name: {
        "gedges_s": value / world, "ms": ms_step, "ms_flushed": ms_flushed, "useful_gbs": gbs,
        "block_colors": st["nblock_colors"], "thread_colors_mean": st["mean_thread_colors"],
        "reuse": st["reuse_all"], "plan_seconds": st["seconds_total"], "parity": head_parity}}
    if not args.no_variants:
        plans = {("hier", "partition", args.layout, False, head_bs): P}
        pick = set(args.variants.split(",")) if args.variants else None
        for key, name, comp_v, staged in res_variants(compute):
            # two-layer plans at their arithmetic's block size; the one-thread-
            # per-iteration baselines do not depend on it
            key = key + ((args.block_size or BLOCK_DEFAULT[comp_v]) if key[0] == "hier" else 256,)
            if name == head_name and key == ("hier", "partition", args.layout, False, head_bs):
                continue
            if pick is not None and name not in pick:
                continue
            try:
                if key not in plans:
                    plans.clear()   # plans are visited grouped: free the previous one
                    plans[key] = make_plan(key[0], key[1], layout=key[2], first_fit=key[3], bs=key[4])
                Pv = plans[key]
                if key[0] == "hier":
                    Pv.res.set_staged(staged)
                dv = make_data(Pv, comp_v)
                fn = caller(Pv, dv, comp_v)
                n_v, msv, _, msfv, _, _ = measure(fn)
            except ml.MeshLoopError as e:
                variants[name] = {"error": str(e)}
                continue
            u = useful_bytes_res_calc(m.ncell, m.nnode, m.nedge, elt_of[comp_v])
            variants[name] = {"gedges_s": m.nedge / msv / 1e6, "ms": msv, "ms_flushed": msfv,
                              "useful_gbs": u / msv / 1e6, "frac_hbm": u / msv / 1e6 / hbm_peak,
                              "colors": Pv.res.stats()["nblock_colors"], "calls_per_rep": n_v,
                              "parity": parity(Pv, dv, fn, comp_v)}
            del dv
        plans.clear()
    del P

    rows = None if args.no_rows else bench_rows(ml, torch, proto, args)
    clk.stop()

    if rank == 0:
        dtype = {"dw": "f64dw", "f64": "f64", "f32": "f32"}[compute]
        line = {
            "metric": METRIC, "value": value, "unit": "Gedges/s", "n_gpus": world, "steps": calls,
            "warmup": warmup, "reps": REPS, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": f"res_calc {args.nx}x{args.ny} jittered renumbered quads, "
                                   + {"f64": "FP64 data and arithmetic", "dw": "FP64 data, double-word arithmetic",
                                      "f32": "FP32 data and arithmetic"}[compute],
                       "cells": m.ncell, "nodes": m.nnode, "edges": m.nedge,
                       "implementation": ("double-word arithmetic, " if compute == "dw" else "")
                                         + "two-layer colouring"
                                         + f" ({'thread-coloured' if head_staged == 'simple' else head_staged}"
                                         + f" increments), RCM + partition, block {head_bs}, "
                                         + args.layout.upper(),
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 (useful bytes {useful / 1e6:.0f} MB > {L2_BYTES / 1e6:.0f} MB); "
                             "value from the warm regime, the L2-flushed regime (a 258 MB write before every "
                             "call) in timing"},
            "timing": {"protocol": f"{warmup} warm-up calls; {REPS} repetitions of {calls} calls; median; "
                                   "CUDA events on the launching stream",
                       "warm_ms_median": ms_step, "warm_ms_reps": reps_warm,
                       "flushed_ms_median": ms_flushed, "flushed_ms_reps": reps_flushed,
                       "flushed_gedges_s": m.nedge / ms_flushed / 1e6},
            "useful_gbs": gbs, "useful_frac_hbm": gbs / hbm_peak, "parity": head_parity,
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": world * m.nedge / e2e_ms / 1e6, "unit": "Gedges/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
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
