"""Autotuner for batched res_calc: picks, per mesh-size class, the
reordering and the race-avoidance strategy (two-layer colouring or
atomics), and one block size for the fused two-layer launch, by timing
res_calc on the batch's own meshes with CUDA events.  Results can be saved
to and loaded from JSON so that tuning is a one-off."""
from __future__ import annotations

import json

import numpy as np

SIZE_CLASSES = ((0, 20_000), (20_000, 100_000), (100_000, 1 << 62))
BLOCK_SIZES = (256, 480)
VARIANTS = (("partition", "hier"), ("rcm", "hier"), ("rcm", "atomic"))


def size_class(ncell: int) -> int:
    for i, (lo, hi) in enumerate(SIZE_CLASSES):
        if lo <= ncell < hi:
            return i
    return len(SIZE_CLASSES) - 1


def _time_res_calc(mesh, q, adt, block_size, reorder, coloring, dtype, reps):
    import torch

    from . import loop_res_calc
    from .mesh import AirfoilPlans
    P = AirfoilPlans(mesh.ncell, mesh.nnode, mesh.edge2node, mesh.edge2cell, mesh.bedge2node, mesh.bedge2cell,
                     mesh.cell2node, block_size=block_size, reorder=reorder, coloring=coloring)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    x = torch.tensor(P.to_plan(mesh.x, "node"), dtype=tdt, device="cuda")
    qd = torch.tensor(P.to_plan(q, "cell"), dtype=tdt, device="cuda")
    ad = torch.tensor(P.to_plan(adt, "cell"), dtype=tdt, device="cuda")
    res = torch.zeros_like(qd)
    for _ in range(3):
        loop_res_calc(P.res, x, qd, ad, res)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        loop_res_calc(P.res, x, qd, ad, res)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(meshes, states, adts, dtype="f32", reps=20):
    """Returns {"block_size": S, "classes": {class: (reorder, coloring)}} and
    the per-mesh choices (block_size, reorder, coloring)."""
    by_class = {}
    for k, m in enumerate(meshes):
        by_class.setdefault(size_class(m.ncell), []).append(k)
    # representative: the median-size mesh of each class present
    reps_of = {c: sorted(ks, key=lambda k: meshes[k].ncell)[len(ks) // 2] for c, ks in by_class.items()}
    timings = {}
    for c, k in reps_of.items():
        for bs in BLOCK_SIZES:
            for ro, co in VARIANTS:
                if co == "atomic" and bs != BLOCK_SIZES[0]:
                    continue
                t = _time_res_calc(meshes[k], states[k], adts[k], bs, ro, co, dtype, reps)
                timings[(c, bs, ro, co)] = t / meshes[k].nedge        # time per edge
    # one block size for the fused two-layer launch: best total over classes,
    # weighting each class by its number of edges
    edges = {c: sum(meshes[k].nedge for k in ks) for c, ks in by_class.items()}

    def best(c, bs):
        opts = [(timings[(c, b, ro, co)], ro, co) for (cc, b, ro, co) in timings
                if cc == c and (b == bs or co == "atomic")]
        return min(opts)

    S = min(BLOCK_SIZES, key=lambda bs: sum(edges[c] * best(c, bs)[0] for c in by_class))
    classes = {c: best(c, S)[1:] for c in by_class}
    choices = [(S if classes[size_class(m.ncell)][1] == "hier" else 256,) + tuple(classes[size_class(m.ncell)])
               for m in meshes]
    return {"block_size": S, "classes": {str(c): list(v) for c, v in classes.items()},
            "timings_ns_per_edge": {f"{c}/{b}/{ro}/{co}": t * 1e6 for (c, b, ro, co), t in timings.items()}}, choices


def save(result, path):
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


def choices_from(result, meshes):
    S = result["block_size"]
    cls = {int(c): tuple(v) for c, v in result["classes"].items()}
    out = []
    for m in meshes:
        ro, co = cls.get(size_class(m.ncell), ("partition", "hier"))
        out.append((S if co == "hier" else 256, ro, co))
    return out
