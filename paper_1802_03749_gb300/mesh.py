"""Plans for the Airfoil-style time step and the hex assembly loop.

Host orchestration only: builds the loop plans with consistent numbering
through the C ABI (``mesh_plan_build``, ``mesh_plan_perm``,
``mesh_map_renumber``) and permutes data into and out of plan numbering.
The res_calc plan decides the reordering of cells and nodes (Sec. 2.3); the
boundary-edge and cell loops reuse that numbering (Sec. 2.3.1: reorder by one
map, renumber the others).
"""
from __future__ import annotations

import numpy as np

from . import Plan, mesh_map_renumber

NODE, CELL = 1, 2


class AirfoilPlans:
    """Plans for res_calc (edges), bres_calc (boundary edges), adt_calc
    (cells) over one quad mesh given by its maps (original numbering)."""

    def __init__(self, ncell, nnode, edge2node, edge2cell, bedge2node, bedge2cell, cell2node,
                 block_size=512, reorder="partition", coloring="hier", layout="aos", adjoint=False, staged=None,
                 recolor=-1):
        self.ncell, self.nnode = int(ncell), int(nnode)
        self.nedge, self.nbedge = int(edge2node.shape[0]), int(bedge2node.shape[0])
        self.layout = layout
        self.res = Plan([{"to_set": NODE, "idx": edge2node, "to_size": nnode, "written": adjoint},
                         {"to_set": CELL, "idx": edge2cell, "to_size": ncell, "written": True}],
                        self.nedge, block_size=block_size, reorder=reorder, coloring=coloring, layout=layout,
                        staged=staged, recolor=recolor)
        self.cell_perm = self.res.perm(CELL)      # new_to_old
        self.node_perm = self.res.perm(NODE)
        self.edge_perm = self.res.perm(0)
        b2n = mesh_map_renumber(bedge2node, None, self.node_perm, nnode)
        b2c = mesh_map_renumber(bedge2cell, None, self.cell_perm, ncell)
        c2n = mesh_map_renumber(cell2node, self.cell_perm, self.node_perm, nnode)
        self.b2n, self.b2c, self.c2n = b2n, b2c, c2n
        self.bres = Plan([{"to_set": NODE, "idx": b2n, "to_size": nnode},
                          {"to_set": CELL, "idx": b2c, "to_size": ncell, "written": True}],
                         self.nbedge, block_size=256, reorder="none", coloring="global", layout=layout)
        self.adt = Plan([{"to_set": NODE, "idx": c2n, "to_size": nnode}], self.ncell, block_size=256,
                        reorder="none", coloring="atomic", layout=layout)

    # data in original numbering [n, dim] <-> plan numbering in the plan's layout
    def to_plan(self, a: np.ndarray, which: str) -> np.ndarray:
        perm = self.cell_perm if which == "cell" else self.node_perm
        b = np.asarray(a)[perm]
        if self.layout == "soa" and b.ndim == 2:
            b = b.T
        return np.ascontiguousarray(b)

    def from_plan(self, b: np.ndarray, which: str, dim: int) -> np.ndarray:
        perm = self.cell_perm if which == "cell" else self.node_perm
        b = np.asarray(b)
        if dim > 1:
            b = b.reshape(dim, -1).T if self.layout == "soa" else b.reshape(-1, dim)
        out = np.empty_like(b)
        out[perm] = b
        return out


class HexPlan:
    """Plan for hex assembly over elements with elem->node[8] (written)."""

    def __init__(self, nnode, elem2node, block_size=256, reorder="partition", coloring="hier", layout="aos",
                 staged=None, block_of=None, recolor=-1):
        self.nnode = int(nnode)
        self.nelem = int(elem2node.shape[0])
        self.layout = layout
        self.plan = Plan([{"to_set": NODE, "idx": elem2node, "to_size": nnode, "written": True}], self.nelem,
                         block_size=block_size, reorder=reorder, coloring=coloring, layout=layout, staged=staged,
                         block_of=block_of, recolor=recolor)
        self.node_perm = self.plan.perm(NODE)
        self.elem_perm = self.plan.perm(0)

    def to_plan(self, a: np.ndarray, which: str) -> np.ndarray:
        perm = self.node_perm if which == "node" else self.elem_perm
        b = np.asarray(a)[perm]
        if self.layout == "soa" and b.ndim == 2:
            b = b.T
        return np.ascontiguousarray(b)

    def from_plan(self, b: np.ndarray, which: str, dim: int) -> np.ndarray:
        perm = self.node_perm if which == "node" else self.elem_perm
        b = np.asarray(b)
        if dim > 1:
            b = b.reshape(dim, -1).T if self.layout == "soa" else b.reshape(-1, dim)
        out = np.empty_like(b)
        out[perm] = b
        return out


class ScatterPlan:
    """Plan of an increment-only loop over a from-set with one written map
    (``loop_space_disc``: edge->cell[2]; ``loop_getacc``: cell->node[4]).
    ``to_plan``/``from_plan`` move per-item ("from") or per-target ("to")
    data between the caller's numbering and the plan's numbering and
    layout."""

    def __init__(self, to_size, from2to, block_size=256, reorder="partition", coloring="hier", layout="aos",
                 staged=None, recolor=-1):
        self.to_size = int(to_size)
        self.from_size = int(from2to.shape[0])
        self.layout = layout
        self.plan = Plan([{"to_set": 1, "idx": from2to, "to_size": to_size, "written": True}], self.from_size,
                         block_size=block_size, reorder=reorder, coloring=coloring, layout=layout, staged=staged,
                         recolor=recolor)
        self.from_perm = self.plan.perm(0)
        self.to_perm = self.plan.perm(1)

    def to_plan(self, a: np.ndarray, which: str) -> np.ndarray:
        perm = self.from_perm if which == "from" else self.to_perm
        b = np.asarray(a)[perm]
        if self.layout == "soa" and b.ndim == 2:
            b = b.T
        return np.ascontiguousarray(b)

    def from_plan(self, b: np.ndarray, which: str, dim: int) -> np.ndarray:
        perm = self.from_perm if which == "from" else self.to_perm
        b = np.asarray(b)
        if dim > 1:
            b = b.reshape(dim, -1).T if self.layout == "soa" else b.reshape(-1, dim)
        out = np.empty_like(b)
        out[perm] = b
        return out


class AirfoilStep:
    """One explicit time step of the Airfoil-style solver on the device:
    save_soln, adt_calc, res_calc, bres_calc, update (K = 1 stage per step).
    Data live in plan numbering and the plans' layout; ``rms`` accumulates
    the FP64 sum of squared updates on the device.  The step can be captured
    in a CUDA graph (``capture``) once the plans are uploaded."""

    def __init__(self, plans: AirfoilPlans, x, q, qinf, dtype="f64", gam=1.4, eps=0.05, cfl=0.9):
        import torch
        from . import loop_adt_calc, loop_bres_calc, loop_res_calc, loop_save_soln, loop_update  # noqa: F401
        self.P = plans
        self.gam, self.eps, self.cfl = gam, eps, cfl
        self.qinf = [float(v) for v in qinf]
        tdt = torch.float64 if dtype == "f64" else torch.float32
        self.x = torch.tensor(plans.to_plan(x, "node"), dtype=tdt, device="cuda")
        self.q = torch.tensor(plans.to_plan(q, "cell"), dtype=tdt, device="cuda")
        self.qold = torch.zeros_like(self.q)
        self.res = torch.zeros_like(self.q)
        self.adt = torch.zeros(plans.ncell, dtype=tdt, device="cuda")
        self.rms = torch.zeros(1, dtype=torch.float64, device="cuda")
        for p in (plans.res, plans.bres, plans.adt):
            p.upload()
        self.graph = None

    def step(self):
        from . import loop_adt_calc, loop_bres_calc, loop_res_calc, loop_save_soln, loop_update
        P = self.P
        loop_save_soln(self.q, self.qold, P.layout)
        loop_adt_calc(P.adt, self.x, self.q, self.adt, self.gam, self.cfl)
        loop_res_calc(P.res, self.x, self.q, self.adt, self.res, self.gam, self.eps)
        loop_bres_calc(P.bres, self.x, self.q, self.adt, self.res, self.qinf, self.gam, self.eps)
        loop_update(self.qold, self.q, self.res, self.adt, self.rms, P.layout)

    def capture(self, steps_per_graph: int = 1):
        """Capture ``steps_per_graph`` steps into one CUDA graph."""
        import torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()                      # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(steps_per_graph):
                self.step()
        self.graph = g
        return g

    def q_original(self):
        return self.P.from_plan(self.q.cpu().numpy().astype("float64"), "cell", 4)


class AirfoilBatch:
    """The Airfoil-style time step over a batch of meshes of uneven size.

    All meshes' data are concatenated (mesh by mesh, each in its own plan
    numbering).  res_calc runs the fused block-descriptor table of the
    meshes planned with two-layer colouring (one launch per colour phase for
    all of them) and one atomic launch for the meshes planned with atomics;
    adt_calc, bres_calc, save_soln and update each run once over the union.
    ``choices[k]`` = (block_size, reorder, coloring) of mesh k; meshes with
    two-layer colouring must share one block size (the fused launch's).
    Storage is FP32 or FP64; the update and the residual sum are FP64.
    ``res_staged="persistent"`` runs the fused res_calc in one persistent
    launch for all colour phases instead of one launch per phase.
    """

    def __init__(self, meshes, states, qinf, choices, dtype="f32", gam=1.4, eps=0.05, cfl=0.9, res_staged=None):
        import numpy as np
        import torch
        order = sorted(range(len(meshes)), key=lambda k: choices[k][2] != "hier")   # hier meshes first
        self.order = order
        self.gam, self.eps, self.cfl = gam, eps, cfl
        self.qinf = [float(v) for v in qinf]
        self.plans = []
        for k in order:
            m = meshes[k]
            bs, ro, co = choices[k]
            self.plans.append(AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell,
                                           m.cell2node, block_size=bs, reorder=ro, coloring=co))
        self.cell_off = np.cumsum([0] + [p.ncell for p in self.plans])
        self.node_off = np.cumsum([0] + [p.nnode for p in self.plans])
        NC, NN = int(self.cell_off[-1]), int(self.node_off[-1])
        self.ncell, self.nnode = NC, NN
        hier = [i for i, k in enumerate(order) if choices[k][2] == "hier"]
        if hier and len({choices[order[i]][0] for i in hier}) != 1:
            raise ValueError("two-layer meshes of one batch must share a block size")
        self.res_hier = Plan.batch([self.plans[i].res for i in hier]) if hier else None
        if self.res_hier is not None and res_staged is not None:
            self.res_hier.set_staged(res_staged)
        atom = [i for i in range(len(order)) if i not in hier]
        self.res_atomic = None
        if atom:
            e2n = np.concatenate([self.plans[i].res.table("map", 0).reshape(-1, 2) + self.node_off[i] for i in atom])
            e2c = np.concatenate([self.plans[i].res.table("map", 1).reshape(-1, 2) + self.cell_off[i] for i in atom])
            self.res_atomic = Plan([{"to_set": NODE, "idx": e2n, "to_size": NN},
                                    {"to_set": CELL, "idx": e2c, "to_size": NC, "written": True}], e2n.shape[0],
                                   block_size=256, reorder="none", coloring="atomic")
        b2n = np.concatenate([p.b2n + self.node_off[i] for i, p in enumerate(self.plans)])
        b2c = np.concatenate([p.b2c + self.cell_off[i] for i, p in enumerate(self.plans)])
        c2n = np.concatenate([p.c2n + self.node_off[i] for i, p in enumerate(self.plans)])
        self.bres = Plan([{"to_set": NODE, "idx": b2n, "to_size": NN},
                          {"to_set": CELL, "idx": b2c, "to_size": NC, "written": True}], b2n.shape[0],
                         block_size=256, reorder="none", coloring="global")
        self.adt_plan = Plan([{"to_set": NODE, "idx": c2n, "to_size": NN}], NC, block_size=256, reorder="none",
                             coloring="atomic")
        tdt = torch.float64 if dtype == "f64" else torch.float32
        x = np.concatenate([p.to_plan(meshes[k].x, "node") for p, k in zip(self.plans, order)])
        q = np.concatenate([p.to_plan(states[k], "cell") for p, k in zip(self.plans, order)])
        self.x = torch.tensor(x, dtype=tdt, device="cuda")
        self.q = torch.tensor(q, dtype=tdt, device="cuda")
        self.qold = torch.zeros_like(self.q)
        self.res = torch.zeros_like(self.q)
        self.adt = torch.zeros(NC, dtype=tdt, device="cuda")
        self.rms = torch.zeros(1, dtype=torch.float64, device="cuda")
        for p in (self.res_hier, self.res_atomic, self.bres, self.adt_plan):
            if p is not None:
                p.upload()
        self.graph = None

    def step(self):
        from . import loop_adt_calc, loop_bres_calc, loop_res_calc, loop_save_soln, loop_update
        loop_save_soln(self.q, self.qold)
        loop_adt_calc(self.adt_plan, self.x, self.q, self.adt, self.gam, self.cfl)
        if self.res_hier is not None:
            loop_res_calc(self.res_hier, self.x, self.q, self.adt, self.res, self.gam, self.eps)
        if self.res_atomic is not None:
            loop_res_calc(self.res_atomic, self.x, self.q, self.adt, self.res, self.gam, self.eps)
        loop_bres_calc(self.bres, self.x, self.q, self.adt, self.res, self.qinf, self.gam, self.eps)
        loop_update(self.qold, self.q, self.res, self.adt, self.rms)

    def capture(self, steps_per_graph: int = 1):
        import torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(steps_per_graph):
                self.step()
        self.graph = g
        return g

    def q_of(self, k):
        """State of mesh k (input order) in its original numbering."""
        i = self.order.index(k)
        a, b = int(self.cell_off[i]), int(self.cell_off[i + 1])
        return self.plans[i].from_plan(self.q[a:b].cpu().numpy().astype("float64"), "cell", 4)
