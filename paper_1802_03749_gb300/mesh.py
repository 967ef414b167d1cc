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
                 block_size=512, reorder="partition", coloring="hier", layout="aos", adjoint=False):
        self.ncell, self.nnode = int(ncell), int(nnode)
        self.nedge, self.nbedge = int(edge2node.shape[0]), int(bedge2node.shape[0])
        self.layout = layout
        self.res = Plan([{"to_set": NODE, "idx": edge2node, "to_size": nnode, "written": adjoint},
                         {"to_set": CELL, "idx": edge2cell, "to_size": ncell, "written": True}],
                        self.nedge, block_size=block_size, reorder=reorder, coloring=coloring, layout=layout)
        self.cell_perm = self.res.perm(CELL)      # new_to_old
        self.node_perm = self.res.perm(NODE)
        self.edge_perm = self.res.perm(0)
        b2n = mesh_map_renumber(bedge2node, None, self.node_perm, nnode)
        b2c = mesh_map_renumber(bedge2cell, None, self.cell_perm, ncell)
        c2n = mesh_map_renumber(cell2node, self.cell_perm, self.node_perm, nnode)
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

    def __init__(self, nnode, elem2node, block_size=256, reorder="partition", coloring="hier", layout="aos"):
        self.nnode = int(nnode)
        self.nelem = int(elem2node.shape[0])
        self.layout = layout
        self.plan = Plan([{"to_set": NODE, "idx": elem2node, "to_size": nnode, "written": True}], self.nelem,
                         block_size=block_size, reorder=reorder, coloring=coloring, layout=layout)
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
