"""Overlapped colour launches (programmatic dependent launch) give the same
bits as plain stream order: every staged and global-colour loop is run in
this process (overlap on) and in a child process with MESHLOOP_NO_PDL set,
on a ragged mesh with small blocks (many colours, many launch boundaries),
and the outputs are compared bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
import meshgen
import paper_1802_03749_gb300 as ml
from paper_1802_03749_gb300.mesh import AirfoilPlans, HexPlan

out = {}
m = meshgen.quad_mesh(97, 53, seed=7)
q = meshgen.quad_state(m.ncell, seed=7, noise=0.01)
adt = 0.5 + meshgen.uniform(8, 1, m.ncell)
rb = meshgen.adjoint_seed(m.ncell, seed=9)
for name, coloring, staged, compute, bs in (("hier_f64", "hier", None, None, 64),
                                            ("hier_f64_gather", "hier", "gather", None, 64),
                                            ("hier_dw", "hier", None, "dw", 64),
                                            ("hier_dw_colour", "hier", "simple", "dw", 64),
                                            ("global_f64", "global", None, None, 256)):
    P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                     block_size=bs, reorder="partition", coloring=coloring, staged=staged)
    t = lambda a, w: torch.tensor(P.to_plan(a, w), device="cuda")
    res = t(0.01 * np.cos(np.arange(q.size)).reshape(q.shape), "cell")
    for _ in range(3):
        ml.loop_res_calc(P.res, t(m.x, "node"), t(q, "cell"), t(adt, "cell"), res, compute=compute)
    out["res_" + name] = res.cpu().numpy()
    if coloring == "hier" and staged is None:
        Pa = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                          block_size=bs, reorder="partition", coloring="hier", adjoint=True)
        ta = lambda a, w: torch.tensor(Pa.to_plan(a, w), device="cuda")
        qb = torch.zeros(m.ncell * 4, dtype=torch.float64, device="cuda")
        xb = torch.zeros(m.nnode * 2, dtype=torch.float64, device="cuda")
        ml.loop_adjoint(Pa.res, ta(m.x, "node"), ta(q, "cell"), ta(adt, "cell"), ta(rb, "cell"), qb, xb,
                        compute=compute)
        out["adj_" + name] = np.concatenate([qb.cpu().numpy().ravel(), xb.cpu().numpy().ravel()])
hm = meshgen.hex_mesh(14, nyz=(9, 11))
sig, v = meshgen.hex_fields(hm)
for name, coloring, staged, compute, bs in (("hier_f64", "hier", "simple", None, 64),
                                            ("hier_f64_atomic", "hier", None, None, 64),
                                            ("hier_dw", "hier", None, "dw", 64),
                                            ("global_f64", "global", None, None, 256)):
    H = HexPlan(hm.nnode, hm.elem2node, block_size=bs, reorder="partition", coloring=coloring, staged=staged)
    t = lambda a, w: torch.tensor(H.to_plan(a, w), device="cuda")
    x = t(hm.x, "node")
    f = torch.zeros_like(x)
    vol = torch.zeros(hm.nelem, dtype=torch.float64, device="cuda")
    ml.loop_elem_assemble(H.plan, x, t(v, "node"), t(sig, "elem"), f, vol, 0.01, compute=compute)
    if staged is None and compute is None and coloring == "hier":
        continue   # shared-memory atomics: the order of additions is not fixed
    out["hex_" + name] = np.concatenate([f.cpu().numpy().ravel(), vol.cpu().numpy().ravel()])
ml.mp_check_device_status()
np.savez(sys.argv[1], **out)
'''


def run(path, no_pdl):
    env = dict(os.environ)
    env.pop("MESHLOOP_NO_PDL", None)
    if no_pdl:
        env["MESHLOOP_NO_PDL"] = "1"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", SCRIPT, path], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return dict(np.load(path))


def test_overlapped_launches_match_stream_order(tmp_path):
    a = run(str(tmp_path / "pdl.npz"), False)
    b = run(str(tmp_path / "plain.npz"), True)
    assert sorted(a) == sorted(b) and len(a) >= 10
    for k in a:
        assert np.array_equal(a[k], b[k]), k
