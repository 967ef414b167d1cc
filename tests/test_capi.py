"""The C ABI library loads and exports every entry point its header
declares; plan files round-trip.  CPU only (no compute call needs a GPU)."""
import os
import re

import numpy as np
import pytest

import meshgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)) - {"if", "sizeof", "while", "for"}
    return names


def test_every_declared_symbol_is_exported():
    import paper_1802_03749_gb300 as ml
    L = ml.lib()
    names = declared_functions()
    assert {"mesh_plan_build", "loop_res_calc", "loop_elem_assemble", "loop_adjoint"} <= names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) <= set(ml.SIGNATURES), sorted(set(names) - set(ml.SIGNATURES))
    assert L.mp_version().startswith(b"meshloop")


def test_plan_save_load_roundtrip(tmp_path):
    import paper_1802_03749_gb300 as ml
    m = meshgen.quad_mesh(30, 20, seed=3)
    P = ml.Plan([{"to_set": 1, "idx": m.edge2node, "to_size": m.nnode},
                 {"to_set": 2, "idx": m.edge2cell, "to_size": m.ncell, "written": True}], m.nedge,
                block_size=128)
    path = str(tmp_path / "p.plan")
    P.save(path)
    Q = ml.Plan.load(path)
    for t in ("block_offsets", "color_offsets", "block_color", "thread_color", "footprint", "local_map"):
        assert np.array_equal(P.table(t), Q.table(t)), t
    for s in (0, 1, 2):
        assert np.array_equal(P.perm(s), Q.perm(s))
    assert P.stats() == Q.stats()
    with open(path, "r+b") as f:
        f.write(b"garbage!")
    with pytest.raises(ml.MeshLoopError) as e:
        ml.Plan.load(path)
    assert e.value.name == "MP_EIO"


def test_error_strings():
    import paper_1802_03749_gb300 as ml
    for code in range(0, -10, -1):
        assert ml.lib().mp_error_string(code)


def test_loop_argument_errors_without_device():
    """Every loop entry point rejects bad arguments before touching a
    device: null data pointers and unknown dtypes give MP_EINVAL, a plan of
    the wrong shape MP_EPLAN (no GPU needed)."""
    import ctypes
    import paper_1802_03749_gb300 as ml
    L = ml.lib()
    EINVAL, EPLAN = -1, -8
    assert ml.lib().mp_error_string(EINVAL) and ml.lib().mp_error_string(EPLAN)
    q = meshgen.quad_mesh(6, 4, seed=2)
    res_plan = ml.Plan([{"to_set": 1, "idx": q.edge2node, "to_size": q.nnode},
                        {"to_set": 2, "idx": q.edge2cell, "to_size": q.ncell, "written": True}], q.nedge,
                       block_size=32)
    cell_plan = ml.Plan([{"to_set": 1, "idx": q.cell2node, "to_size": q.nnode, "written": True}], q.ncell,
                        block_size=32)
    edge_plan = ml.Plan([{"to_set": 1, "idx": q.edge2cell, "to_size": q.ncell, "written": True}], q.nedge,
                        block_size=32)
    N = None
    F64, BAD = 0, 7
    # res_calc on device and host arrays
    assert L.loop_res_calc(res_plan.handle, BAD, N, N, N, N, 1.4, 0.05, N) == EINVAL
    assert L.loop_res_calc_host(res_plan.handle, F64, N, N, N, N, 1.4, 0.05, N) == EINVAL
    assert L.loop_res_calc_host(None, F64, N, N, N, N, 1.4, 0.05, N) == EINVAL
    # increment-only loops and the face flux: null pointers, then wrong plans
    assert L.loop_space_disc(edge_plan.handle, F64, N, N, N, N, N) == EINVAL
    assert L.loop_space_disc(cell_plan.handle, F64, N, N, N, N, N) == EPLAN
    assert L.loop_getacc(cell_plan.handle, F64, N, N, N) == EINVAL
    assert L.loop_getacc(edge_plan.handle, F64, N, N, N) == EPLAN
    assert L.loop_face_flux(edge_plan.handle, F64, N, N, N, 1.4, 1e-3, 0.72, N) == EINVAL
    assert L.loop_face_flux(edge_plan.handle, F64, N, N, N, 1.0, 1e-3, 0.72, N) == EINVAL   # gamma must exceed 1
    assert L.loop_face_flux(cell_plan.handle, F64, N, N, N, 1.4, 1e-3, 0.72, N) == EPLAN
    assert L.loop_elem_assemble(res_plan.handle, F64, N, N, N, N, N, 0.01, N) == EPLAN
    assert L.mesh_plan_set_staged(res_plan.handle, 8) == EINVAL
    assert L.mesh_plan_set_staged(res_plan.handle, 7) == 0
