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
