"""GPU parity of hex assembly (two-layer, global colouring, atomics) against
the FP64 oracle through the C ABI."""
import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import rel_l2, round_to

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {}


def case(n):
    if n not in CASES:
        m = meshgen.hex_mesh(n, seed=31)
        sig, v = meshgen.hex_fields(m, seed=31)
        CASES[n] = (m, sig, v)
    return CASES[n]


def run_hex(m, sig, v, coloring, reorder, layout, dtype, block_size=256):
    import paper_1802_03749_gb300 as ml
    from paper_1802_03749_gb300.mesh import HexPlan
    H = HexPlan(m.nnode, m.elem2node, block_size=block_size, reorder=reorder, coloring=coloring, layout=layout)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    x = torch.tensor(H.to_plan(m.x, "node"), dtype=tdt, device="cuda")
    vd = torch.tensor(H.to_plan(v, "node"), dtype=tdt, device="cuda")
    sd = torch.tensor(H.to_plan(sig, "elem"), dtype=tdt, device="cuda")
    f = torch.zeros_like(x)
    vol = torch.zeros(m.nelem, dtype=tdt, device="cuda")
    ml.loop_elem_assemble(H.plan, x, vd, sd, f, vol, 0.01)
    torch.cuda.synchronize()
    return (H.from_plan(f.cpu().numpy().astype(np.float64), "node", 3),
            H.from_plan(vol.cpu().numpy().astype(np.float64), "elem", 1), H)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("coloring,reorder", [("hier", "partition"), ("hier", "rcm"), ("global", "rcm"),
                                              ("atomic", "none"), ("hier", "none")])
def test_hex_parity(coloring, reorder, layout, dtype):
    m, sig, v = case(14)
    f, vol, _ = run_hex(m, sig, v, coloring, reorder, layout, dtype)
    if dtype == "f64":
        fr, vr = oracle.hex_force(m.elem2node, m.x, v, sig)
        assert rel_l2(vol, vr) <= 1e-12
        assert rel_l2(f, fr) <= 1e-12
    else:
        fr, vr = oracle.hex_force(m.elem2node, round_to(m.x, np.float32), round_to(v, np.float32),
                                  round_to(sig, np.float32))
        assert rel_l2(vol, vr) <= 1e-5
        assert rel_l2(f, fr) <= 1e-5


@pytest.mark.parametrize("block_size", [64, 128, 320, 512])
def test_hex_block_sizes_ragged(block_size):
    """An 11 x 9 x 7 brick: partial blocks and a ragged last block."""
    m = meshgen.hex_mesh(11, seed=32, nyz=(9, 7))
    sig, v = meshgen.hex_fields(m, seed=32)
    fr, vr = oracle.hex_force(m.elem2node, m.x, v, sig)
    f, vol, H = run_hex(m, sig, v, "hier", "partition", "aos", "f64", block_size=block_size)
    assert rel_l2(f, fr) <= 1e-12 and rel_l2(vol, vr) <= 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_hex_smem_atomic_variant(dtype):
    import paper_1802_03749_gb300 as ml
    m, sig, v = case(14)
    ml.mp_set_staged_variant("smem_atomic")
    try:
        f, vol, _ = run_hex(m, sig, v, "hier", "partition", "aos", dtype)
    finally:
        ml.mp_set_staged_variant("simple")
    if dtype == "f64":
        fr, vr = oracle.hex_force(m.elem2node, m.x, v, sig)
        assert rel_l2(f, fr) <= 1e-12
    else:
        fr, vr = oracle.hex_force(m.elem2node, round_to(m.x, np.float32), round_to(v, np.float32),
                                  round_to(sig, np.float32))
        assert rel_l2(f, fr) <= 1e-5
