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


def run_hex(m, sig, v, coloring, reorder, layout, dtype, block_size=256, staged=None):
    import paper_1802_03749_gb300 as ml
    from paper_1802_03749_gb300.mesh import HexPlan
    H = HexPlan(m.nnode, m.elem2node, block_size=block_size, reorder=reorder, coloring=coloring, layout=layout,
                staged=staged)
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
                                              ("atomic", "none"), ("hier", "none"), ("twostep", "rcm")])
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


@pytest.mark.parametrize("staged", ["simple", "warp_agg"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_hex_thread_coloured_variant(dtype, staged):
    """Hex assembly defaults to shared-memory atomics; the thread-coloured
    increments of Algorithm 1 and the warp-aggregated atomics are the other
    staged variants."""
    m, sig, v = case(14)
    f, vol, _ = run_hex(m, sig, v, "hier", "partition", "aos", dtype, staged=staged)
    if dtype == "f64":
        fr, vr = oracle.hex_force(m.elem2node, m.x, v, sig)
        assert rel_l2(f, fr) <= 1e-12
    else:
        fr, vr = oracle.hex_force(m.elem2node, round_to(m.x, np.float32), round_to(v, np.float32),
                                  round_to(sig, np.float32))
        assert rel_l2(f, fr) <= 1e-5


def run_hex_dw(m, sig, v, reorder, layout, block_size=128, staged=None, coloring="hier"):
    import paper_1802_03749_gb300 as ml
    from paper_1802_03749_gb300.mesh import HexPlan
    H = HexPlan(m.nnode, m.elem2node, block_size=block_size, reorder=reorder, coloring=coloring, layout=layout,
                staged=staged)
    x = torch.tensor(H.to_plan(m.x, "node"), device="cuda")
    vd = torch.tensor(H.to_plan(v, "node"), device="cuda")
    sd = torch.tensor(H.to_plan(sig, "elem"), device="cuda")
    f0 = np.cos(np.arange(m.nnode * 3)).reshape(-1, 3)          # increments are "+="
    f = torch.tensor(H.to_plan(f0, "node"), device="cuda")
    vol = torch.zeros(m.nelem, dtype=torch.float64, device="cuda")
    ml.loop_elem_assemble(H.plan, x, vd, sd, f, vol, 0.01, compute="dw")
    ml.mp_check_device_status()
    return (H.from_plan(f.cpu().numpy(), "node", 3) - f0, H.from_plan(vol.cpu().numpy(), "elem", 1))


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("reorder", ["partition", "rcm"])
def test_hex_double_word_parity(reorder, layout):
    """FP64 data with double-word arithmetic, gather (default) and
    thread-coloured increments: within the FP64 bar."""
    m, sig, v = case(14)
    fr, vr = oracle.hex_force(m.elem2node, m.x, v, sig)
    for staged in (None, "simple"):
        f, vol = run_hex_dw(m, sig, v, reorder, layout, staged=staged)
        assert rel_l2(vol, vr) <= 1e-12
        assert rel_l2(f, fr) <= 1e-12


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("reorder", ["none", "rcm"])
@pytest.mark.parametrize("coloring", ["global", "atomic"])
def test_hex_double_word_baselines(coloring, reorder, layout):
    """Global colouring and atomics (Sec. 2.1) in double-word arithmetic on
    FP64 data (a ragged last launch: 13^3 elements): within the FP64 bar."""
    m, sig, v = case(13)
    fr, vr = oracle.hex_force(m.elem2node, m.x, v, sig)
    f, vol = run_hex_dw(m, sig, v, reorder, layout, coloring=coloring)
    assert rel_l2(vol, vr) <= 1e-12
    assert rel_l2(f, fr) <= 1e-12


@pytest.mark.parametrize("block_size", [32, 96, 256])
def test_hex_double_word_gather_ragged_and_deterministic(block_size):
    m, sig, v = case(11)
    fr, _ = oracle.hex_force(m.elem2node, m.x, v, sig)
    a, _ = run_hex_dw(m, sig, v, "partition", "aos", block_size=block_size)
    b, _ = run_hex_dw(m, sig, v, "partition", "aos", block_size=block_size)
    assert rel_l2(a, fr) <= 1e-12 and np.array_equal(a, b)


@pytest.mark.slow
@pytest.mark.parametrize("coloring", ["hier", "atomic"])
def test_hex_double_word_full_size(coloring):
    """The benchmark's hex workload, 120^3 elements, two-layer (partition)
    and atomics (RCM): the oracle computes every node."""
    m = meshgen.hex_mesh(120)
    sig, v = meshgen.hex_fields(m)
    f, vol = run_hex_dw(m, sig, v, "partition" if coloring == "hier" else "rcm", "aos", coloring=coloring)
    fr, vr = oracle.hex_force(m.elem2node, m.x, v, sig)
    assert rel_l2(vol, vr) <= 1e-12
    assert rel_l2(f, fr) <= 1e-12


@pytest.mark.parametrize("shape", [(16, 1, 1), (4, 2, 2)])
def test_hex_handcrafted_blocks(shape):
    """Caller-defined brick blocks (structured-mesh study): parity."""
    dims = (16, 8, 8)
    m = meshgen.hex_mesh(dims[0], seed=33, nyz=dims[1:])
    sig, v = meshgen.hex_fields(m, seed=33)
    import paper_1802_03749_gb300 as ml
    from paper_1802_03749_gb300.mesh import HexPlan
    H = HexPlan(m.nnode, m.elem2node, block_size=32, block_of=meshgen.hex_bricks(m, shape, dims))
    x = torch.tensor(H.to_plan(m.x, "node"), device="cuda")
    vd = torch.tensor(H.to_plan(v, "node"), device="cuda")
    sd = torch.tensor(H.to_plan(sig, "elem"), device="cuda")
    f = torch.zeros_like(x)
    vol = torch.zeros(m.nelem, dtype=torch.float64, device="cuda")
    ml.loop_elem_assemble(H.plan, x, vd, sd, f, vol, 0.01)
    fr, vr = oracle.hex_force(m.elem2node, m.x, v, sig)
    assert rel_l2(H.from_plan(f.cpu().numpy(), "node", 3), fr) <= 1e-12
