"""GPU parity of res_calc (two-layer, global colouring, atomics) against the
FP64 oracle, through the C ABI.  FP64: rel-L2 <= 1e-12; FP32 storage and
arithmetic: rel-L2 <= 1e-5 against the oracle fed the same FP32-rounded
inputs."""
import numpy as np
import pytest

import oracle
from gpu_util import airfoil_case, rel_l2, round_to

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ml():
    import paper_1802_03749_gb300 as ml
    ml.lib()
    return ml


CASES = {}


def case(nx, ny):
    if (nx, ny) not in CASES:
        CASES[(nx, ny)] = airfoil_case(nx, ny)
    return CASES[(nx, ny)]


def run_res_calc(ml, m, q, adt, coloring, reorder, layout, dtype, block_size=480, res0=None, staged=None):
    from paper_1802_03749_gb300.mesh import AirfoilPlans
    P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                     block_size=block_size, reorder=reorder, coloring=coloring, layout=layout, staged=staged)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dev = "cuda"
    x = torch.tensor(P.to_plan(m.x, "node"), dtype=tdt, device=dev)
    qd = torch.tensor(P.to_plan(q, "cell"), dtype=tdt, device=dev)
    ad = torch.tensor(P.to_plan(adt, "cell"), dtype=tdt, device=dev)
    r0 = np.zeros_like(q) if res0 is None else res0
    res = torch.tensor(P.to_plan(r0, "cell"), dtype=tdt, device=dev)
    ml.loop_res_calc(P.res, x, qd, ad, res)
    torch.cuda.synchronize()
    return P.from_plan(res.cpu().numpy().astype(np.float64), "cell", 4), P


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("reorder", ["none", "rcm", "partition"])
@pytest.mark.parametrize("coloring", ["hier", "global", "atomic", "twostep"])
def test_res_calc_parity(ml, coloring, reorder, layout, dtype):
    m, q, adt = case(200, 100)
    r0 = 0.01 * np.cos(np.arange(q.size)).reshape(q.shape)       # increments are "+="
    got, _ = run_res_calc(ml, m, q, adt, coloring, reorder, layout, dtype, res0=r0)
    if dtype == "f64":
        ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt, res=r0.copy())
        assert rel_l2(got - r0, ref - r0) <= 1e-12
    else:
        r0r = round_to(r0, np.float32)
        ref = oracle.res_calc(m.edge2node, m.edge2cell, round_to(m.x, np.float32), round_to(q, np.float32),
                              round_to(adt, np.float32), res=r0r.copy())
        assert rel_l2(got - r0r, ref - r0r) <= 1e-5


@pytest.mark.parametrize("block_size", [64, 128, 256, 480, 1024])
def test_res_calc_ragged_block_sizes(ml, block_size):
    """A 97x53 mesh: many partial blocks and a ragged last block."""
    m, q, adt = case(97, 53)
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    for reorder in ("rcm", "partition"):
        got, P = run_res_calc(ml, m, q, adt, "hier", reorder, "aos", "f64", block_size=block_size)
        assert rel_l2(got, ref) <= 1e-12
        st = P.res.stats()
        assert st["nblocks"] >= m.nedge // block_size


def test_res_calc_two_layer_is_deterministic(ml):
    m, q, adt = case(200, 100)
    a, _ = run_res_calc(ml, m, q, adt, "hier", "partition", "aos", "f64")
    b, _ = run_res_calc(ml, m, q, adt, "hier", "partition", "aos", "f64")
    assert np.array_equal(a, b)


def test_res_calc_tiny_and_empty(ml):
    """A 2x1 mesh (one interior edge) and a plan with no iterations."""
    m, q, adt = case(2, 1)
    assert m.nedge == 1
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    for coloring in ("hier", "global", "atomic"):
        got, _ = run_res_calc(ml, m, q, adt, coloring, "partition", "aos", "f64", block_size=32)
        assert rel_l2(got, ref) <= 1e-12
    P = ml.Plan([{"to_set": 1, "idx": np.zeros((0, 2), np.int32), "to_size": 4},
                 {"to_set": 2, "idx": np.zeros((0, 2), np.int32), "to_size": 4, "written": True}], 0)
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    ml.loop_res_calc(P, z, z, z, z)
    assert P.stats()["nblocks"] == 0


def run_dw(ml, m, q, adt, reorder, layout, block_size=480, res0=None, staged=None, coloring="hier"):
    from paper_1802_03749_gb300.mesh import AirfoilPlans
    P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                     block_size=block_size, reorder=reorder, coloring=coloring, layout=layout, staged=staged)
    x = torch.tensor(P.to_plan(m.x, "node"), device="cuda")
    qd = torch.tensor(P.to_plan(q, "cell"), device="cuda")
    ad = torch.tensor(P.to_plan(adt, "cell"), device="cuda")
    res = torch.tensor(P.to_plan(np.zeros_like(q) if res0 is None else res0, "cell"), device="cuda")
    ml.loop_res_calc(P.res, x, qd, ad, res, compute="dw")
    ml.mp_check_device_status()
    return P.from_plan(res.cpu().numpy(), "cell", 4)


@pytest.mark.parametrize("staged", [None, "simple"])
@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("reorder", ["none", "rcm", "partition"])
def test_res_calc_double_word_parity(ml, reorder, layout, staged):
    """FP64 data with double-word arithmetic, gather (the default) and
    thread-coloured increments: within the FP64 bar."""
    m, q, adt = case(200, 100)
    r0 = 0.01 * np.cos(np.arange(q.size)).reshape(q.shape)
    got = run_dw(ml, m, q, adt, reorder, layout, res0=r0, staged=staged)
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt, res=r0.copy())
    assert rel_l2(got - r0, ref - r0) <= 1e-12


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("reorder", ["none", "rcm"])
@pytest.mark.parametrize("coloring", ["global", "atomic"])
def test_res_calc_double_word_baselines(ml, coloring, reorder, layout):
    """Global colouring and atomics (Sec. 2.1) in double-word arithmetic on
    FP64 data: within the FP64 bar, like the two-layer form."""
    m, q, adt = case(200, 100)
    r0 = 0.01 * np.cos(np.arange(q.size)).reshape(q.shape)
    got = run_dw(ml, m, q, adt, reorder, layout, res0=r0, coloring=coloring)
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt, res=r0.copy())
    assert rel_l2(got - r0, ref - r0) <= 1e-12


@pytest.mark.parametrize("xs,qs", [(1e-12, 1.0), (1e12, 1.0), (1.0, 1e15), (1.0, 1e-15), (1e-6, 1e-10),
                                   (1e6, 1e10)])
def test_res_calc_double_word_scaled_inputs(ml, xs, qs):
    """The double-word arithmetic (FP32 exponent range) on inputs scaled far
    from the unit free stream: coordinates by xs, states by qs (adt follows
    from them): every form stays within the FP64 bar."""
    m0, q0, _ = case(60, 30)
    import copy
    m = copy.copy(m0)
    m.x = m0.x * xs
    q = q0 * qs
    adt = oracle.adt_calc(m.cell2node, m.x, q)
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    for coloring, staged in (("hier", None), ("hier", "simple"), ("global", None), ("atomic", None)):
        got = run_dw(ml, m, q, adt, "partition" if coloring == "hier" else "rcm", "aos", block_size=256,
                     staged=staged, coloring=coloring)
        assert rel_l2(got, ref) <= 1e-12, (coloring, staged)


@pytest.mark.parametrize("xs,qs", [(1e-100, 1.0), (1e100, 1.0), (1.0, 1e150), (1.0, 1e-150), (1e-50, 1e-140),
                                   (1e50, 1e140)])
def test_res_calc_fp64_scaled_inputs(ml, xs, qs):
    """Native FP64 on inputs scaled far from the unit free stream (the
    reciprocal 1/(2 rho) of the flux kernels at densities from 1e-150 to
    1e150): every strategy stays within the FP64 bar.  States above about
    1e154 would overflow the oracle's own |rho u|^2."""
    m0, q0, _ = case(60, 30)
    import copy
    m = copy.copy(m0)
    m.x = m0.x * xs
    q = q0 * qs
    adt = oracle.adt_calc(m.cell2node, m.x, q)
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    for coloring, staged in (("hier", None), ("hier", "simple"), ("hier", "pipelined"), ("global", None),
                             ("atomic", None)):
        got, _ = run_res_calc(ml, m, q, adt, coloring, "partition" if coloring == "hier" else "rcm", "aos", "f64",
                              block_size=256, staged=staged)
        s = np.abs(ref).max()                 # the norm's squares would overflow at 1e186
        assert np.all(np.isfinite(got)) and rel_l2(got / s, ref / s) <= 1e-12, (coloring, staged)


@pytest.mark.slow
@pytest.mark.parametrize("compute", ["f64", "f64_colour", "dw", "dw_colour", "dw_global", "dw_atomic", "f32"])
def test_res_calc_full_size_parity(ml, compute):
    """The benchmark's workload: 2400x1200 quads, two-layer colouring,
    RCM + partition, AoS, in the benchmark's launches: native FP64 at block
    384 with gather increments (the headline), double-word arithmetic
    (gather and thread colours) and FP32 (gather) at block 256; native FP64
    with thread colours at block 480; the double-word global-colour and
    atomic baselines on the RCM order.  The oracle computes every cell."""
    m, q, adt = case(2400, 1200)
    if compute == "dw":
        got = run_dw(ml, m, q, adt, "partition", "aos", block_size=256)
    elif compute == "dw_colour":
        got = run_dw(ml, m, q, adt, "partition", "aos", block_size=256, staged="simple")
    elif compute in ("dw_global", "dw_atomic"):
        got = run_dw(ml, m, q, adt, "rcm", "aos", coloring=compute[3:])
    elif compute == "f32":
        got, _ = run_res_calc(ml, m, q, adt, "hier", "partition", "aos", "f32", block_size=256, staged="gather")
        ref = oracle.res_calc(m.edge2node, m.edge2cell, round_to(m.x, np.float32), round_to(q, np.float32),
                              round_to(adt, np.float32))
        assert rel_l2(got, ref) <= 1e-5
        return
    elif compute == "f64":
        got, _ = run_res_calc(ml, m, q, adt, "hier", "partition", "aos", "f64", block_size=384)
    else:
        got, _ = run_res_calc(ml, m, q, adt, "hier", "partition", "aos", "f64", block_size=480, staged="simple")
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    assert rel_l2(got, ref) <= 1e-12


@pytest.mark.parametrize("variant", ["pipelined", "smem_atomic", "gather", "simple", "warp_agg", "persistent"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("reorder,block_size", [("partition", 480), ("rcm", 256), ("none", 480), ("partition", 1024)])
def test_res_calc_staged_variants(ml, variant, dtype, reorder, block_size):
    """The other staged implementations (pipelined persistent CTAs, shared-
    memory atomics) against the oracle; unfit plans fall back to one block
    per CTA."""
    m, q, adt = case(97, 53)
    got, _ = run_res_calc(ml, m, q, adt, "hier", reorder, "aos", dtype, block_size=block_size, staged=variant)
    ml.mp_check_device_status()
    if dtype == "f64":
        ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
        assert rel_l2(got, ref) <= 1e-12
    else:
        ref = oracle.res_calc(m.edge2node, m.edge2cell, round_to(m.x, np.float32), round_to(q, np.float32),
                              round_to(adt, np.float32))
        assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("block_size", [32, 64, 256, 512])
def test_res_calc_gather_ragged_and_deterministic(ml, block_size):
    """Gather increments on a ragged mesh at several block sizes, native
    FP64 and double-word; two runs give the same bits."""
    m, q, adt = case(97, 53)
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    for reorder in ("rcm", "partition"):
        a, _ = run_res_calc(ml, m, q, adt, "hier", reorder, "aos", "f64", block_size=block_size, staged="gather")
        b, _ = run_res_calc(ml, m, q, adt, "hier", reorder, "aos", "f64", block_size=block_size, staged="gather")
        assert rel_l2(a, ref) <= 1e-12 and np.array_equal(a, b)
        c = run_dw(ml, m, q, adt, reorder, "soa", block_size=block_size, staged="gather")
        d = run_dw(ml, m, q, adt, reorder, "soa", block_size=block_size, staged="gather")
        assert rel_l2(c, ref) <= 1e-12 and np.array_equal(c, d)
    ml.mp_check_device_status()
