"""GPU parity of the increment-only loops against the FP64 oracle, through
the C ABI: the Volna-style edge loop (FP32, the paper's precision, and
FP64) and the BookLeaf-style cell loop (FP64, the paper's precision, and
FP32), with staged two-layer (thread-coloured and gather increments),
global-colour, atomic and owner-computes (two-step) plans.  FP64 rel-L2
<= 1e-12; FP32 <= 1e-5 against the oracle fed the same FP32-rounded
inputs."""
import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import rel_l2, round_to

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VARIANTS = [("hier", "partition", None), ("hier", "partition", "simple"), ("hier", "rcm", None),
            ("global", "rcm", None), ("atomic", "rcm", None), ("atomic", "none", None), ("twostep", "rcm", None),
            ("twostep", "none", None)]


@pytest.fixture(scope="module")
def ml():
    import paper_1802_03749_gb300 as ml
    ml.lib()
    return ml


CASES = {}


def tri_case(nx, ny):
    if ("tri", nx, ny) not in CASES:
        m = meshgen.tri_mesh(nx, ny, seed=11)
        ed, ia = meshgen.volna_fields(m, seed=11)
        CASES[("tri", nx, ny)] = (m, ed, ia)
    return CASES[("tri", nx, ny)]


def quad_case(nx, ny):
    if ("quad", nx, ny) not in CASES:
        m = meshgen.quad_mesh(nx, ny, seed=12)
        CASES[("quad", nx, ny)] = (m, meshgen.bookleaf_fields(m.ncell, seed=12))
    return CASES[("quad", nx, ny)]


def run_space_disc(ml, m, ed, ia, res0, coloring, reorder, staged, layout, dtype, block_size=256):
    from paper_1802_03749_gb300.mesh import ScatterPlan
    S = ScatterPlan(m.ncell, m.edge2cell, block_size=block_size, reorder=reorder, coloring=coloring, layout=layout,
                    staged=staged)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    t = lambda a, w: torch.tensor(S.to_plan(a, w), dtype=tdt, device="cuda")
    res = t(res0, "to")
    fl = torch.tensor(S.to_plan(m.eflag, "from"), dtype=torch.int32, device="cuda")
    ml.loop_space_disc(S.plan, t(ed, "from"), fl, t(ia, "to"), res)
    torch.cuda.synchronize()
    ml.mp_check_device_status()
    return S.from_plan(res.cpu().numpy().astype(np.float64), "to", 4)


def run_getacc(ml, m, cd, nd0, coloring, reorder, staged, layout, dtype, block_size=256):
    from paper_1802_03749_gb300.mesh import ScatterPlan
    S = ScatterPlan(m.nnode, m.cell2node, block_size=block_size, reorder=reorder, coloring=coloring, layout=layout,
                    staged=staged)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    t = lambda a, w: torch.tensor(S.to_plan(a, w), dtype=tdt, device="cuda")
    nd = t(nd0, "to")
    ml.loop_getacc(S.plan, t(cd, "from"), nd)
    torch.cuda.synchronize()
    ml.mp_check_device_status()
    return S.from_plan(nd.cpu().numpy().astype(np.float64), "to", 4)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("coloring,reorder,staged", VARIANTS)
def test_space_disc_parity(ml, coloring, reorder, staged, layout, dtype):
    m, ed, ia = tri_case(97, 53)
    r0 = 0.1 * np.sin(np.arange(4 * m.ncell)).reshape(-1, 4)
    got = run_space_disc(ml, m, ed, ia, r0, coloring, reorder, staged, layout, dtype)
    if dtype == "f64":
        ref = oracle.space_disc(m.edge2cell, ed, m.eflag, ia, res=r0)
        assert rel_l2(got - r0, ref - r0) <= 1e-12
    else:
        r0r = round_to(r0, np.float32)
        ref = oracle.space_disc(m.edge2cell, round_to(ed, np.float32), m.eflag, round_to(ia, np.float32), res=r0r)
        assert rel_l2(got - r0r, ref - r0r) <= 1e-5


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("coloring,reorder,staged", VARIANTS)
def test_getacc_parity(ml, coloring, reorder, staged, layout, dtype):
    m, cd = quad_case(97, 53)
    n0 = 0.1 * np.cos(np.arange(4 * m.nnode)).reshape(-1, 4)
    got = run_getacc(ml, m, cd, n0, coloring, reorder, staged, layout, dtype)
    if dtype == "f64":
        ref = oracle.getacc(m.cell2node, cd, m.nnode, nd=n0)
        assert rel_l2(got - n0, ref - n0) <= 1e-12
    else:
        n0r = round_to(n0, np.float32)
        ref = oracle.getacc(m.cell2node, round_to(cd, np.float32), m.nnode, nd=n0r)
        assert rel_l2(got - n0r, ref - n0r) <= 1e-5


@pytest.mark.parametrize("block_size", [32, 128, 512])
def test_increment_loops_ragged_and_deterministic(ml, block_size):
    """Block sizes from 32 (many colours, corner cells with 5 gather
    entries) to 512; two staged runs give the same bits."""
    m, ed, ia = tri_case(31, 17)
    z = np.zeros((m.ncell, 4))
    ref = oracle.space_disc(m.edge2cell, ed, m.eflag, ia)
    for staged in (None, "simple"):
        a = run_space_disc(ml, m, ed, ia, z, "hier", "partition", staged, "aos", "f64", block_size=block_size)
        b = run_space_disc(ml, m, ed, ia, z, "hier", "partition", staged, "aos", "f64", block_size=block_size)
        assert rel_l2(a, ref) <= 1e-12 and np.array_equal(a, b)
    q, cd = quad_case(29, 19)
    zn = np.zeros((q.nnode, 4))
    refn = oracle.getacc(q.cell2node, cd, q.nnode)
    for staged in (None, "simple"):
        a = run_getacc(ml, q, cd, zn, "hier", "partition", staged, "soa", "f64", block_size=block_size)
        b = run_getacc(ml, q, cd, zn, "hier", "partition", staged, "soa", "f64", block_size=block_size)
        assert rel_l2(a, refn) <= 1e-12 and np.array_equal(a, b)


def test_increment_loops_reject_wrong_plans(ml):
    m, ed, ia = tri_case(5, 4)
    from paper_1802_03749_gb300.mesh import ScatterPlan
    S = ScatterPlan(m.nnode, meshgen.quad_mesh(5, 4).cell2node[:m.ncell % 20 or 1])
    z = torch.zeros(64, dtype=torch.float32, device="cuda")
    zi = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(ml.MeshLoopError):
        ml.loop_space_disc(S.plan, z, zi, z, z)    # arity 4 plan
    T = ScatterPlan(m.ncell, m.edge2cell)
    with pytest.raises(ml.MeshLoopError):
        ml.loop_getacc(T.plan, z, z)               # arity 2 plan


@pytest.mark.slow
def test_increment_loops_full_size(ml):
    """The benchmark's workloads: the edge loop on 1100x1100 quads split
    into 2.42M triangles (3.63M edges), FP32, partitioned, block 256; the
    cell loop on 2000x2000 quads (4M cells), FP64; every output checked."""
    m, ed, ia = tri_case(1100, 1100)
    z = np.zeros((m.ncell, 4))
    got = run_space_disc(ml, m, ed, ia, z, "hier", "partition", None, "aos", "f32")
    ref = oracle.space_disc(m.edge2cell, round_to(ed, np.float32), m.eflag, round_to(ia, np.float32))
    assert rel_l2(got, ref) <= 1e-5
    CASES.clear()
    q, cd = quad_case(2000, 2000)
    got = run_getacc(ml, q, cd, np.zeros((q.nnode, 4)), "hier", "partition", None, "aos", "f64")
    assert rel_l2(got, oracle.getacc(q.cell2node, cd, q.nnode)) <= 1e-12
    CASES.clear()
