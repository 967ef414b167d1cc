"""GPU parity of batched execution: the fused two-layer plan and the batched
time step over meshes of uneven size, against the FP64 oracle mesh by mesh."""
import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import rel_l2, round_to

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def small_batch():
    sizes = [(20, 10), (37, 9), (64, 32), (15, 15), (50, 21)]
    meshes = [meshgen.quad_mesh(nx, ny, seed=100 + i) for i, (nx, ny) in enumerate(sizes)]
    states = [meshgen.quad_state(m.ncell, seed=200 + i) for i, m in enumerate(meshes)]
    return meshes, states


@pytest.mark.parametrize("staged,dtype", [(None, "f64"), ("persistent", "f64"), ("persistent", "f32")])
def test_fused_res_calc_matches_per_mesh_oracle(staged, dtype):
    """The fused plan of meshes of uneven size: one launch per colour phase,
    or one persistent launch for the whole batch (FP64, and FP32 against the
    oracle on FP32-rounded inputs)."""
    import paper_1802_03749_gb300 as ml
    from paper_1802_03749_gb300.mesh import AirfoilPlans
    meshes, states = small_batch()
    adts = [oracle.adt_calc(m.cell2node, m.x, q) for m, q in zip(meshes, states)]
    opts = [(128, "partition"), (256, "rcm"), (480, "partition"), (64, "rcm"), (256, "partition")]
    Ps = [AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                       block_size=bs, reorder=ro) for m, (bs, ro) in zip(meshes, opts)]
    B = ml.Plan.batch([P.res for P in Ps])
    B.set_staged(staged)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    cat = lambda arrs: torch.tensor(np.concatenate(arrs), dtype=tdt, device="cuda")
    x = cat([P.to_plan(m.x, "node") for P, m in zip(Ps, meshes)])
    q = cat([P.to_plan(s, "cell") for P, s in zip(Ps, states)])
    adt = cat([P.to_plan(a, "cell") for P, a in zip(Ps, adts)])
    res = torch.zeros_like(q)
    ml.loop_res_calc(B, x, q, adt, res)
    ml.mp_check_device_status()
    out = res.double().cpu().numpy()
    off = 0
    r = (lambda a: round_to(a, np.float32)) if dtype == "f32" else (lambda a: a)
    for P, m, s, a in zip(Ps, meshes, states, adts):
        got = P.from_plan(out[off:off + m.ncell], "cell", 4)
        off += m.ncell
        ref = oracle.res_calc(m.edge2node, m.edge2cell, r(m.x), r(s), r(a))
        assert rel_l2(got, ref) <= (1e-12 if dtype == "f64" else 1e-5)


def test_persistent_launch_in_a_graph():
    """The persistent (cooperative) res_calc launch captured in a CUDA graph
    and replayed gives the eager launch's bits."""
    import paper_1802_03749_gb300 as ml
    from paper_1802_03749_gb300.mesh import AirfoilPlans
    m = meshgen.quad_mesh(90, 45, seed=7)
    s = meshgen.quad_state(m.ncell, seed=7)
    a = oracle.adt_calc(m.cell2node, m.x, s)
    P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                     block_size=128, reorder="partition", staged="persistent")
    P.res.upload()
    t = lambda v, w: torch.tensor(P.to_plan(v, w), device="cuda")
    x, q, adt = t(m.x, "node"), t(s, "cell"), t(a, "cell")
    eager = torch.zeros_like(q)
    ml.loop_res_calc(P.res, x, q, adt, eager)
    torch.cuda.synchronize()
    res = torch.zeros_like(q)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        ml.loop_res_calc(P.res, x, q, adt, res)
    for _ in range(3):
        res.zero_()
        g.replay()
    torch.cuda.synchronize()
    ml.mp_check_device_status()
    assert torch.equal(res, eager)
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, s, a)
    assert rel_l2(P.from_plan(res.cpu().numpy(), "cell", 4), ref) <= 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_step_matches_oracle(dtype):
    from paper_1802_03749_gb300.mesh import AirfoilBatch
    meshes, states = small_batch()
    qinf = meshgen.freestream()
    choices = [(256, "partition", "hier"), (256, "rcm", "atomic"), (256, "rcm", "hier"),
               (256, "rcm", "atomic"), (256, "partition", "hier")]
    Bt = AirfoilBatch(meshes, states, qinf, choices, dtype=dtype)
    ref = [round_to(s, np.float32) if dtype == "f32" else s.copy() for s in states]
    rms_tot = 0.0
    for step in range(3):
        Bt.rms.zero_()
        Bt.step()
        torch.cuda.synchronize()
        tot = 0.0
        for k, m in enumerate(meshes):
            r, _ = oracle.step(m, ref[k], qinf)
            tot += r * r * m.ncell
            err = rel_l2(Bt.q_of(k), ref[k])
            assert err <= (1e-12 if dtype == "f64" else 1e-5), (step, k, err)
        rms = Bt.rms.item()
        assert abs(rms - tot) <= (1e-12 if dtype == "f64" else 1e-4) * tot


def test_batched_graph_replay_matches_eager():
    from paper_1802_03749_gb300.mesh import AirfoilBatch
    meshes, states = small_batch()
    qinf = meshgen.freestream()
    choices = [(256, "partition", "hier")] * 5
    A = AirfoilBatch(meshes, states, qinf, choices)
    E = AirfoilBatch(meshes, states, qinf, choices)
    A.capture(steps_per_graph=2)
    E.step()
    for _ in range(3):
        A.graph.replay()
        E.step()
        E.step()
    torch.cuda.synchronize()
    assert torch.equal(A.q, E.q)
