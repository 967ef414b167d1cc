"""The failure modes the paper names for the staged scheme (Sec. 3.1.5),
in forms that fault nothing: a block footprint larger than the shared
memory a CTA may opt into is rejected on the host with MP_ESMEM before any
launch, the device error word stays clear, and the same mesh runs once its
blocks are smaller.  (The 256-colour limit, MP_ECOLORS, is a planner error:
tests/test_plan.py.)  And the bounded grid-wide wait of the persistent
launches: a wait that can only run out returns MP_ETIMEOUT through the
device error word after its limit, and the GPU stays usable."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def no_reuse_mesh(nedge, seed=5):
    """nedge edges that share no node and no cell: edge i joins nodes 2i,
    2i+1 and cells 2i, 2i+1, so a block of S edges stages 2S cells and 2S
    nodes (reuse factor 1, the worst case for shared memory)."""
    rng = np.random.default_rng(seed)
    e2n = np.arange(2 * nedge, dtype=np.int32).reshape(-1, 2)
    e2c = np.arange(2 * nedge, dtype=np.int32).reshape(-1, 2)
    x = rng.uniform(0.0, 1.0, (2 * nedge, 2))
    q = np.column_stack([rng.uniform(0.9, 1.1, 2 * nedge), rng.uniform(-0.1, 0.5, 2 * nedge),
                         rng.uniform(-0.1, 0.1, 2 * nedge), rng.uniform(1.8, 2.0, 2 * nedge)])
    adt = rng.uniform(0.5, 1.0, 2 * nedge)
    return e2n, e2c, x, q, adt


def run(ml, e2n, e2c, x, q, adt, block_size, block_of):
    P = ml.Plan([{"to_set": 1, "idx": e2n, "to_size": x.shape[0]},
                 {"to_set": 2, "idx": e2c, "to_size": q.shape[0], "written": True}], e2n.shape[0],
                block_size=block_size, coloring="hier", block_of=block_of, staged="simple")
    cp, npm = P.perm(2), P.perm(1)
    xd = torch.tensor(x[npm], device="cuda")
    qd = torch.tensor(q[cp], device="cuda")
    ad = torch.tensor(adt[cp], device="cuda")
    res = torch.zeros_like(qd)
    ml.loop_res_calc(P, xd, qd, ad, res)
    torch.cuda.synchronize()
    out = np.empty_like(q)
    out[cp] = res.cpu().numpy()
    return P, out


def test_footprint_beyond_shared_memory_is_rejected_before_launch():
    import paper_1802_03749_gb300 as ml
    n = 1024
    e2n, e2c, x, q, adt = no_reuse_mesh(n)
    # one block of 1024 edges: 2048 cells x 108 B + 2048 nodes x 16 B of FP64
    # staging = 253,952 B, above the 227 KB a CTA may opt into
    with pytest.raises(ml.MeshLoopError) as e:
        run(ml, e2n, e2c, x, q, adt, 1024, np.zeros(n, np.int32))
    assert e.value.name == "MP_ESMEM"
    ml.mp_check_device_status()   # nothing was launched: the device error word is clear
    # the same edges in two blocks of 512 fit, and match the oracle
    P, got = run(ml, e2n, e2c, x, q, adt, 1024, (np.arange(n) >= n // 2).astype(np.int32))
    assert P.stats()["nblocks"] == 2
    ref = oracle.res_calc(e2n, e2c, x, q, adt)
    assert rel_l2(got, ref) <= 1e-12
    ml.mp_check_device_status()


def test_footprint_limit_is_per_kernel_layout():
    """The FP32 kernel stages half the bytes per point: the block of 1024
    edges that FP64 rejects fits in FP32."""
    import paper_1802_03749_gb300 as ml
    n = 1024
    e2n, e2c, x, q, adt = no_reuse_mesh(n, seed=6)
    P = ml.Plan([{"to_set": 1, "idx": e2n, "to_size": x.shape[0]},
                 {"to_set": 2, "idx": e2c, "to_size": q.shape[0], "written": True}], n,
                block_size=1024, coloring="hier", block_of=np.zeros(n, np.int32), staged="simple")
    cp, npm = P.perm(2), P.perm(1)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    xd, qd, ad = t(x[npm]), t(q[cp]), t(adt[cp])
    res = torch.zeros_like(qd)
    ml.loop_res_calc(P, xd, qd, ad, res)
    torch.cuda.synchronize()
    ml.mp_check_device_status()
    got = np.empty_like(q)
    got[cp] = res.double().cpu().numpy()
    r = lambda a: a.astype(np.float32).astype(np.float64)
    ref = oracle.res_calc(e2n, e2c, r(x), r(q), r(adt))
    assert rel_l2(got, ref) <= 1e-5


def test_grid_wait_runs_out_and_reports_timeout():
    import paper_1802_03749_gb300 as ml
    ml.mp_grid_wait_test(8, 50_000_000, 0)        # every arrival comes: no error
    ml.mp_check_device_status()
    ml.mp_grid_wait_test(8, 20_000_000, 1)        # one arrival never comes: 20 ms, then MP_ETIMEOUT
    with pytest.raises(ml.MeshLoopError) as e:
        ml.mp_check_device_status()
    assert e.value.name == "MP_ETIMEOUT"
    ml.mp_check_device_status()                   # the status word was cleared
    ml.mp_grid_wait_test(8, 50_000_000, 0)        # and the device still works
    ml.mp_check_device_status()
    with pytest.raises(ml.MeshLoopError) as e:
        ml.mp_grid_wait_test(0, 1000, 0)
    assert e.value.name == "MP_EINVAL"
