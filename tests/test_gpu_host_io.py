"""loop_res_calc_host: res_calc on host arrays through the C ABI gives the
same bits as the device-array call, with pinned and pageable memory, and
consecutive calls on two streams (two device buffer slots) stay correct."""
import numpy as np
import pytest

import oracle
from gpu_util import airfoil_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    import paper_1802_03749_gb300 as ml
    from paper_1802_03749_gb300.mesh import AirfoilPlans
    m, q, adt = airfoil_case(97, 53)
    P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                     block_size=256, reorder="partition")
    return ml, m, q, adt, P


@pytest.mark.parametrize("dtype,compute", [("f64", None), ("f64", "dw"), ("f32", None)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_call_matches_device_call(setup, dtype, compute, pinned):
    ml, m, q, adt, P = setup
    tdt = torch.float64 if dtype == "f64" else torch.float32
    r0 = 0.01 * np.cos(np.arange(q.size)).reshape(q.shape)
    host = [torch.tensor(P.to_plan(a, w), dtype=tdt) for a, w in ((m.x, "node"), (q, "cell"), (adt, "cell"),
                                                                     (r0, "cell"))]
    if pinned:
        host = [h.pin_memory() for h in host]
    dev = [h.cuda() for h in host]
    ml.loop_res_calc(P.res, *dev, compute=compute)
    ml.loop_res_calc_host(P.res, *host, compute=compute)
    torch.cuda.synchronize()
    assert torch.equal(host[3], dev[3].cpu())
    ml.mp_check_device_status()


def test_two_streams_alternating(setup):
    """Four calls alternating two streams, each with its own host arrays and
    a different res, against the oracle."""
    ml, m, q, adt, P = setup
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ref = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    outs = []
    for k in range(4):
        r0 = (k + 1) * 0.01 * np.sin(np.arange(q.size) + k).reshape(q.shape)
        host = [torch.tensor(P.to_plan(a, w)).pin_memory() for a, w in ((m.x, "node"), (q, "cell"),
                                                                        (adt, "cell"), (r0, "cell"))]
        ml.loop_res_calc_host(P.res, *host, stream=streams[k % 2], compute="dw")
        outs.append((r0, host[3]))
    torch.cuda.synchronize()
    for r0, hres in outs:
        got = P.from_plan(hres.numpy(), "cell", 4)
        assert rel_l2(got - r0, ref) <= 1e-12
    ml.mp_check_device_status()
