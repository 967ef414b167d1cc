"""GPU parity of the res_calc adjoint against the oracle's hand-derived
adjoint, the complex-step dot-product identity and central finite
differences (h = 1e-6, 100 directions), through the C ABI and autograd."""
import numpy as np
import pytest

import meshgen
import oracle
from gpu_util import airfoil_case, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def setup(nx, ny, coloring="hier", reorder="partition", layout="aos", block_size=480):
    from paper_1802_03749_gb300.mesh import AirfoilPlans
    m, q, adt = airfoil_case(nx, ny, noise=0.05)
    rb = meshgen.adjoint_seed(m.ncell)
    P = AirfoilPlans(m.ncell, m.nnode, m.edge2node, m.edge2cell, m.bedge2node, m.bedge2cell, m.cell2node,
                     block_size=block_size, reorder=reorder, coloring=coloring, layout=layout, adjoint=True)
    return m, q, adt, rb, P


def gpu_adjoint(m, q, adt, rb, P, compute=None):
    import paper_1802_03749_gb300 as ml
    t = lambda a, w: torch.tensor(P.to_plan(a, w), dtype=torch.float64, device="cuda")
    x, qd, ad, rbd = t(m.x, "node"), t(q, "cell"), t(adt, "cell"), t(rb, "cell")
    qb = torch.zeros_like(qd)
    xb = torch.zeros_like(x)
    ml.loop_adjoint(P.res, x, qd, ad, rbd, qb, xb, compute=compute)
    ml.mp_check_device_status()
    torch.cuda.synchronize()
    return P.from_plan(qb.cpu().numpy(), "cell", 4), P.from_plan(xb.cpu().numpy(), "node", 2)


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("coloring,reorder", [("hier", "partition"), ("hier", "rcm"), ("global", "rcm"),
                                              ("atomic", "none")])
def test_adjoint_matches_oracle(coloring, reorder, layout):
    m, q, adt, rb, P = setup(200, 100, coloring, reorder, layout)
    qb, xb = gpu_adjoint(m, q, adt, rb, P)
    qr, xr = oracle.res_calc_adjoint(m.edge2node, m.edge2cell, m.x, q, adt, rb)
    assert rel_l2(qb, qr) <= 1e-12
    assert rel_l2(xb, xr) <= 1e-12


def test_adjoint_dot_product_and_fd():
    """<res_bar, J d> (complex step) = <q_bar, d_q> + <x_bar, d_x> to 1e-13
    and central differences agree to FD accuracy, on 100 directions; both
    relative to the sum of the absolute terms of the dot product, the scale
    of its rounding error (some directions cancel by a factor of 1e5, where
    even the oracle's own adjoint misses the identity by 3e-12 of the sum)."""
    m, q, adt, rb, P = setup(60, 30)
    qb, xb = gpu_adjoint(m, q, adt, rb, P)
    worst_cs, worst_fd = 0.0, 0.0
    h = 1e-6
    for d in meshgen.directions(m.ncell * 4 + m.nnode * 2, 100, seed=41):
        dq = d[:4 * m.ncell].reshape(-1, 4) * q.std(axis=0)
        dx = d[4 * m.ncell:].reshape(-1, 2) * m.h * 0.1
        ad = float((qb * dq).sum() + (xb * dx).sum())
        # rounding in a dot product is bounded relative to the sum of its
        # absolute terms, not to |ad| (which may nearly cancel)
        scale = float(np.abs(qb * dq).sum() + np.abs(xb * dx).sum())
        _, jd = oracle.res_calc_cstep(m.edge2node, m.edge2cell, m.x, dx, q, dq, adt)
        worst_cs = max(worst_cs, abs(float((rb * jd).sum()) - ad) / scale)
        rp = oracle.res_calc(m.edge2node, m.edge2cell, m.x + h * dx, q + h * dq, adt)
        rm = oracle.res_calc(m.edge2node, m.edge2cell, m.x - h * dx, q - h * dq, adt)
        fd = float((rb * (rp - rm)).sum()) / (2 * h)
        worst_fd = max(worst_fd, abs(fd - ad) / scale)
    assert worst_cs <= 1e-13
    assert worst_fd <= 1e-7


def test_autograd_function():
    """torch.autograd through ResCalc: grad of <res, res_bar> is the adjoint."""
    from paper_1802_03749_gb300.autograd import res_calc
    m, q, adt, rb, P = setup(80, 40)
    t = lambda a, w: torch.tensor(P.to_plan(a, w), dtype=torch.float64, device="cuda")
    x = t(m.x, "node").requires_grad_(True)
    qd = t(q, "cell").requires_grad_(True)
    ad = t(adt, "cell")
    res = res_calc(x, qd, ad, P.res)
    np.testing.assert_allclose(P.from_plan(res.detach().cpu().numpy(), "cell", 4),
                               oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt), rtol=0, atol=1e-13)
    (res * t(rb, "cell")).sum().backward()
    qr, xr = oracle.res_calc_adjoint(m.edge2node, m.edge2cell, m.x, q, adt, rb)
    assert rel_l2(P.from_plan(qd.grad.cpu().numpy(), "cell", 4), qr) <= 1e-12
    assert rel_l2(P.from_plan(x.grad.cpu().numpy(), "node", 2), xr) <= 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("reorder,block_size", [("partition", 128), ("partition", 384), ("rcm", 256),
                                                ("none", 480), ("partition", 1024)])
def test_adjoint_native_gather_and_colours(reorder, block_size, layout, dtype):
    """Native arithmetic, gather increments (the default) and thread colours
    (Algorithm 1): FP64 within the FP64 bar, FP32 storage and arithmetic
    within 1e-5 of the FP64 oracle fed the same FP32-rounded inputs; the
    gather form is deterministic."""
    import paper_1802_03749_gb300 as ml
    from gpu_util import round_to
    m, q, adt, rb, P = setup(97, 53, "hier", reorder, layout, block_size=block_size)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        m.x, q, adt, rb = (round_to(a, np.float32) for a in (m.x, q, adt, rb))
    qr, xr = oracle.res_calc_adjoint(m.edge2node, m.edge2cell, m.x, q, adt, rb)
    t = lambda a, w: torch.tensor(P.to_plan(a, w), dtype=tdt, device="cuda")
    x, qd, ad, rbd = t(m.x, "node"), t(q, "cell"), t(adt, "cell"), t(rb, "cell")
    bar = 1e-12 if dtype == "f64" else 1e-5
    out = {}
    for staged in ("gather", None, "simple"):
        P.res.set_staged(staged)
        qb, xb = torch.zeros_like(qd), torch.zeros_like(x)
        ml.loop_adjoint(P.res, x, qd, ad, rbd, qb, xb)
        ml.mp_check_device_status()
        qb = P.from_plan(qb.double().cpu().numpy(), "cell", 4)
        xb = P.from_plan(xb.double().cpu().numpy(), "node", 2)
        assert rel_l2(qb, qr) <= bar, staged
        assert rel_l2(xb, xr) <= bar, staged
        out[staged] = (qb, xb)
    # the default is the gather form, and it gives the same bits every call
    assert all(np.array_equal(a, b) for a, b in zip(out["gather"], out[None]))


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("reorder,block_size", [("partition", 128), ("rcm", 256), ("none", 480)])
def test_adjoint_double_word_parity(reorder, block_size, layout):
    """FP64 data with double-word arithmetic, gather (default) and
    thread-coloured increments: within the FP64 bar; the gather form is
    deterministic."""
    m, q, adt, rb, P = setup(200, 100, "hier", reorder, layout, block_size=block_size)
    qr, xr = oracle.res_calc_adjoint(m.edge2node, m.edge2cell, m.x, q, adt, rb)
    for staged in (None, "simple"):
        P.res.set_staged(staged)
        qb, xb = gpu_adjoint(m, q, adt, rb, P, compute="dw")
        assert rel_l2(qb, qr) <= 1e-12
        assert rel_l2(xb, xr) <= 1e-12
        if staged is None:
            qb2, xb2 = gpu_adjoint(m, q, adt, rb, P, compute="dw")
            assert np.array_equal(qb, qb2) and np.array_equal(xb, xb2)


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("coloring,reorder", [("global", "rcm"), ("atomic", "rcm"), ("atomic", "none")])
def test_adjoint_double_word_baselines(coloring, reorder, layout):
    """Global colouring and atomics (Sec. 2.1) in double-word arithmetic on
    FP64 data: within the FP64 bar, like the two-layer form."""
    m, q, adt, rb, P = setup(200, 100, coloring, reorder, layout)
    qr, xr = oracle.res_calc_adjoint(m.edge2node, m.edge2cell, m.x, q, adt, rb)
    qb, xb = gpu_adjoint(m, q, adt, rb, P, compute="dw")
    assert rel_l2(qb, qr) <= 1e-12
    assert rel_l2(xb, xr) <= 1e-12


@pytest.mark.slow
def test_adjoint_full_size():
    """The adjoint workload, 1200x600 quads, native FP64 and double-word."""
    m, q, adt, rb, P = setup(1200, 600, "hier", "partition", "aos", block_size=128)
    qr, xr = oracle.res_calc_adjoint(m.edge2node, m.edge2cell, m.x, q, adt, rb)
    for compute in (None, "dw"):
        qb, xb = gpu_adjoint(m, q, adt, rb, P, compute=compute)
        assert rel_l2(qb, qr) <= 1e-12
        assert rel_l2(xb, xr) <= 1e-12


@pytest.mark.slow
@pytest.mark.parametrize("compute", [None, "dw"])
def test_adjoint_fd_full_size(compute):
    """The adjoint workload (1200x600 quads, res_bar ~ N(0,1)): central
    finite differences of the oracle's forward res_calc (h = 1e-6) on 100
    random directions agree with the GPU adjoint, native FP64 and
    double-word, to FD accuracy."""
    m, q, adt, rb, P = setup(1200, 600, "hier", "partition", "aos", block_size=128)
    qb, xb = gpu_adjoint(m, q, adt, rb, P, compute=compute)
    h = 1e-6
    worst = 0.0
    for d in meshgen.directions(m.ncell * 4 + m.nnode * 2, 100, seed=43):
        dq = d[:4 * m.ncell].reshape(-1, 4) * q.std(axis=0)
        dx = d[4 * m.ncell:].reshape(-1, 2) * m.h * 0.1
        ad = float((qb * dq).sum() + (xb * dx).sum())
        rp = oracle.res_calc(m.edge2node, m.edge2cell, m.x + h * dx, q + h * dq, adt)
        rm = oracle.res_calc(m.edge2node, m.edge2cell, m.x - h * dx, q - h * dq, adt)
        fd = float((rb * (rp - rm)).sum()) / (2 * h)
        scale = float(np.abs(qb * dq).sum() + np.abs(xb * dx).sum())
        worst = max(worst, abs(fd - ad) / scale)
    assert worst <= 1e-7
