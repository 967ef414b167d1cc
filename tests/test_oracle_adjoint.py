"""Pins of the oracle's hand-derived res_calc adjoint: the complex-step
forward derivative (exact to rounding, since the flux is rational), the
dot-product test and central finite differences.  CPU only."""
import numpy as np
import pytest

import meshgen
import oracle


@pytest.fixture(scope="module")
def case():
    m = meshgen.quad_mesh(24, 12, seed=21)
    q = meshgen.quad_state(m.ncell, seed=21, noise=0.05)
    adt = meshgen.positive_field(m.ncell, 0.05, 0.15, seed=21)
    rb = meshgen.adjoint_seed(m.ncell, seed=21)
    return m, q, adt, rb


def test_complex_step_real_part_is_res(case):
    m, q, adt, _ = case
    d = meshgen.directions(m.ncell * 4 + m.nnode * 2, 1, seed=21)[0]
    re, _ = oracle.res_calc_cstep(m.edge2node, m.edge2cell, m.x, d[4 * m.ncell:].reshape(-1, 2), q,
                                  d[:4 * m.ncell].reshape(-1, 4), adt)
    res = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    np.testing.assert_allclose(re, res, rtol=1e-14, atol=1e-17)


def test_dot_product_identity(case):
    """<res_bar, J d> = <q_bar, d_q> + <x_bar, d_x> for random d."""
    m, q, adt, rb = case
    qb, xb = oracle.res_calc_adjoint(m.edge2node, m.edge2cell, m.x, q, adt, rb)
    for k, d in enumerate(meshgen.directions(m.ncell * 4 + m.nnode * 2, 5, seed=22)):
        dq = d[:4 * m.ncell].reshape(-1, 4)
        dx = d[4 * m.ncell:].reshape(-1, 2) * 1e-3
        _, jd = oracle.res_calc_cstep(m.edge2node, m.edge2cell, m.x, dx, q, dq, adt)
        lhs = float((rb * jd).sum())
        rhs = float((qb * dq).sum() + (xb * dx).sum())
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-14)


def test_central_differences_100_directions(case):
    """Central FD, h = 1e-6, on 100 random directions: agreement limited by
    the FD truncation and cancellation error."""
    m, q, adt, rb = case
    qb, xb = oracle.res_calc_adjoint(m.edge2node, m.edge2cell, m.x, q, adt, rb)
    h = 1e-6
    worst = 0.0
    for d in meshgen.directions(m.ncell * 4 + m.nnode * 2, 100, seed=23):
        dq = d[:4 * m.ncell].reshape(-1, 4) * q.std(axis=0)
        dx = d[4 * m.ncell:].reshape(-1, 2) * m.h * 0.1
        rp = oracle.res_calc(m.edge2node, m.edge2cell, m.x + h * dx, q + h * dq, adt)
        rm = oracle.res_calc(m.edge2node, m.edge2cell, m.x - h * dx, q - h * dq, adt)
        fd = float((rb * (rp - rm)).sum()) / (2 * h)
        ad = float((qb * dq).sum() + (xb * dx).sum())
        scale = float(np.abs(qb * dq).sum() + np.abs(xb * dx).sum())
        worst = max(worst, abs(fd - ad) / scale)
    assert worst < 1e-7
