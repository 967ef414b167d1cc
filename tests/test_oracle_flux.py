"""Pins of the FP64 oracle's 2D loops (res_calc, bres_calc, adt_calc,
update, step) against hand-computed values, closed forms, invariants and
brute force.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import meshgen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GAM, EPS, CFL = oracle.GAMMA, oracle.EPS, oracle.CFL


@pytest.fixture(scope="module")
def small():
    m = meshgen.quad_mesh(40, 20, seed=7)
    q = meshgen.quad_state(m.ncell, seed=7)
    adt = meshgen.positive_field(m.ncell, 0.05, 0.15, seed=7)
    return m, q, adt


def test_edge_flux_worked_example():
    """Hand-computed single edge between motionless cells (fixture)."""
    g = json.load(open(os.path.join(GOLD, "flux_quiescent.json")))
    f = oracle.edge_flux(g["xa"], g["xb"], g["q1"], g["q2"], g["adt1"], g["adt2"], g["gam"], g["eps"])
    np.testing.assert_allclose(f, g["f"], rtol=0, atol=1e-15)


def test_edge_flux_uniform_state_primitive_form():
    """q1 = q2: the dissipation vanishes and f is the textbook Euler normal
    flux written from primitive variables (rho, u, v, p)."""
    rho, u, v, p = 1.3, 0.25, -0.4, 0.9
    E = p / (GAM - 1) + 0.5 * rho * (u * u + v * v)
    q = [rho, rho * u, rho * v, E]
    xa, xb = [0.2, 0.9], [0.5, 0.1]
    nx, ny = xa[1] - xb[1], -(xa[0] - xb[0])
    un = u * nx + v * ny
    expect = [rho * un, rho * u * un + p * nx, rho * v * un + p * ny, (E + p) * un]
    f = oracle.edge_flux(xa, xb, q, q, 0.7, 0.3)
    np.testing.assert_allclose(f, expect, rtol=1e-14, atol=1e-15)


def test_swap_orientation_is_bitwise_neutral(small):
    """Swapping c1<->c2 together with a<->b flips n and f exactly, so res is
    bit-identical."""
    m, q, adt = small
    r1 = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    e2n = m.edge2node.copy()
    e2c = m.edge2cell.copy()
    sel = np.arange(m.nedge) % 3 == 0
    e2n[sel] = e2n[sel][:, ::-1]
    e2c[sel] = e2c[sel][:, ::-1]
    r2 = oracle.res_calc(e2n, e2c, m.x, q, adt)
    assert np.array_equal(r1, r2)


def test_conservation(small):
    """Each interior flux is added to one cell and subtracted from another:
    the increments sum to zero."""
    m, q, adt = small
    res = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    scale = np.abs(res).sum(axis=0)
    assert np.all(np.abs(res.sum(axis=0)) <= 1e-13 * scale)


def test_cell_gather_equals_edge_scatter():
    """Brute force in another loop order: for each cell, sum +f over edges
    where it is c1 and -f where it is c2, one edge flux at a time."""
    m = meshgen.quad_mesh(12, 7, seed=3)
    q = meshgen.quad_state(m.ncell, seed=3)
    adt = meshgen.positive_field(m.ncell, 0.05, 0.15, seed=3)
    res = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    f = np.array([oracle.edge_flux(m.x[a], m.x[b], q[c1], q[c2], adt[c1], adt[c2])
                  for (a, b), (c1, c2) in zip(m.edge2node, m.edge2cell)])
    gather = np.zeros_like(res)
    for c in range(m.ncell):
        for e in range(m.nedge):
            if m.edge2cell[e, 0] == c:
                gather[c] += f[e]
            if m.edge2cell[e, 1] == c:
                gather[c] -= f[e]
    np.testing.assert_allclose(gather, res, rtol=1e-13, atol=1e-16)
    # every cell of a 12x7 grid with boundary has at least two interior edges
    assert np.all(np.abs(res).sum(axis=1) > 0)


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_freestream_residual_vanishes(jitter):
    """q = q_inf everywhere: every cell is closed by its interior and
    boundary edges, so res = F(q_inf) . sum(n_out) = 0 and the dissipation
    terms vanish (q1 = q2 = q_inf)."""
    m = meshgen.quad_mesh(30, 17, seed=11, jitter=jitter)
    qinf = meshgen.freestream()
    q = np.tile(qinf, (m.ncell, 1))
    adt = meshgen.positive_field(m.ncell, 0.05, 0.15, seed=11)
    res = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    res = oracle.bres_calc(m.bedge2node, m.bedge2cell, m.x, q, adt, qinf, res=res)
    fscale = np.abs(qinf).max() * m.h
    assert np.abs(res).max() <= 1e-13 * fscale
    # and the interior-edge loop alone does not vanish on boundary cells
    res2 = oracle.res_calc(m.edge2node, m.edge2cell, m.x, q, adt)
    assert np.abs(res2).max() > 1e-3 * fscale


def test_bres_single_edge_is_boundary_flux():
    """q_c = q_inf: f = F(q_inf).n exactly (textbook primitive form)."""
    qinf = meshgen.freestream()
    rho, u, v = qinf[0], qinf[1] / qinf[0], qinf[2] / qinf[0]
    p = 1.0 / GAM
    x = np.array([[0.4, 0.0], [0.1, 0.0]])   # bottom edge, a=(0.4,0), b=(0.1,0): n = (0, -0.3)
    res = oracle.bres_calc(np.array([[0, 1]]), np.array([[0]]), x, qinf[None, :], np.array([0.3]), qinf)
    nx, ny = 0.0, -0.3
    un = u * nx + v * ny
    expect = [rho * un, rho * u * un + p * nx, rho * v * un + p * ny, (qinf[3] + p) * un]
    np.testing.assert_allclose(res[0], expect, rtol=1e-14, atol=1e-16)
    # a state away from q_inf adds eps * adt * (q_c - q_inf) on top of F(q_b).n
    qc = qinf * np.array([1.1, 0.9, 1.2, 1.05])
    qb = 0.5 * (qc + qinf)
    rb, ub, vb = qb[0], qb[1] / qb[0], qb[2] / qb[0]
    pb = (GAM - 1) * (qb[3] - 0.5 * rb * (ub * ub + vb * vb))
    unb = ub * nx + vb * ny
    expect = np.array([rb * unb, rb * ub * unb + pb * nx, rb * vb * unb + pb * ny, (qb[3] + pb) * unb])
    expect += EPS * 0.3 * (qc - qinf)
    res = oracle.bres_calc(np.array([[0, 1]]), np.array([[0]]), x, qc[None, :], np.array([0.3]), qinf)
    np.testing.assert_allclose(res[0], expect, rtol=1e-14, atol=1e-16)


def test_adt_closed_form_unjittered():
    """Unjittered h x h cell, free stream: sides (h,0),(0,h),(-h,0),(0,-h)
    give adt = (2h(|u| + |v|) + 4 h c) / cfl with c = sqrt(gam p/rho) = 1."""
    m = meshgen.quad_mesh(20, 10, seed=5, jitter=0.0)
    qinf = meshgen.freestream()
    q = np.tile(qinf, (m.ncell, 1))
    adt = oracle.adt_calc(m.cell2node, m.x, q)
    u, v = qinf[1], qinf[2]
    expect = (2 * m.h * (abs(u) + abs(v)) + 4 * m.h * 1.0) / CFL
    np.testing.assert_allclose(adt, expect, rtol=1e-13)


def test_update_closed_form():
    qold = np.array([[1.0, 2.0, 3.0, 4.0], [0.5, -1.0, 0.25, 8.0]])
    res = np.array([[0.5, -1.0, 0.25, 2.0], [1.0, 1.0, -3.0, 0.0]])
    adt = np.array([2.0, 4.0])
    q = np.zeros_like(qold)
    s = oracle.update(qold, q, res, adt)
    d = np.array([[0.25, -0.5, 0.125, 1.0], [0.25, 0.25, -0.75, 0.0]])
    assert np.array_equal(q, qold - d)
    assert np.all(res == 0)
    assert s == pytest.approx(float((d * d).sum()), rel=0, abs=1e-15)


def test_step_freestream_is_fixed_point():
    m = meshgen.quad_mesh(16, 9, seed=9)
    qinf = meshgen.freestream()
    q = np.tile(qinf, (m.ncell, 1))
    rms, work = oracle.step(m, q, qinf)
    assert rms < 1e-14
    np.testing.assert_allclose(q, np.tile(qinf, (m.ncell, 1)), rtol=1e-14)


def test_step_decreases_residual():
    """The explicit step is a damped iteration towards steady state: the
    residual of a perturbed free stream falls over the first steps."""
    m = meshgen.quad_mesh(40, 20, seed=2)
    qinf = meshgen.freestream()
    q = meshgen.quad_state(m.ncell, seed=2)
    rms = [oracle.step(m, q, qinf)[0] for _ in range(20)]
    assert all(np.isfinite(rms))
    assert rms[-1] < 0.5 * rms[0]
