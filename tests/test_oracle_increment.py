"""Pins of the oracle's increment-only loops (Volna-style edge loop,
Sec. 3.1.2; BookLeaf-style cell loop, Sec. 3.1.3) against closed forms,
conservation and cell- or node-centric brute force.  CPU only."""
import numpy as np
import pytest

import meshgen
import oracle


@pytest.fixture(scope="module")
def tri():
    m = meshgen.tri_mesh(9, 6, seed=5)
    ed, ia = meshgen.volna_fields(m, seed=5)
    return m, ed, ia


def test_tri_mesh_is_a_triangulation(tri):
    """Every triangle counter-clockwise with positive area; every interior
    edge shared by two triangles and seen in opposite directions; the
    boundary is the rectangle's perimeter (2 (nx + ny) edges)."""
    m, ed, ia = tri
    assert np.all(ia > 0)
    assert m.ncell == 2 * 9 * 6 and m.nnode == 10 * 7
    assert m.eflag.sum() == 2 * (9 + 6)
    assert 3 * m.ncell == 2 * m.nedge - m.eflag.sum()      # each triangle has 3 edges
    # each edge's nodes appear consecutively (counter-clockwise) in c1, reversed in c2
    for e in range(m.nedge):
        a, b = m.edge2node[e]
        t1 = list(m.cell2node[m.edge2cell[e, 0]])
        i = t1.index(a)
        assert t1[(i + 1) % 3] == b
        if not m.eflag[e]:
            t2 = list(m.cell2node[m.edge2cell[e, 1]])
            j = t2.index(b)
            assert t2[(j + 1) % 3] == a
        else:
            assert m.edge2cell[e, 0] == m.edge2cell[e, 1]


def test_space_disc_cell_centric_brute_force(tri):
    """Cell by cell, each incident edge's contribution: the edge scatter
    must give the same result as this gather in another loop order."""
    m, ed, ia = tri
    got = oracle.space_disc(m.edge2cell, ed, m.eflag, ia)
    ref = np.zeros((m.ncell, 4))
    inc = {c: [] for c in range(m.ncell)}
    for e in range(m.nedge):
        inc[m.edge2cell[e, 0]].append((e, -1.0))
        if not m.eflag[e]:
            inc[m.edge2cell[e, 1]].append((e, 1.0))
    for c in range(m.ncell):
        for e, sgn in inc[c]:
            F0, F1, F2, P, L, nx, ny = ed[e]
            ref[c] += sgn * ia[c] * L * np.array([F0, F1 + P * nx, F2 + P * ny, P])
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_space_disc_linear_pressure_divergence_theorem(tri):
    """F = 0 and P the value of p(x, y) = x + 2 y at each edge's midpoint:
    the midpoint rule integrates a linear p exactly on straight edges, so by
    the divergence theorem the sum over a triangle's edges of L p n_out is
    A grad p = A (1, 2).  Every cell (interior or on the boundary) then gets
    momentum increments -(1, 2) and no mass increment."""
    m, ed, ia = tri
    e = ed.copy()
    mid = 0.5 * (m.x[m.edge2node[:, 0]] + m.x[m.edge2node[:, 1]])
    e[:, 0:3] = 0.0
    e[:, 3] = mid[:, 0] + 2.0 * mid[:, 1]
    r = oracle.space_disc(m.edge2cell, e, m.eflag, ia)
    assert np.abs(r[:, 0]).max() == 0.0
    np.testing.assert_allclose(r[:, 1], -1.0, rtol=0, atol=1e-11)
    np.testing.assert_allclose(r[:, 2], -2.0, rtol=0, atol=1e-11)


def test_space_disc_conservation(tri):
    """Interior edges add and subtract the same w: sum_c A_c res_c equals
    minus the boundary edges' w (and the flag is what keeps a boundary
    edge from counting twice)."""
    m, ed, ia = tri
    r = oracle.space_disc(m.edge2cell, ed, m.eflag, ia)
    lhs = (r / ia[:, None]).sum(0)
    b = m.eflag == 1
    F0, F1, F2, P, L, nx, ny = ed[b].T
    rhs = -np.array([(L * F0).sum(), (L * (F1 + P * nx)).sum(), (L * (F2 + P * ny)).sum(), (L * P).sum()])
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_getacc_uniform_closed_form():
    """Unpermuted structured quads, the same corner values in every cell:
    interior nodes collect 4 corners, edge nodes 2, corners 1, each corner
    k of a cell counter-clockwise from the lower left."""
    m = meshgen.quad_mesh(5, 4, seed=1, permute=False, jitter=0.0)
    cd = np.tile(np.array([2.0] + [1, 2, 3, 4] + [0.5, 0.25, 1, 2] + [1, -1, 2, -2] + [3, 1, -3, -1.0]), (m.ncell, 1))
    nd = oracle.getacc(m.cell2node, cd, m.nnode)
    ii, jj = np.meshgrid(np.arange(6), np.arange(5), indexing="xy")
    ii, jj = ii.ravel(), jj.ravel()
    # node (i, j) is corner 0 of cell (i, j), 1 of (i-1, j), 2 of (i-1, j-1), 3 of (i, j-1)
    exp = np.zeros((m.nnode, 4))
    for k, (di, dj) in enumerate([(0, 0), (-1, 0), (-1, -1), (0, -1)]):
        ci, cj = ii + di, jj + dj
        ok = (ci >= 0) & (ci < 5) & (cj >= 0) & (cj < 4)
        exp[ok] += np.array([cd[0, 1 + k], cd[0, 0] * cd[0, 5 + k], cd[0, 9 + k], cd[0, 13 + k]])
    np.testing.assert_array_equal(nd, exp)


def test_getacc_node_centric_brute_force_and_conservation():
    m = meshgen.quad_mesh(7, 5, seed=3)
    cd = meshgen.bookleaf_fields(m.ncell, seed=3)
    nd = oracle.getacc(m.cell2node, cd, m.nnode)
    ref = np.zeros((m.nnode, 4))
    for n in range(m.nnode):
        for c, k in zip(*np.nonzero(m.cell2node == n)):
            ref[n] += [cd[c, 1 + k], cd[c, 0] * cd[c, 5 + k], cd[c, 9 + k], cd[c, 13 + k]]
    np.testing.assert_allclose(nd, ref, rtol=1e-14, atol=1e-14)
    tot = np.array([cd[:, 1:5].sum(), (cd[:, :1] * cd[:, 5:9]).sum(), cd[:, 9:13].sum(), cd[:, 13:17].sum()])
    np.testing.assert_allclose(nd.sum(0), tot, rtol=1e-13)
