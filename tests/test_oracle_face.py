"""Pins of the oracle's miniAero-style face flux (Sec. 3.1.5): freestream
preservation on closed cells, conservation, antisymmetry, the dissipative
sign of the Rusanov term, rotation invariance, exactness for linear fields,
and a cell-centric brute force.  CPU only."""
import numpy as np
import pytest

import meshgen
import oracle

GAM, MU, PR = oracle.GAMMA, oracle.MU, oracle.PR


@pytest.fixture(scope="module")
def case():
    hm = meshgen.hex_mesh(5, nyz=(4, 6), seed=3)
    f2c, fd = meshgen.hex_faces(hm, (5, 4, 6), seed=3)
    cd = meshgen.aero_cells(hm, seed=3)
    return hm, f2c, fd, cd


def one_face(fd_row, cd1, cd2):
    """The flux of a single face between two cells (c1 = 0, c2 = 1)."""
    r = oracle.face_flux(np.array([[0, 1]]), fd_row[None, :], np.stack([cd1, cd2]))
    return r[0]


def test_faces_close_every_interior_cell(case):
    """The bilinear faces' area vectors of a hexahedron sum to zero."""
    hm, f2c, fd, cd = case
    s = np.zeros((hm.nelem, 3))
    np.add.at(s, f2c[:, 0], fd[:, :3])
    np.add.at(s, f2c[:, 1], -fd[:, :3])
    inner = np.bincount(f2c.ravel(), minlength=hm.nelem) == 6
    assert inner.sum() == 3 * 2 * 4 and np.abs(s[inner]).max() < 1e-15


def test_freestream_is_preserved(case):
    """Uniform state, zero gradients: F_inv = |A| F(Q).nhat on every face
    and no viscous flux, so every closed cell's residual vanishes."""
    hm, f2c, fd, cd = case
    c = cd.copy()
    c[:, :5] = cd[0, :5]
    c[:, 5:20] = 0.0
    r = oracle.face_flux(f2c, fd, c)
    inner = np.bincount(f2c.ravel(), minlength=hm.nelem) == 6
    assert np.abs(r[inner]).max() < 1e-15
    assert np.abs(r[~inner]).max() > 1e-4      # open cells do see the flux


def test_conservation(case):
    hm, f2c, fd, cd = case
    r = oracle.face_flux(f2c, fd, cd)
    assert np.abs(r.sum(0)).max() < 1e-15 * max(1.0, np.abs(r).sum())


def test_antisymmetry(case):
    """Swapping a face's cells and reversing its orientation (A, nhat, dx)
    gives the same residual."""
    hm, f2c, fd, cd = case
    r = oracle.face_flux(f2c, fd, cd)
    fs = fd.copy()
    fs[:, 0:3] *= -1
    fs[:, 6:12] *= -1
    r2 = oracle.face_flux(f2c[:, ::-1], fs, cd)
    np.testing.assert_allclose(r2, r, rtol=1e-13, atol=1e-15)


def test_rusanov_term_is_dissipative(case):
    """A density jump at rest (u = 0, equal pressure, no gradients): the
    mass crosses the face from the denser cell to the lighter one."""
    hm, f2c, fd, cd = case
    c1, c2 = cd[0].copy(), cd[0].copy()
    for c, rho in ((c1, 1.0), (c2, 2.0)):
        c[5:20] = 0.0
        c[0] = rho
        c[1:4] = 0.0
        c[4] = 1.0 / GAM / (GAM - 1.0)
    f = one_face(fd[0], c1, c2)
    # flux from c1 into c2 is negative: mass moves from c2 (rho 2) to c1
    assert f[0] < 0 and abs(f[0]) > 1e-6


def rotation(a, b, c):
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rx = np.array([[1, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return Rz @ Ry @ Rx


def test_rotation_invariance(case):
    """Rotating every vector (geometry, velocity) and every gradient (scalar
    gradients as vectors, the velocity gradient as R grad(u) R^T) leaves
    mass and energy residuals unchanged and rotates the momentum residual.
    (Component-wise limiters of u, v, w are not rotation invariant, so the
    three velocity limiters are set equal here.)"""
    hm, f2c, fd, cd = case
    cd = cd.copy()
    cd[:, 22:24] = cd[:, 21:22]
    R = rotation(0.3, -0.7, 1.1)
    fr = fd.copy()
    for s in (0, 3, 6, 9):
        fr[:, s:s + 3] = fd[:, s:s + 3] @ R.T
    cr = cd.copy()
    cr[:, 1:4] = cd[:, 1:4] @ R.T
    G = cd[:, 5:20].reshape(-1, 5, 3)
    Gr = G @ R.T                                       # each gradient (row) rotated
    Gu = G[:, 1:4, :]                                  # d u_a / d x_d
    Gr[:, 1:4, :] = np.einsum("ab,nbc,dc->nad", R, Gu, R)
    cr[:, 5:20] = Gr.reshape(-1, 15)
    cr[:, 25:28] = cd[:, 25:28] @ R.T
    r = oracle.face_flux(f2c, fd, cd)
    rr = oracle.face_flux(f2c, fr, cr)
    np.testing.assert_allclose(rr[:, [0, 4]], r[:, [0, 4]], rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(rr[:, 1:4], r[:, 1:4] @ R.T, rtol=1e-11, atol=1e-14)


def test_linear_fields_are_exact():
    """Constant density, velocity and pressure linear in x, limiters 1, the
    true gradients: both reconstructions give the field's value at the face
    (no dissipation), and the corrected face gradients are the field's, so
    one face's flux is |A| F(V(xf)).nhat minus the Newtonian viscous and heat
    flux of those gradients."""
    hm = meshgen.hex_mesh(3, seed=9)
    f2c, fd = meshgen.hex_faces(hm, seed=9)
    xc = hm.x[hm.elem2node].mean(axis=1)
    rho0, u0, p0 = 1.1, np.array([0.3, -0.2, 0.1]), 0.8
    B = np.array([[0.2, -0.1, 0.05], [0.03, 0.1, -0.2], [-0.15, 0.02, 0.07]])   # d u_a / d x_d
    gp = np.array([0.05, -0.03, 0.02])

    def V(x):
        return rho0, u0 + B @ x, p0 + gp @ x

    cd = np.zeros((hm.nelem, 28))
    for c in range(hm.nelem):
        rho, u, p = V(xc[c])
        cd[c, :5] = [rho, *(rho * u), p / (GAM - 1) + 0.5 * rho * u @ u]
        cd[c, 5 + 3:5 + 12] = B.ravel()
        cd[c, 5 + 12:5 + 15] = gp
        cd[c, 20:25] = 1.0
        cd[c, 25:28] = xc[c]
    for f in range(0, f2c.shape[0], 7):
        A, xf, n = fd[f, :3], fd[f, 3:6], fd[f, 6:9]
        rho, u, p = V(xf)
        E = p / (GAM - 1) + 0.5 * rho * u @ u
        un = u @ n
        Finv = np.linalg.norm(A) * np.array([rho * un, *(rho * u * un + p * n), (E + p) * un])
        tau = MU * (B + B.T) - 2.0 / 3.0 * MU * np.trace(B) * np.eye(3)
        tA = tau @ A
        uf = 0.5 * (V(xc[f2c[f, 0]])[1] + V(xc[f2c[f, 1]])[1])
        k = MU * GAM / ((GAM - 1) * PR)
        Fv = np.array([0.0, *tA, uf @ tA + k * (gp / rho0) @ A])
        got = one_face(fd[f], cd[f2c[f, 0]], cd[f2c[f, 1]])
        np.testing.assert_allclose(got, Finv - Fv, rtol=1e-12, atol=1e-16)


def test_cell_centric_brute_force(case):
    """Each cell's residual as the sum over its faces of the single-face
    flux, +F where it is the first cell, -F where it is the second."""
    hm, f2c, fd, cd = case
    r = oracle.face_flux(f2c, fd, cd)
    ref = np.zeros_like(r)
    for c in range(hm.nelem):
        for f in np.flatnonzero((f2c == c).any(axis=1)):
            F = one_face(fd[f], cd[f2c[f, 0]], cd[f2c[f, 1]])
            ref[c] += F if f2c[f, 0] == c else -F
    np.testing.assert_allclose(r, ref, rtol=1e-13, atol=1e-16)


def test_face_gradient_correction_without_cell_gradients():
    """Cell gradients all zero, velocity and temperature linear in the cell
    centres: the corrected face gradient is the difference quotient along
    dx, (phi_2 - phi_1) dx / |dx|^2.  The viscous part of the flux (the
    difference of the fluxes with mu = 0 and mu) must be the Newtonian flux
    of that gradient."""
    hm = meshgen.hex_mesh(3, seed=9, jitter=0.0)
    f2c, fd = meshgen.hex_faces(hm, seed=9)
    xc = hm.x[hm.elem2node].mean(axis=1)
    rho0 = 1.2
    B = np.array([[0.2, -0.1, 0.05], [0.03, 0.1, -0.2], [-0.15, 0.02, 0.07]])
    gp = np.array([0.05, -0.03, 0.02])
    cd = np.zeros((hm.nelem, 28))
    for c in range(hm.nelem):
        u = np.array([0.3, -0.2, 0.1]) + B @ xc[c]
        p = 0.8 + gp @ xc[c]
        cd[c, :5] = [rho0, *(rho0 * u), p / (GAM - 1) + 0.5 * rho0 * u @ u]
        cd[c, 25:28] = xc[c]
    mu = 0.01
    full = oracle.face_flux(f2c, fd, cd, mu=mu)
    inv = oracle.face_flux(f2c, fd, cd, mu=0.0)
    Fv = inv - full                                   # res[c1] += F_inv - F_v
    k = mu * GAM / ((GAM - 1) * PR)
    exp = np.zeros_like(Fv)
    for f in range(f2c.shape[0]):
        A, dx = fd[f, :3], fd[f, 9:12]
        c1, c2 = f2c[f]
        dd = dx @ dx
        gu = np.outer(B @ dx, dx) / dd
        gT = (gp @ dx / rho0) * dx / dd
        tau = mu * (gu + gu.T) - 2.0 / 3.0 * mu * np.trace(gu) * np.eye(3)
        tA = tau @ A
        uf = 0.5 * (cd[c1, 1:4] + cd[c2, 1:4]) / rho0
        F = np.array([0.0, *tA, uf @ tA + k * gT @ A])
        exp[c1] += F
        exp[c2] -= F
    np.testing.assert_allclose(Fv, exp, rtol=1e-10, atol=1e-15)
