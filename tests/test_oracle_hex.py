"""Pins of the oracle's hex8 assembly: closed forms on cubes and
parallelepipeds, exact identities, a finite-difference derivative of the
volume and the hourglass null space.  CPU only."""
import json
import os

import numpy as np
import pytest

import meshgen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
XI = meshgen.HEX_CORNERS.astype(float)


def test_cube_hourglass_fixture():
    g = json.load(open(os.path.join(GOLD, "hex_hourglass_cube.json")))
    h, c, e = g["h"], np.array(g["centre"]), np.array(g["e"])
    xe = c + 0.5 * h * XI
    gamma4 = XI[:, 0] * XI[:, 1] * XI[:, 2]
    ve = gamma4[:, None] * e[None, :]
    fe, vol = oracle.hex_element(xe, ve, g["sig"], g["kappa"])
    assert vol == pytest.approx(g["vol"], rel=1e-15)
    np.testing.assert_allclose(fe, g["f"], rtol=0, atol=1e-15)


def test_parallelepiped_volume_is_exact():
    """Affine element x_i = c + A xi_i: the one-point volume 8 det J equals
    the parallelepiped volume det(2A) exactly (J = A)."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        A = np.eye(3) * 0.3 + 0.05 * rng.standard_normal((3, 3))
        xe = np.array([1.0, -2.0, 0.5]) + XI @ A.T
        _, vol = oracle.hex_element(xe, np.zeros((8, 3)), [0, 0, 0])
        assert vol == pytest.approx(np.linalg.det(2 * A), rel=1e-13)


def _jittered_element(seed):
    rng = np.random.default_rng(seed)
    return 0.5 * XI + 0.08 * rng.uniform(-1, 1, (8, 3)), rng


def test_stress_force_is_minus_volume_gradient():
    """B_i = dV/dx_i, so for isotropic stress s the force is -s dV/dx_i:
    checked against central differences of the oracle's own volume."""
    xe, _ = _jittered_element(1)
    s = -0.7
    fe, _ = oracle.hex_element(xe, np.zeros((8, 3)), [s, s, s])
    d = 1e-6
    grad = np.zeros((8, 3))
    for i in range(8):
        for a in range(3):
            xp, xm = xe.copy(), xe.copy()
            xp[i, a] += d
            xm[i, a] -= d
            grad[i, a] = (oracle.hex_element(xp, np.zeros((8, 3)), [0, 0, 0])[1]
                          - oracle.hex_element(xm, np.zeros((8, 3)), [0, 0, 0])[1]) / (2 * d)
    np.testing.assert_allclose(fe, -s * grad, rtol=1e-7, atol=1e-10)


def test_forces_sum_to_zero_and_moment_identity():
    """sum_i B_i = 0 gives sum_i f_i^s = 0; sum_i g_{k,i} = 0 gives
    sum_i f_i^hg = 0."""
    xe, rng = _jittered_element(2)
    ve = rng.standard_normal((8, 3))
    fe, _ = oracle.hex_element(xe, ve, [-1.0, -0.6, -1.3], 0.05)
    np.testing.assert_allclose(fe.sum(axis=0), 0.0, atol=1e-14)


def test_hourglass_vanishes_for_affine_velocity():
    xe, rng = _jittered_element(3)
    A = rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    ve = xe @ A.T + b
    f_with, _ = oracle.hex_element(xe, ve, [0.0, 0.0, 0.0], 0.5)
    np.testing.assert_allclose(f_with, 0.0, atol=1e-13)
    # a non-affine field does produce hourglass forces
    f_hg, _ = oracle.hex_element(xe, ve + 0.1 * rng.standard_normal((8, 3)), [0.0, 0.0, 0.0], 0.5)
    assert np.abs(f_hg).max() > 1e-4


def test_uniform_stress_zero_at_interior_nodes():
    """Unjittered grid, uniform sigma, v = 0: neighbouring elements' forces
    cancel at every interior node; boundary nodes carry the traction."""
    m = meshgen.hex_mesh(5, seed=4, jitter=0.0)
    sig = np.tile([-1.0, -0.5, -2.0], (m.nelem, 1))
    f, vol = oracle.hex_force(m.elem2node, m.x, np.zeros_like(m.x), sig)
    np.testing.assert_allclose(vol, m.h ** 3, rtol=1e-13)
    inner = np.all((m.x > 1e-9) & (m.x < 1 - 1e-9), axis=1)
    assert inner.sum() == 4 ** 3
    np.testing.assert_allclose(f[inner], 0.0, atol=1e-15)
    assert np.abs(f[~inner]).max() > 1e-3


def test_mesh_total_force_zero_and_volume_sum():
    """Per-element forces sum to zero, so the assembled forces do too; the
    volumes of an unjittered-boundary mesh of [0,1]^3 sum to 1 up to the
    one-point rule's error on jittered interior elements."""
    m = meshgen.hex_mesh(6, seed=5)
    sig, v = meshgen.hex_fields(m, seed=5)
    f, vol = oracle.hex_force(m.elem2node, m.x, v, sig)
    np.testing.assert_allclose(f.sum(axis=0), 0.0, atol=1e-13)
    assert vol.min() > 0
    assert abs(vol.sum() - 1.0) < 1e-2
