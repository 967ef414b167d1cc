"""Shared helpers of the GPU parity tests (inputs from meshgen, expected
values from the oracle, results through the C ABI)."""
import numpy as np

import meshgen
import oracle


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def airfoil_case(nx, ny, seed=1802, noise=0.01):
    m = meshgen.quad_mesh(nx, ny, seed=seed)
    q = meshgen.quad_state(m.ncell, seed=seed, noise=noise)
    adt = oracle.adt_calc(m.cell2node, m.x, q)
    return m, q, adt


def round_to(a, dtype):
    """Inputs as the storage precision sees them (float32 storage rounds)."""
    return np.asarray(a).astype(dtype).astype(np.float64)
