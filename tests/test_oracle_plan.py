"""Pins of the plain-Python plan oracle (colourings, RCM, data-point key,
reuse factor) against brute force and known orderings.  CPU only."""
import itertools

import numpy as np

import meshgen
from oracle import plan as P


def test_first_fit_matches_brute_force_definition():
    """Tiny conflict structure: item i conflicts with j iff they share a
    point.  First fit = smallest colour unused by earlier neighbours."""
    rows = [[0, 1], [1, 2], [2, 3], [3, 0], [0, 2], [4], [4, 1]]
    col = P.first_fit_items(rows)
    # item 6 = [4, 1] meets item 5 (colour 0 via 4), items 0, 1 (colours 0, 1 via 1)
    assert col == [0, 1, 0, 1, 2, 0, 2]
    assert P.check_coloring(rows, col)
    # greedy never uses more colours than max degree + 1
    for perm in itertools.islice(itertools.permutations(range(len(rows))), 50):
        c = P.first_fit_items(rows, order=perm)
        assert P.check_coloring(rows, c)
        assert max(c) + 1 <= 4


def _bandwidth(idx, new_of_old):
    r = new_of_old[idx]
    return int(np.abs(r[:, 0] - r[:, 1]).max())


def test_rcm_on_permuted_chain_recovers_the_path():
    n = 50
    perm = meshgen.permutation(3, 1, n)
    idx = np.stack([perm[:-1], perm[1:]], axis=1)     # chain perm[0]-perm[1]-...
    order = P.rcm_order(P.clique_graph(idx, n))
    new = np.empty(n, dtype=int)
    new[order] = np.arange(n)
    assert _bandwidth(idx, new) == 1
    assert order[0] in (perm[0], perm[-1])            # starts at an end (peripheral)


def test_rcm_bandwidth_on_permuted_grid():
    """Cell adjacency of an nx*ny quad grid: RCM bandwidth is at most about
    the short side (level sets are anti-diagonals of length <= ny)."""
    m = meshgen.quad_mesh(30, 12, seed=8)
    order = P.rcm_order(P.clique_graph(m.edge2cell, m.ncell))
    new = np.empty(m.ncell, dtype=int)
    new[order] = np.arange(m.ncell)
    assert P.is_permutation(order, m.ncell)
    before = _bandwidth(m.edge2cell, np.arange(m.ncell))
    after = _bandwidth(m.edge2cell, new)
    assert after <= 2 * 12 + 2 < before
    # pseudo-peripheral start: a corner cell (degree 2) ends the RCM order
    deg = np.bincount(m.edge2cell.ravel(), minlength=m.ncell)
    assert deg[order[-1]] == 2


def test_data_point_key_hand_example():
    # items 0,1 in block 0; items 2,3 in block 1; points 0..5
    idx = np.array([[0, 1], [1, 2], [2, 3], [4, 3]])
    blk = [0, 0, 1, 1]
    order = P.data_point_order(blk, [idx], 6)
    # 1-block points: block 0 -> {0,1}, block 1 -> {3,4}; 2-block: {2}; unused {5}
    assert order == [0, 1, 3, 4, 2, 5]


def test_reuse_factor_brute_force():
    idx = np.array([[0, 1], [1, 2], [2, 3], [4, 3]])
    # blocks [0,2), [2,4): block0 accesses 4 over {0,1,2}, block1 4 over {2,3,4}
    assert P.reuse_factor([0, 2, 4], [idx]) == 8 / 6
