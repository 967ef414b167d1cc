"""Host planner (C++ through the C ABI) against the plain-Python plan oracle
and the plan invariants.  CPU only: mesh_plan_build touches no GPU."""
import numpy as np
import pytest

import meshgen
from oracle import plan as PO

ml = pytest.importorskip("paper_1802_03749_gb300")


@pytest.fixture(scope="module")
def mesh():
    return meshgen.quad_mesh(60, 30, seed=4)


def res_maps(m, adjoint=False):
    return [{"to_set": 1, "idx": m.edge2node, "to_size": m.nnode, "written": adjoint},
            {"to_set": 2, "idx": m.edge2cell, "to_size": m.ncell, "written": True}]


def oracle_maps(m, P, adjoint=False):
    """Plan-numbered maps as dicts for the Python oracle."""
    e2n = P.table("map", 0).reshape(-1, 2)
    e2c = P.table("map", 1).reshape(-1, 2)
    return [{"to_set": 1, "idx": e2n, "to_size": m.nnode, "written": adjoint},
            {"to_set": 2, "idx": e2c, "to_size": m.ncell, "written": True}]


def check_perm_consistency(m, P):
    """Plan-numbered maps = original maps renumbered by the plan's perms."""
    pe, pn, pc = P.perm(0), P.perm(1), P.perm(2)
    assert PO.is_permutation(pe, m.nedge)
    assert PO.is_permutation(pn, m.nnode)
    assert PO.is_permutation(pc, m.ncell)
    inv_n = np.empty_like(pn)
    inv_n[pn] = np.arange(m.nnode)
    inv_c = np.empty_like(pc)
    inv_c[pc] = np.arange(m.ncell)
    assert np.array_equal(P.table("map", 0).reshape(-1, 2), inv_n[m.edge2node[pe]])
    assert np.array_equal(P.table("map", 1).reshape(-1, 2), inv_c[m.edge2cell[pe]])


@pytest.mark.parametrize("reorder", ["none", "rcm", "partition"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_hier_plan_matches_oracle(mesh, reorder, adjoint):
    """The paper's colouring steps alone (no sparse-colour elimination)
    against the Python first-fit oracle."""
    m = mesh
    P = ml.Plan(res_maps(m, adjoint), m.nedge, block_size=256, reorder=reorder, coloring="hier", recolor=0)
    check_perm_consistency(m, P)
    st = P.stats()
    bo = P.table("block_offsets")
    co = P.table("color_offsets")
    bc = P.table("block_color")
    tc = P.table("thread_color")
    assert bo[0] == 0 and bo[-1] == m.nedge and np.all(np.diff(bo) >= 1)
    sprime = int(256 / 1.001) if reorder == "partition" else 256
    assert np.diff(bo).max() <= sprime and st["sprime"] == int(256 / 1.001)
    maps = oracle_maps(m, P, adjoint)
    wrows = PO.written_rows_of(maps)
    blocks = [list(range(bo[b], bo[b + 1])) for b in range(len(bo) - 1)]
    # block colours: bit-exact first fit in the plan's block order, and sorted
    # by colour (the plan renumbers blocks colour-major after colouring, a
    # stable sort of the first-fit order, so first fit on the sorted order
    # gives the same colours)
    assert list(bc) == PO.block_colors(blocks, wrows)
    assert np.all(np.diff(bc) >= 0)
    assert np.array_equal(co, np.searchsorted(bc, np.arange(bc.max() + 2)))
    # thread colours: first fit within each block (items are colour-sorted,
    # and a stable sort of first-fit colours reproduces itself)
    for b in blocks:
        assert [tc[i] for i in b] == PO.thread_colors(b, wrows)
        assert all(tc[b[i]] <= tc[b[i + 1]] for i in range(len(b) - 1))
    assert PO.check_coloring(wrows, list(tc), groups=blocks)
    # block colouring invariant: same-colour blocks share no written point
    owner = {}
    for b, items in enumerate(blocks):
        for i in items:
            for p in wrows[i]:
                k = (bc[b], p)
                assert owner.get(k, b) == b
                owner[k] = b
    assert st["reuse_all"] == pytest.approx(PO.reuse_factor(bo, [maps[0]["idx"], maps[1]["idx"]]))


@pytest.mark.parametrize("reorder", ["rcm", "partition"])
def test_footprints_and_local_maps(mesh, reorder):
    """What the staged kernels index: fp[start[b,slot] + local[it,k]] is the
    plan-numbered point of map slot k of iteration it, and each block's
    footprint is sorted and duplicate-free."""
    m = mesh
    P = ml.Plan(res_maps(m), m.nedge, block_size=480, reorder=reorder, coloring="hier")
    bo = P.table("block_offsets")
    fp = P.table("footprint")
    fs = P.table("fp_start").reshape(-1, 2)
    fc = P.table("fp_count").reshape(-1, 2)
    lm = P.table("local_map").reshape(m.nedge, -1)
    e2n = P.table("map", 0).reshape(-1, 2)
    e2c = P.table("map", 1).reshape(-1, 2)
    slot_of = [0, 0, 1, 1]
    glob = np.concatenate([e2n, e2c], axis=1)
    st = P.stats()
    for b in range(len(bo) - 1):
        for s in range(2):
            lst = fp[fs[b, s]:fs[b, s] + fc[b, s]]
            assert np.all(np.diff(lst) > 0)
        for it in range(bo[b], bo[b + 1]):
            for k in range(4):
                s = slot_of[k]
                assert lm[it, k] < fc[b, s]
                assert fp[fs[b, s] + lm[it, k]] == glob[it, k]
    assert fc[:, 0].max() == st["footprint_max"][0] and fc[:, 1].max() == st["footprint_max"][1]


def test_rcm_matches_oracle(mesh):
    m = mesh
    P = ml.Plan(res_maps(m), m.nedge, block_size=256, reorder="rcm", coloring="atomic")
    maps = [{"to_set": 1, "idx": m.edge2node, "to_size": m.nnode, "written": False},
            {"to_set": 2, "idx": m.edge2cell, "to_size": m.ncell, "written": True}]
    ref = PO.rcm_plan_perms(maps, m.nedge, primary=1)
    assert np.array_equal(P.perm(2), ref[2])
    assert np.array_equal(P.perm(0), ref[0])
    assert np.array_equal(P.perm(1), ref[1])


@pytest.mark.parametrize("case", ["bedge_arity1", "cell2node_arity4"])
def test_rcm_matches_oracle_other_arities(mesh, case):
    """The RCM reorder with a primary map of arity 1 (boundary edge -> cell)
    and of arity 4 (cell -> node): iteration order by the sorted tuple of
    renumbered primary points, ties by old id."""
    m = mesh
    if case == "bedge_arity1":
        maps = [{"to_set": 1, "idx": m.bedge2node, "to_size": m.nnode, "written": False},
                {"to_set": 2, "idx": m.bedge2cell.reshape(-1, 1), "to_size": m.ncell, "written": True}]
        n, primary, sets = m.bedge2cell.shape[0], 1, (0, 1, 2)
    else:
        maps = [{"to_set": 1, "idx": m.cell2node, "to_size": m.nnode, "written": True}]
        n, primary, sets = m.ncell, 0, (0, 1)
    P = ml.Plan(maps, n, block_size=64, reorder="rcm", coloring="atomic")
    ref = PO.rcm_plan_perms(maps, n, primary=primary)
    for s in sets:
        assert np.array_equal(P.perm(s), ref[s])


def test_global_coloring_matches_oracle(mesh):
    m = mesh
    P = ml.Plan(res_maps(m), m.nedge, block_size=256, reorder="rcm", coloring="global")
    check_perm_consistency(m, P)
    co = P.table("color_offsets")
    tc = P.table("thread_color")
    maps = oracle_maps(m, P)
    wrows = PO.written_rows_of(maps)
    # items are sorted by colour: first fit over the RCM order, stably sorted
    Pr = ml.Plan(res_maps(m), m.nedge, block_size=256, reorder="rcm", coloring="atomic")
    wr = PO.written_rows_of(oracle_maps(m, Pr))
    col = PO.first_fit_items(wr)
    assert sorted(col) == list(tc)
    assert PO.check_coloring(wrows, list(tc))
    assert np.array_equal(co, np.searchsorted(tc, np.arange(tc.max() + 2)))


def test_partition_data_reorder_groups_points(mesh):
    """After the data-point reorder, points are sorted by the key (number of
    accessing blocks, accessing block ids)."""
    m = mesh
    P = ml.Plan(res_maps(m), m.nedge, block_size=256, reorder="partition", coloring="hier")
    bo = P.table("block_offsets")
    blk = np.repeat(np.arange(len(bo) - 1), np.diff(bo))
    e2c = P.table("map", 1).reshape(-1, 2)
    order = PO.data_point_order(blk, [e2c], m.ncell)
    assert order == list(range(m.ncell))


@pytest.mark.parametrize("reorder", ["rcm", "partition"])
def test_data_point_order_all_key_groups(reorder):
    """Data-point order of both to-sets on a random map with points of one,
    two, three or more blocks and points no iteration touches (unused ids
    at the top of each set), against the oracle's key."""
    rng = np.random.default_rng(7)
    n, nn, nc = 3000, 900, 700
    e2n = rng.integers(0, nn - 60, size=(n, 2), dtype=np.int32)
    e2c = rng.integers(0, nc - 40, size=(n, 3), dtype=np.int32)
    maps = [{"to_set": 1, "idx": e2n, "to_size": nn, "written": False},
            {"to_set": 2, "idx": e2c, "to_size": nc, "written": True}]
    P = ml.Plan(maps, n, block_size=64, reorder=reorder, coloring="hier", data_reorder=1)
    bo = P.table("block_offsets")
    blk = np.repeat(np.arange(len(bo) - 1), np.diff(bo))
    pn = P.table("map", 0).reshape(-1, 2)
    pc = P.table("map", 1).reshape(-1, 3)
    counts = [len({int(b) for b in blk[np.any(pc == p, axis=1)]}) for p in range(nc)]
    assert max(counts) >= 3 and min(counts) == 0
    assert PO.data_point_order(blk, [pn], nn) == list(range(nn))
    assert PO.data_point_order(blk, [pc], nc) == list(range(nc))


def test_many_block_colours_keep_first_fit():
    """Above 64 block colours the default plan keeps the first-fit block
    colouring (no trailing-colour removal): same colours as recolor=0."""
    rng = np.random.default_rng(11)
    n, nc = 20000, 5000  # about 100 block colours
    e2c = rng.integers(0, nc, size=(n, 2), dtype=np.int32)
    maps = [{"to_set": 1, "idx": e2c, "to_size": nc, "written": True}]
    P = ml.Plan(maps, n, block_size=32, reorder="none", coloring="hier")
    Q = ml.Plan(maps, n, block_size=32, reorder="none", coloring="hier", recolor=0)
    assert P.stats()["nblock_colors"] > 64
    for t in ("block_offsets", "block_color", "thread_color"):
        assert np.array_equal(P.table(t), Q.table(t))
    bo = P.table("block_offsets")
    wrows = PO.written_rows_of([{"to_set": 1, "idx": P.table("map", 0).reshape(-1, 2), "to_size": nc,
                                 "written": True}])
    blocks = [list(range(bo[b], bo[b + 1])) for b in range(len(bo) - 1)]
    assert list(P.table("block_color")) == PO.block_colors(blocks, wrows)


def test_errors():
    idx = np.array([[0, 1], [1, 5]], dtype=np.int32)
    with pytest.raises(ml.MeshLoopError) as e:
        ml.Plan([{"to_set": 1, "idx": idx, "to_size": 3, "written": True}], 2)
    assert e.value.name == "MP_EMAPRANGE"
    with pytest.raises(ml.MeshLoopError) as e:
        ml.Plan([{"to_set": 1, "idx": idx, "to_size": 6, "written": True}], 2, block_size=100)
    assert e.value.name == "MP_EINVAL"
    # a star: 300 iterations all writing point 0 need 300 colours > 256
    star = np.stack([np.zeros(300, np.int32), np.arange(1, 301, dtype=np.int32)], axis=1)
    with pytest.raises(ml.MeshLoopError) as e:
        ml.Plan([{"to_set": 1, "idx": star, "to_size": 301, "written": True}], 300, reorder="none",
                coloring="global")
    assert e.value.name == "MP_ECOLORS"
    # more than 64 thread colours inside one block
    with pytest.raises(ml.MeshLoopError) as e:
        ml.Plan([{"to_set": 1, "idx": star[:100], "to_size": 301, "written": True}], 100, reorder="none",
                coloring="hier", block_size=128)
    assert e.value.name == "MP_ECOLORS"


def test_map_renumber_roundtrip():
    m = meshgen.quad_mesh(10, 6, seed=1)
    pc = meshgen.permutation(5, 1, m.ncell).astype(np.int32)
    pn = meshgen.permutation(5, 2, m.nnode).astype(np.int32)
    out = ml.mesh_map_renumber(m.cell2node, pc, pn, m.nnode)
    inv = np.empty_like(pn)
    inv[pn] = np.arange(m.nnode)
    assert np.array_equal(out, inv[m.cell2node[pc]])


def test_batch_fuses_plans():
    """mesh_batch_build: one block table over the disjoint union of meshes;
    the staged-kernel indexing invariant holds on the fused tables and
    blocks are grouped by colour phase."""
    meshes = [meshgen.quad_mesh(nx, ny, seed=s) for nx, ny, s in [(20, 10, 1), (33, 7, 2), (12, 12, 3)]]
    opts = [(128, "partition"), (256, "rcm"), (64, "partition")]
    plans = [ml.Plan(res_maps(m), m.nedge, block_size=bs, reorder=ro) for m, (bs, ro) in zip(meshes, opts)]
    B = ml.Plan.batch(plans)
    st = B.stats()
    ne = sum(m.nedge for m in meshes)
    nc = sum(m.ncell for m in meshes)
    nn = sum(m.nnode for m in meshes)
    assert st["from_size"] == ne and st["block_size"] == 256
    assert st["nblocks"] == sum(p.stats()["nblocks"] for p in plans)
    assert st["nblock_colors"] == max(p.stats()["nblock_colors"] for p in plans)
    bo = B.table("block_offsets")
    bc = B.table("block_color")
    assert bo[0] == 0 and bo[-1] == ne and np.all(np.diff(bo) >= 1) and np.all(np.diff(bc) >= 0)
    fp = B.table("footprint")
    fs = B.table("fp_start").reshape(-1, 2)
    fc = B.table("fp_count").reshape(-1, 2)
    lm = B.table("local_map").reshape(ne, -1)
    glob = np.concatenate([B.table("map", 0).reshape(-1, 2), B.table("map", 1).reshape(-1, 2)], axis=1)
    for b in range(len(bo) - 1):
        for it in range(bo[b], bo[b + 1]):
            for k, s in enumerate([0, 0, 1, 1]):
                assert fp[fs[b, s] + lm[it, k]] == glob[it, k]
    # the fused maps are the per-mesh plan maps, offset into the concatenation
    pe = B.perm(0)
    assert PO.is_permutation(pe, ne) and PO.is_permutation(B.perm(2), nc) and PO.is_permutation(B.perm(1), nn)
    offs_c = np.cumsum([0] + [m.ncell for m in meshes])
    offs_n = np.cumsum([0] + [m.nnode for m in meshes])
    offs_e = np.cumsum([0] + [m.nedge for m in meshes])
    e2c_orig = np.concatenate([m.edge2cell + offs_c[i] for i, m in enumerate(meshes)])
    inv_c = np.empty(nc, dtype=np.int64)
    inv_c[B.perm(2)] = np.arange(nc)
    assert np.array_equal(glob[:, 2:], inv_c[e2c_orig[pe]])
    assert offs_e[-1] == ne and offs_n[-1] == nn
    # same-colour blocks share no written cell
    wr = PO.written_rows_of([{"to_set": 1, "idx": glob[:, :2], "to_size": nn, "written": False},
                             {"to_set": 2, "idx": glob[:, 2:], "to_size": nc, "written": True}])
    owner = {}
    for b in range(len(bo) - 1):
        for i in range(bo[b], bo[b + 1]):
            for p in wr[i]:
                assert owner.setdefault((bc[b], p), b) == b


@pytest.mark.parametrize("reorder", ["none", "rcm", "partition"])
def test_twostep_inverse_map(mesh, reorder):
    """TWOSTEP plans: the inverse of the written map lists, for every point,
    exactly its (item, slot) pairs in ascending order, in the final point
    numbering (after the data-point reordering of partitioned plans)."""
    m = mesh
    P = ml.Plan(res_maps(m), m.nedge, block_size=256, reorder=reorder, coloring="twostep")
    check_perm_consistency(m, P)
    off = P.table("inv_offsets")
    idx = P.table("inv_index")
    e2c = P.table("map", 1).reshape(-1, 2)
    assert off[0] == 0 and off[-1] == 2 * m.nedge and np.all(np.diff(off) >= 0)
    for c in range(m.ncell):
        ent = idx[off[c]:off[c + 1]]
        assert np.all(np.diff(ent) > 0)
        assert np.all(e2c.ravel()[ent] == c)
    assert np.array_equal(np.bincount(e2c.ravel(), minlength=m.ncell), np.diff(off))
    with pytest.raises(ml.MeshLoopError):   # two written maps: not a two-step loop
        ml.Plan(res_maps(m, adjoint=True), m.nedge, coloring="twostep")


@pytest.mark.parametrize("shape", [(16, 1, 1), (4, 4, 1), (2, 2, 4), (4, 2, 2)])
def test_caller_defined_brick_blocks(shape):
    """Handcrafted bricks of bx x by x bz elements on a structured hex grid:
    every block is one brick and the node reuse is exactly
    8 bx by bz / ((bx+1)(by+1)(bz+1))."""
    dims = (16, 8, 8)
    m = meshgen.hex_mesh(dims[0], seed=2, nyz=dims[1:])
    blk = meshgen.hex_bricks(m, shape, dims)
    bx, by, bz = shape
    P = ml.Plan([{"to_set": 1, "idx": m.elem2node, "to_size": m.nnode, "written": True}], m.nelem,
                block_size=64, block_of=blk)
    st = P.stats()
    assert st["nblocks"] == m.nelem // (bx * by * bz)
    bo = P.table("block_offsets")
    pe = P.perm(0)
    for b in range(len(bo) - 1):
        assert len(set(blk[pe[bo[b]:bo[b + 1]]])) == 1
    assert st["reuse_all"] == pytest.approx(8 * bx * by * bz / ((bx + 1) * (by + 1) * (bz + 1)))
    wr = PO.written_rows_of([{"to_set": 1, "idx": P.table("map", 0).reshape(-1, 8), "to_size": m.nnode,
                              "written": True}])
    blocks = [list(range(bo[b], bo[b + 1])) for b in range(len(bo) - 1)]
    assert PO.check_coloring(wr, list(P.table("thread_color")), groups=blocks)
    big = meshgen.hex_bricks(m, (4, 4, 4), dims)                # 64 elements per brick
    with pytest.raises(ml.MeshLoopError):     # a brick larger than the block size
        ml.Plan([{"to_set": 1, "idx": m.elem2node, "to_size": m.nnode, "written": True}], m.nelem,
                block_size=32, block_of=big)


def check_gather_rows(P, nitems, written_slots, slot_of):
    """Every footprint point's gather row lists, ascending, t * 16 + k of
    each written map slot k of each block-local iteration t that maps to
    it, then -1; points of unwritten to-sets have empty rows."""
    bo = P.table("block_offsets")
    fs = P.table("fp_start").reshape(-1, 2)
    fc = P.table("fp_count").reshape(-1, 2)
    lm = P.table("local_map").reshape(nitems, -1)
    gat = P.table("gather")
    nfp = len(P.table("footprint"))
    assert len(gat) % nfp == 0
    w = len(gat) // nfp
    assert w in (4, 8, 16)
    gat = gat.reshape(nfp, w)
    seen = np.zeros(nfp, dtype=bool)
    for b in range(len(bo) - 1):
        t0, t1 = bo[b], bo[b + 1]
        for s in range(2):
            rows = {i: [] for i in range(fc[b, s])}
            for k in written_slots:
                if slot_of[k] != s:
                    continue
                for t in range(t1 - t0):
                    rows[lm[t0 + t, k]].append(t * 16 + k)
            for i, lst in rows.items():
                r = gat[fs[b, s] + i]
                lst = sorted(lst)
                assert list(r[:len(lst)]) == lst and np.all(r[len(lst):] == -1)
                seen[fs[b, s] + i] = True
    assert seen.all()
    return w


@pytest.mark.parametrize("reorder", ["rcm", "partition"])
def test_gather_rows(mesh, reorder):
    """The block-local inverse map read by the gather form of the staged
    kernels: cells list their edges' slot-2/3 increments, nodes none (the
    forward plan) or their slot-0/1 increments (the adjoint plan)."""
    m = mesh
    P = ml.Plan(res_maps(m), m.nedge, block_size=256, reorder=reorder)
    assert check_gather_rows(P, m.nedge, [2, 3], [0, 0, 1, 1]) == 4
    Pa = ml.Plan(res_maps(m, adjoint=True), m.nedge, block_size=128, reorder=reorder)
    check_gather_rows(Pa, m.nedge, [0, 1, 2, 3], [0, 0, 1, 1])


def test_gather_rows_batch():
    """Fused batch plans carry the members' gather rows in the fused
    footprint numbering."""
    meshes = [meshgen.quad_mesh(nx, ny, seed=s) for nx, ny, s in [(20, 10, 1), (33, 7, 2)]]
    plans = [ml.Plan(res_maps(m), m.nedge, block_size=bs, reorder="partition") for m, bs in zip(meshes, (128, 64))]
    B = ml.Plan.batch(plans)
    check_gather_rows(B, sum(m.nedge for m in meshes), [2, 3], [0, 0, 1, 1])


def block_coloring_valid(P, wrows):
    bo = P.table("block_offsets")
    bc = P.table("block_color")
    owner = {}
    for b in range(len(bo) - 1):
        for i in range(bo[b], bo[b + 1]):
            for p in wrows[i]:
                if owner.setdefault((bc[b], p), b) != b:
                    return False
    return True


@pytest.mark.parametrize("nx,ny,bs", [(200, 100, 64), (200, 100, 256), (600, 300, 480), (97, 53, 32)])
def test_sparse_colors_eliminated(nx, ny, bs):
    """Recolouring after first fit (Kempe interchanges, dissolving the
    blocks of a sparse last colour into pieces of earlier colours): a valid
    block colouring with no more colours than first fit, every iteration in
    exactly one block of at most S' iterations, thread colours valid, and
    on these meshes one launch fewer."""
    m = meshgen.quad_mesh(nx, ny, seed=4)
    P0 = ml.Plan(res_maps(m), m.nedge, block_size=bs, reorder="partition", recolor=0)
    P1 = ml.Plan(res_maps(m), m.nedge, block_size=bs, reorder="partition", recolor=1)
    st0, st1 = P0.stats(), P1.stats()
    assert st1["nblock_colors"] <= st0["nblock_colors"]
    if (nx, ny, bs) != (97, 53, 32):
        assert st1["nblock_colors"] <= st0["nblock_colors"] - 1
    check_perm_consistency(m, P1)
    wrows = PO.written_rows_of(oracle_maps(m, P1))
    assert block_coloring_valid(P1, wrows)
    bo = P1.table("block_offsets")
    bc = P1.table("block_color")
    co = P1.table("color_offsets")
    assert bo[0] == 0 and bo[-1] == m.nedge and np.all(np.diff(bo) >= 1)
    assert np.diff(bo).max() <= st1["sprime"]
    assert np.all(np.diff(bc) >= 0) and np.array_equal(co, np.searchsorted(bc, np.arange(bc.max() + 2)))
    tc = P1.table("thread_color")
    blocks = [list(range(bo[b], bo[b + 1])) for b in range(len(bo) - 1)]
    assert PO.check_coloring(wrows, list(tc), groups=blocks)
    # default options recolour
    assert ml.Plan(res_maps(m), m.nedge, block_size=bs, reorder="partition").stats()["nblock_colors"] == \
        st1["nblock_colors"]
