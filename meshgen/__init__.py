"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the mesh method itself: it only draws
random numbers and lays out meshes and fields.  Both sides of every parity
check read their inputs from here, and nothing here reads either side.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: the value at counter i of stream k is mix64(seed_k + (i+1)*G)
with seed_k = mix64(seed + k) and G the 64-bit golden-ratio increment.

Meshes (Sec. 1.1 of the paper: sets, fixed-arity maps and data on sets):

* ``quad_mesh(nx, ny, ...)``  -- 2D Airfoil-style mesh on a structured
  nx*ny quad grid, jittered and randomly renumbered.  Sets: nodes, cells,
  interior edges, boundary edges.  Maps (all int32, row-major ``n x arity``):
  edge->node[2], edge->cell[2], bedge->node[2], bedge->cell[1],
  cell->node[4].  Orientation convention (the paper is silent): for an
  interior edge with nodes (a, b) the vector n = (y_a - y_b, -(x_a - x_b))
  points from cell c1 = edge->cell[0] into c2 = edge->cell[1]; for a
  boundary edge it points out of the domain.  cell->node lists the corners
  counter-clockwise.
* ``hex_mesh(n, ...)`` -- 3D n^3 hex grid on [0,1]^3, elem->node[8] with the
  corner order (-,-,-), (+,-,-), (+,+,-), (-,+,-), (-,-,+), (+,-,+),
  (+,+,+), (-,+,+) in (xi, eta, zeta).
* ``batch_sizes(...)`` -- quad counts and aspect ratios for a batch of meshes.
* ``tri_mesh(nx, ny, ...)`` -- 2D triangle mesh (each quad of a jittered
  nx*ny grid split along a diagonal, alternating), renumbered.  One edge set
  holds interior and boundary edges: edge->cell[2] with the edge's first
  cell c1 (the triangle that lists the edge's nodes counter-clockwise) and
  c2 = the neighbour, or c2 = c1 with flag 1 on the boundary.
* ``volna_fields`` / ``bookleaf_fields`` -- direct data of the increment-only
  loops (Sec. 3.1.2 and 3.1.3): per edge 7 floats and 1 integer, per cell 17
  doubles.
* ``hex_faces(mesh, dims)`` / ``aero_cells(mesh)`` -- the interior faces of a
  structured hex grid (face->cell[2], from the cell on the low side to the
  cell on the high side, renumbered) with 12 doubles of face geometry each,
  and 28 doubles of cell data (state, gradients, limiters, centroid) for the
  face-flux loop (Sec. 3.1.5).

Stream ids (``seed + k``): 1 node jitter, 2 cell permutation, 3 node
permutation, 4 edge permutation, 5 boundary-edge permutation, 6 state noise,
7 adjoint seeds, 8 hex fields, 9 batch sizes, 10 free directions for tests,
11 increment-only loop fields, 12 face-flux cell data and face permutation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DEFAULT_SEED = 1802

S_JITTER, S_PERM_CELL, S_PERM_NODE, S_PERM_EDGE, S_PERM_BEDGE = 1, 2, 3, 4, 5
S_NOISE, S_ADJ, S_HEX, S_BATCH, S_DIR = 6, 7, 8, 9, 10
S_INC = 11
S_FACE = 12


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n raw 64-bit SplitMix64 outputs of stream ``stream`` from counter ``offset``."""
    with np.errstate(over="ignore"):
        s = _mix64(np.array([(seed + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix64(s + ctr * _G)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (stream_u64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform on pairs of uniforms."""
    u = uniform(seed, stream, 2 * n, offset)
    u1 = 1.0 - u[0::2]                     # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def permutation(seed: int, stream: int, n: int) -> np.ndarray:
    """A seeded random permutation (new_to_old) of range(n): argsort of random keys."""
    keys = stream_u64(seed, stream, n)
    return np.argsort(keys, kind="stable").astype(np.int64)


def _inverse(p: np.ndarray) -> np.ndarray:
    inv = np.empty_like(p)
    inv[p] = np.arange(p.size, dtype=p.dtype)
    return inv


# --------------------------------------------------------------------------
# 2D quad mesh
# --------------------------------------------------------------------------

GAMMA = 1.4
EPS = 0.05
MACH = 0.4
ALPHA_DEG = 3.0


def freestream(gam: float = GAMMA, mach: float = MACH, alpha_deg: float = ALPHA_DEG) -> np.ndarray:
    """Conserved free-stream state (rho, rho u, rho v, E) with rho = 1,
    |u| = mach, p = 1/gam (so that the sound speed is 1) and total energy
    E = p/(gam-1) + rho |u|^2 / 2."""
    a = math.radians(alpha_deg)
    u, v, rho, p = mach * math.cos(a), mach * math.sin(a), 1.0, 1.0 / gam
    return np.array([rho, rho * u, rho * v, p / (gam - 1.0) + 0.5 * rho * (u * u + v * v)])


@dataclass
class QuadMesh:
    nx: int
    ny: int
    h: float
    x: np.ndarray          # [nnode, 2] float64
    cell2node: np.ndarray  # [ncell, 4] int32, counter-clockwise
    edge2node: np.ndarray  # [nedge, 2] int32
    edge2cell: np.ndarray  # [nedge, 2] int32, n points from [:,0] into [:,1]
    bedge2node: np.ndarray  # [nbedge, 2] int32
    bedge2cell: np.ndarray  # [nbedge, 1] int32, n points out of the domain
    # new_to_old permutations that were applied (identity when unpermuted)
    perms: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return self.cell2node.shape[0]

    @property
    def nnode(self) -> int:
        return self.x.shape[0]

    @property
    def nedge(self) -> int:
        return self.edge2node.shape[0]

    @property
    def nbedge(self) -> int:
        return self.bedge2node.shape[0]


def quad_mesh(nx: int, ny: int, lx: float | None = None, ly: float | None = None,
              seed: int = DEFAULT_SEED, jitter: float = 0.2, permute: bool = True) -> QuadMesh:
    """Jittered, renumbered nx*ny quad grid on [0,lx]x[0,ly] (default h = 1/ny).

    Interior nodes move by U(-jitter*h, jitter*h) per coordinate; boundary
    nodes stay on the rectangle.  With ``permute`` the cells, nodes, interior
    edges and boundary edges are renumbered by seeded random permutations.
    """
    if lx is None:
        lx = nx / ny
    if ly is None:
        ly = 1.0
    h = ly / ny
    nnx = nx + 1
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    x = np.stack([ii * (lx / nx), jj * h], axis=1).astype(np.float64)
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
    nnode = x.shape[0]
    if jitter > 0:
        u = uniform(seed, S_JITTER, 2 * nnode).reshape(nnode, 2)
        d = h * jitter * (2.0 * u - 1.0)
        x[interior] += d[interior]

    def nid(i, j):
        return j * nnx + i

    def cid(i, j):
        return j * nx + i

    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()
    cell2node = np.stack([nid(ci, cj), nid(ci + 1, cj), nid(ci + 1, cj + 1), nid(ci, cj + 1)], axis=1)

    # vertical interior edges between (i-1,j) and (i,j): n points +x
    vi, vj = np.meshgrid(np.arange(1, nx), np.arange(ny), indexing="xy")
    vi = vi.ravel()
    vj = vj.ravel()
    v_e2n = np.stack([nid(vi, vj + 1), nid(vi, vj)], axis=1)
    v_e2c = np.stack([cid(vi - 1, vj), cid(vi, vj)], axis=1)
    # horizontal interior edges between (i,j-1) and (i,j): n points +y
    hi, hj = np.meshgrid(np.arange(nx), np.arange(1, ny), indexing="xy")
    hi = hi.ravel()
    hj = hj.ravel()
    h_e2n = np.stack([nid(hi, hj), nid(hi + 1, hj)], axis=1)
    h_e2c = np.stack([cid(hi, hj - 1), cid(hi, hj)], axis=1)
    edge2node = np.concatenate([v_e2n, h_e2n])
    edge2cell = np.concatenate([v_e2c, h_e2c])

    # boundary edges, n out of the domain
    bi = np.arange(nx)
    bj = np.arange(ny)
    b_e2n = np.concatenate([
        np.stack([nid(bi + 1, 0), nid(bi, 0)], axis=1),             # bottom: -y
        np.stack([nid(bi, ny), nid(bi + 1, ny)], axis=1),           # top: +y
        np.stack([nid(0, bj), nid(0, bj + 1)], axis=1),             # left: -x
        np.stack([nid(nx, bj + 1), nid(nx, bj)], axis=1),           # right: +x
    ])
    b_e2c = np.concatenate([cid(bi, 0), cid(bi, ny - 1), cid(0, bj), cid(nx - 1, bj)])[:, None]

    ncell = nx * ny
    nedge = edge2node.shape[0]
    nbedge = b_e2n.shape[0]
    perms = {}
    if permute:
        pc = permutation(seed, S_PERM_CELL, ncell)
        pn = permutation(seed, S_PERM_NODE, nnode)
        pe = permutation(seed, S_PERM_EDGE, nedge)
        pb = permutation(seed, S_PERM_BEDGE, nbedge)
        ic, inn = _inverse(pc), _inverse(pn)
        x = x[pn]
        cell2node = inn[cell2node[pc]]
        edge2node = inn[edge2node[pe]]
        edge2cell = ic[edge2cell[pe]]
        b_e2n = inn[b_e2n[pb]]
        b_e2c = ic[b_e2c[pb]]
        perms = {"cell": pc, "node": pn, "edge": pe, "bedge": pb}
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    return QuadMesh(nx, ny, h, np.ascontiguousarray(x), i32(cell2node), i32(edge2node), i32(edge2cell),
                    i32(b_e2n), i32(b_e2c), perms)


def quad_state(ncell: int, seed: int = DEFAULT_SEED, noise: float = 0.01,
               qinf: np.ndarray | None = None) -> np.ndarray:
    """Cell states q = qinf * (1 + noise * U(-1,1)) per component, [ncell, 4]."""
    if qinf is None:
        qinf = freestream()
    u = uniform(seed, S_NOISE, 4 * ncell).reshape(ncell, 4)
    return np.ascontiguousarray(qinf[None, :] * (1.0 + noise * (2.0 * u - 1.0)))


def adjoint_seed(ncell: int, seed: int = DEFAULT_SEED, ncomp: int = 4) -> np.ndarray:
    """Adjoint seeds res_bar ~ N(0,1), [ncell, ncomp]."""
    return np.ascontiguousarray(normal(seed, S_ADJ, ncomp * ncell).reshape(ncell, ncomp))


def directions(n: int, count: int, seed: int = DEFAULT_SEED, offset: int = 0) -> np.ndarray:
    """``count`` random N(0,1) direction vectors of length n (for derivative checks)."""
    return normal(seed, S_DIR, n * count, offset).reshape(count, n)


def positive_field(n: int, lo: float, hi: float, seed: int = DEFAULT_SEED, stream: int = S_DIR,
                   offset: int = 0) -> np.ndarray:
    """U(lo, hi) draws, for synthetic per-cell scalars such as a time-step field."""
    return lo + (hi - lo) * uniform(seed, stream, n, offset)


# --------------------------------------------------------------------------
# 3D hex mesh
# --------------------------------------------------------------------------

HEX_CORNERS = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                        [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.int64)


@dataclass
class HexMesh:
    n: int
    h: float
    x: np.ndarray          # [nnode, 3] float64
    elem2node: np.ndarray  # [nelem, 8] int32
    perms: dict = field(default_factory=dict)

    @property
    def nelem(self) -> int:
        return self.elem2node.shape[0]

    @property
    def nnode(self) -> int:
        return self.x.shape[0]


def hex_mesh(n: int, seed: int = DEFAULT_SEED, jitter: float = 0.2, permute: bool = True,
             nyz: tuple | None = None) -> HexMesh:
    """Jittered, renumbered hex grid of n x ny x nz elements on [0,1]x[0,ny h]x[0,nz h], h = 1/n."""
    ny, nz = (n, n) if nyz is None else nyz
    h = 1.0 / n
    nn = (n + 1, ny + 1, nz + 1)
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(n + 1), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    x = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    nnode = x.shape[0]
    interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz)
    if jitter > 0:
        u = uniform(seed, S_JITTER, 3 * nnode).reshape(nnode, 3)
        d = h * jitter * (2.0 * u - 1.0)
        x[interior] += d[interior]
    ek, ej, ei = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(n), indexing="ij")
    ei, ej, ek = ei.ravel(), ej.ravel(), ek.ravel()
    cols = []
    for s in HEX_CORNERS:
        di, dj, dk = (s + 1) // 2
        cols.append(((ek + dk) * nn[1] + (ej + dj)) * nn[0] + (ei + di))
    elem2node = np.stack(cols, axis=1)
    perms = {}
    if permute:
        pe = permutation(seed, S_PERM_CELL, elem2node.shape[0])
        pn = permutation(seed, S_PERM_NODE, nnode)
        inn = _inverse(pn)
        x = x[pn]
        elem2node = inn[elem2node[pe]]
        perms = {"elem": pe, "node": pn}
    return HexMesh(n, h, np.ascontiguousarray(x), np.ascontiguousarray(elem2node, dtype=np.int32), perms)


def hex_bricks(mesh: HexMesh, shape: tuple, dims: tuple) -> np.ndarray:
    """Block id of every element (in the mesh's numbering) for handcrafted
    brick-shaped blocks of shape = (bx, by, bz) elements on a structured grid
    of dims = (nx, ny, nz) elements: element (i, j, k) belongs to brick
    (i // bx, j // by, k // bz), numbered x fastest."""
    nx, ny, nz = dims
    bx, by, bz = shape
    orig = mesh.perms.get("elem", np.arange(mesh.nelem))
    i = orig % nx
    j = (orig // nx) % ny
    k = orig // (nx * ny)
    gx, gy = -(-nx // bx), -(-ny // by)
    return ((k // bz) * gy + (j // by)) * gx + (i // bx)


def hex_fields(mesh: HexMesh, seed: int = DEFAULT_SEED):
    """Element stresses sig = diag(sxx, syy, szz) ~ U(-1.5, -0.5) and nodal
    velocities v = A x + b + 0.1 N(0,1), with A, b ~ U(-1, 1)."""
    ne, nn = mesh.nelem, mesh.nnode
    u = uniform(seed, S_HEX, 3 * ne + 12)
    sig = (-1.5 + u[: 3 * ne]).reshape(ne, 3)
    ab = 2.0 * u[3 * ne:] - 1.0
    A = ab[:9].reshape(3, 3)
    b = ab[9:12]
    v = mesh.x @ A.T + b[None, :] + 0.1 * normal(seed, S_HEX, 3 * nn, offset=3 * ne + 12).reshape(nn, 3)
    return np.ascontiguousarray(sig), np.ascontiguousarray(v)


# --------------------------------------------------------------------------
# batches of meshes
# --------------------------------------------------------------------------

def batch_sizes(count: int = 64, qmin: int = 2000, qmax: int = 400000, amin: float = 1.0,
                amax: float = 4.0, seed: int = DEFAULT_SEED):
    """(nx, ny) per mesh: Q log-uniform in [qmin, qmax], aspect a ~ U(amin, amax),
    nx = round(sqrt(Q a)), ny = round(Q / nx)."""
    u = uniform(seed, S_BATCH, 2 * count)
    q = np.exp(math.log(qmin) + u[0::2] * (math.log(qmax) - math.log(qmin)))
    a = amin + (amax - amin) * u[1::2]
    nx = np.maximum(2, np.rint(np.sqrt(q * a))).astype(int)
    ny = np.maximum(2, np.rint(q / nx)).astype(int)
    return list(zip(nx.tolist(), ny.tolist()))


# --------------------------------------------------------------------------
# 2D triangle mesh and the increment-only loops' direct data
# --------------------------------------------------------------------------

@dataclass
class TriMesh:
    nx: int
    ny: int
    h: float
    x: np.ndarray          # [nnode, 2] float64
    cell2node: np.ndarray  # [ncell, 3] int32, counter-clockwise
    edge2node: np.ndarray  # [nedge, 2] int32, counter-clockwise in edge2cell[:, 0]
    edge2cell: np.ndarray  # [nedge, 2] int32; boundary edges repeat the cell
    eflag: np.ndarray      # [nedge] int32, 1 on boundary edges

    @property
    def ncell(self) -> int:
        return self.cell2node.shape[0]

    @property
    def nnode(self) -> int:
        return self.x.shape[0]

    @property
    def nedge(self) -> int:
        return self.edge2node.shape[0]


def tri_mesh(nx: int, ny: int, seed: int = DEFAULT_SEED, jitter: float = 0.2, permute: bool = True) -> TriMesh:
    """Each quad (i, j) of a jittered nx*ny grid on [0, nx/ny] x [0, 1] is
    split along the diagonal (i,j)-(i+1,j+1) when i+j is even, else along
    (i+1,j)-(i,j+1): 2 nx ny triangles, counter-clockwise."""
    q = quad_mesh(nx, ny, seed=seed, jitter=jitter, permute=False)
    nnx = nx + 1
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ci, cj = ci.ravel(), cj.ravel()
    n00, n10 = cj * nnx + ci, cj * nnx + ci + 1
    n01, n11 = (cj + 1) * nnx + ci, (cj + 1) * nnx + ci + 1
    even = (ci + cj) % 2 == 0
    t1 = np.where(even[:, None], np.stack([n00, n10, n11], 1), np.stack([n00, n10, n01], 1))
    t2 = np.where(even[:, None], np.stack([n00, n11, n01], 1), np.stack([n10, n11, n01], 1))
    tri = np.concatenate([t1, t2]).astype(np.int64)
    ntri = tri.shape[0]
    # half-edges (a -> b counter-clockwise in triangle t), grouped by node pair
    a = tri.ravel()
    b = tri[:, [1, 2, 0]].ravel()
    t = np.repeat(np.arange(ntri), 3)
    nnode = q.x.shape[0]
    key = np.minimum(a, b) * nnode + np.maximum(a, b)
    order = np.argsort(key, kind="stable")
    key, a, b, t = key[order], a[order], b[order], t[order]
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    idx = np.flatnonzero(first)
    cnt = np.diff(np.append(idx, key.size))
    e2n = np.stack([a[idx], b[idx]], 1)
    c1 = t[idx]
    c2 = np.where(cnt == 2, t[np.minimum(idx + 1, key.size - 1)], c1)
    flag = (cnt == 1).astype(np.int32)
    x = q.x
    if permute:
        pc = permutation(seed, S_PERM_CELL, ntri)
        pn = permutation(seed, S_PERM_NODE, nnode)
        pe = permutation(seed, S_PERM_EDGE, e2n.shape[0])
        ic, inn = _inverse(pc), _inverse(pn)
        x = x[pn]
        tri = inn[tri[pc]]
        e2n = inn[e2n[pe]]
        c1, c2, flag = ic[c1[pe]], ic[c2[pe]], flag[pe]
    i32 = lambda v: np.ascontiguousarray(v, dtype=np.int32)
    return TriMesh(nx, ny, q.h, np.ascontiguousarray(x), i32(tri), i32(e2n), i32(np.stack([c1, c2], 1)), i32(flag))


def volna_fields(mesh: TriMesh, seed: int = DEFAULT_SEED):
    """Direct data of the edge loop: per edge (F0, F1, F2, P, L, nx, ny) with
    F ~ N(0,1), P ~ U(0.5, 1.5), L the edge length and (nx, ny) the unit normal
    out of the edge's first cell; the cells' inverse areas.  float64 arrays;
    the loop runs on their float32 roundings."""
    xa = mesh.x[mesh.edge2node[:, 0]]
    xb = mesh.x[mesh.edge2node[:, 1]]
    d = xb - xa
    L = np.hypot(d[:, 0], d[:, 1])
    ne = mesh.nedge
    F = normal(seed, S_INC, 3 * ne).reshape(ne, 3)
    P = 0.5 + uniform(seed, S_INC, ne, offset=6 * ne)
    ed = np.column_stack([F, P, L, d[:, 1] / L, -d[:, 0] / L])
    p = mesh.x[mesh.cell2node]
    area = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    return np.ascontiguousarray(ed), 1.0 / area


def bookleaf_fields(ncell: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Direct data of the cell loop: per cell (rho, m[4], w[4], fx[4], fy[4])
    with rho ~ U(0.5, 2), m, w ~ U(0, 1), fx, fy ~ N(0, 1); [ncell, 17]."""
    u = uniform(seed, S_INC, 9 * ncell, offset=1 << 40).reshape(ncell, 9)
    g = normal(seed, S_INC, 8 * ncell, offset=1 << 41).reshape(ncell, 8)
    return np.ascontiguousarray(np.column_stack([0.5 + 1.5 * u[:, :1], u[:, 1:], g]))


# --------------------------------------------------------------------------
# hex faces and the face-flux loop's data
# --------------------------------------------------------------------------

# corners of the +x, +y and +z faces of an element (HEX_CORNERS order), listed
# so that A = (p2 - p0) x (p3 - p1) / 2 points to +x, +y, +z
_FACE_CORNERS = ((1, 2, 6, 5), (3, 7, 6, 2), (4, 5, 6, 7))


def hex_faces(mesh: HexMesh, dims: tuple | None = None, seed: int = DEFAULT_SEED):
    """Interior faces of the structured grid under ``mesh`` (dims = element
    counts, default n^3): face->cell[2] (int32; the first cell is on the low
    side, the area normal points into the second) and per face 12 doubles
    (A[3] area normal of the bilinear face, xf[3] mean of its corners,
    nhat[3] = A/|A|, dx[3] = centroid of cell 2 minus centroid of cell 1).
    Faces are renumbered by a seeded permutation."""
    nx, ny, nz = dims if dims is not None else (mesh.n, mesh.n, mesh.n)
    perm = mesh.perms.get("elem", np.arange(mesh.nelem))
    new_of = _inverse(perm)                      # original element id -> mesh id
    ek, ej, ei = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ei, ej, ek = ei.ravel(), ej.ravel(), ek.ravel()
    orig = (ek * ny + ej) * nx + ei
    c1s, c2s, corners = [], [], []
    for axis, (lim, step) in enumerate(((nx, 1), (ny, nx), (nz, nx * ny))):
        pos = (ei, ej, ek)[axis]
        sel = pos < lim - 1
        c1 = new_of[orig[sel]]
        c2 = new_of[orig[sel] + step]
        c1s.append(c1)
        c2s.append(c2)
        corners.append(mesh.elem2node[c1][:, list(_FACE_CORNERS[axis])])
    c1, c2, fc = np.concatenate(c1s), np.concatenate(c2s), np.concatenate(corners)
    pf = permutation(seed, S_FACE, c1.size)
    c1, c2, fc = c1[pf], c2[pf], fc[pf]
    p = mesh.x[fc]                               # [nf, 4, 3]
    A = 0.5 * np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 1])
    xf = p.mean(axis=1)
    nhat = A / np.linalg.norm(A, axis=1)[:, None]
    xc = mesh.x[mesh.elem2node].mean(axis=1)
    dx = xc[c2] - xc[c1]
    f2c = np.ascontiguousarray(np.stack([c1, c2], 1), dtype=np.int32)
    return f2c, np.ascontiguousarray(np.column_stack([A, xf, nhat, dx]))


def aero_cells(mesh: HexMesh, seed: int = DEFAULT_SEED, gam: float = GAMMA) -> np.ndarray:
    """Per cell 28 doubles: conserved state Q = (rho, rho u, rho v, rho w, E)
    with rho ~ U(0.9, 1.1), velocity ~ (0.3, 0.1, 0.05) + U(-0.05, 0.05),
    p = (1 + 0.1 U(-1, 1)) / gam; gradients of the primitives (rho, u, v, w,
    p) along x, y, z ~ 0.5 N(0, 1) (index 5 + 3 v + d); limiters ~ U(0.5, 1)
    (index 20 + v); the cell centroid (index 25..27)."""
    ne = mesh.nelem
    u = uniform(seed, S_FACE, 10 * ne, offset=1 << 40).reshape(ne, 10)
    rho = 0.9 + 0.2 * u[:, 0]
    vel = np.array([0.3, 0.1, 0.05]) + 0.1 * (u[:, 1:4] - 0.5)
    p = (1.0 + 0.1 * (2.0 * u[:, 4] - 1.0)) / gam
    E = p / (gam - 1.0) + 0.5 * rho * (vel ** 2).sum(1)
    Q = np.column_stack([rho, rho[:, None] * vel, E])
    G = 0.5 * normal(seed, S_FACE, 15 * ne, offset=1 << 41).reshape(ne, 15)
    phi = 0.5 + 0.5 * u[:, 5:10]
    xc = mesh.x[mesh.elem2node].mean(axis=1)
    return np.ascontiguousarray(np.column_stack([Q, G, phi, xc]))
