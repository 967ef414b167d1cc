"""Plain-Python restatements of the planner's integer objects -- TEST
INFRASTRUCTURE ONLY (see the package docstring).

Written from the definitions the planner documents, independently of its
C++ code, for bit-exact comparison on small meshes:

* first-fit colourings (Sec. 2.1 global colouring; Sec. 2.2 two-layer
  colouring: block colours on written points, then thread colours within
  each block, threads sorted by colour, Sec. 2.4);
* the reverse Cuthill-McKee ordering used as the bandwidth-reducing BFS
  renumbering of Sec. 2.3.1: George-Liu pseudo-peripheral start from the
  lowest-id minimum-degree vertex, neighbours visited by (degree, id),
  the whole sequence reversed; iterations then sorted lexicographically by
  their renumbered points and secondary points numbered by first touch;
* the data-point key of Sec. 2.3.2 (number of accessing blocks, then the
  sorted accessing block ids);
* the data reuse factor of Sec. 3.1 and the plan invariants.
"""
from __future__ import annotations

from collections import deque

import numpy as np


# ------------------------------------------------------------------ colouring

def first_fit_items(rows, order=None):
    """First-fit colours of items visited in ``order``: an item takes the
    smallest colour not held by an earlier item sharing a point.
    ``rows[i]`` is the list of written points of item i."""
    n = len(rows)
    order = range(n) if order is None else order
    used = {}
    color = [-1] * n
    for i in order:
        taken = set()
        for p in rows[i]:
            taken |= used.get(p, set())
        c = 0
        while c in taken:
            c += 1
        color[i] = c
        for p in rows[i]:
            used.setdefault(p, set()).add(c)
    return color


def block_colors(blocks, written_rows):
    """First-fit block colours: blocks in id order, a conflict iff two blocks
    share a written point.  ``blocks[b]`` lists the items of block b."""
    brows = []
    for items in blocks:
        pts = set()
        for i in items:
            pts.update(written_rows[i])
        brows.append(sorted(pts))
    return first_fit_items(brows)


def thread_colors(items, written_rows):
    """First-fit colours of the items of one block in the given order."""
    return first_fit_items([written_rows[i] for i in items])


def written_rows_of(maps):
    """Per item, the written points as (map_to_set, point) tuples."""
    n = maps[0]["idx"].shape[0]
    rows = [[] for _ in range(n)]
    for m in maps:
        if not m["written"]:
            continue
        idx = m["idx"]
        for i in range(n):
            rows[i].extend((m["to_set"], int(p)) for p in idx[i])
    return rows


# ------------------------------------------------------------------ RCM

def clique_graph(idx, npoints):
    """Adjacency sets of the graph whose vertices are the to-set points and
    whose edges join points that appear in one row of the map (each row is a
    clique, Sec. 2.3.1)."""
    adj = [set() for _ in range(npoints)]
    for row in idx:
        row = [int(p) for p in row]
        for a in row:
            for b in row:
                if a != b:
                    adj[a].add(b)
    return adj


def _bfs_levels(adj, start, alive):
    levels = [[start]]
    seen = {start}
    while True:
        nxt = []
        for u in levels[-1]:
            for w in sorted(adj[u]):
                if alive[w] and w not in seen:
                    seen.add(w)
                    nxt.append(w)
        if not nxt:
            return levels
        levels.append(nxt)


def rcm_order(adj):
    """Reverse Cuthill-McKee order (list of old ids, new id = position)."""
    n = len(adj)
    deg = [len(a) for a in adj]
    alive = [True] * n
    cm = []
    by_degree = sorted(range(n), key=lambda v: (deg[v], v))
    for v0 in by_degree:
        if not alive[v0]:
            continue
        # George-Liu pseudo-peripheral vertex
        r = v0
        levels = _bfs_levels(adj, r, alive)
        while True:
            last = levels[-1]
            w = min(last, key=lambda v: (deg[v], v))
            lw = _bfs_levels(adj, w, alive)
            if len(lw) > len(levels):
                r, levels = w, lw
            else:
                break
        # Cuthill-McKee BFS from r
        alive[r] = False
        q = deque([r])
        while q:
            u = q.popleft()
            cm.append(u)
            nb = [w for w in adj[u] if alive[w]]
            nb.sort(key=lambda v: (deg[v], v))
            for w in nb:
                alive[w] = False
                q.append(w)
    return cm[::-1]


def rcm_plan_perms(maps, from_size, primary):
    """Permutations (new_to_old) of the from-set and every to-set under the
    RCM reorder: primary to-set by RCM, iterations sorted by the ascending
    tuple of their renumbered primary points (ties by old id), other to-sets
    numbered by first touch over the sorted iterations (map order, slot
    order), untouched points last in old order."""
    pm = maps[primary]
    order = rcm_order(clique_graph(pm["idx"], pm["to_size"]))
    new_p = np.empty(pm["to_size"], dtype=np.int64)
    new_p[np.array(order, dtype=np.int64)] = np.arange(len(order))
    keys = [(tuple(sorted(int(new_p[p]) for p in pm["idx"][i])), i) for i in range(from_size)]
    items = [i for _, i in sorted(keys)]
    perms = {0: np.array(items, dtype=np.int64), pm["to_set"]: np.array(order, dtype=np.int64)}
    for m in maps:
        t = m["to_set"]
        if t in perms:
            continue
        seen = np.zeros(m["to_size"], dtype=bool)
        seq = []
        for i in items:
            for m2 in maps:
                if m2["to_set"] != t:
                    continue
                for p in m2["idx"][i]:
                    p = int(p)
                    if not seen[p]:
                        seen[p] = True
                        seq.append(p)
        seq.extend(int(p) for p in np.nonzero(~seen)[0])
        perms[t] = np.array(seq, dtype=np.int64)
    return perms


# ------------------------------------------------------------------ data reorder

def data_point_order(block_of_item, idx_list, npoints):
    """Order of points by key (number of distinct accessing blocks, sorted
    accessing block ids), ties by id; unaccessed points last (Sec. 2.3.2)."""
    acc = [set() for _ in range(npoints)]
    for idx in idx_list:
        for i, row in enumerate(idx):
            for p in row:
                acc[int(p)].add(int(block_of_item[i]))
    def key(p):
        s = sorted(acc[p])
        return (len(s) if s else 1 << 30, s, p)
    return sorted(range(npoints), key=key)


# ------------------------------------------------------------------ metrics

def reuse_factor(block_offsets, idx_list, to_sets=None):
    """Accesses to staged points over distinct staged points, summed over
    blocks (Sec. 3.1's data reuse factor).  ``to_sets[k]`` names the to-set
    of ``idx_list[k]`` (maps into one to-set share its points); by default
    every map has its own to-set."""
    to_sets = list(range(len(idx_list))) if to_sets is None else to_sets
    acc = 0
    uniq = 0
    for b in range(len(block_offsets) - 1):
        s, e = block_offsets[b], block_offsets[b + 1]
        pts = set()
        for t, idx in zip(to_sets, idx_list):
            rows = idx[s:e]
            acc += rows.size
            pts.update((t, int(p)) for p in rows.ravel())
        uniq += len(pts)
    return acc / max(uniq, 1)


def check_coloring(rows, color, groups=None):
    """True iff no two items of one colour (within one group) share a point."""
    groups = [range(len(rows))] if groups is None else groups
    for g in groups:
        owner = {}
        for i in g:
            for p in rows[i]:
                k = (color[i], p)
                if k in owner and owner[k] != i:
                    return False
                owner[k] = i
    return True


def is_permutation(p, n):
    p = np.asarray(p)
    return p.shape == (n,) and np.array_equal(np.sort(p), np.arange(n))
