// Host planner for indirect-increment mesh loops (Sec. 2.2 and 2.3 of
// Sulyok et al., "Locality Optimized Unstructured Mesh Algorithms on GPUs").
//
// Steps, in order:
//   1. validation of the maps (fixed arity, indices in range; Sec. 1.1.1)
//   2. reordering (Sec. 2.3.1): reverse Cuthill-McKee on the clique graph of
//      the primary map's to-set, iterations sorted lexicographically by their
//      renumbered points, other to-sets numbered by first touch
//   3. blocks: contiguous chunks of S iterations, or (Sec. 2.3.2) a greedy
//      graph-growing partition into compact blocks of at most S' = floor(S/l)
//      iterations (Eq. 1); the paper used METIS k-way partitioning here
//   4. colouring: first-fit block colours on written points, blocks sorted by
//      colour, first-fit thread colours inside each block, threads sorted by
//      colour (Sec. 2.2, 2.4); or first-fit iteration colours (global
//      colouring, Sec. 2.1); or none (atomics)
//   5. data-point reordering by (number of accessing blocks, accessing block
//      ids) (Sec. 2.3.2)
//   6. per-block footprint lists and 16-bit block-local maps
// Everything here is host code and touches no GPU.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <queue>
#include <stdexcept>

#include "plan_internal.h"

namespace {

struct plan_error {
    int code;
};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Stable LSD radix sort of idx by key (11-bit digits, as many passes as the
// largest key needs): equal keys keep their order in idx.
void radix_sort(std::vector<uint64_t> &key, std::vector<int32_t> &idx)
{
    const size_t n = key.size();
    uint64_t all = 0;
    for (uint64_t k : key) all |= k;
    int bits = 0;
    while (bits < 64 && (all >> bits) != 0) ++bits;
    std::vector<uint64_t> k2(n);
    std::vector<int32_t> i2(n);
    for (int shift = 0; shift < bits; shift += 11) {
        size_t cnt[2049] = {0};
        for (uint64_t k : key) cnt[((k >> shift) & 2047) + 1]++;
        for (int d = 0; d < 2048; ++d) cnt[d + 1] += cnt[d];
        for (size_t j = 0; j < n; ++j) {
            const size_t to = cnt[(key[j] >> shift) & 2047]++;
            k2[to] = key[j];
            i2[to] = idx[j];
        }
        key.swap(k2);
        idx.swap(i2);
    }
}

// ----------------------------------------------------------------- CSR utils

struct csr {
    std::vector<int64_t> off;
    std::vector<int32_t> adj;
};

// point -> iterations incidence of the given maps into one to-set (with
// repetition if an iteration references a point twice).
csr point_to_items(const mp_plan &P, int slot, const std::vector<int32_t> *map_idx_override = nullptr)
{
    csr g;
    int64_t n = P.toset_size[slot];
    g.off.assign(n + 1, 0);
    for (int m = 0; m < P.nmaps; ++m) {
        if (P.maps[m].slot != slot) continue;
        const auto &idx = map_idx_override ? map_idx_override[m] : P.maps[m].idx;
        for (int32_t p : idx) g.off[p + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) g.off[i + 1] += g.off[i];
    g.adj.resize(g.off[n]);
    std::vector<int64_t> pos(g.off.begin(), g.off.end() - 1);
    for (int m = 0; m < P.nmaps; ++m) {
        if (P.maps[m].slot != slot) continue;
        const auto &idx = map_idx_override ? map_idx_override[m] : P.maps[m].idx;
        int a = P.maps[m].arity;
        for (int64_t i = 0; i < P.from_size; ++i)
            for (int k = 0; k < a; ++k) g.adj[pos[idx[i * a + k]]++] = (int32_t)i;
    }
    return g;
}

// Clique graph of one map (Sec. 2.3.1, mesh-to-graph): vertices are the
// to-set points, u ~ v iff they appear in a common row.  Adjacency lists are
// sorted and free of duplicates and self loops.
csr clique_graph(const std::vector<int32_t> &idx, int64_t from_size, int arity, int64_t npts)
{
    csr g;
    g.off.assign(npts + 1, 0);
    for (int64_t i = 0; i < from_size; ++i)
        for (int k = 0; k < arity; ++k) g.off[idx[i * arity + k] + 1] += arity - 1;
    for (int64_t i = 0; i < npts; ++i) g.off[i + 1] += g.off[i];
    std::vector<int32_t> tmp(g.off[npts]);
    std::vector<int64_t> pos(g.off.begin(), g.off.end() - 1);
    for (int64_t i = 0; i < from_size; ++i)
        for (int k = 0; k < arity; ++k)
            for (int l = 0; l < arity; ++l)
                if (l != k) tmp[pos[idx[i * arity + k]]++] = idx[i * arity + l];
    // sort + unique each list, drop self loops
    std::vector<int64_t> noff(npts + 1, 0);
    int64_t w = 0;
    for (int64_t v = 0; v < npts; ++v) {
        auto b = tmp.begin() + g.off[v], e = tmp.begin() + g.off[v + 1];
        std::sort(b, e);
        int32_t last = -1;
        noff[v] = w;
        for (auto it = b; it != e; ++it) {
            if (*it == last || *it == v) continue;
            last = *it;
            tmp[w++] = *it;
        }
    }
    noff[npts] = w;
    tmp.resize(w);
    g.off.swap(noff);
    g.adj.swap(tmp);
    return g;
}

// BFS level structure restricted to unnumbered vertices; returns the
// number of levels and the last level's vertices.
int bfs_levels(const csr &g, int32_t start, const std::vector<uint8_t> &done, std::vector<int32_t> &stamp,
               int32_t mark, std::vector<int32_t> &queue, std::vector<int32_t> &last_level)
{
    queue.clear();
    queue.push_back(start);
    stamp[start] = mark;
    size_t level_begin = 0;
    int nlevels = 0;
    while (level_begin < queue.size()) {
        size_t level_end = queue.size();
        ++nlevels;
        for (size_t i = level_begin; i < level_end; ++i) {
            int32_t u = queue[i];
            for (int64_t j = g.off[u]; j < g.off[u + 1]; ++j) {
                int32_t w = g.adj[j];
                if (done[w] || stamp[w] == mark) continue;
                stamp[w] = mark;
                queue.push_back(w);
            }
        }
        if (queue.size() == level_end) {
            last_level.assign(queue.begin() + level_begin, queue.begin() + level_end);
            break;
        }
        level_begin = level_end;
    }
    return nlevels;
}

// Reverse Cuthill-McKee: each component starts at a George-Liu
// pseudo-peripheral vertex found from the lowest-id minimum-degree vertex
// still unnumbered; neighbours are appended by (degree, id); the whole
// Cuthill-McKee sequence is reversed.  Returns new_to_old.
std::vector<int32_t> rcm(const csr &g)
{
    int64_t n = (int64_t)g.off.size() - 1;
    std::vector<int32_t> deg(n);
    for (int64_t v = 0; v < n; ++v) deg[v] = (int32_t)(g.off[v + 1] - g.off[v]);
    std::vector<int32_t> by_deg(n);
    for (int64_t v = 0; v < n; ++v) by_deg[v] = (int32_t)v;
    std::stable_sort(by_deg.begin(), by_deg.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
    std::vector<uint8_t> done(n, 0);
    std::vector<int32_t> stamp(n, -1), queue, last, cm;
    cm.reserve(n);
    int32_t mark = 0;
    std::vector<int32_t> nb;
    for (int32_t v0 : by_deg) {
        if (done[v0]) continue;
        int32_t r = v0;
        int h = bfs_levels(g, r, done, stamp, mark++, queue, last);
        for (;;) {
            int32_t w = last[0];
            for (int32_t c : last)
                if (deg[c] < deg[w] || (deg[c] == deg[w] && c < w)) w = c;
            std::vector<int32_t> last_w;
            int hw = bfs_levels(g, w, done, stamp, mark++, queue, last_w);
            if (hw > h) {
                r = w;
                h = hw;
                last.swap(last_w);
            } else {
                break;
            }
        }
        size_t head = cm.size();
        cm.push_back(r);
        done[r] = 1;
        while (head < cm.size()) {
            int32_t u = cm[head++];
            nb.clear();
            for (int64_t j = g.off[u]; j < g.off[u + 1]; ++j)
                if (!done[g.adj[j]]) nb.push_back(g.adj[j]);
            std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
                return deg[a] < deg[b] || (deg[a] == deg[b] && a < b);
            });
            for (int32_t w : nb) {
                done[w] = 1;
                cm.push_back(w);
            }
        }
    }
    std::reverse(cm.begin(), cm.end());
    return cm;
}

std::vector<int32_t> inverse(const std::vector<int32_t> &p)
{
    std::vector<int32_t> inv(p.size());
    for (size_t i = 0; i < p.size(); ++i) inv[p[i]] = (int32_t)i;
    return inv;
}

// Apply new_to_old permutations of the from-set and one to-set to a map.
void renumber(std::vector<int32_t> &idx, int arity, const std::vector<int32_t> *from_n2o,
              const std::vector<int32_t> *to_n2o)
{
    int64_t n = (int64_t)idx.size() / arity;
    std::vector<int32_t> out(idx.size());
    std::vector<int32_t> to_o2n;
    if (to_n2o) to_o2n = inverse(*to_n2o);
    for (int64_t i = 0; i < n; ++i) {
        int64_t src = from_n2o ? (*from_n2o)[i] : i;
        for (int k = 0; k < arity; ++k) {
            int32_t p = idx[src * arity + k];
            out[i * arity + k] = to_n2o ? to_o2n[p] : p;
        }
    }
    idx.swap(out);
}

void compose(std::vector<int32_t> &total, const std::vector<int32_t> &step)
{
    // total: new_to_old so far; step: new_to_old of a further renumbering
    std::vector<int32_t> out(step.size());
    for (size_t i = 0; i < step.size(); ++i) out[i] = total[step[i]];
    total.swap(out);
}

// Apply an iteration permutation (new_to_old) to every map and to the
// accumulated from-set permutation.
void permute_items(mp_plan &P, const std::vector<int32_t> &n2o)
{
    for (int m = 0; m < P.nmaps; ++m) renumber(P.maps[m].idx, P.maps[m].arity, &n2o, nullptr);
    compose(P.perm_from, n2o);
}

void permute_points(mp_plan &P, int slot, const std::vector<int32_t> &n2o)
{
    for (int m = 0; m < P.nmaps; ++m)
        if (P.maps[m].slot == slot) renumber(P.maps[m].idx, P.maps[m].arity, nullptr, &n2o);
    compose(P.perm_to[slot], n2o);
}

// ----------------------------------------------------------- 2. reordering

void reorder_rcm(mp_plan &P, int primary)
{
    const mp_map_info &pm = P.maps[primary];
    int ps = pm.slot;
    csr g = clique_graph(pm.idx, P.from_size, pm.arity, P.toset_size[ps]);
    std::vector<int32_t> order = rcm(g);
    permute_points(P, ps, order);
    // iterations sorted by the ascending tuple of their primary points
    int a = pm.arity;
    int64_t n = P.from_size;
    std::vector<int32_t> keys((size_t)n * a);
    for (int64_t i = 0; i < n; ++i) {
        std::copy(pm.idx.begin() + i * a, pm.idx.begin() + (i + 1) * a, keys.begin() + i * a);
        std::sort(keys.begin() + i * a, keys.begin() + (i + 1) * a);
    }
    std::vector<int32_t> items(n);
    for (int64_t i = 0; i < n; ++i) items[i] = (int32_t)i;
    if (a <= 2) {
        // the (at most two) non-negative 31-bit keys packed in one word:
        // a stable radix sort from ascending ids gives the same order
        std::vector<uint64_t> packed(n);
        for (int64_t i = 0; i < n; ++i)
            packed[i] = a == 1 ? (uint64_t)keys[i] : ((uint64_t)keys[2 * i] << 31) | (uint64_t)keys[2 * i + 1];
        radix_sort(packed, items);
    } else {
        std::sort(items.begin(), items.end(), [&](int32_t x, int32_t y) {
            for (int k = 0; k < a; ++k) {
                int32_t kx = keys[(int64_t)x * a + k], ky = keys[(int64_t)y * a + k];
                if (kx != ky) return kx < ky;
            }
            return x < y;
        });
    }
    permute_items(P, items);
    // other to-sets: first touch over the sorted iterations, map then slot order
    for (int s = 0; s < P.ntosets; ++s) {
        if (s == ps) continue;
        std::vector<uint8_t> seen(P.toset_size[s], 0);
        std::vector<int32_t> seq;
        seq.reserve(P.toset_size[s]);
        for (int64_t i = 0; i < n; ++i)
            for (int m = 0; m < P.nmaps; ++m) {
                if (P.maps[m].slot != s) continue;
                for (int k = 0; k < P.maps[m].arity; ++k) {
                    int32_t p = P.maps[m].idx[i * P.maps[m].arity + k];
                    if (!seen[p]) {
                        seen[p] = 1;
                        seq.push_back(p);
                    }
                }
            }
        for (int64_t p = 0; p < P.toset_size[s]; ++p)
            if (!seen[p]) seq.push_back((int32_t)p);
        permute_points(P, s, seq);
    }
}

// -------------------------------------------------------- 3. partitioning

// Greedy graph growing on G_M (iterations adjacent iff they share a point,
// Sec. 2.3.2).  A block starts at the lowest-numbered free iteration and
// repeatedly takes the free iteration with the most points already in the
// block's footprint; ties go to the iteration that reached that gain first
// (first in, first out), which grows the block as a compact ball around its
// seed rather than along the numbering.  Blocks hold at most S' iterations;
// when a block's neighbourhood is exhausted it continues from the next free
// iteration.  Returns the block of each iteration; blocks are numbered in
// creation order.
std::vector<int32_t> partition_greedy(const mp_plan &P, int sprime, int32_t &nblocks)
{
    int64_t n = P.from_size;
    std::vector<int32_t> block(n, -1);
    csr p2i[MP_MAX_TOSETS];
    std::vector<int32_t> mark[MP_MAX_TOSETS];
    for (int s = 0; s < P.ntosets; ++s) {
        p2i[s] = point_to_items(P, s);
        mark[s].assign(P.toset_size[s], -1);
    }
    int maxgain = 0;
    for (int m = 0; m < P.nmaps; ++m) maxgain += P.maps[m].arity;
    std::vector<int16_t> gain(n, 0);
    std::vector<std::vector<int32_t>> bucket(maxgain + 1);   // FIFO per gain level
    std::vector<size_t> head(maxgain + 1, 0);
    std::vector<int32_t> touched;
    int64_t next_free = 0;
    int32_t b = 0;
    int64_t assigned = 0;
    while (assigned < n) {
        int count = 0;
        touched.clear();
        int top = -1;
        auto add = [&](int32_t it) {
            block[it] = b;
            ++count;
            ++assigned;
            for (int m = 0; m < P.nmaps; ++m) {
                const mp_map_info &mi = P.maps[m];
                int s = mi.slot;
                for (int k = 0; k < mi.arity; ++k) {
                    int32_t p = mi.idx[(int64_t)it * mi.arity + k];
                    if (mark[s][p] == b) continue;
                    mark[s][p] = b;
                    for (int64_t j = p2i[s].off[p]; j < p2i[s].off[p + 1]; ++j) {
                        int32_t o = p2i[s].adj[j];
                        if (block[o] >= 0) continue;
                        if (gain[o] == 0) touched.push_back(o);
                        int g = ++gain[o];
                        if (g > maxgain) g = maxgain;
                        bucket[g].push_back(o);
                        if (g > top) top = g;
                    }
                }
            }
        };
        while (count < sprime && assigned < n) {
            int32_t pick = -1;
            while (top > 0 && pick < 0) {
                auto &q = bucket[top];
                while (head[top] < q.size()) {
                    int32_t o = q[head[top]++];
                    if (block[o] < 0 && gain[o] == top) {
                        pick = o;
                        break;
                    }
                }
                if (pick < 0) --top;
            }
            if (pick < 0) {
                while (next_free < n && block[next_free] >= 0) ++next_free;
                pick = (int32_t)next_free;
            }
            add(pick);
        }
        for (int32_t o : touched) gain[o] = 0;
        for (int g = 0; g <= maxgain; ++g) {
            bucket[g].clear();
            head[g] = 0;
        }
        ++b;
    }
    nblocks = b;
    return block;
}

// ----------------------------------------------------------- 4. colouring

// First-fit colouring of groups in order: a group takes the smallest colour
// not held by an earlier group sharing a written point.  points_of(g, out)
// lists the written points of group g as (slot, point).  masks hold up to
// 256 colours per point.
template <class F>
std::vector<int32_t> first_fit(const mp_plan &P, int64_t ngroups, F points_of, int max_colors, int32_t &ncolors)
{
    constexpr int W = MP_MAX_BLOCK_COLORS / 64;
    std::vector<uint64_t> mask[MP_MAX_TOSETS];
    for (int s = 0; s < P.ntosets; ++s) mask[s].assign((size_t)P.toset_size[s] * W, 0);
    std::vector<int32_t> color(ngroups, -1);
    std::vector<std::pair<int, int32_t>> pts;
    ncolors = 0;
    for (int64_t g = 0; g < ngroups; ++g) {
        pts.clear();
        points_of(g, pts);
        uint64_t used[W] = {0, 0, 0, 0};
        for (auto &sp : pts)
            for (int w = 0; w < W; ++w) used[w] |= mask[sp.first][(size_t)sp.second * W + w];
        int c = -1;
        for (int w = 0; w < W && c < 0; ++w)
            if (~used[w]) c = w * 64 + __builtin_ctzll(~used[w]);
        if (c < 0 || c >= max_colors) throw plan_error{MP_ECOLORS};
        color[g] = c;
        for (auto &sp : pts) mask[sp.first][(size_t)sp.second * W + c / 64] |= 1ull << (c % 64);
        if (c + 1 > ncolors) ncolors = c + 1;
    }
    return color;
}

void written_points(const mp_plan &P, int64_t it, std::vector<std::pair<int, int32_t>> &out)
{
    for (int m = 0; m < P.nmaps; ++m) {
        const mp_map_info &mi = P.maps[m];
        if (!mi.written) continue;
        for (int k = 0; k < mi.arity; ++k) out.emplace_back(mi.slot, mi.idx[it * mi.arity + k]);
    }
}

// Dissolves the blocks of a sparse last block colour (at most nblocks/32)
// into pieces of earlier colours: each iteration of such a block joins the
// first colour c < K-1 whose other blocks touch none of its written points
// (points the block's own pieces took in c do not count); the iterations
// that chose c form one new block of colour c.  A block with an iteration
// that fits no colour stays whole, and then the colour stays.  Pieces are
// subsets of their block, so no piece exceeds the block size.
void split_last_color(const mp_plan &P, std::vector<int32_t> &color, int32_t &ncolors,
                      std::vector<std::vector<int32_t>> &pieces, std::vector<int32_t> &piece_color,
                      std::vector<char> &dissolved)
{
    const int32_t nb = P.nblocks;
    pieces.clear();
    piece_color.clear();
    dissolved.assign(nb, 0);
    if (ncolors < 2 || ncolors > 64) return;
    const int last = ncolors - 1;
    std::vector<int32_t> todo;
    for (int32_t b = 0; b < nb; ++b)
        if (color[b] == last) todo.push_back(b);
    if (todo.empty() || (int64_t)todo.size() * 32 > nb) return;
    // colours of the blocks touching each written point
    std::vector<uint64_t> mask[MP_MAX_TOSETS];
    for (int s = 0; s < P.ntosets; ++s) mask[s].assign(P.toset_size[s], 0);
    std::vector<std::pair<int, int32_t>> pts;
    for (int32_t b = 0; b < nb; ++b) {
        if (color[b] == last) continue;
        pts.clear();
        for (int32_t it = P.block_offsets[b]; it < P.block_offsets[b + 1]; ++it) written_points(P, it, pts);
        for (auto &sp : pts) mask[sp.first][sp.second] |= 1ull << color[b];
    }
    bool all = true;
    std::vector<std::pair<int, int32_t>> mine;  // (slot, point) this block took, per colour below
    std::vector<uint64_t> mine_mask;
    for (int32_t B : todo) {
        const int32_t s0 = P.block_offsets[B], s1 = P.block_offsets[B + 1];
        std::vector<std::vector<int32_t>> part(last);
        std::vector<std::pair<std::pair<int, int32_t>, uint64_t>> took;  // point -> colours B took it in
        auto took_in = [&](const std::pair<int, int32_t> &sp) -> uint64_t {
            for (auto &t : took)
                if (t.first == sp) return t.second;
            return 0;
        };
        bool ok = true;
        for (int32_t it = s0; it < s1 && ok; ++it) {
            pts.clear();
            written_points(P, it, pts);
            int chosen = -1;
            for (int c = 0; c < last && chosen < 0; ++c) {
                bool fits = true;
                for (auto &sp : pts)
                    if ((mask[sp.first][sp.second] >> c & 1) && !(took_in(sp) >> c & 1)) fits = false;
                if (fits) chosen = c;
            }
            if (chosen < 0) {
                ok = false;
                break;
            }
            part[chosen].push_back(it);
            for (auto &sp : pts) {
                bool found = false;
                for (auto &t : took)
                    if (t.first == sp) {
                        t.second |= 1ull << chosen;
                        found = true;
                    }
                if (!found) took.push_back({sp, 1ull << chosen});
            }
        }
        if (!ok) {
            all = false;
            continue;
        }
        // the pieces now own their points in their colours
        for (auto &t : took) mask[t.first.first][t.first.second] |= t.second;
        dissolved[B] = 1;
        for (int c = 0; c < last; ++c)
            if (!part[c].empty()) {
                pieces.push_back(std::move(part[c]));
                piece_color.push_back(c);
            }
    }
    if (all) ncolors = last;
}

// Empties sparse trailing block colours after first fit.  First fit on a
// partitioned mesh typically leaves a last colour or two with a handful of
// blocks, each a launch of its own.  For every block B of the last colour K-1
// (while it holds at most nblocks/32 blocks), in order:
//  1. an earlier colour c whose blocks conflicting with B (sharing a written
//     point) are at most two and can each move to a colour c' < K-1,
//     c' != c, free of conflicts: apply the moves, B takes c;
//  2. otherwise a Kempe-chain interchange: for colours c != c2 below K-1,
//     the connected set of c- and c2-coloured blocks reachable from B's
//     c-neighbours; if it holds none of B's c2-neighbours, swapping c and c2
//     inside it frees c for B (the swap keeps the colouring valid).
// Stops at the first colour that cannot be emptied completely (the blocks
// already moved stay moved: still a valid colouring).  Deterministic.
// Plans with more than 64 colours (blocks of an unordered mesh) keep their
// first-fit colours: one launch in that many matters little, and the colour
// pairs the interchanges try (quadratic in the colours, each over the
// block's neighbours) would dominate the build.
void reduce_sparse_colors(const mp_plan &P, std::vector<int32_t> &color, int32_t &ncolors)
{
    const int32_t nb = P.nblocks;
    if (nb < 2 || ncolors < 2 || ncolors > 64) return;
    // block adjacency through shared written points
    std::vector<int32_t> off[MP_MAX_TOSETS], lst[MP_MAX_TOSETS];
    std::vector<std::pair<int, int32_t>> pts;
    std::vector<std::vector<std::pair<int, int32_t>>> bpts(nb);
    for (int s = 0; s < P.ntosets; ++s) off[s].assign(P.toset_size[s] + 1, 0);
    for (int32_t b = 0; b < nb; ++b) {
        pts.clear();
        for (int32_t it = P.block_offsets[b]; it < P.block_offsets[b + 1]; ++it) written_points(P, it, pts);
        std::sort(pts.begin(), pts.end());
        pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
        for (auto &sp : pts) off[sp.first][sp.second + 1]++;
        bpts[b] = pts;
    }
    for (int s = 0; s < P.ntosets; ++s) {
        for (int64_t i = 0; i < P.toset_size[s]; ++i) off[s][i + 1] += off[s][i];
        lst[s].assign(off[s].back(), 0);
    }
    {
        std::vector<int32_t> pos[MP_MAX_TOSETS];
        for (int s = 0; s < P.ntosets; ++s) pos[s].assign(off[s].begin(), off[s].end() - 1);
        for (int32_t b = 0; b < nb; ++b)
            for (auto &sp : bpts[b]) lst[sp.first][pos[sp.first][sp.second]++] = b;
    }
    std::vector<std::vector<int32_t>> adj(nb);
    for (int32_t b = 0; b < nb; ++b) {
        std::vector<int32_t> &a = adj[b];
        for (auto &sp : bpts[b])
            for (int32_t j = off[sp.first][sp.second]; j < off[sp.first][sp.second + 1]; ++j)
                if (lst[sp.first][j] != b) a.push_back(lst[sp.first][j]);
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    auto free_in = [&](int32_t b, int c) {
        for (int32_t n : adj[b])
            if (color[n] == c) return false;
        return true;
    };
    std::vector<int32_t> chain, mark(nb, 0);
    int32_t stamp = 1;
    while (ncolors > 1) {
        const int last = ncolors - 1;
        std::vector<int32_t> todo;
        for (int32_t b = 0; b < nb; ++b)
            if (color[b] == last) todo.push_back(b);
        if ((int64_t)todo.size() * 32 > nb) return;
        // a few sweeps: a later placement can open a way for an earlier block
        for (int sweep = 0; sweep < 4 && !todo.empty(); ++sweep) {
        std::vector<int32_t> left;
        for (int32_t B : todo) {
            bool placed = false;
            for (int c = 0; c < last && !placed; ++c) {
                std::vector<int32_t> conf;
                for (int32_t n : adj[B])
                    if (color[n] == c) conf.push_back(n);
                if (conf.size() > 2) continue;
                std::vector<std::pair<int32_t, int>> undo;
                bool ok = true;
                for (int32_t N : conf) {
                    int to = -1;
                    for (int c2 = 0; c2 < last && to < 0; ++c2)
                        if (c2 != c && free_in(N, c2)) to = c2;
                    if (to < 0) {
                        ok = false;
                        break;
                    }
                    undo.emplace_back(N, color[N]);
                    color[N] = to;
                }
                if (ok && free_in(B, c)) {
                    color[B] = c;
                    placed = true;
                } else {
                    for (auto it = undo.rbegin(); it != undo.rend(); ++it) color[it->first] = it->second;
                }
            }
            for (int c = 0; c < last && !placed; ++c)
                for (int c2 = 0; c2 < last && !placed; ++c2) {
                    if (c2 == c) continue;
                    // the (c, c2) chain from B's c-neighbours
                    chain.clear();
                    for (int32_t n : adj[B])
                        if (color[n] == c && mark[n] != stamp) {
                            mark[n] = stamp;
                            chain.push_back(n);
                        }
                    bool blocked = false;
                    for (size_t h = 0; h < chain.size() && !blocked; ++h)
                        for (int32_t n : adj[chain[h]]) {
                            if (n == B || (color[n] != c && color[n] != c2) || mark[n] == stamp) continue;
                            mark[n] = stamp;
                            chain.push_back(n);
                        }
                    for (int32_t n : adj[B])
                        if (color[n] == c2 && mark[n] == stamp) blocked = true;
                    ++stamp;
                    if (blocked || chain.empty()) continue;
                    for (int32_t n : chain) color[n] = color[n] == c ? c2 : c;
                    color[B] = c;
                    placed = true;
                }
            if (!placed) left.push_back(B);
        }
        const bool progress = left.size() < todo.size();
        todo.swap(left);
        if (!progress) break;
        }
        if (!todo.empty()) return;
        ncolors = last;
    }
}

// Thread colours inside each block: first fit over the block's iterations
// in order, on written points (64-bit masks, reset per block).  Then the
// iterations of each block are stably sorted by colour (Sec. 2.4).
// Returns the iteration permutation (new_to_old) and fills thread colours.
std::vector<int32_t> color_threads(mp_plan &P)
{
    std::vector<uint64_t> mask[MP_MAX_TOSETS];
    for (int s = 0; s < P.ntosets; ++s) mask[s].assign(P.toset_size[s], 0);
    std::vector<int32_t> n2o(P.from_size);
    std::vector<uint8_t> tc(P.from_size);
    P.block_ncolors.assign(P.nblocks, 0);
    std::vector<std::pair<int, int32_t>> pts;
    std::vector<std::pair<int, int32_t>> all;
    std::vector<int32_t> col;
    for (int32_t b = 0; b < P.nblocks; ++b) {
        int32_t s0 = P.block_offsets[b], s1 = P.block_offsets[b + 1];
        col.assign(s1 - s0, 0);
        all.clear();
        int nc = 0;
        for (int32_t it = s0; it < s1; ++it) {
            pts.clear();
            written_points(P, it, pts);
            uint64_t used = 0;
            for (auto &sp : pts) used |= mask[sp.first][sp.second];
            if (used == ~0ull) throw plan_error{MP_ECOLORS};
            int c = __builtin_ctzll(~used);
            if (c >= MP_MAX_THREAD_COLORS) throw plan_error{MP_ECOLORS};
            col[it - s0] = c;
            for (auto &sp : pts) {
                mask[sp.first][sp.second] |= 1ull << c;
                all.push_back(sp);
            }
            if (c + 1 > nc) nc = c + 1;
        }
        for (auto &sp : all) mask[sp.first][sp.second] = 0;
        P.block_ncolors[b] = nc;
        std::vector<int32_t> ord(s1 - s0);
        for (int32_t i = 0; i < s1 - s0; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return col[x] < col[y]; });
        for (int32_t i = 0; i < s1 - s0; ++i) {
            n2o[s0 + i] = s0 + ord[i];
            tc[s0 + i] = (uint8_t)col[ord[i]];
        }
    }
    P.thread_color.swap(tc);
    return n2o;
}

// ------------------------------------------------------ 5. data reordering

// Points ordered by (number of distinct accessing blocks, the sorted list
// of accessing blocks, id); points no block accesses go last (Sec. 2.3.2).
std::vector<int32_t> data_point_order(const mp_plan &P, int slot)
{
    int64_t np = P.toset_size[slot];
    std::vector<int32_t> last(np, -1), cnt(np, 0);
    for (int32_t b = 0; b < P.nblocks; ++b)
        for (int32_t it = P.block_offsets[b]; it < P.block_offsets[b + 1]; ++it)
            for (int m = 0; m < P.nmaps; ++m) {
                const mp_map_info &mi = P.maps[m];
                if (mi.slot != slot) continue;
                for (int k = 0; k < mi.arity; ++k) {
                    int32_t p = mi.idx[(int64_t)it * mi.arity + k];
                    if (last[p] != b) {
                        last[p] = b;
                        cnt[p]++;
                    }
                }
            }
    std::vector<int64_t> off(np + 1, 0);
    for (int64_t p = 0; p < np; ++p) off[p + 1] = off[p] + cnt[p];
    std::vector<int32_t> lst(off[np]);
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    std::fill(last.begin(), last.end(), -1);
    for (int32_t b = 0; b < P.nblocks; ++b)   // blocks visited in order: lists come out sorted
        for (int32_t it = P.block_offsets[b]; it < P.block_offsets[b + 1]; ++it)
            for (int m = 0; m < P.nmaps; ++m) {
                const mp_map_info &mi = P.maps[m];
                if (mi.slot != slot) continue;
                for (int k = 0; k < mi.arity; ++k) {
                    int32_t p = mi.idx[(int64_t)it * mi.arity + k];
                    if (last[p] != b) {
                        last[p] = b;
                        lst[pos[p]++] = b;
                    }
                }
            }
    // Points of one or two blocks (most of them) are ordered by a packed key
    // (count, first block, second block) with a stable radix sort from
    // ascending ids; points of three or more blocks follow, compared list by
    // list; points of no block go last, by id.
    std::vector<uint64_t> key;
    std::vector<int32_t> order, many, none;
    key.reserve(np);
    order.reserve(np);
    for (int64_t p = 0; p < np; ++p) {
        if (cnt[p] == 1 || cnt[p] == 2) {
            const uint64_t b0 = (uint64_t)lst[off[p]], b1 = cnt[p] == 2 ? (uint64_t)lst[off[p] + 1] : 0;
            key.push_back(((uint64_t)cnt[p] << 62) | (b0 << 31) | b1);
            order.push_back((int32_t)p);
        } else if (cnt[p] > 2) {
            many.push_back((int32_t)p);
        } else {
            none.push_back((int32_t)p);
        }
    }
    radix_sort(key, order);
    std::sort(many.begin(), many.end(), [&](int32_t x, int32_t y) {
        if (cnt[x] != cnt[y]) return cnt[x] < cnt[y];
        for (int32_t k = 0; k < cnt[x]; ++k)
            if (lst[off[x] + k] != lst[off[y] + k]) return lst[off[x] + k] < lst[off[y] + k];
        return x < y;
    });
    order.insert(order.end(), many.begin(), many.end());
    order.insert(order.end(), none.begin(), none.end());
    return order;
}

// ------------------------------------------------------------ 6. footprints

void build_footprints(mp_plan &P)
{
    int slots = 0;
    for (int m = 0; m < P.nmaps; ++m) slots += P.maps[m].arity;
    P.lmap_stride = slots <= 4 ? 4 : (slots <= 8 ? 8 : 16);
    P.lmap.assign((size_t)P.from_size * P.lmap_stride, 0);
    std::vector<int32_t> stamp[MP_MAX_TOSETS], local[MP_MAX_TOSETS];
    for (int s = 0; s < P.ntosets; ++s) {
        stamp[s].assign(P.toset_size[s], -1);
        local[s].assign(P.toset_size[s], 0);
        P.fp_offsets[s].assign(P.nblocks + 1, 0);
        P.fp_ids[s].clear();
    }
    P.desc.assign(P.nblocks, mp_block_desc{});
    std::vector<int32_t> pts;
    for (int32_t b = 0; b < P.nblocks; ++b) {
        int32_t s0 = P.block_offsets[b], s1 = P.block_offsets[b + 1];
        mp_block_desc &d = P.desc[b];
        d.item_start = s0;
        d.nitems = s1 - s0;
        d.ncolors = P.block_ncolors.empty() ? 1 : P.block_ncolors[b];
        for (int s = 0; s < P.ntosets; ++s) {
            pts.clear();
            for (int32_t it = s0; it < s1; ++it)
                for (int m = 0; m < P.nmaps; ++m) {
                    const mp_map_info &mi = P.maps[m];
                    if (mi.slot != s) continue;
                    for (int k = 0; k < mi.arity; ++k) {
                        int32_t p = mi.idx[(int64_t)it * mi.arity + k];
                        if (stamp[s][p] != b) {
                            stamp[s][p] = b;
                            pts.push_back(p);
                        }
                    }
                }
            std::sort(pts.begin(), pts.end());
            if (pts.size() > 65535) throw plan_error{MP_ESMEM};
            for (size_t i = 0; i < pts.size(); ++i) local[s][pts[i]] = (int32_t)i;
            d.fp_start[s] = (int32_t)P.fp_ids[s].size();
            d.fp_count[s] = (int32_t)pts.size();
            P.fp_ids[s].insert(P.fp_ids[s].end(), pts.begin(), pts.end());
            P.fp_offsets[s][b + 1] = (int32_t)P.fp_ids[s].size();
        }
        for (int32_t it = s0; it < s1; ++it) {
            int slot = 0;
            for (int m = 0; m < P.nmaps; ++m) {
                const mp_map_info &mi = P.maps[m];
                for (int k = 0; k < mi.arity; ++k)
                    P.lmap[(size_t)it * P.lmap_stride + slot++] =
                        (uint16_t)local[mi.slot][mi.idx[(int64_t)it * mi.arity + k]];
            }
        }
    }
    // the device holds the footprint lists of all to-sets back to back:
    // descriptors index that concatenation
    int64_t base = 0;
    for (int s = 0; s < P.ntosets; ++s) {
        if (base + (int64_t)P.fp_ids[s].size() > INT32_MAX) throw plan_error{MP_ENOMEM};
        for (auto &d : P.desc) d.fp_start[s] += (int32_t)base;
        base += (int64_t)P.fp_ids[s].size();
    }
    // block-local inverse of the written maps, for the gather form of the
    // increments: per footprint point the (local iteration, map slot) pairs
    // that increment it, ascending, in a row of gat_w entries padded with
    // 0xFFFF (gat_w = 0: some point has more than 16 and the form is off)
    int slot_of_map[MP_MAX_MAPS];
    for (int m = 0, sl = 0; m < P.nmaps; ++m) {
        slot_of_map[m] = sl;
        sl += P.maps[m].arity;
    }
    auto for_each_written = [&](auto fn) {
        for (int32_t b = 0; b < P.nblocks; ++b) {
            const mp_block_desc &d = P.desc[b];
            for (int32_t t = 0; t < d.nitems; ++t) {
                const int64_t it = d.item_start + t;
                for (int m = 0; m < P.nmaps; ++m) {
                    const mp_map_info &mi = P.maps[m];
                    if (!mi.written) continue;
                    for (int k = 0; k < mi.arity; ++k) {
                        const int slot = slot_of_map[m] + k;
                        const int64_t fpi = d.fp_start[mi.slot] + P.lmap[(size_t)it * P.lmap_stride + slot];
                        fn(fpi, (uint16_t)(t * 16 + slot));
                    }
                }
            }
        }
    };
    std::vector<uint8_t> cnt(base, 0);
    int maxc = 0;
    for_each_written([&](int64_t fpi, uint16_t) {
        if (cnt[fpi] < 255) cnt[fpi]++;
        maxc = std::max(maxc, (int)cnt[fpi]);
    });
    P.gat_w = maxc <= 4 ? 4 : (maxc <= 8 ? 8 : (maxc <= 16 ? 16 : 0));
    P.gat_tab.clear();
    if (P.gat_w > 0 && P.opts.block_size <= 4096) {
        P.gat_tab.assign((size_t)base * P.gat_w, 0xFFFF);
        std::fill(cnt.begin(), cnt.end(), 0);
        for_each_written([&](int64_t fpi, uint16_t e) { P.gat_tab[(size_t)fpi * P.gat_w + cnt[fpi]++] = e; });
    } else {
        P.gat_w = 0;
    }
}

void compute_stats(mp_plan &P)
{
    mp_plan_stats &S = P.stats;
    S.from_size = P.from_size;
    S.nblocks = P.nblocks;
    S.nblock_colors = P.ncolors;
    S.block_size = P.opts.block_size;
    S.sprime = (int32_t)(P.opts.block_size / P.opts.imbalance);
    S.lprime = (P.opts.block_size + P.opts.eps) / (double)S.sprime;
    S.ntosets = P.ntosets;
    int maxtc = 0;
    double sumtc = 0;
    for (int32_t c : P.block_ncolors) {
        maxtc = std::max(maxtc, c);
        sumtc += c;
    }
    S.max_thread_colors = maxtc;
    S.mean_thread_colors = P.block_ncolors.empty() ? 0.0 : sumtc / P.block_ncolors.size();
    int64_t acc_all = 0, uniq_all = 0;
    for (int s = 0; s < MP_MAX_TOSETS; ++s) {
        S.reuse[s] = 0;
        S.footprint_total[s] = 0;
        S.footprint_max[s] = 0;
        S.to_set_id[s] = s < P.ntosets ? P.toset_id[s] : 0;
        S.to_set_size[s] = s < P.ntosets ? P.toset_size[s] : 0;
    }
    // reuse: accesses per distinct staged point within a block (Sec. 3.1),
    // evaluated on the plan's blocks (chunks of S for GLOBAL/ATOMIC plans)
    std::vector<int32_t> stamp;
    for (int s = 0; s < P.ntosets; ++s) {
        int64_t acc = 0, uniq = 0;
        int32_t fmax = 0;
        stamp.assign(P.toset_size[s], -1);
        for (int32_t b = 0; b < P.nblocks; ++b) {
            int32_t u = 0;
            for (int32_t it = P.block_offsets[b]; it < P.block_offsets[b + 1]; ++it)
                for (int m = 0; m < P.nmaps; ++m) {
                    const mp_map_info &mi = P.maps[m];
                    if (mi.slot != s) continue;
                    for (int k = 0; k < mi.arity; ++k) {
                        int32_t p = mi.idx[(int64_t)it * mi.arity + k];
                        ++acc;
                        if (stamp[p] != b) {
                            stamp[p] = b;
                            ++u;
                        }
                    }
                }
            uniq += u;
            fmax = std::max(fmax, u);
        }
        S.reuse[s] = uniq ? (double)acc / (double)uniq : 0.0;
        S.footprint_total[s] = uniq;
        S.footprint_max[s] = fmax;
        acc_all += acc;
        uniq_all += uniq;
    }
    S.reuse_all = uniq_all ? (double)acc_all / (double)uniq_all : 0.0;
    int64_t bytes = 0;
    if (P.opts.coloring == MP_COLOR_HIER) {
        bytes += (int64_t)P.desc.size() * sizeof(mp_block_desc);
        bytes += (int64_t)P.lmap.size() * 2 + P.from_size;
        bytes += (int64_t)P.gat_tab.size() * 2;
        for (int s = 0; s < P.ntosets; ++s) bytes += (int64_t)P.fp_ids[s].size() * 4;
    } else {
        for (int m = 0; m < P.nmaps; ++m) bytes += (int64_t)P.maps[m].idx.size() * 4;
        bytes += (int64_t)(P.inv_off.size() + P.inv_idx.size()) * 4;
    }
    S.plan_bytes = bytes;
}

int build(const mp_map *maps, int32_t nmaps, int64_t from_size, const mp_plan_opts *opts, mp_plan *P)
{
    double t0 = now_s();
    if (!maps || nmaps < 1 || nmaps > MP_MAX_MAPS || from_size < 0 || from_size > INT32_MAX) return MP_EINVAL;
    mp_plan_opts o;
    mp_plan_opts_default(&o);
    if (opts) o = *opts;
    if (o.block_size < 32 || o.block_size > 1024 || o.block_size % 32) return MP_EINVAL;
    if (o.reorder < 0 || o.reorder > 2 || o.coloring < 0 || o.coloring > 3 || o.layout < 0 || o.layout > 1)
        return MP_EINVAL;
    if (!(o.imbalance >= 1.0) || o.imbalance > 2.0) return MP_EINVAL;
    if (o.staged < -1 || o.staged > 7 || o.recolor < -1 || o.recolor > 1) return MP_EINVAL;
    if (o.data_reorder < 0) o.data_reorder = (o.reorder == MP_REORDER_PARTITION || o.block_of) ? 1 : 0;
    P->opts = o;
    P->opts.block_of = nullptr;  // read during the build only
    P->from_size = from_size;
    P->nmaps = nmaps;
    // 1. validation and to-set slots
    for (int m = 0; m < nmaps; ++m) {
        const mp_map &mm = maps[m];
        if (mm.arity < 1 || mm.arity > 8 || mm.to_size <= 0 || mm.to_size > INT32_MAX || mm.to_set < 1)
            return MP_EINVAL;
        if (from_size > 0 && !mm.idx) return MP_EINVAL;
        int slot = -1;
        for (int s = 0; s < P->ntosets; ++s)
            if (P->toset_id[s] == mm.to_set) slot = s;
        if (slot < 0) {
            if (P->ntosets == MP_MAX_TOSETS) return MP_EINVAL;
            slot = P->ntosets++;
            P->toset_id[slot] = mm.to_set;
            P->toset_size[slot] = mm.to_size;
        } else if (P->toset_size[slot] != mm.to_size) {
            return MP_EINVAL;
        }
        mp_map_info &mi = P->maps[m];
        mi.to_set = mm.to_set;
        mi.arity = mm.arity;
        mi.written = mm.written ? 1 : 0;
        mi.slot = slot;
        mi.to_size = mm.to_size;
        mi.idx.assign(mm.idx, mm.idx + from_size * mm.arity);
        for (int32_t p : mi.idx)
            if (p < 0 || p >= mm.to_size) return MP_EMAPRANGE;
    }
    int primary = o.primary_map;
    if (primary < 0) {
        primary = 0;
        for (int m = nmaps - 1; m >= 0; --m)
            if (P->maps[m].written) primary = m;
    }
    if (primary >= nmaps) return MP_EINVAL;
    P->perm_from.resize(from_size);
    for (int64_t i = 0; i < from_size; ++i) P->perm_from[i] = (int32_t)i;
    for (int s = 0; s < P->ntosets; ++s) {
        P->perm_to[s].resize(P->toset_size[s]);
        for (int64_t i = 0; i < P->toset_size[s]; ++i) P->perm_to[s][i] = (int32_t)i;
    }
    // 2. reordering
    double t1 = now_s();
    if (o.reorder != MP_REORDER_NONE && from_size > 0 && !o.block_of) reorder_rcm(*P, primary);
    double t2 = now_s();
    // 3. blocks
    int S = o.block_size;
    int sprime = (int)(S / o.imbalance);
    if (sprime < 1) sprime = 1;
    std::vector<int32_t> blk;
    if (o.block_of && from_size > 0) {
        // caller-defined blocks: iterations grouped by ascending block value
        std::vector<int32_t> n2o(from_size);
        for (int64_t i = 0; i < from_size; ++i) n2o[i] = (int32_t)i;
        std::stable_sort(n2o.begin(), n2o.end(), [&](int32_t a, int32_t b) { return o.block_of[a] < o.block_of[b]; });
        P->block_offsets.assign(1, 0);
        for (int64_t i = 0; i < from_size; ++i)
            if (i > 0 && o.block_of[n2o[i]] != o.block_of[n2o[i - 1]]) P->block_offsets.push_back((int32_t)i);
        P->block_offsets.push_back((int32_t)from_size);
        P->nblocks = (int32_t)P->block_offsets.size() - 1;
        for (int32_t b = 0; b < P->nblocks; ++b)
            if (P->block_offsets[b + 1] - P->block_offsets[b] > S) return MP_EINVAL;
        permute_items(*P, n2o);
    } else if (o.reorder == MP_REORDER_PARTITION && from_size > 0) {
        blk = partition_greedy(*P, sprime, P->nblocks);
        // iterations grouped by block, ascending within a block
        std::vector<int32_t> cnt(P->nblocks + 1, 0);
        for (int32_t b : blk) cnt[b + 1]++;
        for (int32_t b = 0; b < P->nblocks; ++b) cnt[b + 1] += cnt[b];
        P->block_offsets = cnt;
        std::vector<int32_t> n2o(from_size);
        std::vector<int32_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t i = 0; i < from_size; ++i) n2o[pos[blk[i]]++] = (int32_t)i;
        permute_items(*P, n2o);
    } else {
        P->nblocks = (int32_t)((from_size + S - 1) / S);
        P->block_offsets.resize(P->nblocks + 1);
        for (int32_t b = 0; b <= P->nblocks; ++b) P->block_offsets[b] = (int32_t)std::min<int64_t>((int64_t)b * S, from_size);
    }
    double t3 = now_s();
    // 4. colouring
    if (o.coloring == MP_COLOR_HIER) {
        const std::vector<int32_t> &bo = P->block_offsets;
        P->block_color = first_fit(*P, P->nblocks,
                                   [&](int64_t b, std::vector<std::pair<int, int32_t>> &out) {
                                       for (int32_t it = bo[b]; it < bo[b + 1]; ++it) written_points(*P, it, out);
                                   },
                                   MP_MAX_BLOCK_COLORS, P->ncolors);
        std::vector<std::vector<int32_t>> pieces;
        std::vector<int32_t> piece_color;
        std::vector<char> dissolved(P->nblocks, 0);
        if (o.recolor != 0) {
            reduce_sparse_colors(*P, P->block_color, P->ncolors);
            split_last_color(*P, P->block_color, P->ncolors, pieces, piece_color, dissolved);
        }
        // blocks stably sorted by colour (pieces of dissolved blocks after
        // the whole blocks of their colour)
        const int32_t nwhole = P->nblocks, nall = nwhole + (int32_t)pieces.size();
        auto color_of = [&](int32_t x) { return x < nwhole ? P->block_color[x] : piece_color[x - nwhole]; };
        std::vector<int32_t> border;
        for (int32_t b = 0; b < nall; ++b)
            if (b >= nwhole || !dissolved[b]) border.push_back(b);
        std::stable_sort(border.begin(), border.end(), [&](int32_t x, int32_t y) { return color_of(x) < color_of(y); });
        std::vector<int32_t> n2o;
        n2o.reserve(from_size);
        std::vector<int32_t> nbo(1, 0), nbc;
        for (int32_t b : border) {
            if (b < nwhole)
                for (int32_t it = bo[b]; it < bo[b + 1]; ++it) n2o.push_back(it);
            else
                n2o.insert(n2o.end(), pieces[b - nwhole].begin(), pieces[b - nwhole].end());
            nbo.push_back((int32_t)n2o.size());
            nbc.push_back(color_of(b));
        }
        if ((int64_t)n2o.size() != from_size) throw plan_error{MP_EINVAL};
        P->nblocks = (int32_t)border.size();
        permute_items(*P, n2o);
        P->block_offsets = nbo;
        P->block_color = nbc;
        P->color_offsets.assign(P->ncolors + 1, 0);
        for (int32_t c : P->block_color) P->color_offsets[c + 1]++;
        for (int c = 0; c < P->ncolors; ++c) P->color_offsets[c + 1] += P->color_offsets[c];
        std::vector<int32_t> tperm = color_threads(*P);
        permute_items(*P, tperm);
    } else if (o.coloring == MP_COLOR_GLOBAL) {
        std::vector<int32_t> col = first_fit(*P, from_size,
                                             [&](int64_t it, std::vector<std::pair<int, int32_t>> &out) {
                                                 written_points(*P, it, out);
                                             },
                                             MP_MAX_BLOCK_COLORS, P->ncolors);
        std::vector<int32_t> n2o(from_size);
        for (int64_t i = 0; i < from_size; ++i) n2o[i] = (int32_t)i;
        std::stable_sort(n2o.begin(), n2o.end(), [&](int32_t x, int32_t y) { return col[x] < col[y]; });
        permute_items(*P, n2o);
        P->color_offsets.assign(P->ncolors + 1, 0);
        for (int32_t c : col) P->color_offsets[c + 1]++;
        for (int c = 0; c < P->ncolors; ++c) P->color_offsets[c + 1] += P->color_offsets[c];
        P->thread_color.assign(from_size, 0);
        for (int64_t i = 0; i < from_size; ++i) P->thread_color[i] = (uint8_t)col[n2o[i]];
        // launch chunks of S within each colour
        P->block_offsets.assign(1, 0);
        P->block_color.clear();
        for (int c = 0; c < P->ncolors; ++c)
            for (int32_t s = P->color_offsets[c]; s < P->color_offsets[c + 1]; s += S) {
                P->block_offsets.push_back(std::min(s + S, P->color_offsets[c + 1]));
                P->block_color.push_back(c);
            }
        P->nblocks = (int32_t)P->block_color.size();
    } else {
        P->ncolors = from_size > 0 ? 1 : 0;
        P->color_offsets = {0, (int32_t)from_size};
        P->block_color.assign(P->nblocks, 0);
        P->thread_color.assign(from_size, 0);
    }
    double t4 = now_s();
    // 5. data-point reordering
    if (o.data_reorder && from_size > 0)
        for (int s = 0; s < P->ntosets; ++s) permute_points(*P, s, data_point_order(*P, s));
    // 6. footprints and local maps (HIER), inverse map (TWOSTEP), both in
    // the final point numbering
    if (o.coloring == MP_COLOR_HIER) build_footprints(*P);
    if (o.coloring == MP_COLOR_TWOSTEP) {
        // inverse of the (single) written map: point -> sorted (item, slot)
        int w = -1, nw = 0;
        for (int m = 0; m < nmaps; ++m)
            if (P->maps[m].written) {
                w = m;
                ++nw;
            }
        if (nw != 1) return MP_EINVAL;
        const mp_map_info &mi = P->maps[w];
        P->inv_map = w;
        P->inv_off.assign(mi.to_size + 1, 0);
        for (int32_t p : mi.idx) P->inv_off[p + 1]++;
        for (int64_t i = 0; i < mi.to_size; ++i) P->inv_off[i + 1] += P->inv_off[i];
        P->inv_idx.resize(mi.idx.size());
        std::vector<int32_t> pos(P->inv_off.begin(), P->inv_off.end() - 1);
        for (int64_t e = 0; e < from_size; ++e)  // items ascending, slots ascending
            for (int k = 0; k < mi.arity; ++k)
                P->inv_idx[pos[mi.idx[e * mi.arity + k]]++] = (int32_t)(e * mi.arity + k);
    }
    compute_stats(*P);
    double t5 = now_s();
    P->stats.seconds_reorder = t2 - t1;
    P->stats.seconds_partition = t3 - t2;
    P->stats.seconds_color = t4 - t3;
    P->stats.seconds_total = t5 - t0;
    return MP_OK;
}

}  // namespace

extern "C" {

void mp_plan_opts_default(mp_plan_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->block_size = 512;
    o->reorder = MP_REORDER_PARTITION;
    o->coloring = MP_COLOR_HIER;
    o->layout = MP_LAYOUT_AOS;
    o->imbalance = 1.001;
    o->eps = 0.0;
    o->primary_map = -1;
    o->data_reorder = -1;
    o->staged = -1;
    o->recolor = -1;
    o->block_of = nullptr;
}

int mesh_plan_build(const mp_map *maps, int32_t nmaps, int64_t from_size, const mp_plan_opts *opts, mp_plan **out)
{
    if (!out) return MP_EINVAL;
    *out = nullptr;
    mp_plan *P = new (std::nothrow) mp_plan();
    if (!P) return MP_ENOMEM;
    int rc;
    try {
        rc = build(maps, nmaps, from_size, opts, P);
    } catch (const plan_error &e) {
        rc = e.code;
    } catch (const std::bad_alloc &) {
        rc = MP_ENOMEM;
    }
    if (rc != MP_OK) {
        delete P;
        return rc;
    }
    *out = P;
    return MP_OK;
}

void mesh_plan_destroy(mp_plan *P)
{
    if (!P) return;
    mp_plan_free_device(P);
    delete P;
}

int mesh_plan_set_staged(mp_plan *P, int32_t staged)
{
    if (!P || staged < -1 || staged > 7) return MP_EINVAL;
    P->opts.staged = staged;
    return MP_OK;
}

int mesh_plan_query(const mp_plan *P, mp_plan_stats *s)
{
    if (!P || !s) return MP_EINVAL;
    *s = P->stats;
    return MP_OK;
}

int mesh_plan_perm(const mp_plan *P, int32_t set_id, int32_t *n2o)
{
    if (!P || !n2o) return MP_EINVAL;
    if (set_id == 0) {
        std::copy(P->perm_from.begin(), P->perm_from.end(), n2o);
        return MP_OK;
    }
    for (int s = 0; s < P->ntosets; ++s)
        if (P->toset_id[s] == set_id) {
            std::copy(P->perm_to[s].begin(), P->perm_to[s].end(), n2o);
            return MP_OK;
        }
    return MP_EINVAL;
}

int mesh_plan_table(const mp_plan *P, int32_t table, int32_t arg, int32_t *out, int64_t cap, int64_t *count)
{
    if (!P || !count) return MP_EINVAL;
    std::vector<int32_t> tmp;
    const std::vector<int32_t> *src = nullptr;
    switch (table) {
    case MP_TAB_BLOCK_OFFSETS: src = &P->block_offsets; break;
    case MP_TAB_COLOR_OFFSETS: src = &P->color_offsets; break;
    case MP_TAB_BLOCK_COLOR: src = &P->block_color; break;
    case MP_TAB_THREAD_COLOR:
        tmp.assign(P->thread_color.begin(), P->thread_color.end());
        src = &tmp;
        break;
    case MP_TAB_MAP:
        if (arg < 0 || arg >= P->nmaps) return MP_EINVAL;
        src = &P->maps[arg].idx;
        break;
    case MP_TAB_FOOTPRINT:
        for (int s = 0; s < P->ntosets; ++s) tmp.insert(tmp.end(), P->fp_ids[s].begin(), P->fp_ids[s].end());
        src = &tmp;
        break;
    case MP_TAB_FP_START:
    case MP_TAB_FP_COUNT:
        for (const auto &d : P->desc)
            for (int s = 0; s < MP_MAX_TOSETS; ++s)
                tmp.push_back(table == MP_TAB_FP_START ? d.fp_start[s] : d.fp_count[s]);
        src = &tmp;
        break;
    case MP_TAB_LOCAL_MAP:
        tmp.assign(P->lmap.begin(), P->lmap.end());
        src = &tmp;
        break;
    case MP_TAB_GATHER:
        tmp.assign(P->gat_tab.begin(), P->gat_tab.end());
        for (auto &v : tmp)
            if (v == 0xFFFF) v = -1;
        src = &tmp;
        break;
    case MP_TAB_INV_OFFSETS: src = &P->inv_off; break;
    case MP_TAB_INV_INDEX: src = &P->inv_idx; break;
    default: return MP_EINVAL;
    }
    *count = (int64_t)src->size();
    if (!out) return MP_OK;
    if (cap < (int64_t)src->size()) return MP_EINVAL;
    std::copy(src->begin(), src->end(), out);
    return MP_OK;
}

int mesh_map_renumber(const int32_t *idx, int64_t from_size, int32_t arity, const int32_t *from_perm,
                      const int32_t *to_perm, int64_t to_size, int32_t *out)
{
    if ((!idx && from_size > 0) || (!out && from_size > 0) || arity < 1 || from_size < 0 || to_size <= 0)
        return MP_EINVAL;
    std::vector<int32_t> o2n;
    if (to_perm) {
        o2n.assign(to_size, -1);
        for (int64_t i = 0; i < to_size; ++i) {
            if (to_perm[i] < 0 || to_perm[i] >= to_size || o2n[to_perm[i]] >= 0) return MP_EINVAL;
            o2n[to_perm[i]] = (int32_t)i;
        }
    }
    for (int64_t i = 0; i < from_size; ++i) {
        int64_t src = from_perm ? from_perm[i] : i;
        if (src < 0 || src >= from_size) return MP_EINVAL;
        for (int k = 0; k < arity; ++k) {
            int32_t p = idx[src * arity + k];
            if (p < 0 || p >= to_size) return MP_EMAPRANGE;
            out[i * arity + k] = to_perm ? o2n[p] : p;
        }
    }
    return MP_OK;
}

const char *mp_error_string(int code)
{
    switch (code) {
    case MP_OK: return "ok";
    case MP_EINVAL: return "invalid argument (null or misaligned pointer, bad arity, size or option)";
    case MP_EMAPRANGE: return "map index out of range of its to-set";
    case MP_ECOLORS: return "too many colours (block colours > 256 or thread colours > 64)";
    case MP_ESMEM: return "block footprint exceeds shared memory";
    case MP_ECUDA: return "CUDA runtime error";
    case MP_ETIMEOUT: return "device-side wait timed out";
    case MP_ENOMEM: return "host allocation failed";
    case MP_EPLAN: return "plan does not fit this loop";
    case MP_EIO: return "plan file could not be read or written";
    case MP_ETOOBIG: return "size exceeds the fixed static scratch of an allocation-free entry point";
    default: return "unknown error";
    }
}

const char *mp_version(void) { return "meshloop 0.1 (sm_103a)"; }

}  // extern "C"
