// Adjoint of res_calc with FP64 data and double-word (FP32 pair)
// arithmetic, the FP64-accurate variant for GB300 (see loops_res_dw.cu).
// Same staged two-layer structure and formulas as adjoint_hier
// (loops_adj.cu): per edge, with f_bar = res_bar[c1] - res_bar[c2] and
// h = f_bar / 2, each side's reverse sweep of F(q).n is
//   V = u . n,  Vb = h0 rho + h1 rho u + h2 rho v + h3 H,
//   pb = h1 n_x + h2 n_y + h3 V,  Wb = Vb / rho,  gpb = (gam-1) pb,
//   q_b = (h0 V - Wb V + gpb |u|^2/2,  h1 V + Wb n_x - gpb u,
//          h2 V + Wb n_y - gpb v,  h3 V + gpb),
//   n_b += (h1 p + Wb rho u,  h2 p + Wb rho v),
// plus mu f_bar on q1 and -mu f_bar on q2; each component is one
// compensated sum of products.  The edge normal is formed in FP64.
#include <algorithm>

#include "common.cuh"
#include "dw.cuh"

namespace {

__device__ __forceinline__ dw ldw(const float2 *a, int i)
{
    float2 v = a[i];
    return {v.x, v.y};
}
__device__ __forceinline__ void stw(float2 *a, int i, dw v) { a[i] = make_float2(v.hi, v.lo); }

// Dynamic shared memory for cap_c cells and cap_n nodes:
//   double x, y, xbar[2]                  (32 B per node)
//   double qbar[4]                        (32 B per cell)
//   dw rho, ru, rv, H, ri, u, v, p, K, a' (10 x 8 B per cell; K = |u|^2/2,
//                                          a' = eps adt / 2)
//   dw rb[4], qinc[4]                     (64 B per cell)
//   dw xinc[2]                            (16 B per node)
//   (gather form: no qinc / xinc; a [10][cap_f] buffer of per-edge
//    increments over the cell arrays and rb, then the gather rows)
//   int gid per cell and node
constexpr int kAdjDwCellBytes = 32 + 80 + 64 + 4;
constexpr int kAdjDwNodeBytes = 32 + 16 + 4;

// Per-cell values of the reverse sweep from q = (rho, ru, rv, E): H = E + p,
// 1/rho, u, v, p and K = |u|^2 / 2.
__device__ __forceinline__ void dw_adj_prims(const dw qq[4], dw gm1, dw &H, dw &ri, dw &u, dw &v, dw &p, dw &K)
{
    ri = dw_recip(qq[0]);
    u = dw_mul(qq[1], ri);
    v = dw_mul(qq[2], ri);
    dw_acc A = dw_dot_begin(u, u);
    dw_dot_add(A, v, v);
    K = dw_scale2(dw_dot_end(A), 0.5f);
    p = dw_mul(gm1, dw_sub(qq[3], dw_mul(qq[0], K)));
    H = dw_add(qq[3], p);
}

// One side's reverse sweep; accumulates n_b.
__device__ __forceinline__ void flux_rev_dw(dw r, dw ru, dw rv, dw H, dw ri, dw u, dw v, dw p, dw K, dw nx, dw ny,
                                            const dw h[4], dw gm1, dw qb[4], dw_acc &nbx, dw_acc &nby, bool first)
{
    dw_acc A = dw_dot_begin(u, nx);
    dw_dot_add(A, v, ny);
    const dw V = dw_dot_end(A);
    A = dw_dot_begin(h[0], r);
    dw_dot_add(A, h[1], ru);
    dw_dot_add(A, h[2], rv);
    dw_dot_add(A, h[3], H);
    const dw Wb = dw_mul(dw_dot_end(A), ri);
    A = dw_dot_begin(h[1], nx);
    dw_dot_add(A, h[2], ny);
    dw_dot_add(A, h[3], V);
    const dw gpb = dw_mul(gm1, dw_dot_end(A));
    A = dw_dot_begin(h[0], V);
    dw_dot_add(A, dw_neg(Wb), V);
    dw_dot_add(A, gpb, K);
    qb[0] = dw_dot_end(A);
    A = dw_dot_begin(h[1], V);
    dw_dot_add(A, Wb, nx);
    dw_dot_add(A, dw_neg(gpb), u);
    qb[1] = dw_dot_end(A);
    A = dw_dot_begin(h[2], V);
    dw_dot_add(A, Wb, ny);
    dw_dot_add(A, dw_neg(gpb), v);
    qb[2] = dw_dot_end(A);
    qb[3] = dw_add_fast(dw_mul(h[3], V), gpb);
    if (first) {
        nbx = dw_dot_begin(h[1], p);
        nby = dw_dot_begin(h[2], p);
    } else {
        dw_dot_add(nbx, h[1], p);
        dw_dot_add(nby, h[2], p);
    }
    dw_dot_add(nbx, Wb, ru);
    dw_dot_add(nby, Wb, rv);
}

// GATHER: the per-edge adjoint increments (q_bar of both cells, the normal
// adjoint) go to a shared buffer over the dead staged cell data, and each
// cell and node sums its edges' entries through the plan's gather rows.
template <bool SOA, bool GATHER>
__global__ void __launch_bounds__(512, 2) adjoint_hier_dw(const mp_block_desc *__restrict__ desc, int block0,
                                                          const ushort4 *__restrict__ lmap,
                                                          const uint8_t *__restrict__ tcolor,
                                                          const ushort4 *__restrict__ gat, int gw4, int cap_f,
                                                          const int32_t *__restrict__ fp, const double *__restrict__ x,
                                                          const double *__restrict__ q,
                                                          const double *__restrict__ adt,
                                                          const double *__restrict__ rbar, double *__restrict__ qbar,
                                                          double *__restrict__ xbar, int64_t nnode, int64_t ncell,
                                                          int cap_c, int cap_n, dw gm1, dw half_eps,
                                                          int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *s_x = reinterpret_cast<double *>(smem_raw);  // [2][cap_n]
    double *s_xb = s_x + 2 * cap_n;                       // [2][cap_n] x_bar (FP64, prefetched)
    double *s_qb = s_xb + 2 * cap_n;                      // [4][cap_c] q_bar (FP64, prefetched)
    float2 *s_cell = reinterpret_cast<float2 *>(s_qb + 4 * cap_c);  // [10][cap_c]
    float2 *s_rb = s_cell + 10 * cap_c;                   // [4][cap_c]
    float2 *s_qi = s_rb + 4 * cap_c;                      // coloured: [4][cap_c] q_bar increments
    float2 *s_xi = s_qi + 4 * cap_c;                      // coloured: [2][cap_n] x_bar increments
    // gather: [10][cap_f] per-edge increments over s_cell and s_rb, rows
    float2 *s_fb = s_cell;
    ushort4 *s_ge = reinterpret_cast<ushort4 *>(GATHER ? s_cell + max(14 * cap_c, 10 * cap_f) : s_xi + 2 * cap_n);
    int *s_gc = reinterpret_cast<int *>(s_ge + (GATHER ? gw4 * (cap_c + cap_n) : 0));
    int *s_gn = s_gc + cap_c;
    const float2 *S[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) S[k] = s_cell + k * cap_c;

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nn = d.fp_count[0], nc = d.fp_count[1];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gn + cap_n) - smem_raw) > dynamic_smem_bytes() ||
        nc > cap_c || nn > cap_n || d.nitems > (int)blockDim.x ||
        (GATHER && ((int)blockDim.x > cap_f || gw4 < 1 || gw4 > 4))) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpn = fp + d.fp_start[0];
    const int32_t *fpc = fp + d.fp_start[1];
    const bool active = tid < d.nitems;
    ushort4 l = make_ushort4(0, 0, 0, 0);
    int my_color = -1;
    if (active) {
        l = lmap[d.item_start + tid];
        if (!GATHER) my_color = tcolor[d.item_start + tid];
    }
    for (int i = tid; i < nc; i += blockDim.x) {
        const int64_t g = fpc[i];
        dw qq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t j = SOA ? k * ncell + g : 4 * g + k;
            qq[k] = dw_from_double_int(q[j]);
            stw(s_rb, k * cap_c + i, dw_from_double_int(rbar[j]));
            if (!GATHER) s_qi[k * cap_c + i] = make_float2(0.f, 0.f);
        }
        mp_pdl_wait();  // q_bar, x_bar: written by the previous colour's launch
#pragma unroll
        for (int k = 0; k < 4; ++k) s_qb[k * cap_c + i] = qbar[SOA ? k * ncell + g : 4 * g + k];
        dw H, ri, u, v, p, K;
        dw_adj_prims(qq, gm1, H, ri, u, v, p, K);
        float2 *W = s_cell;
        stw(W, 0 * cap_c + i, qq[0]);
        stw(W, 1 * cap_c + i, qq[1]);
        stw(W, 2 * cap_c + i, qq[2]);
        stw(W, 3 * cap_c + i, H);
        stw(W, 4 * cap_c + i, ri);
        stw(W, 5 * cap_c + i, u);
        stw(W, 6 * cap_c + i, v);
        stw(W, 7 * cap_c + i, p);
        stw(W, 8 * cap_c + i, K);
        stw(W, 9 * cap_c + i, dw_mul(dw_from_double_int(adt[g]), half_eps));
        if (GATHER) {
            const ushort4 *row = gat + (int64_t)(d.fp_start[1] + i) * gw4;
            for (int h = 0; h < gw4; ++h) s_ge[h * cap_c + i] = row[h];  // cell rows
        }
        s_gc[i] = (int)g;
    }
    // nodes: on the warps that stage no cell when there are enough of them
    // (at most two nodes per thread), so that the node loads do not follow the cell
    // arithmetic on the cell warps
    auto stage_node = [&](int i) {
        const int64_t g = fpn[i];
        s_x[i] = SOA ? x[g] : x[2 * g];
        s_x[cap_n + i] = SOA ? x[nnode + g] : x[2 * g + 1];
        mp_pdl_wait();
        s_xb[i] = SOA ? xbar[g] : xbar[2 * g];
        s_xb[cap_n + i] = SOA ? xbar[nnode + g] : xbar[2 * g + 1];
        if (GATHER) {
            const ushort4 *row = gat + (int64_t)(d.fp_start[0] + i) * gw4;
            for (int h = 0; h < gw4; ++h) s_ge[gw4 * cap_c + h * cap_n + i] = row[h];  // node rows
        } else {
            s_xi[i] = make_float2(0.f, 0.f);
            s_xi[cap_n + i] = make_float2(0.f, 0.f);
        }
        s_gn[i] = (int)g;
    };
    const int ncw = (nc + 31) & ~31, nfree = (int)blockDim.x - ncw;
    if (nfree >= 32 && 2 * nfree >= nn) {
        if (tid >= ncw) {
            const int i = tid - ncw;
            if (i < nn) stage_node(i);
            if (i + nfree < nn) stage_node(i + nfree);
        }
    } else {
        for (int i = tid; i < nn; i += blockDim.x) stage_node(i);
    }
    __syncthreads();
    int na = 0, nb = 0, c1 = 0, c2 = 0;
    dw qb1[4], qb2[4], nbx, nby;
    if (active) {
        na = l.x;
        nb = l.y;
        c1 = l.z;
        c2 = l.w;
        const dw nx = dw_from_double_int(s_x[cap_n + na] - s_x[cap_n + nb]);  // exact in FP64
        const dw ny = dw_from_double_int(s_x[nb] - s_x[na]);
        dw fb[4], h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            fb[k] = dw_add_fast(ldw(s_rb, k * cap_c + c1), dw_neg(ldw(s_rb, k * cap_c + c2)));
            h[k] = dw_scale2(fb[k], 0.5f);
        }
        dw_acc NX, NY;
        auto side = [&](int c, dw qb[4], bool first) {
            flux_rev_dw(ldw(S[0], c), ldw(S[1], c), ldw(S[2], c), ldw(S[3], c), ldw(S[4], c), ldw(S[5], c),
                        ldw(S[6], c), ldw(S[7], c), ldw(S[8], c), nx, ny, h, gm1, qb, NX, NY, first);
        };
        side(c1, qb1, true);
        side(c2, qb2, false);
        nbx = dw_dot_end(NX);
        nby = dw_dot_end(NY);
        const dw mu = dw_add_fast(ldw(S[9], c1), ldw(S[9], c2));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const dw m = dw_mul(mu, fb[k]);
            qb1[k] = dw_add_fast(qb1[k], m);
            qb2[k] = dw_add_fast(qb2[k], dw_neg(m));
        }
    }
    if constexpr (GATHER) {
        __syncthreads();  // every edge is computed: the staged cell data are dead
        if (active) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                stw(s_fb, k * cap_f + tid, qb1[k]);
                stw(s_fb, (4 + k) * cap_f + tid, qb2[k]);
            }
            stw(s_fb, 8 * cap_f + tid, nbx);
            stw(s_fb, 9 * cap_f + tid, nby);
        }
        __syncthreads();
        // cells: q_bar of the edges' first (map slot 2) or second (slot 3) cell
        // (compensated double-word sums, branch-free: a padding entry adds 0
        // times the values of thread 0, computed in every block)
        for (int i = tid; i < nc; i += blockDim.x) {
            dw_acc S[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            for (int h = 0; h < gw4; ++h) {
                const ushort4 e4 = s_ge[h * cap_c + i];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned en = es[j];
                    const bool valid = en != 0xFFFFu;
                    const int t = valid ? (int)(en >> 4) : 0, base = (en & 15u) == 3u ? 4 : 0;
                    const float sg = valid ? 1.0f : 0.0f;
#pragma unroll
                    for (int k = 0; k < 4; ++k) dw_sum_add(S[k], ldw(s_fb, (base + k) * cap_f + t), sg);
                }
            }
            const int64_t g = s_gc[i];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                qbar[SOA ? k * ncell + g : 4 * g + k] = f64_add_dw(s_qb[k * cap_c + i], dw_sum_end(S[k]));
        }
        // nodes: node a (slot 0) gets (-n_y_bar, n_x_bar), node b (slot 1) the opposite
        for (int i = tid; i < nn; i += blockDim.x) {
            dw_acc Sx = {0.f, 0.f}, Sy = {0.f, 0.f};
            for (int h = 0; h < gw4; ++h) {
                const ushort4 e4 = s_ge[gw4 * cap_c + h * cap_n + i];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned en = es[j];
                    const bool valid = en != 0xFFFFu;
                    const int t = valid ? (int)(en >> 4) : 0;
                    const float sg = !valid ? 0.0f : ((en & 15u) == 0u ? 1.0f : -1.0f);
                    const dw bx = ldw(s_fb, 8 * cap_f + t), by = ldw(s_fb, 9 * cap_f + t);
                    dw_sum_add(Sx, by, -sg);
                    dw_sum_add(Sy, bx, sg);
                }
            }
            const int64_t g = s_gn[i];
            xbar[SOA ? g : 2 * g] = f64_add_dw(s_xb[i], dw_sum_end(Sx));
            xbar[SOA ? nnode + g : 2 * g + 1] = f64_add_dw(s_xb[cap_n + i], dw_sum_end(Sy));
        }
    } else {
    for (int c = 0; c < d.ncolors; ++c) {
        if (my_color == c) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                stw(s_qi, k * cap_c + c1, dw_add_fast(ldw(s_qi, k * cap_c + c1), qb1[k]));
                stw(s_qi, k * cap_c + c2, dw_add_fast(ldw(s_qi, k * cap_c + c2), qb2[k]));
            }
            // n_x = y_a - y_b, n_y = x_b - x_a
            stw(s_xi, na, dw_add_fast(ldw(s_xi, na), dw_neg(nby)));
            stw(s_xi, nb, dw_add_fast(ldw(s_xi, nb), nby));
            stw(s_xi, cap_n + na, dw_add_fast(ldw(s_xi, cap_n + na), nbx));
            stw(s_xi, cap_n + nb, dw_add_fast(ldw(s_xi, cap_n + nb), dw_neg(nbx)));
        }
        __syncthreads();
    }
    for (int i = tid; i < nc; i += blockDim.x) {
        const int64_t g = s_gc[i];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            qbar[SOA ? k * ncell + g : 4 * g + k] = f64_add_dw(s_qb[k * cap_c + i], ldw(s_qi, k * cap_c + i));
    }
    for (int i = tid; i < nn; i += blockDim.x) {
        const int64_t g = s_gn[i];
        xbar[SOA ? g : 2 * g] = f64_add_dw(s_xb[i], ldw(s_xi, i));
        xbar[SOA ? nnode + g : 2 * g + 1] = f64_add_dw(s_xb[cap_n + i], ldw(s_xi, cap_n + i));
    }
    }
}

// Global colouring and atomics (Sec. 2.1) in the same arithmetic: one thread
// per edge of [e0, e1) reads its two nodes and two cells from global memory,
// forms the per-cell values and both sides' reverse sweeps as the staged
// kernel does, and writes q_bar (4 per cell) and x_bar (2 per node) either
// with two FP64 additions (GLOBAL: edges of one colour share no cell or
// node) or with one FP64 atomicAdd of the nearest double (ATOMIC).
template <bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256) adjoint_direct_dw(int e0, int e1, const int32_t *__restrict__ e2n,
                                                         const int32_t *__restrict__ e2c,
                                                         const double *__restrict__ x, const double *__restrict__ q,
                                                         const double *__restrict__ adt,
                                                         const double *__restrict__ rbar, double *__restrict__ qbar,
                                                         double *__restrict__ xbar, int64_t nnode, int64_t ncell,
                                                         dw gm1, dw half_eps)
{
    mp_pdl_trigger();
    const int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    const int2 nab = reinterpret_cast<const int2 *>(e2n)[e];
    const int2 cc = reinterpret_cast<const int2 *>(e2c)[e];
    auto X = [&](int64_t g, int k) { return SOA ? x[k * nnode + g] : x[2 * g + k]; };
    const dw nx = dw_from_double_int(X(nab.x, 1) - X(nab.y, 1));  // exact in FP64
    const dw ny = dw_from_double_int(X(nab.y, 0) - X(nab.x, 0));
    dw qq[2][4], fb[4], h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t j1 = SOA ? k * ncell + cc.x : 4 * (int64_t)cc.x + k;
        const int64_t j2 = SOA ? k * ncell + cc.y : 4 * (int64_t)cc.y + k;
        qq[0][k] = dw_from_double_int(q[j1]);
        qq[1][k] = dw_from_double_int(q[j2]);
        fb[k] = dw_add_fast(dw_from_double_int(rbar[j1]), dw_neg(dw_from_double_int(rbar[j2])));
        h[k] = dw_scale2(fb[k], 0.5f);
    }
    dw qb[2][4];
    dw_acc NX, NY;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        dw H, ri, u, v, p, K;
        dw_adj_prims(qq[sd], gm1, H, ri, u, v, p, K);
        flux_rev_dw(qq[sd][0], qq[sd][1], qq[sd][2], H, ri, u, v, p, K, nx, ny, h, gm1, qb[sd], NX, NY, sd == 0);
    }
    const dw nbx = dw_dot_end(NX), nby = dw_dot_end(NY);
    const dw mu = dw_add_fast(dw_mul(dw_from_double_int(adt[cc.x]), half_eps),
                              dw_mul(dw_from_double_int(adt[cc.y]), half_eps));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const dw m = dw_mul(mu, fb[k]);
        qb[0][k] = dw_add_fast(qb[0][k], m);
        qb[1][k] = dw_add_fast(qb[1][k], dw_neg(m));
    }
    // n_x = y_a - y_b, n_y = x_b - x_a: node a gets (-n_y_bar, n_x_bar), node b the opposite
    const dw xi[2][2] = {{dw_neg(nby), nbx}, {nby, dw_neg(nbx)}};
    const int node[2] = {nab.x, nab.y}, cell[2] = {cc.x, cc.y};
    if (!ATOMIC) mp_pdl_wait();  // q_bar, x_bar: read-add-written by the previous colour's launch
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double *t = qbar + (SOA ? k * ncell + cell[sd] : 4 * (int64_t)cell[sd] + k);
            if (ATOMIC)
                atomicAdd(t, f32_to_f64_int(qb[sd][k].hi) + f32_to_f64_int(qb[sd][k].lo));
            else
                *t = f64_add_dw(*t, qb[sd][k]);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            double *t = xbar + (SOA ? k * nnode + node[sd] : 2 * (int64_t)node[sd] + k);
            if (ATOMIC)
                atomicAdd(t, f32_to_f64_int(xi[sd][k].hi) + f32_to_f64_int(xi[sd][k].lo));
            else
                *t = f64_add_dw(*t, xi[sd][k]);
        }
    }
}

template <bool SOA>
int adjoint_dw_t(const mp_plan *P, const void *x, const void *q, const void *adt, const void *rbar, void *qbar,
                 void *xbar, double gam, double eps, cudaStream_t s)
{
    const int64_t nnode = P->maps[0].to_size, ncell = P->maps[1].to_size;
    const double g1 = gam - 1.0, he = 0.5 * eps;
    const float g1h = (float)g1, heh = (float)he;
    const dw gm1{g1h, (float)(g1 - (double)g1h)}, half_eps{heh, (float)(he - (double)heh)};
    if (P->opts.coloring == MP_COLOR_GLOBAL || P->opts.coloring == MP_COLOR_ATOMIC) {
        const bool atomic = P->opts.coloring == MP_COLOR_ATOMIC;
        auto kern = atomic ? adjoint_direct_dw<SOA, true> : adjoint_direct_dw<SOA, false>;
        bool overlap = false;  // global colours: overlapped like the staged launches
        for (int c = 0; c < P->ncolors; ++c) {
            const int e0 = P->color_offsets[c], e1 = P->color_offsets[c + 1];
            if (e1 <= e0) continue;
            MP_CUDA_TRY(mp_launch(kern, (e1 - e0 + 255) / 256, 256, 0, s, overlap && !atomic, e0, e1,
                                  P->dev.map[0], P->dev.map[1], (const double *)x, (const double *)q,
                                  (const double *)adt, (const double *)rbar, (double *)qbar, (double *)xbar, nnode,
                                  ncell, gm1, half_eps));
            overlap = true;
        }
        MP_CUDA_TRY(cudaGetLastError());
        return MP_OK;
    }
    if (P->opts.coloring != MP_COLOR_HIER || P->maps[0].slot != 0 || P->maps[1].slot != 1) return MP_EPLAN;
    if (P->opts.block_size > 512) return MP_EINVAL;
    const int cap_n = P->stats.footprint_max[0], cap_c = P->stats.footprint_max[1];
    const bool gather = mp_staged(P, MP_STAGED_GATHER) == MP_STAGED_GATHER && mp_gather_ready(P);
    const int gw4 = gather ? P->gat_w / 4 : 0, cap_f = gather ? P->opts.block_size : 0;
    // gather: no increment arrays (32 B per cell, 16 B per node); the edge
    // buffer (80 B per thread) reuses the staged cell data (112 B per cell)
    const int smem = gather ? cap_c * (kAdjDwCellBytes - 32) + cap_n * (kAdjDwNodeBytes - 16) +
                                  std::max(0, 80 * cap_f - 112 * cap_c) + 8 * gw4 * (cap_c + cap_n)
                            : cap_c * kAdjDwCellBytes + cap_n * kAdjDwNodeBytes;
    auto kern = gather ? adjoint_hier_dw<SOA, true> : adjoint_hier_dw<SOA, false>;
    int rc = mp_allow_smem(kern, smem);
    if (rc != MP_OK) return rc;
    int *err = nullptr;
    if ((rc = mp_device_error_word(&err)) != MP_OK) return rc;
    bool overlap = false;
    for (int c = 0; c < P->ncolors; ++c) {
        const int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
        if (nb == 0) continue;
        MP_CUDA_TRY(mp_launch(kern, nb, P->opts.block_size, smem, s, overlap, P->dev.desc, b0,
                              reinterpret_cast<const ushort4 *>(P->dev.lmap), P->dev.tcolor,
                              reinterpret_cast<const ushort4 *>(P->dev.gat), gw4, cap_f, P->dev.fp,
                              (const double *)x, (const double *)q, (const double *)adt, (const double *)rbar,
                              (double *)qbar, (double *)xbar, nnode, ncell, cap_c, cap_n, gm1, half_eps, err));
        overlap = true;
    }
    return MP_OK;
}

}  // namespace

int mp_adjoint_dw(const mp_plan *P, const void *x, const void *q, const void *adt, const void *rbar, void *qbar,
                  void *xbar, double gam, double eps, void *stream)
{
    return P->opts.layout == MP_LAYOUT_SOA
               ? adjoint_dw_t<true>(P, x, q, adt, rbar, qbar, xbar, gam, eps, as_stream(stream))
               : adjoint_dw_t<false>(P, x, q, adt, rbar, qbar, xbar, gam, eps, as_stream(stream));
}
