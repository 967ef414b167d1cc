// Adjoint of res_calc with x, q, adt held fixed (adt not differentiated):
//   q_bar += (d res / d q)^T res_bar,   x_bar += (d res / d x)^T res_bar.
// Every edge increments q_bar on its 2 cells and x_bar on its 2 nodes, so
// the plan is coloured on both maps.  HIER stages q, adt, res_bar and the
// per-cell primitives of the block's cells and x of its nodes in shared
// memory and writes each footprint cell and node back once, applying both
// increment sets either through the plan's gather rows (the default) or one
// thread colour at a time (Algorithm 1); GLOBAL / ATOMIC read global memory.
//
// Per edge, with n = (y_a - y_b, x_b - x_a), f_bar = res_bar[c1] - res_bar[c2]
// and h = f_bar / 2, the reverse sweep of F(q).n (V = W / rho,
// W = rho u . n, p = (gam-1)(E - K), K = |rho u|^2 / (2 rho)) for each side:
//   Vb = h0 rho + h1 rho u + h2 rho v + h3 H,  pb = h1 n_x + h2 n_y + h3 V
//   rho_b = h0 V - Vb V / rho + (gam-1) pb |u|^2 / 2
//   (rho u)_b = h1 V + (Vb / rho) n_x - (gam-1) pb u   (likewise rho v)
//   E_b = h3 V + (gam-1) pb
//   n_b += (h1 p + (Vb / rho) rho u,  h2 p + (Vb / rho) rho v)
// plus the dissipation mu f_bar on q1 and -mu f_bar on q2.
#include "common.cuh"
#include "rows.cuh"

namespace {

// One side's reverse sweep (K2 = |u|^2 / 2) with the side's share of the
// dissipation mu (q1 - q2) folded in, as in the forward flux: its q_bar
// part is s mu f_bar = s mu2 h (h = f_bar / 2, mu2 = 2 mu, s = +1 for the
// edge's first cell, -1 for its second), and with Vd = V + s mu2
//   q_bar = (h0 Vd - Wb V + gpb K2, h1 Vd + Wb n_x - gpb u,
//            h2 Vd + Wb n_y - gpb v, h3 Vd + gpb),
// 3 operations fewer than adding s mu2 h afterwards.  hn = h1 n_x + h2 n_y
// is common to both sides; the side's n_b is stored (first side) or added
// (second side).
template <typename T>
__device__ __forceinline__ void flux_rev(T r, T ru, T rv, T u, T v, T p, T H, T ri, T K2, T nx, T ny, T hn, T smu2,
                                         T gm1, const T h[4], T qb[4], T &nbx, T &nby, bool first)
{
    const T V = u * nx + v * ny;
    const T Vd = V + smu2;
    const T Vb = h[0] * r + h[1] * ru + h[2] * rv + h[3] * H;
    const T pb = h[3] * V + hn;
    const T Wb = Vb * ri;
    const T gpb = gm1 * pb;
    qb[0] = h[0] * Vd - Wb * V + gpb * K2;
    qb[1] = h[1] * Vd + Wb * nx - gpb * u;
    qb[2] = h[2] * Vd + Wb * ny - gpb * v;
    qb[3] = h[3] * Vd + gpb;
    if (first) {
        nbx = h[1] * p + Wb * ru;
        nby = h[2] * p + Wb * rv;
    } else {
        nbx = fma(h[1], p, fma(Wb, ru, nbx));
        nby = fma(h[2], p, fma(Wb, rv, nby));
    }
}

// Thread-coloured kernel (Algorithm 1), smem per cell: q[4], adt, u, v, p,
// H, ri, rb[4], inc[4] (18 T) + gid; per node: x[2], inc[2] (4 T) + gid
template <typename T>
__host__ __device__ constexpr int adj_smem_per_cell()
{
    return 18 * (int)sizeof(T) + 4;
}
template <typename T>
__host__ __device__ constexpr int adj_smem_per_node()
{
    return 4 * (int)sizeof(T) + 4;
}

template <typename T, bool SOA>
__global__ void __launch_bounds__(1024) adjoint_hier(const mp_block_desc *__restrict__ desc, int block0,
                                                     const ushort4 *__restrict__ lmap,
                                                     const uint8_t *__restrict__ tcolor,
                                                     const int32_t *__restrict__ fp, const T *__restrict__ x,
                                                     const T *__restrict__ q, const T *__restrict__ adt,
                                                     const T *__restrict__ rbar, T *__restrict__ qbar,
                                                     T *__restrict__ xbar, int64_t nnode, int64_t ncell, int cap_c,
                                                     int cap_n, T gm1, T eps, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_q = reinterpret_cast<T *>(smem_raw);  // [4][cap_c]
    T *s_adt = s_q + 4 * cap_c;
    T *s_u = s_adt + cap_c;
    T *s_v = s_u + cap_c;
    T *s_p = s_v + cap_c;
    T *s_H = s_p + cap_c;
    T *s_ri = s_H + cap_c;
    T *s_rb = s_ri + cap_c;   // [4][cap_c]
    T *s_qi = s_rb + 4 * cap_c;  // [4][cap_c] q_bar (prefetched, incremented)
    T *s_x = s_qi + 4 * cap_c;   // [2][cap_n]
    T *s_xi = s_x + 2 * cap_n;   // [2][cap_n] x_bar (prefetched, incremented)
    int *s_gc = reinterpret_cast<int *>(s_xi + 2 * cap_n);
    int *s_gn = s_gc + cap_c;

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nn = d.fp_count[0], nc = d.fp_count[1];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gn + cap_n) - smem_raw) > dynamic_smem_bytes() ||
        nc > cap_c || nn > cap_n || d.nitems > (int)blockDim.x) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpn = fp + d.fp_start[0];
    const int32_t *fpc = fp + d.fp_start[1];
    const bool active = tid < d.nitems;
    ushort4 l = make_ushort4(0, 0, 0, 0);
    int my_color = -1;
    if (active) {  // independent of the staging: issued first
        l = lmap[d.item_start + tid];
        my_color = tcolor[d.item_start + tid];
    }
    // stage q, adt, res_bar, primitives and the current q_bar / x_bar
    // (increments accumulate onto them; the write-back is a plain store)
    for (int i = tid; i < nc; i += blockDim.x) {
        int64_t g = fpc[i];
        T qq[4], rb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int64_t j = SOA ? k * ncell + g : 4 * g + k;
            qq[k] = q[j];
            rb[k] = rbar[j];
        }
        mp_pdl_wait();  // q_bar, x_bar: written by the previous colour's launch
#pragma unroll
        for (int k = 0; k < 4; ++k) s_qi[k * cap_c + i] = qbar[SOA ? k * ncell + g : 4 * g + k];
        T ri = rcp(qq[0]);
        T u = qq[1] * ri, v = qq[2] * ri;
        T p = gm1 * (qq[3] - half_of(qq[1] * u + qq[2] * v));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s_q[k * cap_c + i] = qq[k];
            s_rb[k * cap_c + i] = rb[k];
        }
        s_adt[i] = adt[g];
        s_u[i] = u;
        s_v[i] = v;
        s_p[i] = p;
        s_H[i] = qq[3] + p;
        s_ri[i] = ri;
        s_gc[i] = (int)g;
    }
    // nodes: on the warps that stage no cell when there are enough of them
    // (at most two nodes per thread), so that the node loads do not follow the cell
    // arithmetic on the cell warps
    auto stage_node = [&](int i) {
        int64_t g = fpn[i];
        s_x[i] = SOA ? x[g] : x[2 * g];
        s_x[cap_n + i] = SOA ? x[nnode + g] : x[2 * g + 1];
        mp_pdl_wait();
        s_xi[i] = SOA ? xbar[g] : xbar[2 * g];
        s_xi[cap_n + i] = SOA ? xbar[nnode + g] : xbar[2 * g + 1];
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
    T qb1[4], qb2[4], nbx = T(0), nby = T(0);
    if (active) {
        na = l.x;
        nb = l.y;
        c1 = l.z;
        c2 = l.w;
        T nx = s_x[cap_n + na] - s_x[cap_n + nb];
        T ny = s_x[nb] - s_x[na];
        T h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = half_of(s_rb[k * cap_c + c1] - s_rb[k * cap_c + c2]);
        auto K2 = [&](int c) { return half_of(s_u[c] * s_u[c] + s_v[c] * s_v[c]); };
        const T hn = h[1] * nx + h[2] * ny, mu2 = (s_adt[c1] + s_adt[c2]) * eps;
        flux_rev(s_q[c1], s_q[cap_c + c1], s_q[2 * cap_c + c1], s_u[c1], s_v[c1], s_p[c1], s_H[c1], s_ri[c1], K2(c1),
                 nx, ny, hn, mu2, gm1, h, qb1, nbx, nby, true);
        flux_rev(s_q[c2], s_q[cap_c + c2], s_q[2 * cap_c + c2], s_u[c2], s_v[c2], s_p[c2], s_H[c2], s_ri[c2], K2(c2),
                 nx, ny, hn, -mu2, gm1, h, qb2, nbx, nby, false);
    }
    for (int c = 0; c < d.ncolors; ++c) {
        if (my_color == c) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s_qi[k * cap_c + c1] += qb1[k];
                s_qi[k * cap_c + c2] += qb2[k];
            }
            // n_x = y_a - y_b, n_y = x_b - x_a
            s_xi[na] -= nby;
            s_xi[nb] += nby;
            s_xi[cap_n + na] += nbx;
            s_xi[cap_n + nb] -= nbx;
        }
        __syncthreads();
    }
    for (int i = tid; i < nc; i += blockDim.x) {
        int64_t g = s_gc[i];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int64_t j = SOA ? k * ncell + g : 4 * g + k;
            qbar[j] = s_qi[k * cap_c + i];
        }
    }
    for (int i = tid; i < nn; i += blockDim.x) {
        int64_t g = s_gn[i];
        xbar[SOA ? g : 2 * g] = s_xi[i];
        xbar[SOA ? nnode + g : 2 * g + 1] = s_xi[cap_n + i];
    }
}

// Gather form (native FP64 and FP32), laid out like res_calc's: vector
// records per cell and node, one reverse sweep per thread whose increments
// are all stored, one barrier, then each footprint cell and node sums its
// edges' increments through the plan's gather rows (the block-local inverse
// of both written maps) onto the prefetched q_bar / x_bar and stores them:
// no thread colours, a fixed order of additions.
// Dynamic shared memory, cap_c cells, cap_n nodes, S = blockDim edges:
//   T  cq[cap_c][4]    rho, ru, rv, H
//   T  cp[cap_c][4]    u, v, p, 1/rho
//   T  ch[cap_c][4]    res_bar / 2
//   T  cb[cap_c][4]    q_bar, prefetched
//   T  eq[2 S + 1][4]  q_bar increments: of the edge's first cell at [e], of
//                      its second at [S + e], zeros at [2 S]
//   T  en[S + 1][2]    x_bar increment of the edge's first node,
//                      (-n_y_bar, n_x_bar), at [e]; zeros at [S]
//   T  ck[cap_c][2]    |u|^2 / 2, eps adt
//   T  xn[cap_n][2]    node coordinates
//   T  xb[cap_n][2]    x_bar, prefetched
//   ushort4 gc[nrow][cap_c]  cell gather rows as rows of eq
//   ushort4 gn[nrow][cap_n]  node gather rows as rows of en, bit 15 set for
//                            the edge's second node (the negated increment)
//   int idc[cap_c], idn[cap_n]
template <typename T>
struct adj_g_args {
    const mp_block_desc *desc;
    const ushort4 *lmap, *gat;
    const int32_t *fp;
    const T *x, *q, *adt, *rbar;
    T *qbar, *xbar;
    int64_t nnode, ncell;
    int gw4, cap_c, cap_n;
    T gm1, eps;
    int *err;
};

template <typename T>
__host__ __device__ constexpr int adj_g_smem(int cap_c, int cap_n, int S, int nrow)
{
    return cap_c * (18 * (int)sizeof(T) + 8 * nrow + 4) + cap_n * (4 * (int)sizeof(T) + 8 * nrow + 4) +
           (2 * S + 1) * 4 * (int)sizeof(T) + (S + 1) * 2 * (int)sizeof(T);
}

template <typename T, bool SOA, bool GW1>
__global__ void __maxnreg__(64) adjoint_hier_g(adj_g_args<T> A, int block0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = blockDim.x, tid = threadIdx.x, cap_c = A.cap_c, cap_n = A.cap_n;
    const int nrow = GW1 ? 1 : A.gw4;
    T *s_cq = reinterpret_cast<T *>(smem_raw);
    T *s_cp = s_cq + 4 * cap_c;
    T *s_ch = s_cp + 4 * cap_c;
    T *s_cb = s_ch + 4 * cap_c;
    T *s_eq = s_cb + 4 * cap_c;
    T *s_en = s_eq + 4 * (2 * S + 1);
    T *s_ck = s_en + 2 * (S + 1);
    T *s_xn = s_ck + 2 * cap_c;
    T *s_xb = s_xn + 2 * cap_n;
    ushort4 *s_gc = reinterpret_cast<ushort4 *>(s_xb + 2 * cap_n);
    ushort4 *s_gn = s_gc + nrow * cap_c;
    int *s_idc = reinterpret_cast<int *>(s_gn + nrow * cap_n);
    int *s_idn = s_idc + cap_c;

    mp_pdl_trigger();
    const mp_block_desc d = A.desc[block0 + blockIdx.x];
    const int nn = d.fp_count[0], nc = d.fp_count[1];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_idn + cap_n) - smem_raw) > dynamic_smem_bytes() ||
        nc > cap_c || nn > cap_n || d.nitems > S || A.gw4 < 1 || A.gw4 > (GW1 ? 1 : 4)) {
        if (tid == 0) atomicExch(A.err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpn = A.fp + d.fp_start[0];
    const int32_t *fpc = A.fp + d.fp_start[1];
    const bool active = tid < d.nitems;
    ushort4 l = make_ushort4(0, 0, 0, 0);
    if (active) l = A.lmap[d.item_start + tid];  // independent of the staging: issued first
    if (tid == 0) {
        st_row4(s_eq, 2 * S, T(0), T(0), T(0), T(0));
        st_row2(s_en, S, T(0), T(0));
    }
    // gather entries "local edge x 16 + map slot": cells (slots 2, 3, the
    // edge's first and second cell) -> rows of eq; nodes (slots 0, 1) ->
    // rows of en, bit 15 for the second node; padding -> the zero rows
    auto cell_row = [&](unsigned e) -> unsigned short {
        return (unsigned short)(e == 0xFFFFu ? 2u * S : (e >> 4) + ((e & 15u) == 3u ? (unsigned)S : 0u));
    };
    auto node_row = [&](unsigned e) -> unsigned short {
        return (unsigned short)(e == 0xFFFFu ? (unsigned)S : (e >> 4) | ((e & 15u) == 1u ? 0x8000u : 0u));
    };
    const T gm1 = A.gm1, eps = A.eps;
    // cells: q, res_bar, adt and the gather rows, then q_bar after the
    // dependent-launch wait (the previous colour's launch writes it)
    for (int i = tid; i < nc; i += S) {
        const int g = fpc[i];
        T r, ru, rv, E, b0, b1, b2, b3;
        load_cell<T, SOA>(A.q, A.ncell, g, r, ru, rv, E);
        load_cell<T, SOA>(A.rbar, A.ncell, g, b0, b1, b2, b3);
        const T a = A.adt[g];
        const ushort4 *rw = A.gat + (int64_t)(d.fp_start[1] + i) * A.gw4;
        for (int h = 0; h < nrow; ++h) {
            const ushort4 e4 = rw[h];
            s_gc[h * cap_c + i] = make_ushort4(cell_row(e4.x), cell_row(e4.y), cell_row(e4.z), cell_row(e4.w));
        }
        s_idc[i] = g;
        mp_pdl_wait();
        T c0, c1, c2, c3;
        load_cell<T, SOA>(A.qbar, A.ncell, g, c0, c1, c2, c3);
        const T ri = rcp(r);
        const T u = ru * ri, v = rv * ri;
        const T K2 = half_of(u * u + v * v);
        const T p = gm1 * (E - r * K2);
        st_row4(s_cq, i, r, ru, rv, E + p);
        st_row4(s_cp, i, u, v, p, ri);
        st_row4(s_ch, i, half_of(b0), half_of(b1), half_of(b2), half_of(b3));
        st_row4(s_cb, i, c0, c1, c2, c3);
        st_row2(s_ck, i, K2, eps * a);
    }
    // nodes: on the warps that stage no cell when they are enough
    auto stage_node = [&](int i) {
        const int g = fpn[i];
        T px, py;
        load_node<T, SOA>(A.x, A.nnode, g, px, py);
        const ushort4 *rw = A.gat + (int64_t)(d.fp_start[0] + i) * A.gw4;
        for (int h = 0; h < nrow; ++h) {
            const ushort4 e4 = rw[h];
            s_gn[h * cap_n + i] = make_ushort4(node_row(e4.x), node_row(e4.y), node_row(e4.z), node_row(e4.w));
        }
        s_idn[i] = g;
        st_row2(s_xn, i, px, py);
        mp_pdl_wait();
        load_node<T, SOA>(A.xbar, A.nnode, g, px, py);
        st_row2(s_xb, i, px, py);
    };
    const int ncw = (nc + 31) & ~31, nfree = S - ncw;
    if (nfree >= 32 && 2 * nfree >= nn) {
        if (tid >= ncw) {
            const int i = tid - ncw;
            if (i < nn) stage_node(i);
            if (i + nfree < nn) stage_node(i + nfree);
        }
    } else {
        for (int i = tid; i < nn; i += S) stage_node(i);
    }
    // every thread: the write-back below must follow the previous colour's
    mp_pdl_wait();
    __syncthreads();

    if (active) {
        const int na = l.x, nb = l.y, c1 = l.z, c2 = l.w;
        T xa, ya, xb, yb;
        ld_row2(s_xn, na, xa, ya);
        ld_row2(s_xn, nb, xb, yb);
        const T nx = ya - yb, ny = xb - xa;
        T h[4], t0, t1, t2, t3;
        ld_row4(s_ch, c1, h[0], h[1], h[2], h[3]);
        ld_row4(s_ch, c2, t0, t1, t2, t3);
        h[0] -= t0;  // f_bar / 2 = (res_bar1 - res_bar2) / 2
        h[1] -= t1;
        h[2] -= t2;
        h[3] -= t3;
        T K1, a1, K2, a2;
        ld_row2(s_ck, c1, K1, a1);
        ld_row2(s_ck, c2, K2, a2);
        const T mu2 = a1 + a2, hn = h[1] * nx + h[2] * ny;  // 2 mu = eps (adt1 + adt2)
        T qb[4], nbx, nby, r, ru, rv, H, u, v, p, ri;
        ld_row4(s_cq, c1, r, ru, rv, H);
        ld_row4(s_cp, c1, u, v, p, ri);
        flux_rev(r, ru, rv, u, v, p, H, ri, K1, nx, ny, hn, mu2, gm1, h, qb, nbx, nby, true);
        st_row4(s_eq, tid, qb[0], qb[1], qb[2], qb[3]);
        ld_row4(s_cq, c2, r, ru, rv, H);
        ld_row4(s_cp, c2, u, v, p, ri);
        flux_rev(r, ru, rv, u, v, p, H, ri, K2, nx, ny, hn, -mu2, gm1, h, qb, nbx, nby, false);
        st_row4(s_eq, S + tid, qb[0], qb[1], qb[2], qb[3]);
        st_row2(s_en, tid, flip_sign(nby), nbx);  // n_x = y_a - y_b, n_y = x_b - x_a
    }
    __syncthreads();

    // the cells, then the nodes, one per thread: sums in gather-row order
    for (int i = tid; i < nc + nn; i += S) {
        if (i < nc) {
            T a0, a1, a2, a3;
            ld_row4(s_cb, i, a0, a1, a2, a3);
            for (int h = 0; h < nrow; ++h) {
                const ushort4 e4 = s_gc[h * cap_c + i];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // padding (the zero row) comes last in a row, and halo
                    // cells after interior ones: their warps skip it whole
                    if (sizeof(T) == 8 && !__any_sync(__activemask(), es[j] != 2 * S)) continue;
                    T v0, v1, v2, v3;
                    ld_row4(s_eq, es[j], v0, v1, v2, v3);
                    a0 += v0;
                    a1 += v1;
                    a2 += v2;
                    a3 += v3;
                }
            }
            store_cell<T, SOA>(A.qbar, A.ncell, s_idc[i], a0, a1, a2, a3);
        } else {
            const int k = i - nc;
            T b0, b1;
            ld_row2(s_xb, k, b0, b1);
            for (int h = 0; h < nrow; ++h) {
                const ushort4 e4 = s_gn[h * cap_n + k];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (sizeof(T) == 8 && !__any_sync(__activemask(), es[j] != S)) continue;
                    const T sg = (es[j] & 0x8000u) ? T(-1) : T(1);
                    T v0, v1;
                    ld_row2(s_en, es[j] & 0x7fff, v0, v1);
                    b0 += sg * v0;
                    b1 += sg * v1;
                }
            }
            store_node<T, SOA>(A.xbar, A.nnode, s_idn[k], b0, b1);
        }
    }
}

template <typename T, bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256) adjoint_direct(int e0, int e1, const int32_t *__restrict__ e2n,
                                                      const int32_t *__restrict__ e2c, const T *__restrict__ x,
                                                      const T *__restrict__ q, const T *__restrict__ adt,
                                                      const T *__restrict__ rbar, T *__restrict__ qbar,
                                                      T *__restrict__ xbar, int64_t nnode, int64_t ncell, T gm1,
                                                      T eps)
{
    int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    int2 nab = reinterpret_cast<const int2 *>(e2n)[e];
    int2 cc = reinterpret_cast<const int2 *>(e2c)[e];
    auto X = [&](int64_t g, int k) { return SOA ? x[k * nnode + g] : x[2 * g + k]; };
    T nx = X(nab.x, 1) - X(nab.y, 1);
    T ny = X(nab.y, 0) - X(nab.x, 0);
    T q1[4], q2[4], h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int64_t j1 = SOA ? k * ncell + cc.x : 4 * (int64_t)cc.x + k;
        int64_t j2 = SOA ? k * ncell + cc.y : 4 * (int64_t)cc.y + k;
        q1[k] = q[j1];
        q2[k] = q[j2];
        h[k] = half_of(rbar[j1] - rbar[j2]);
    }
    const T hn = h[1] * nx + h[2] * ny, mu2 = (adt[cc.x] + adt[cc.y]) * eps;
    T qb1[4], qb2[4], nbx, nby;
    {
        T ri = rcp(q1[0]), u = q1[1] * ri, v = q1[2] * ri;
        T K2 = half_of(u * u + v * v);
        T p = gm1 * (q1[3] - q1[0] * K2);
        flux_rev(q1[0], q1[1], q1[2], u, v, p, q1[3] + p, ri, K2, nx, ny, hn, mu2, gm1, h, qb1, nbx, nby, true);
    }
    {
        T ri = rcp(q2[0]), u = q2[1] * ri, v = q2[2] * ri;
        T K2 = half_of(u * u + v * v);
        T p = gm1 * (q2[3] - q2[0] * K2);
        flux_rev(q2[0], q2[1], q2[2], u, v, p, q2[3] + p, ri, K2, nx, ny, hn, -mu2, gm1, h, qb2, nbx, nby, false);
    }
    T xa0 = -nby, xb0 = nby, xa1 = nbx, xb1 = -nbx;
    int64_t ja0 = SOA ? nab.x : 2 * (int64_t)nab.x, ja1 = SOA ? nnode + nab.x : 2 * (int64_t)nab.x + 1;
    int64_t jb0 = SOA ? nab.y : 2 * (int64_t)nab.y, jb1 = SOA ? nnode + nab.y : 2 * (int64_t)nab.y + 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int64_t j1 = SOA ? k * ncell + cc.x : 4 * (int64_t)cc.x + k;
        int64_t j2 = SOA ? k * ncell + cc.y : 4 * (int64_t)cc.y + k;
        T a = qb1[k], b = qb2[k];
        if (ATOMIC) {
            atomicAdd(qbar + j1, a);
            atomicAdd(qbar + j2, b);
        } else {
            qbar[j1] += a;
            qbar[j2] += b;
        }
    }
    if (ATOMIC) {
        atomicAdd(xbar + ja0, xa0);
        atomicAdd(xbar + jb0, xb0);
        atomicAdd(xbar + ja1, xa1);
        atomicAdd(xbar + jb1, xb1);
    } else {
        xbar[ja0] += xa0;
        xbar[jb0] += xb0;
        xbar[ja1] += xa1;
        xbar[jb1] += xb1;
    }
}

template <typename T, bool SOA>
int adjoint_t(const mp_plan *P, const void *x, const void *q, const void *adt, const void *rbar, void *qbar,
              void *xbar, double gam, double eps, cudaStream_t s)
{
    const int64_t nnode = P->maps[0].to_size, ncell = P->maps[1].to_size;
    const T gm1 = (T)(gam - 1.0), teps = (T)eps;
    if (P->opts.coloring == MP_COLOR_HIER) {
        if (P->maps[0].slot != 0 || P->maps[1].slot != 1) return MP_EPLAN;
        const int cap_n = P->stats.footprint_max[0], cap_c = P->stats.footprint_max[1];
        int *err = nullptr;
        int rc = mp_device_error_word(&err);
        if (rc != MP_OK) return rc;
        bool overlap = false;
        if (mp_staged(P, MP_STAGED_GATHER) == MP_STAGED_GATHER && mp_gather_ready(P)) {
            const int gw4 = P->gat_w / 4, bs = P->opts.block_size;
            const bool gw1 = gw4 == 1;
            const int smem = adj_g_smem<T>(cap_c, cap_n, bs, gw1 ? 1 : gw4);
            auto kern = gw1 ? adjoint_hier_g<T, SOA, true> : adjoint_hier_g<T, SOA, false>;
            if ((rc = mp_allow_smem(kern, smem)) != MP_OK) return rc;
            const adj_g_args<T> A{P->dev.desc, reinterpret_cast<const ushort4 *>(P->dev.lmap),
                                  reinterpret_cast<const ushort4 *>(P->dev.gat), P->dev.fp, (const T *)x,
                                  (const T *)q, (const T *)adt, (const T *)rbar, (T *)qbar, (T *)xbar, nnode, ncell,
                                  gw4, cap_c, cap_n, gm1, teps, err};
            for (int c = 0; c < P->ncolors; ++c) {
                int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
                if (nb == 0) continue;
                MP_CUDA_TRY(mp_launch(kern, nb, bs, smem, s, overlap, A, b0));
                overlap = true;
            }
            MP_CUDA_TRY(cudaGetLastError());
            return MP_OK;
        }
        const int smem = cap_c * adj_smem_per_cell<T>() + cap_n * adj_smem_per_node<T>();
        auto kern = adjoint_hier<T, SOA>;
        if ((rc = mp_allow_smem(kern, smem)) != MP_OK) return rc;
        for (int c = 0; c < P->ncolors; ++c) {
            int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
            if (nb == 0) continue;
            MP_CUDA_TRY(mp_launch(kern, nb, P->opts.block_size, smem, s, overlap, P->dev.desc, b0,
                                  reinterpret_cast<const ushort4 *>(P->dev.lmap), P->dev.tcolor, P->dev.fp,
                                  (const T *)x, (const T *)q, (const T *)adt, (const T *)rbar, (T *)qbar, (T *)xbar,
                                  nnode, ncell, cap_c, cap_n, gm1, teps, err));
            overlap = true;
        }
    } else {
        const bool atomic = P->opts.coloring == MP_COLOR_ATOMIC;
        for (int c = 0; c < P->ncolors; ++c) {
            int e0 = P->color_offsets[c], e1 = P->color_offsets[c + 1];
            if (e1 <= e0) continue;
            auto kern = atomic ? adjoint_direct<T, SOA, true> : adjoint_direct<T, SOA, false>;
            kern<<<(e1 - e0 + 255) / 256, 256, 0, s>>>(e0, e1, P->dev.map[0], P->dev.map[1], (const T *)x,
                                                       (const T *)q, (const T *)adt, (const T *)rbar, (T *)qbar,
                                                       (T *)xbar, nnode, ncell, gm1, teps);
        }
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

extern "C" int loop_adjoint(const mp_plan *P, int32_t dtype, const void *x, const void *q, const void *adt,
                            const void *res_bar, void *q_bar, void *x_bar, double gam, double eps, void *stream)
{
    if (!P || (dtype != MP_F64 && dtype != MP_F32 && dtype != MP_F64_DW)) return MP_EINVAL;
    if (P->nmaps != 2 || P->maps[0].arity != 2 || P->maps[1].arity != 2 || !P->maps[0].written ||
        !P->maps[1].written)
        return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    for (const void *p : {x, q, adt, res_bar, (const void *)q_bar, (const void *)x_bar})
        if (!p || !aligned16(p)) return MP_EINVAL;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    if (dtype == MP_F64_DW) return mp_adjoint_dw(P, x, q, adt, res_bar, q_bar, x_bar, gam, eps, stream);
    cudaStream_t s = as_stream(stream);
    bool soa = P->opts.layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64)
        return soa ? adjoint_t<double, true>(P, x, q, adt, res_bar, q_bar, x_bar, gam, eps, s)
                   : adjoint_t<double, false>(P, x, q, adt, res_bar, q_bar, x_bar, gam, eps, s);
    return soa ? adjoint_t<float, true>(P, x, q, adt, res_bar, q_bar, x_bar, gam, eps, s)
               : adjoint_t<float, false>(P, x, q, adt, res_bar, q_bar, x_bar, gam, eps, s);
}
