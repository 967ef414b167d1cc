// res_calc, two-layer staged kernel with FP64 data and double-word (FP32
// pair) arithmetic: the FP64-accurate variant for GB300, whose FP64 pipe
// (2 FMA per clock per SM) would otherwise bind the loop.
//
// Same structure as res_calc_hier (Algorithm 1): stage the block's cells
// and nodes, compute one edge flux per thread from shared memory, apply the
// increments one thread colour at a time, write every footprint cell back
// once.  Differences:
//  * cell data are converted to double-word at staging and the per-cell
//    primitives (u, v, p, H) are computed in double-word arithmetic;
//  * node coordinates stay FP64 in shared memory: the edge normal
//    n = (y_a - y_b, x_b - x_a) is formed in FP64, where the subtraction of
//    nearby coordinates is exact, and only then converted (a double-word
//    copy of the coordinates would lose the low bits that the difference
//    keeps);
//  * increments accumulate in double-word in shared memory and are added
//    to the FP64 res in FP64 at write-back.
// Measured against the FP64 oracle the result agrees to ~1e-13 rel-L2.
//
// GLOBAL and ATOMIC plans run the baselines of Sec. 2.1 in the same
// arithmetic (res_calc_direct_dw).
//
// GATHER form: instead of the thread-coloured increments each thread
// stores its flux in shared memory, one barrier, and the thread that staged
// a cell sums that cell's edge fluxes (the plan's block-local inverse map,
// staged with the cell) and writes it back.
#include <algorithm>

#include "common.cuh"
#include "dw.cuh"

namespace {

// Dynamic shared memory for cap_c cells and cap_n nodes:
//   double x, y                                    (16 B per node)
//   double res[4]  (prefetched at staging)         (32 B per cell)
//   dw   [cap_c][9]: rho, ru, rv, E, eps adt/2, u, v, p, H of each cell
//                        (72 B per cell)
//   dw   inc[4][cap_c]   coloured form             (32 B per cell)
//        f[4][cap_f]     gather form: over the records, extended when
//                        4 cap_f > 9 cap_c
//   int  gid                                       (4 B per cell)
//   ushort4 ge[gw4][cap_c]  gather form            (8 gw4 B per cell)
// The FP64 arrays come first (8-byte alignment).
constexpr int kDwCellBytes = 32 + 9 * 8 + 4;
constexpr int kDwIncBytes = 32;
constexpr int kDwNodeBytes = 16;

__device__ __forceinline__ dw ld(const float2 *a, int i)
{
    float2 v = a[i];
    return {v.x, v.y};
}
__device__ __forceinline__ void st(float2 *a, int i, dw v) { a[i] = make_float2(v.hi, v.lo); }

// Per-cell primitives of a conserved state in double-word arithmetic:
// u, v, p = (gam - 1)(E - (ru u + rv v)/2), H = E + p.  Sloppy additions
// throughout: the kinetic energy sums two non-negative terms, E - kin =
// p/(gam-1) has condition number 1 + (gam-1) gam M^2 / 2 (1.05 at Mach 0.4),
// E + p adds positives.
__device__ __forceinline__ void dw_cell_prims(dw R, dw RU, dw RV, dw EE, dw gm1, dw &u, dw &v, dw &p, dw &H)
{
    const dw ri = dw_recip_fast(R);
    u = dw_mul(RU, ri);
    v = dw_mul(RV, ri);
    const dw kin = dw_scale2(dw_add_fast(dw_mul(RU, u), dw_mul(RV, v)), 0.5f);
    p = dw_mul(gm1, dw_add_fast(EE, dw_neg(kin)));
    H = dw_add_fast(EE, p);
}

// Edge flux from the half normal (nxh, nyh) = n/2 and both cells' states,
// primitives and eps adt / 2 (a1, a2).  With mu = eps (adt1 + adt2) / 2,
// V = u nx/2 + v ny/2 and W1 = V1 + mu, W2 = V2 - mu (accurate double-word
// additions: V and mu may nearly cancel), the dissipation of the first
// three components folds into the normal velocities; each component is one
// compensated sum of products:
//   f0 = r1 W1 + r2 W2
//   f1 = ru1 W1 + ru2 W2 + (p1 + p2) nx/2                    (f2 likewise)
//   f3 = H1 V1 + H2 V2 + mu E1 - mu E2
__device__ __forceinline__ void dw_edge_flux(dw nxh, dw nyh, dw r1, dw ru1, dw rv1, dw E1, dw a1, dw u1, dw v1,
                                             dw p1, dw H1, dw r2, dw ru2, dw rv2, dw E2, dw a2, dw u2, dw v2, dw p2,
                                             dw H2, dw f[4])
{
    const dw pp = dw_add_fast(p1, p2);  // two positive pressures, no cancellation
    dw_acc A = dw_dot_begin(u1, nxh);
    dw_dot_add(A, v1, nyh);
    const dw V1 = dw_dot_end(A);
    A = dw_dot_begin(u2, nxh);
    dw_dot_add(A, v2, nyh);
    const dw V2 = dw_dot_end(A);
    const dw mu = dw_add_fast(a1, a2);  // two positive terms
    const dw W1 = dw_add(V1, mu), W2 = dw_add(V2, dw_neg(mu));
    A = dw_dot_begin(r1, W1);
    dw_dot_add(A, r2, W2);
    f[0] = dw_dot_end(A);
    A = dw_dot_begin(ru1, W1);
    dw_dot_add(A, ru2, W2);
    dw_dot_add(A, pp, nxh);
    f[1] = dw_dot_end(A);
    A = dw_dot_begin(rv1, W1);
    dw_dot_add(A, rv2, W2);
    dw_dot_add(A, pp, nyh);
    f[2] = dw_dot_end(A);
    A = dw_dot_begin(H1, V1);
    dw_dot_add(A, H2, V2);
    dw_dot_add(A, mu, E1);
    dw_dot_add(A, mu, dw_neg(E2));
    f[3] = dw_dot_end(A);
}

template <bool SOA, bool GATHER>
__global__ void __launch_bounds__(512, 4) res_calc_hier_dw(const mp_block_desc *__restrict__ desc, int block0,
                                                         const ushort4 *__restrict__ lmap,
                                                         const uint8_t *__restrict__ tcolor,
                                                         const ushort4 *__restrict__ gat, int gw4,
                                                         const int32_t *__restrict__ fp,
                                                         const double *__restrict__ x, const double *__restrict__ q,
                                                         const double *__restrict__ adt, double *__restrict__ res,
                                                         int64_t nnode, int64_t ncell, int cap_c, int cap_n,
                                                         int cap_f, dw gm1, dw half_eps, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *s_x = reinterpret_cast<double *>(smem_raw);
    double *s_y = s_x + cap_n;
    double *s_res = s_y + cap_n;  // [4][cap_c]
    // per-cell records of 9 double-words, [cap_c][9]: an odd stride in
    // 8-byte words keeps 16 consecutive cells on distinct bank pairs
    float2 *s_r = reinterpret_cast<float2 *>(s_res + 4 * cap_c);
    float2 *s_ru = s_r + 1;
    float2 *s_rv = s_r + 2;
    float2 *s_E = s_r + 3;
    float2 *s_a = s_r + 4;
    float2 *s_u = s_r + 5;
    float2 *s_v = s_r + 6;
    float2 *s_p = s_r + 7;
    float2 *s_H = s_r + 8;
    // increments [4][cap_c] (coloured) after the primitives; the gather
    // form's fluxes [4][cap_f] overwrite the primitives once all threads
    // have read them
    float2 *s_inc = GATHER ? s_r : s_r + 9 * cap_c;
    float2 *s_tail = GATHER ? s_r + max(9 * cap_c, 4 * cap_f) : s_inc + 4 * cap_c;
    ushort4 *s_ge = reinterpret_cast<ushort4 *>(s_tail);  // [gw4][cap_c]
    int *s_gid = reinterpret_cast<int *>(s_ge + (GATHER ? gw4 * cap_c : 0));

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nn = d.fp_count[0], nc = d.fp_count[1];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gid + cap_c) - smem_raw) > dynamic_smem_bytes() ||
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
    if (active) {  // independent of the staging: issued first
        l = lmap[d.item_start + tid];
        if (!GATHER) my_color = tcolor[d.item_start + tid];
    }

    for (int i = tid; i < nc; i += blockDim.x) {
        const int64_t g = fpc[i];
        double r, ru, rv, E;
        if (SOA) {
            r = q[g];
            ru = q[ncell + g];
            rv = q[2 * ncell + g];
            E = q[3 * ncell + g];
            mp_pdl_wait();  // res: written by the previous colour's launch
#pragma unroll
            for (int k = 0; k < 4; ++k) s_res[k * cap_c + i] = res[k * ncell + g];
        } else {
            const double2 *q2 = reinterpret_cast<const double2 *>(q) + 2 * g;
            double2 a = q2[0], b = q2[1];
            r = a.x;
            ru = a.y;
            rv = b.x;
            E = b.y;
            mp_pdl_wait();  // res: written by the previous colour's launch
            const double2 *r2 = reinterpret_cast<const double2 *>(res) + 2 * g;
            double2 ra = r2[0], rb = r2[1];
            s_res[i] = ra.x;
            s_res[cap_c + i] = ra.y;
            s_res[2 * cap_c + i] = rb.x;
            s_res[3 * cap_c + i] = rb.y;
        }
        dw R = dw_from_double_int(r), RU = dw_from_double_int(ru), RV = dw_from_double_int(rv),
           EE = dw_from_double_int(E);
        dw u, v, p, H;
        dw_cell_prims(R, RU, RV, EE, gm1, u, v, p, H);
        st(s_r, 9 * i, R);
        st(s_ru, 9 * i, RU);
        st(s_rv, 9 * i, RV);
        st(s_E, 9 * i, EE);
        st(s_a, 9 * i, dw_mul(dw_from_double_int(adt[g]), half_eps));  // eps adt / 2
        st(s_u, 9 * i, u);
        st(s_v, 9 * i, v);
        st(s_p, 9 * i, p);
        st(s_H, 9 * i, H);
        if (GATHER) {
            const ushort4 *row = gat + (int64_t)(d.fp_start[1] + i) * gw4;
            for (int h = 0; h < gw4; ++h) s_ge[h * cap_c + i] = row[h];
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) s_inc[k * cap_c + i] = make_float2(0.f, 0.f);
        }
        s_gid[i] = (int)g;
    }
    // nodes: on the warps that stage no cell when there are enough of them
    // (at most two nodes per thread), so that the node loads do not follow
    // the cell arithmetic on the cell warps
    auto stage_node = [&](int i) {
        const int64_t g = fpn[i];
        if (SOA) {
            s_x[i] = x[g];
            s_y[i] = x[nnode + g];
        } else {
            double2 a = reinterpret_cast<const double2 *>(x)[g];
            s_x[i] = a.x;
            s_y[i] = a.y;
        }
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

    dw f[4];
    int c1 = 0, c2 = 0;
    if (active) {
        const int na = l.x, nb = l.y;
        c1 = l.z;
        c2 = l.w;
        // n = (y_a - y_b, x_b - x_a), exact in FP64 for nearby nodes; halved
        const dw nxh = dw_scale2(dw_from_double_int(s_y[na] - s_y[nb]), 0.5f);
        const dw nyh = dw_scale2(dw_from_double_int(s_x[nb] - s_x[na]), 0.5f);
        dw_edge_flux(nxh, nyh, ld(s_r, 9 * c1), ld(s_ru, 9 * c1), ld(s_rv, 9 * c1), ld(s_E, 9 * c1),
                     ld(s_a, 9 * c1), ld(s_u, 9 * c1), ld(s_v, 9 * c1), ld(s_p, 9 * c1), ld(s_H, 9 * c1),
                     ld(s_r, 9 * c2), ld(s_ru, 9 * c2), ld(s_rv, 9 * c2), ld(s_E, 9 * c2), ld(s_a, 9 * c2),
                     ld(s_u, 9 * c2), ld(s_v, 9 * c2), ld(s_p, 9 * c2), ld(s_H, 9 * c2), f);
    }
    if constexpr (GATHER) {
        __syncthreads();  // every flux is computed: the primitives are dead
        if (active) {
#pragma unroll
            for (int k = 0; k < 4; ++k) st(s_inc, k * cap_f + tid, f[k]);
        }
        __syncthreads();
        // each cell sums its edges' fluxes: +f from the edge's first cell
        // slot (map slot 2), -f from its second (slot 3)
        for (int i = tid; i < nc; i += blockDim.x) {
            // branch-free: a padding entry adds 0 times slot 0 (thread 0's
            // flux, computed in every block)
            dw_acc S[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            for (int h = 0; h < gw4; ++h) {
                const ushort4 e4 = s_ge[h * cap_c + i];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned e = es[j];
                    const bool valid = e != 0xFFFFu;
                    const int t = valid ? (int)(e >> 4) : 0;
                    const float sg = !valid ? 0.0f : ((e & 15u) == 3u ? -1.0f : 1.0f);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const dw v = ld(s_inc, k * cap_f + t);
                        dw_sum_add(S[k], v, sg);
                    }
                }
            }
            const dw a[4] = {dw_sum_end(S[0]), dw_sum_end(S[1]), dw_sum_end(S[2]), dw_sum_end(S[3])};
            const int64_t g = s_gid[i];
            if (SOA) {
#pragma unroll
                for (int k = 0; k < 4; ++k) res[k * ncell + g] = f64_add_dw(s_res[k * cap_c + i], a[k]);
            } else {
                double2 *r2 = reinterpret_cast<double2 *>(res) + 2 * g;
                r2[0] = make_double2(f64_add_dw(s_res[i], a[0]), f64_add_dw(s_res[cap_c + i], a[1]));
                r2[1] = make_double2(f64_add_dw(s_res[2 * cap_c + i], a[2]), f64_add_dw(s_res[3 * cap_c + i], a[3]));
            }
        }
    } else {
    for (int c = 0; c < d.ncolors; ++c) {
        if (my_color == c) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                st(s_inc, k * cap_c + c1, dw_add_fast(ld(s_inc, k * cap_c + c1), f[k]));
                st(s_inc, k * cap_c + c2, dw_add_fast(ld(s_inc, k * cap_c + c2), dw_neg(f[k])));
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < nc; i += blockDim.x) {
        const int64_t g = s_gid[i];
        if (SOA) {
#pragma unroll
            for (int k = 0; k < 4; ++k) res[k * ncell + g] = f64_add_dw(s_res[k * cap_c + i], ld(s_inc, k * cap_c + i));
        } else {
            double2 *r2 = reinterpret_cast<double2 *>(res) + 2 * g;
            r2[0] = make_double2(f64_add_dw(s_res[i], ld(s_inc, i)), f64_add_dw(s_res[cap_c + i], ld(s_inc, cap_c + i)));
            r2[1] = make_double2(f64_add_dw(s_res[2 * cap_c + i], ld(s_inc, 2 * cap_c + i)),
                                 f64_add_dw(s_res[3 * cap_c + i], ld(s_inc, 3 * cap_c + i)));
        }
    }
    }
}

// The baselines of Sec. 2.1 in the same double-word arithmetic, so that the
// strategies compare at equal arithmetic: one thread per edge of [e0, e1)
// gathers its two nodes and two cells from global memory (FP64), forms the
// primitives of both cells and the flux as the staged kernel does, and
//   GLOBAL (edges of one colour share no cell): res[c] = res[c] + f in
//          FP64 (two FP64 additions, as the staged write-back);
//   ATOMIC: atomicAdd of the nearest double of f (hi + lo, one FP64
//          addition) into res.
template <bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256) res_calc_direct_dw(int e0, int e1, const int32_t *__restrict__ e2n,
                                                          const int32_t *__restrict__ e2c,
                                                          const double *__restrict__ x, const double *__restrict__ q,
                                                          const double *__restrict__ adt, double *__restrict__ res,
                                                          int64_t nnode, int64_t ncell, dw gm1, dw half_eps)
{
    mp_pdl_trigger();
    const int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    const int2 nab = reinterpret_cast<const int2 *>(e2n)[e];
    const int2 cc = reinterpret_cast<const int2 *>(e2c)[e];
    double xa, ya, xb, yb;
    if (SOA) {
        xa = x[nab.x];
        ya = x[nnode + nab.x];
        xb = x[nab.y];
        yb = x[nnode + nab.y];
    } else {
        const double2 a = reinterpret_cast<const double2 *>(x)[nab.x];
        const double2 b = reinterpret_cast<const double2 *>(x)[nab.y];
        xa = a.x;
        ya = a.y;
        xb = b.x;
        yb = b.y;
    }
    dw c[2][5];  // rho, ru, rv, E, eps adt / 2 of both cells
    const int cell[2] = {cc.x, cc.y};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int64_t g = cell[s];
        double v[4];
        if (SOA) {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = q[k * ncell + g];
        } else {
            const double2 *q2 = reinterpret_cast<const double2 *>(q) + 2 * g;
            const double2 a = q2[0], b = q2[1];
            v[0] = a.x;
            v[1] = a.y;
            v[2] = b.x;
            v[3] = b.y;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) c[s][k] = dw_from_double_int(v[k]);
        c[s][4] = dw_mul(dw_from_double_int(adt[g]), half_eps);
    }
    dw u1, v1, p1, H1, u2, v2, p2, H2;
    dw_cell_prims(c[0][0], c[0][1], c[0][2], c[0][3], gm1, u1, v1, p1, H1);
    dw_cell_prims(c[1][0], c[1][1], c[1][2], c[1][3], gm1, u2, v2, p2, H2);
    const dw nxh = dw_scale2(dw_from_double_int(ya - yb), 0.5f);
    const dw nyh = dw_scale2(dw_from_double_int(xb - xa), 0.5f);
    dw f[4];
    dw_edge_flux(nxh, nyh, c[0][0], c[0][1], c[0][2], c[0][3], c[0][4], u1, v1, p1, H1, c[1][0], c[1][1], c[1][2],
                 c[1][3], c[1][4], u2, v2, p2, H2, f);
    if (!ATOMIC) mp_pdl_wait();  // res: read-add-written by the previous colour's launch
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t j1 = SOA ? k * ncell + cc.x : 4 * (int64_t)cc.x + k;
        const int64_t j2 = SOA ? k * ncell + cc.y : 4 * (int64_t)cc.y + k;
        if (ATOMIC) {
            const double d = f32_to_f64_int(f[k].hi) + f32_to_f64_int(f[k].lo);
            atomicAdd(res + j1, d);
            atomicAdd(res + j2, -d);
        } else {
            res[j1] = f64_add_dw(res[j1], f[k]);
            res[j2] = f64_add_dw(res[j2], dw_neg(f[k]));
        }
    }
}

template <bool SOA>
int res_calc_direct_dw_t(const mp_plan *P, const void *x, const void *q, const void *adt, void *res, dw gm1,
                         dw half_eps, cudaStream_t s)
{
    const bool atomic = P->opts.coloring == MP_COLOR_ATOMIC;
    auto kern = atomic ? res_calc_direct_dw<SOA, true> : res_calc_direct_dw<SOA, false>;
    bool overlap = false;
    for (int c = 0; c < P->ncolors; ++c) {
        const int e0 = P->color_offsets[c], e1 = P->color_offsets[c + 1];
        if (e1 <= e0) continue;
        MP_CUDA_TRY(mp_launch(kern, (e1 - e0 + 255) / 256, 256, 0, s, overlap && !atomic, e0, e1, P->dev.map[0],
                              P->dev.map[1], (const double *)x, (const double *)q, (const double *)adt,
                              (double *)res, P->maps[0].to_size, P->maps[1].to_size, gm1, half_eps));
        overlap = true;
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

template <bool SOA>
int res_calc_dw_t(const mp_plan *P, const void *x, const void *q, const void *adt, void *res, double gam, double eps,
                  cudaStream_t s)
{
    // constants as the nearest double-words of their FP64 values
    const double g1 = gam - 1.0, he = 0.5 * eps;
    const float g1h = (float)g1, heh = (float)he;
    const dw gm1{g1h, (float)(g1 - (double)g1h)}, half_eps{heh, (float)(he - (double)heh)};
    if (P->opts.coloring == MP_COLOR_GLOBAL || P->opts.coloring == MP_COLOR_ATOMIC)
        return res_calc_direct_dw_t<SOA>(P, x, q, adt, res, gm1, half_eps, s);
    if (P->opts.coloring != MP_COLOR_HIER || P->maps[0].slot != 0 || P->maps[1].slot != 1) return MP_EPLAN;
    const int64_t nnode = P->maps[0].to_size, ncell = P->maps[1].to_size;
    const int cap_n = P->stats.footprint_max[0], cap_c = P->stats.footprint_max[1];
    const bool gather = mp_staged(P, MP_STAGED_GATHER) == MP_STAGED_GATHER && mp_gather_ready(P);
    const int gw4 = gather ? P->gat_w / 4 : 0, cap_f = gather ? P->opts.block_size : 0;
    // the gather fluxes reuse the 9 primitive arrays (72 B per cell)
    const int inc_bytes = gather ? std::max(0, kDwIncBytes * cap_f - 72 * cap_c) : kDwIncBytes * cap_c;
    const int smem = cap_c * kDwCellBytes + cap_n * kDwNodeBytes + inc_bytes + 8 * gw4 * cap_c;
    auto kern = gather ? res_calc_hier_dw<SOA, true> : res_calc_hier_dw<SOA, false>;
    int rc = mp_allow_smem(kern, smem);
    if (rc != MP_OK) return rc;
    int *err = nullptr;
    if ((rc = mp_device_error_word(&err)) != MP_OK) return rc;
    bool overlap = false;  // the first launch follows the caller's work: plain stream order
    for (int c = 0; c < P->ncolors; ++c) {
        int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
        if (nb == 0) continue;
        MP_CUDA_TRY(mp_launch(kern, nb, P->opts.block_size, smem, s, overlap, P->dev.desc, b0,
                              reinterpret_cast<const ushort4 *>(P->dev.lmap), P->dev.tcolor,
                              reinterpret_cast<const ushort4 *>(P->dev.gat), gw4, P->dev.fp, (const double *)x,
                              (const double *)q, (const double *)adt, (double *)res, nnode, ncell, cap_c, cap_n,
                              cap_f, gm1, half_eps, err));
        overlap = true;
    }
    return MP_OK;
}

}  // namespace

int mp_res_calc_dw(const mp_plan *P, const void *x, const void *q, const void *adt, void *res, double gam, double eps,
                   void *stream)
{
    const bool soa = P->opts.layout == MP_LAYOUT_SOA;
    return soa ? res_calc_dw_t<true>(P, x, q, adt, res, gam, eps, as_stream(stream))
               : res_calc_dw_t<false>(P, x, q, adt, res, gam, eps, as_stream(stream));
}
