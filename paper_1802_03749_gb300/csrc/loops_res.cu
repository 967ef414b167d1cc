// Airfoil-style edge loops: res_calc (three race-avoidance strategies),
// bres_calc and adt_calc.
//
// res_calc strategies (Sec. 2.1 and 2.2 of the paper):
//   HIER   staged two-layer colouring (Algorithm 1): one CTA per block of a
//          block colour; the block's cell and node footprint is gathered into
//          shared memory with coalesced (vector) loads and per-cell
//          primitives are computed once per staged cell; each thread computes
//          one edge flux from shared memory; increments are applied to shared
//          memory one thread colour at a time; every footprint cell is
//          written back once with a plain read-add-write (no atomics: blocks
//          of one colour share no cell).
//   GLOBAL one launch per edge colour; every thread gathers its two cells and
//          two nodes from global memory and read-add-writes res directly.
//   ATOMIC one launch; increments with FP64/FP32 atomicAdd.
#include "common.cuh"
#include "rows.cuh"

namespace {

// ------------------------------------------------------------------ HIER

// Dynamic shared memory layout for a block with cap_c cells and cap_n nodes:
//   T  q[4][cap_c], adt[cap_c], u[cap_c], v[cap_c], p[cap_c], H[cap_c]
//                            (u, v, p halved: cell_prims_half)
//   T  inc[4][cap_c]         (res prefetched at staging, increments added on)
//   T  x[2][cap_n]           (node coordinates)
//   int gid[cap_c]
//
// Increment forms (template INC):
//   kIncColor   thread colours, one colour per barrier (Algorithm 1)
//   kIncAtomic  shared-memory atomics, one barrier
//   kIncShuffle warp-aggregated atomics: lanes of a warp with the same
//               target reduce by shuffles, one atomic per target and warp
// The gather form (every thread stores its flux, one barrier, then each
// cell sums the fluxes of its edges from the plan's block-local inverse
// map) is res_calc_hier_g below.
template <typename T>
__host__ __device__ constexpr int res_smem_per_cell()
{
    return 13 * (int)sizeof(T) + 4;
}
template <typename T>
__host__ __device__ constexpr int res_smem_per_node()
{
    return 2 * (int)sizeof(T);
}
constexpr int kIncColor = 0, kIncAtomic = 1, kIncShuffle = 3;


// CG: read through L2 only (ld.global.cg), for values another CTA of the
// same launch wrote (this SM's L1 may hold an older copy)
template <typename T, bool SOA, bool CG = false>
__device__ __forceinline__ void load_res(const T *__restrict__ res, int64_t ncell, int g, T &r0, T &r1, T &r2, T &r3)
{
    if (SOA) {
        r0 = CG ? __ldcg(res + g) : res[g];
        r1 = CG ? __ldcg(res + ncell + g) : res[ncell + g];
        r2 = CG ? __ldcg(res + 2 * ncell + g) : res[2 * ncell + g];
        r3 = CG ? __ldcg(res + 3 * ncell + g) : res[3 * ncell + g];
    } else if (sizeof(T) == 8) {
        const double2 *p = reinterpret_cast<const double2 *>(res) + 2 * (int64_t)g;
        double2 a = CG ? __ldcg(p) : p[0], b = CG ? __ldcg(p + 1) : p[1];
        r0 = (T)a.x;
        r1 = (T)a.y;
        r2 = (T)b.x;
        r3 = (T)b.y;
    } else {
        const float4 *p = reinterpret_cast<const float4 *>(res) + g;
        float4 a = CG ? __ldcg(p) : p[0];
        r0 = (T)a.x;
        r1 = (T)a.y;
        r2 = (T)a.z;
        r3 = (T)a.w;
    }
}

template <typename T, bool SOA, int INC>
__global__ void __launch_bounds__(1024) res_calc_hier(const mp_block_desc *__restrict__ desc, int block0,
                                                      const ushort4 *__restrict__ lmap,
                                                      const uint8_t *__restrict__ tcolor,
                                                      const int32_t *__restrict__ fp, const T *__restrict__ x,
                                                      const T *__restrict__ q, const T *__restrict__ adt,
                                                      T *__restrict__ res, int64_t nnode, int64_t ncell, int cap_c,
                                                      int cap_n, T gm1h, T half_eps, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_q = reinterpret_cast<T *>(smem_raw);
    T *s_adt = s_q + 4 * cap_c;
    T *s_u = s_adt + cap_c;
    T *s_v = s_u + cap_c;
    T *s_p = s_v + cap_c;
    T *s_H = s_p + cap_c;
    T *s_inc = s_H + cap_c;
    T *s_x = s_inc + 4 * cap_c;
    int *s_gid = reinterpret_cast<int *>(s_x + 2 * cap_n);

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nn = d.fp_count[0], nc = d.fp_count[1];
    // the carve-up above must fit the launch's dynamic shared memory and
    // the block's footprint its capacity; otherwise record and return
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gid + cap_c) - smem_raw) > dynamic_smem_bytes() ||
        nc > cap_c || nn > cap_n || d.nitems > (int)blockDim.x) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpn = fp + d.fp_start[0];
    const int32_t *fpc = fp + d.fp_start[1];
    // the thread's own local map and colour do not depend on the staging:
    // issue their loads first so they overlap it
    const bool active = tid < d.nitems;
    ushort4 l = make_ushort4(0, 0, 0, 0);
    int my_color = -1;
    if (active) {
        l = lmap[d.item_start + tid];
        if (INC == kIncColor) my_color = tcolor[d.item_start + tid];
    }

    // Staging: the cells (q, adt, per-cell primitives, the current res,
    // global id, gather row) and the nodes.  When the warps that hold no
    // cell are enough, they take the nodes (at most two per thread), so
    // that node loads do not follow the cell arithmetic on the cell warps.
    auto stage_prims = [&](int i, int g) {
        T r, ru, rv, E;
        if (SOA) {
            r = q[g];
            ru = q[ncell + g];
            rv = q[2 * ncell + g];
            E = q[3 * ncell + g];
        } else if (sizeof(T) == 8) {
            const double2 *q2 = reinterpret_cast<const double2 *>(q) + 2 * (int64_t)g;
            double2 a = q2[0], b = q2[1];
            r = (T)a.x;
            ru = (T)a.y;
            rv = (T)b.x;
            E = (T)b.y;
        } else {
            float4 a = reinterpret_cast<const float4 *>(q)[g];
            r = (T)a.x;
            ru = (T)a.y;
            rv = (T)a.z;
            E = (T)a.w;
        }
        T u, v, p, H;
        cell_prims_half(r, ru, rv, E, gm1h, u, v, p, H);
        s_q[i] = r;
        s_q[cap_c + i] = ru;
        s_q[2 * cap_c + i] = rv;
        s_q[3 * cap_c + i] = E;
        s_u[i] = u;
        s_v[i] = v;
        s_p[i] = p;
        s_H[i] = H;
    };
    auto stage_aux = [&](int i, int g) {  // before the dependent-launch wait
        s_adt[i] = adt[g];
        s_gid[i] = g;
    };
    // res is prefetched: increments accumulate onto it in shared memory and
    // the write-back is a plain store (blocks of one colour share no cell,
    // so no other block touches these values meanwhile); the previous
    // colour's launch writes it, so this follows the dependent-launch wait
    auto stage_res = [&](int i, int g) {
        T r0, r1, r2, r3;
        load_res<T, SOA>(res, ncell, g, r0, r1, r2, r3);
        s_inc[i] = r0;
        s_inc[cap_c + i] = r1;
        s_inc[2 * cap_c + i] = r2;
        s_inc[3 * cap_c + i] = r3;
    };
    auto stage_node = [&](int i) {
        int g = fpn[i];
        T px, py;
        if (SOA) {
            px = x[g];
            py = x[nnode + g];
        } else if (sizeof(T) == 8) {
            double2 a = reinterpret_cast<const double2 *>(x)[g];
            px = (T)a.x;
            py = (T)a.y;
        } else {
            float2 a = reinterpret_cast<const float2 *>(x)[g];
            px = (T)a.x;
            py = (T)a.y;
        }
        s_x[i] = px;
        s_x[cap_n + i] = py;
    };
    const int ncw = (nc + 31) & ~31, nfree = (int)blockDim.x - ncw;
    const bool split = nfree >= 32 && 2 * nfree >= nn;
    for (int i = tid; i < nc; i += blockDim.x) {
        const int g = fpc[i];
        stage_prims(i, g);
        stage_aux(i, g);
        mp_pdl_wait();
        stage_res(i, g);
    }
    if (split) {
        if (tid >= ncw) {
            const int i = tid - ncw;
            if (i < nn) stage_node(i);
            if (i + nfree < nn) stage_node(i + nfree);
        }
    } else {
        for (int i = tid; i < nn; i += blockDim.x) stage_node(i);
    }
    __syncthreads();

    T f[4] = {T(0), T(0), T(0), T(0)};
    int c1 = 0, c2 = 0;
    if (active) {
        const int na = l.x, nb = l.y;
        c1 = l.z;
        c2 = l.w;
        T nx = s_x[cap_n + na] - s_x[cap_n + nb];
        T ny = s_x[nb] - s_x[na];
        edge_flux(nx, ny, s_q[c1], s_q[cap_c + c1], s_q[2 * cap_c + c1], s_q[3 * cap_c + c1], s_u[c1], s_v[c1],
                  s_p[c1], s_H[c1], s_adt[c1], s_q[c2], s_q[cap_c + c2], s_q[2 * cap_c + c2], s_q[3 * cap_c + c2],
                  s_u[c2], s_v[c2], s_p[c2], s_H[c2], s_adt[c2], half_eps, f);
    }
    if (INC == kIncShuffle) {
        // warp-aggregated shared-memory atomics: one barrier
        const unsigned act = __ballot_sync(0xffffffffu, active);
        if (active) {
            T g[4] = {-f[0], -f[1], -f[2], -f[3]};
            warp_aggregated_add<T, 4>(act, c1, f, s_inc, cap_c);
            warp_aggregated_add<T, 4>(act, c2, g, s_inc, cap_c);
        }
        __syncthreads();
    } else if (INC == kIncAtomic) {
        // shared-memory atomics instead of thread colours: one barrier
        if (active) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                atomicAdd(s_inc + k * cap_c + c1, f[k]);
                atomicAdd(s_inc + k * cap_c + c2, -f[k]);
            }
        }
        __syncthreads();
    } else {
        // thread-coloured increments in shared memory (Algorithm 1)
        for (int c = 0; c < d.ncolors; ++c) {
            if (my_color == c) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    s_inc[k * cap_c + c1] += f[k];
                    s_inc[k * cap_c + c2] -= f[k];
                }
            }
            __syncthreads();
        }
    }
    // one coalesced store per footprint cell
    for (int i = tid; i < nc; i += blockDim.x) {
        int g = s_gid[i];
        if (SOA) {
#pragma unroll
            for (int k = 0; k < 4; ++k) res[k * ncell + g] = s_inc[k * cap_c + i];
        } else if (sizeof(T) == 8) {
            double2 *r2 = reinterpret_cast<double2 *>(res) + 2 * (int64_t)g;
            r2[0] = make_double2((double)s_inc[i], (double)s_inc[cap_c + i]);
            r2[1] = make_double2((double)s_inc[2 * cap_c + i], (double)s_inc[3 * cap_c + i]);
        } else {
            reinterpret_cast<float4 *>(res)[g] = make_float4((float)s_inc[i], (float)s_inc[cap_c + i],
                                                              (float)s_inc[2 * cap_c + i], (float)s_inc[3 * cap_c + i]);
        }
    }
}

// ------------------------------------------------------- GLOBAL / ATOMIC

// The gather form of the staged kernel, with every value another thread
// reads stored as one vector record in shared memory:
//   T  cq[cap_c][4]   rho, ru, rv, E
//   T  cp[cap_c][4]   u/2, v/2, p/2, H        (cell_prims_half)
//   T  cr[cap_c][4]   res, prefetched at staging
//   T  f[2 S + 1][4]  FP32: the flux of every edge of the block (S =
//                     blockDim) at [e], its negation at [S + e], zeros at
//                     [2 S];  FP64: [S + 1][4], the fluxes (and a zero row)
//   T  x[cap_n][2]    coordinates of the nodes
//   ushort4 ge[gw4][cap_c]  the cells' gather rows, as indices into f
//   int gid[cap_c]
//   T  ca[cap_c]      eps adt / 2
// Per block: stage (cells on the first warps, nodes on the warps that hold
// no cell when they are enough; each gather entry "local edge x 16 + map
// slot" becomes the index of +f (the edge's first cell slot) or -f (its
// second), padding the zero row), barrier, one flux per thread stored with
// its negation, barrier, and the thread that staged a cell adds the rows
// its entries index onto the prefetched res and stores it: a fixed order,
// deterministic, with no sign or padding test after the last barrier.  In
// FP64, whose pipe bounds the kernel, no negated copy is stored and the
// rows keep the plan's entries: the gather adds sign x flux (one FMA per
// value, padding entries 0 times row 0), measured 3 % faster there.
// GW1: every cell has at most 4 increments in the block (one gather row),
// the case of quadrilateral meshes.
template <typename T>
__host__ __device__ constexpr int res_g_smem_per_cell()
{
    return 13 * (int)sizeof(T) + 4;
}

// Arguments of the gather-form kernels.
template <typename T>
struct res_g_args {
    const mp_block_desc *desc;
    const ushort4 *lmap;
    const ushort4 *gat;
    const int32_t *fp;
    const T *x, *q, *adt;
    T *res;
    int64_t nnode, ncell;
    int gw4, cap_c, cap_n;
    T gm1h, half_eps;  // (gam-1)/2, eps/2
    int *err;
};

// One block (index b of the descriptor table) of the gather form.
// PERSIST: the block runs inside a persistent launch: no dependent-launch
// wait, and res is read through L2 (another CTA of the launch may have
// written it before the last grid barrier).  Returns false, with the error
// word set, when the block does not fit the launch.
template <typename T, bool SOA, bool GW1, bool PERSIST>
__device__ __forceinline__ bool res_block_g(const res_g_args<T> &A, int b)
{
    const ushort4 *__restrict__ lmap = A.lmap;
    const ushort4 *__restrict__ gat = A.gat;
    const int32_t *__restrict__ fp = A.fp;
    const T *__restrict__ x = A.x;
    const T *__restrict__ q = A.q;
    const T *__restrict__ adt = A.adt;
    T *__restrict__ res = A.res;
    const int64_t nnode = A.nnode, ncell = A.ncell;
    const int gw4 = A.gw4, cap_c = A.cap_c, cap_n = A.cap_n;
    const T gm1h = A.gm1h, half_eps = A.half_eps;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bd = blockDim.x, tid = threadIdx.x;
    const int nrow = GW1 ? 1 : gw4;
    T *s_cq = reinterpret_cast<T *>(smem_raw);
    T *s_cp = s_cq + 4 * cap_c;
    T *s_cr = s_cp + 4 * cap_c;
    T *s_f = s_cr + 4 * cap_c;
    constexpr bool NEG_ROWS = sizeof(T) == 4;  // negated copies of the fluxes in f
    const int nfrow = NEG_ROWS ? 2 * bd + 1 : bd + 1;
    T *s_x = s_f + 4 * nfrow;
    ushort4 *s_ge = reinterpret_cast<ushort4 *>(s_x + 2 * cap_n);
    int *s_gid = reinterpret_cast<int *>(s_ge + nrow * cap_c);
    T *s_ca = reinterpret_cast<T *>(s_gid + cap_c + (sizeof(T) == 8 ? (cap_c & 1) : 0));

    const mp_block_desc d = A.desc[b];
    const int nn = d.fp_count[0], nc = d.fp_count[1];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_ca + cap_c) - smem_raw) > dynamic_smem_bytes() ||
        nc > cap_c || nn > cap_n || d.nitems > bd || gw4 < 1 || gw4 > (GW1 ? 1 : 4)) {
        if (tid == 0) atomicExch(A.err, MP_DEVERR_SMEM);
        return false;
    }
    const int32_t *fpn = fp + d.fp_start[0];
    const int32_t *fpc = fp + d.fp_start[1];
    const bool active = tid < d.nitems;
    ushort4 l = make_ushort4(0, 0, 0, 0);
    if (active) l = lmap[d.item_start + tid];  // independent of the staging: issued first
    if (tid == 0) st_row4(s_f, nfrow - 1, T(0), T(0), T(0), T(0));

    // gather entry -> index of the row of f it adds
    const unsigned zero_row = (unsigned)nfrow - 1u;
    auto to_row = [&](unsigned e) -> unsigned short {
        const unsigned minus = (e & 15u) == 3u ? (NEG_ROWS ? (unsigned)bd : 0x8000u) : 0u;
        return (unsigned short)(e == 0xFFFFu ? zero_row : (e >> 4) + minus);
    };
    // cells: q, adt and the gather rows, then res after the dependent-launch
    // wait (the previous colour's launch writes it), then the primitives
    for (int i = tid; i < nc; i += bd) {
        const int g = fpc[i];
        T r, ru, rv, E;
        load_cell<T, SOA>(q, ncell, g, r, ru, rv, E);
        const T a = adt[g];
        const ushort4 *rw = gat + (int64_t)(d.fp_start[1] + i) * gw4;
        for (int h = 0; h < nrow; ++h) {
            const ushort4 e4 = rw[h];
            s_ge[h * cap_c + i] =
                NEG_ROWS ? make_ushort4(to_row(e4.x), to_row(e4.y), to_row(e4.z), to_row(e4.w)) : e4;
        }
        s_gid[i] = g;
        if (!PERSIST) mp_pdl_wait();
        T r0, r1, r2, r3;
        load_res<T, SOA, PERSIST>(res, ncell, g, r0, r1, r2, r3);
        T u, v, p, H;
        cell_prims_half(r, ru, rv, E, gm1h, u, v, p, H);
        st_row4(s_cq, i, r, ru, rv, E);
        st_row4(s_cp, i, u, v, p, H);
        st_row4(s_cr, i, r0, r1, r2, r3);
        s_ca[i] = a * half_eps;
    }
    // nodes: on the warps that stage no cell when they are enough (at most
    // two nodes per thread, both loads issued before either is stored)
    auto stage_nodes = [&](int i0, int i1) {
        T px0 = T(0), py0 = T(0), px1 = T(0), py1 = T(0);
        if (i0 < nn) load_node<T, SOA>(x, nnode, fpn[i0], px0, py0);
        if (i1 < nn) load_node<T, SOA>(x, nnode, fpn[i1], px1, py1);
        if (i0 < nn) {
            s_x[2 * i0] = px0;
            s_x[2 * i0 + 1] = py0;
        }
        if (i1 < nn) {
            s_x[2 * i1] = px1;
            s_x[2 * i1 + 1] = py1;
        }
    };
    const int ncw = (nc + 31) & ~31, nfree = bd - ncw;
    if (nfree >= 32 && 2 * nfree >= nn) {
        if (tid >= ncw) stage_nodes(tid - ncw, tid - ncw + nfree);
    } else {
        for (int i = tid; i < nn; i += 2 * bd) stage_nodes(i, i + bd);
    }
    __syncthreads();

    if (active) {
        const int na = l.x, nb = l.y, c1 = l.z, c2 = l.w;
        const T nx = s_x[2 * na + 1] - s_x[2 * nb + 1];
        const T ny = s_x[2 * nb] - s_x[2 * na];
        T r1, ru1, rv1, E1, u1, v1, p1, H1, r2, ru2, rv2, E2, u2, v2, p2, H2;
        ld_row4(s_cq, c1, r1, ru1, rv1, E1);
        ld_row4(s_cp, c1, u1, v1, p1, H1);
        ld_row4(s_cq, c2, r2, ru2, rv2, E2);
        ld_row4(s_cp, c2, u2, v2, p2, H2);
        T f[4];
        // eps adt / 2 is folded in per cell: mu = a1 + a2
        edge_flux(nx, ny, r1, ru1, rv1, E1, u1, v1, p1, H1, s_ca[c1], r2, ru2, rv2, E2, u2, v2, p2, H2, s_ca[c2],
                  T(1), f);
        st_row4(s_f, tid, f[0], f[1], f[2], f[3]);
        if (NEG_ROWS) st_row4(s_f, bd + tid, flip_sign(f[0]), flip_sign(f[1]), flip_sign(f[2]), flip_sign(f[3]));
    }
    __syncthreads();

    for (int i = tid; i < nc; i += bd) {
        T a0, a1, a2, a3;
        ld_row4(s_cr, i, a0, a1, a2, a3);
        for (int h = 0; h < nrow; ++h) {
            const ushort4 e4 = s_ge[h * cap_c + i];
            const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                T v0, v1, v2, v3;
                if (NEG_ROWS) {
                    ld_row4(s_f, es[j], v0, v1, v2, v3);
                    a0 += v0;
                    a1 += v1;
                    a2 += v2;
                    a3 += v3;
                } else {  // raw entry: +f, -f, or padding (0 times row 0)
                    const unsigned e = es[j];
                    const bool valid = e != 0xFFFFu;
                    // entries ascend, padding last, and the data-point order
                    // puts a block's halo cells (fewer in-block edges) after
                    // its interior cells: warps of halo cells skip their
                    // trailing padding entries as a whole (FP64 only: in the
                    // issue-bound FP32 and double-word sums the vote costs
                    // more than the skipped additions)
                    if (__any_sync(__activemask(), valid)) {
                        const T sg = !valid ? T(0) : ((e & 15u) == 3u ? T(-1) : T(1));
                        ld_row4(s_f, valid ? (int)(e >> 4) : 0, v0, v1, v2, v3);
                        a0 += sg * v0;
                        a1 += sg * v1;
                        a2 += sg * v2;
                        a3 += sg * v3;
                    }
                }
            }
        }
        const int64_t g = s_gid[i];
        if (SOA) {
            res[g] = a0;
            res[ncell + g] = a1;
            res[2 * ncell + g] = a2;
            res[3 * ncell + g] = a3;
        } else if (sizeof(T) == 8) {
            double2 *r2p = reinterpret_cast<double2 *>(res) + 2 * g;
            r2p[0] = make_double2((double)a0, (double)a1);
            r2p[1] = make_double2((double)a2, (double)a3);
        } else {
            reinterpret_cast<float4 *>(res)[g] = make_float4((float)a0, (float)a1, (float)a2, (float)a3);
        }
    }
    return true;
}

// One launch per block colour: CTA k takes block block0 + k.
template <typename T, bool SOA, bool GW1>
__global__ void __maxnreg__(sizeof(T) == 4 ? 32 : 48) res_calc_hier_g(res_g_args<T> A, int block0)
{
    mp_pdl_trigger();
    res_block_g<T, SOA, GW1, false>(A, block0 + (int)blockIdx.x);
}

// One persistent (cooperative) launch for all block colours: the resident
// CTAs take the blocks of a colour one at a time from a counter (a CTA that
// finishes early takes the next block, so the colour's end is not held back
// by a fixed share) and meet at a bounded grid-wide barrier before the next
// colour, whose blocks may share cells with this one's.  A barrier that runs
// out leaves MP_ETIMEOUT in the error word and the CTAs return.
// bar[0]: barrier arrivals; bar[1 + c]: blocks of colour c taken; all 0 at
// launch.
template <typename T, bool SOA, bool GW1>
__global__ void __maxnreg__(sizeof(T) == 4 ? 32 : 48) res_calc_hier_gp(res_g_args<T> A,
                                                                       const int32_t *__restrict__ color_off,
                                                                       int ncolors, unsigned *bar)
{
    __shared__ int s_next;
    for (int c = 0; c < ncolors; ++c) {
        const int b0 = color_off[c], nb = color_off[c + 1] - b0;
        for (;;) {
            if (threadIdx.x == 0) s_next = (int)atomicAdd(bar + 1 + c, 1u);
            __syncthreads();
            const int k = s_next;
            if (k >= nb) break;
            if (!res_block_g<T, SOA, GW1, true>(A, b0 + k)) return;
            __syncthreads();  // the next block reuses the shared memory and s_next
        }
        if (c + 1 < ncolors && !mp_grid_barrier(bar, (unsigned)(c + 1) * gridDim.x, MP_GRID_WAIT_NS, A.err)) return;
    }
}

// One thread per edge of [e0, e1): gather from global, flux, then either a
// plain read-add-write (edges of one colour share no cell) or atomics.
template <typename T, bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256) res_calc_direct(int e0, int e1, const int32_t *__restrict__ e2n,
                                                       const int32_t *__restrict__ e2c, const T *__restrict__ x,
                                                       const T *__restrict__ q, const T *__restrict__ adt,
                                                       T *__restrict__ res, int64_t nnode, int64_t ncell, T gm1h,
                                                       T half_eps)
{
    mp_pdl_trigger();
    int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    int2 nab = reinterpret_cast<const int2 *>(e2n)[e];
    int2 cc = reinterpret_cast<const int2 *>(e2c)[e];
    T xa, ya, xb, yb;
    load_node<T, SOA>(x, nnode, nab.x, xa, ya);
    load_node<T, SOA>(x, nnode, nab.y, xb, yb);
    T r1, ru1, rv1, E1, r2, ru2, rv2, E2;
    load_cell<T, SOA>(q, ncell, cc.x, r1, ru1, rv1, E1);
    load_cell<T, SOA>(q, ncell, cc.y, r2, ru2, rv2, E2);
    T a1 = adt[cc.x], a2 = adt[cc.y];
    T u1, v1, p1, H1, u2, v2, p2, H2;
    cell_prims_half(r1, ru1, rv1, E1, gm1h, u1, v1, p1, H1);
    cell_prims_half(r2, ru2, rv2, E2, gm1h, u2, v2, p2, H2);
    T f[4];
    edge_flux(ya - yb, xb - xa, r1, ru1, rv1, E1, u1, v1, p1, H1, a1, r2, ru2, rv2, E2, u2, v2, p2, H2, a2, half_eps, f);
    if (!ATOMIC) mp_pdl_wait();  // res: read-add-written by the previous colour's launch
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int64_t j1 = SOA ? k * ncell + cc.x : 4 * (int64_t)cc.x + k;
        int64_t j2 = SOA ? k * ncell + cc.y : 4 * (int64_t)cc.y + k;
        if (ATOMIC) {
            atomicAdd(res + j1, f[k]);
            atomicAdd(res + j2, -f[k]);
        } else {
            res[j1] += f[k];
            res[j2] -= f[k];
        }
    }
}

// Step 1 of the temporary-array method (Sec. 2.1): the increments of edge
// e for its two cells go to scratch[(2e + slot) * 4 + k] (+f, -f).
template <typename T, bool SOA>
__global__ void __launch_bounds__(256) res_calc_step1(int n, const int32_t *__restrict__ e2n,
                                                      const int32_t *__restrict__ e2c, const T *__restrict__ x,
                                                      const T *__restrict__ q, const T *__restrict__ adt,
                                                      T *__restrict__ scratch, int64_t nnode, int64_t ncell, T gm1h,
                                                      T half_eps)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int2 nab = reinterpret_cast<const int2 *>(e2n)[e];
    int2 cc = reinterpret_cast<const int2 *>(e2c)[e];
    T xa, ya, xb, yb;
    load_node<T, SOA>(x, nnode, nab.x, xa, ya);
    load_node<T, SOA>(x, nnode, nab.y, xb, yb);
    T r1, ru1, rv1, E1, r2, ru2, rv2, E2;
    load_cell<T, SOA>(q, ncell, cc.x, r1, ru1, rv1, E1);
    load_cell<T, SOA>(q, ncell, cc.y, r2, ru2, rv2, E2);
    T u1, v1, p1, H1, u2, v2, p2, H2;
    cell_prims_half(r1, ru1, rv1, E1, gm1h, u1, v1, p1, H1);
    cell_prims_half(r2, ru2, rv2, E2, gm1h, u2, v2, p2, H2);
    T f[4];
    edge_flux(ya - yb, xb - xa, r1, ru1, rv1, E1, u1, v1, p1, H1, adt[cc.x], r2,
              ru2, rv2, E2, u2, v2, p2, H2, adt[cc.y], half_eps, f);
    T *o = scratch + 8 * (int64_t)e;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        o[k] = f[k];
        o[4 + k] = -f[k];
    }
}

// ------------------------------------------------------------- bres_calc

// Far-field boundary edges: q_b = (q_c + qinf)/2,
// res[c] += F(q_b).n + eps adt_c (q_c - qinf).
template <typename T, bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256) bres_calc_direct(int e0, int e1, const int32_t *__restrict__ b2n,
                                                        const int32_t *__restrict__ b2c, const T *__restrict__ x,
                                                        const T *__restrict__ q, const T *__restrict__ adt,
                                                        T *__restrict__ res, int64_t nnode, int64_t ncell, T gm1,
                                                        T eps, T qi0, T qi1, T qi2, T qi3)
{
    int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    int2 nab = reinterpret_cast<const int2 *>(b2n)[e];
    int c = b2c[e];
    T xa, ya, xb, yb;
    load_node<T, SOA>(x, nnode, nab.x, xa, ya);
    load_node<T, SOA>(x, nnode, nab.y, xb, yb);
    T qc[4];
    load_cell<T, SOA>(q, ncell, c, qc[0], qc[1], qc[2], qc[3]);
    const T qi[4] = {qi0, qi1, qi2, qi3};
    T qb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) qb[k] = T(0.5) * (qc[k] + qi[k]);
    T u, v, p, H;
    cell_prims(qb[0], qb[1], qb[2], qb[3], gm1, u, v, p, H);
    T nx = ya - yb, ny = xb - xa;
    T V = u * nx + v * ny;
    T ea = eps * adt[c];
    T f[4];
    f[0] = qb[0] * V + ea * (qc[0] - qi[0]);
    f[1] = qb[1] * V + p * nx + ea * (qc[1] - qi[1]);
    f[2] = qb[2] * V + p * ny + ea * (qc[2] - qi[2]);
    f[3] = H * V + ea * (qc[3] - qi[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int64_t j = SOA ? k * ncell + c : 4 * (int64_t)c + k;
        if (ATOMIC)
            atomicAdd(res + j, f[k]);
        else
            res[j] += f[k];
    }
}

// ------------------------------------------------------------- adt_calc

// Cell loop with read-only indirection: adt = sum over the 4 sides of
// (|u dy - v dx| + c sqrt(dx^2 + dy^2)) / cfl,  c = sqrt(gam p / rho).
template <typename T, bool SOA>
__global__ void __launch_bounds__(256) adt_calc_kernel(int64_t n, const int32_t *__restrict__ c2n,
                                                       const T *__restrict__ x, const T *__restrict__ q,
                                                       T *__restrict__ adt, int64_t nnode, T gam, T gm1,
                                                       T inv_cfl)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    int4 nd = reinterpret_cast<const int4 *>(c2n)[c];
    T r, ru, rv, E;
    load_cell<T, SOA>(q, n, (int)c, r, ru, rv, E);
    T ri = T(1) / r;
    T u = ru * ri, v = rv * ri;
    T p = gm1 * (E - T(0.5) * (ru * u + rv * v));
    T cs = sqrt(gam * p * ri);
    T px[4], py[4];
    load_node<T, SOA>(x, nnode, nd.x, px[0], py[0]);
    load_node<T, SOA>(x, nnode, nd.y, px[1], py[1]);
    load_node<T, SOA>(x, nnode, nd.z, px[2], py[2]);
    load_node<T, SOA>(x, nnode, nd.w, px[3], py[3]);
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T dx = px[(k + 1) & 3] - px[k];
        T dy = py[(k + 1) & 3] - py[k];
        s += fabs(u * dy - v * dx) + cs * sqrt(dx * dx + dy * dy);
    }
    adt[c] = s * inv_cfl;
}

// --------------------------------------------------------------- drivers

bool check_maps(const mp_plan *P, int a0, int w0, int a1, int w1)
{
    return P->nmaps == 2 && P->maps[0].arity == a0 && P->maps[1].arity == a1 && P->maps[0].written == w0 &&
           P->maps[1].written == w1;
}

template <typename T, bool SOA>
int res_calc_t(const mp_plan *P, const void *x, const void *q, const void *adt, void *res, double gam, double eps,
               cudaStream_t s)
{
    const int64_t nnode = P->maps[0].to_size, ncell = P->maps[1].to_size;
    const T gm1h = (T)(0.5 * (gam - 1.0)), half_eps = (T)(0.5 * eps);
    const int co = P->opts.coloring;
    if (co == MP_COLOR_HIER) {
        if (P->maps[0].slot != 0 || P->maps[1].slot != 1) return MP_EPLAN;
        const int cap_n = P->stats.footprint_max[0], cap_c = P->stats.footprint_max[1];
        // default increments: gather (measured faster on GB300 in both
        // precisions: FP64 0.487 against 0.554 ms for thread colours)
        const int variant = mp_staged(P, MP_STAGED_GATHER);
        const bool gather =
            (variant == MP_STAGED_GATHER || variant == MP_STAGED_PERSISTENT) && mp_gather_ready(P);
        int *err = nullptr;
        int rc = mp_device_error_word(&err);
        if (rc != MP_OK) return rc;
        const int32_t *fp = P->dev.fp;
        const int bs = P->opts.block_size;
        bool overlap = false;  // the first launch follows the caller's work: plain stream order
        if (gather) {
            const int gw4 = P->gat_w / 4;
            const bool gw1 = gw4 == 1;
            const int smem = cap_c * res_g_smem_per_cell<T>() + cap_n * 2 * (int)sizeof(T) +
                             (sizeof(T) == 4 ? 2 * bs + 1 : bs + 1) * 4 * (int)sizeof(T) + (gw1 ? 1 : gw4) * cap_c * 8 +
                             (sizeof(T) == 8 ? 4 : 0);
            const res_g_args<T> A{P->dev.desc, reinterpret_cast<const ushort4 *>(P->dev.lmap),
                                  reinterpret_cast<const ushort4 *>(P->dev.gat), fp, (const T *)x, (const T *)q,
                                  (const T *)adt, (T *)res, nnode, ncell, gw4, cap_c, cap_n, gm1h, half_eps, err};
            if (variant == MP_STAGED_PERSISTENT) {
                auto kern = gw1 ? res_calc_hier_gp<T, SOA, true> : res_calc_hier_gp<T, SOA, false>;
                if ((rc = mp_allow_smem(kern, smem)) != MP_OK) return rc;
                int dev = 0, sms = 0, occ = 0;
                MP_CUDA_TRY(cudaGetDevice(&dev));
                MP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
                MP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, bs, smem));
                if (occ < 1) return MP_ESMEM;
                MP_CUDA_TRY(cudaMemsetAsync(P->dev.bar, 0, sizeof(unsigned) * (1 + P->ncolors), s));
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)(sms * occ));
                cfg.blockDim = dim3((unsigned)bs);
                cfg.dynamicSmemBytes = (size_t)smem;
                cfg.stream = s;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeCooperative;
                at[0].val.cooperative = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                MP_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, A, (const int32_t *)P->dev.color_off, P->ncolors,
                                               P->dev.bar));
                MP_CUDA_TRY(cudaGetLastError());
                return MP_OK;
            }
            auto kern = gw1 ? res_calc_hier_g<T, SOA, true> : res_calc_hier_g<T, SOA, false>;
            if ((rc = mp_allow_smem(kern, smem)) != MP_OK) return rc;
            for (int c = 0; c < P->ncolors; ++c) {
                int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
                if (nb == 0) continue;
                MP_CUDA_TRY(mp_launch(kern, nb, bs, smem, s, overlap, A, b0));
                overlap = true;
            }
            MP_CUDA_TRY(cudaGetLastError());
            return MP_OK;
        }
        const int smem = cap_c * res_smem_per_cell<T>() + cap_n * res_smem_per_node<T>();
        auto kern = variant == MP_STAGED_SMEM_ATOMIC ? res_calc_hier<T, SOA, kIncAtomic>
                    : variant == MP_STAGED_WARP_AGG  ? res_calc_hier<T, SOA, kIncShuffle>
                                                     : res_calc_hier<T, SOA, kIncColor>;
        if ((rc = mp_allow_smem(kern, smem)) != MP_OK) return rc;
        for (int c = 0; c < P->ncolors; ++c) {
            int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
            if (nb == 0) continue;
            MP_CUDA_TRY(mp_launch(kern, nb, bs, smem, s, overlap, P->dev.desc, b0,
                                  reinterpret_cast<const ushort4 *>(P->dev.lmap), P->dev.tcolor, fp, (const T *)x,
                                  (const T *)q, (const T *)adt, (T *)res, nnode, ncell, cap_c, cap_n, gm1h, half_eps,
                                  err));
            overlap = true;
        }
    } else if (co == MP_COLOR_TWOSTEP) {
        void *scratch = nullptr;
        int rc = mp_twostep_scratch(P, (size_t)P->from_size * 8 * sizeof(T), &scratch);
        if (rc != MP_OK) return rc;
        const int n = (int)P->from_size;
        res_calc_step1<T, SOA><<<(n + 255) / 256, 256, 0, s>>>(n, P->dev.map[0], P->dev.map[1], (const T *)x,
                                                                (const T *)q, (const T *)adt, (T *)scratch, nnode,
                                                                ncell, gm1h, half_eps);
        MP_CUDA_TRY(cudaGetLastError());
        return mp_twostep_gather(P, sizeof(T) == 8 ? MP_F64 : MP_F32, 4, scratch, res, s);
    } else {
        const bool atomic = co == MP_COLOR_ATOMIC;
        bool overlap = false;  // global colours: the same overlap as the staged launches
        for (int c = 0; c < P->ncolors; ++c) {
            int e0 = P->color_offsets[c], e1 = P->color_offsets[c + 1];
            if (e1 <= e0) continue;
            int grid = (e1 - e0 + 255) / 256;
            auto kern = atomic ? res_calc_direct<T, SOA, true> : res_calc_direct<T, SOA, false>;
            MP_CUDA_TRY(mp_launch(kern, grid, 256, 0, s, overlap && !atomic, e0, e1, P->dev.map[0], P->dev.map[1],
                                  (const T *)x, (const T *)q, (const T *)adt, (T *)res, nnode, ncell, gm1h,
                                  half_eps));
            overlap = true;
        }
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

template <typename T, bool SOA>
int bres_calc_t(const mp_plan *P, const void *x, const void *q, const void *adt, void *res, const double *qinf,
                double gam, double eps, cudaStream_t s)
{
    const int64_t nnode = P->maps[0].to_size, ncell = P->maps[1].to_size;
    const bool atomic = P->opts.coloring == MP_COLOR_ATOMIC;
    // HIER plans of this loop run their block colours as global colours
    // would: each block colour's iterations share no cell.
    for (int c = 0; c < P->ncolors; ++c) {
        int e0, e1;
        if (P->opts.coloring == MP_COLOR_HIER) {
            e0 = P->block_offsets[P->color_offsets[c]];
            e1 = P->block_offsets[P->color_offsets[c + 1]];
        } else {
            e0 = P->color_offsets[c];
            e1 = P->color_offsets[c + 1];
        }
        if (e1 <= e0) continue;
        int grid = (e1 - e0 + 255) / 256;
        auto kern = atomic ? bres_calc_direct<T, SOA, true> : bres_calc_direct<T, SOA, false>;
        kern<<<grid, 256, 0, s>>>(e0, e1, P->dev.map[0], P->dev.map[1], (const T *)x, (const T *)q, (const T *)adt,
                                  (T *)res, nnode, ncell, (T)(gam - 1.0), (T)eps, (T)qinf[0], (T)qinf[1], (T)qinf[2],
                                  (T)qinf[3]);
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

bool data_ok(std::initializer_list<const void *> ptrs)
{
    for (const void *p : ptrs)
        if (!p || !aligned16(p)) return false;
    return true;
}

}  // namespace

extern "C" int loop_res_calc(const mp_plan *P, int32_t dtype, const void *x, const void *q, const void *adt,
                             void *res, double gam, double eps, void *stream)
{
    if (!P || (dtype != MP_F64 && dtype != MP_F32 && dtype != MP_F64_DW)) return MP_EINVAL;
    // edge->node may be marked written: an adjoint plan (both maps coloured)
    // also runs the forward loop in the same numbering
    if (!check_maps(P, 2, 0, 2, 1) && !check_maps(P, 2, 1, 2, 1)) return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    if (!data_ok({x, q, adt, res})) return MP_EINVAL;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    if (dtype == MP_F64_DW) return mp_res_calc_dw(P, x, q, adt, res, gam, eps, stream);
    if (P->opts.coloring == MP_COLOR_HIER && mp_staged(P, MP_STAGED_SIMPLE) == MP_STAGED_PIPELINED) {
        rc = mp_res_calc_pipe(P, dtype, x, q, adt, res, gam, eps, stream);
        if (rc != MP_EPLAN) return rc;  // otherwise the layout does not fit: one block per CTA
    }
    cudaStream_t s = as_stream(stream);
    bool soa = P->opts.layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64)
        return soa ? res_calc_t<double, true>(P, x, q, adt, res, gam, eps, s)
                   : res_calc_t<double, false>(P, x, q, adt, res, gam, eps, s);
    return soa ? res_calc_t<float, true>(P, x, q, adt, res, gam, eps, s)
               : res_calc_t<float, false>(P, x, q, adt, res, gam, eps, s);
}

extern "C" int loop_bres_calc(const mp_plan *P, int32_t dtype, const void *x, const void *q, const void *adt,
                              void *res, const double *qinf, double gam, double eps, void *stream)
{
    if (!P || !qinf || (dtype != MP_F64 && dtype != MP_F32)) return MP_EINVAL;
    if (!check_maps(P, 2, 0, 1, 1)) return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    if (!data_ok({x, q, adt, res})) return MP_EINVAL;
    // the direct kernels read the global maps: GLOBAL or ATOMIC plans; HIER
    // plans (which keep no global maps) and TWOSTEP plans are rejected here
    if (P->opts.coloring == MP_COLOR_HIER || P->opts.coloring == MP_COLOR_TWOSTEP) return MP_EPLAN;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    cudaStream_t s = as_stream(stream);
    bool soa = P->opts.layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64)
        return soa ? bres_calc_t<double, true>(P, x, q, adt, res, qinf, gam, eps, s)
                   : bres_calc_t<double, false>(P, x, q, adt, res, qinf, gam, eps, s);
    return soa ? bres_calc_t<float, true>(P, x, q, adt, res, qinf, gam, eps, s)
               : bres_calc_t<float, false>(P, x, q, adt, res, qinf, gam, eps, s);
}

extern "C" int loop_adt_calc(const mp_plan *P, int32_t dtype, const void *x, const void *q, void *adt, double gam,
                             double cfl, void *stream)
{
    if (!P || (dtype != MP_F64 && dtype != MP_F32) || !(cfl > 0)) return MP_EINVAL;
    if (P->nmaps != 1 || P->maps[0].arity != 4) return MP_EPLAN;
    if (P->opts.coloring == MP_COLOR_HIER) return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    if (!data_ok({x, q, adt})) return MP_EINVAL;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    cudaStream_t s = as_stream(stream);
    bool soa = P->opts.layout == MP_LAYOUT_SOA;
    int64_t n = P->from_size, nnode = P->maps[0].to_size;
    int grid = (int)((n + 255) / 256);
    if (dtype == MP_F64) {
        auto k = soa ? adt_calc_kernel<double, true> : adt_calc_kernel<double, false>;
        k<<<grid, 256, 0, s>>>(n, P->dev.map[0], (const double *)x, (const double *)q, (double *)adt, nnode, gam,
                               gam - 1.0, 1.0 / cfl);
    } else {
        auto k = soa ? adt_calc_kernel<float, true> : adt_calc_kernel<float, false>;
        k<<<grid, 256, 0, s>>>(n, P->dev.map[0], (const float *)x, (const float *)q, (float *)adt, nnode,
                               (float)gam, (float)(gam - 1.0), (float)(1.0 / cfl));
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}
