// Increment-only loops: indirect increments with (almost) no indirect reads.
//
//   space_disc  edges -> 2 cells (Sec. 3.1.2, the access pattern of Volna's
//               SpaceDiscretization): per edge 7 values and 1 integer read
//               directly, per cell 1 value read (the inverse area) and 4
//               incremented.  With d = (F0, F1, F2, P, L, nx, ny):
//                 w = L (F0, F1 + P nx, F2 + P ny, P)
//                 res[c1] -= w / A[c1];  res[c2] += w / A[c2] unless the
//                 edge is a boundary edge (flag 1, its cell listed twice).
//   getacc      cells -> 4 nodes (Sec. 3.1.3, the access pattern of
//               BookLeaf's getacc_scatter): per cell 17 values read directly,
//               (rho, m[4], w[4], fx[4], fy[4]); node k of the cell gets
//               (m_k, rho w_k, fx_k, fy_k).
//
// The staged (HIER) kernels stage only the written set: its current values
// (prefetched, so the write-back is a plain store) and, for space_disc, the
// one value read per cell.  The direct data are read once, by their own
// thread.  TWOSTEP plans run the owner-computes form below.  Increments: gather (the default: each thread stores its
// increments in shared memory, one barrier, every footprint point sums them
// through the plan's block-local inverse map) or thread colours (Algorithm
// 1, MP_STAGED_SIMPLE).  GLOBAL plans run one launch per colour with plain
// read-add-writes, ATOMIC plans one launch with atomics.
#include "common.cuh"

namespace {

constexpr int kIncColor = 0, kIncGather = 2;

// -------------------------------------------------------------- space_disc

template <typename T, bool SOA>
__device__ __forceinline__ void space_disc_w(const T *__restrict__ ed, int64_t nedge, int64_t e, T w[4])
{
    T d[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) d[k] = SOA ? ed[k * nedge + e] : ed[7 * e + k];
    const T L = d[4];
    w[0] = L * d[0];
    w[1] = L * (d[1] + d[3] * d[5]);
    w[2] = L * (d[2] + d[3] * d[6]);
    w[3] = L * d[3];
}

template <typename T, bool SOA>
__device__ __forceinline__ T *res_at(T *res, int64_t ncell, int64_t c, int k)
{
    return SOA ? res + k * ncell + c : res + 4 * c + k;
}

// Shared memory for cap cells and cap_f threads:
//   ushort4 ge[gw4][cap]   (gather only)
//   T inc[4][cap]          (res prefetched, incremented)
//   T ia[cap]
//   T f[4][cap_f]          (gather only)
//   int flag[cap_f]        (gather only)
//   int gid[cap]
template <typename T, bool SOA, int INC>
__global__ void __launch_bounds__(1024) space_disc_hier(const mp_block_desc *__restrict__ desc, int block0,
                                                        const ushort4 *__restrict__ lmap,
                                                        const uint8_t *__restrict__ tcolor,
                                                        const ushort4 *__restrict__ gat, int gw4,
                                                        const int32_t *__restrict__ fp, const T *__restrict__ ed,
                                                        const int32_t *__restrict__ eflag,
                                                        const T *__restrict__ inv_area, T *__restrict__ res,
                                                        int64_t nedge, int64_t ncell, int cap, int cap_f,
                                                        int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ushort4 *s_ge = reinterpret_cast<ushort4 *>(smem_raw);
    T *s_inc = reinterpret_cast<T *>(s_ge + (INC == kIncGather ? gw4 * cap : 0));
    T *s_ia = s_inc + 4 * cap;
    T *s_f = s_ia + cap;
    int *s_flag = reinterpret_cast<int *>(s_f + (INC == kIncGather ? 4 * cap_f : 0));
    int *s_gid = s_flag + (INC == kIncGather ? cap_f : 0);

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nc = d.fp_count[0];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gid + cap) - smem_raw) > dynamic_smem_bytes() || nc > cap ||
        d.nitems > (int)blockDim.x ||
        (INC == kIncGather && ((int)blockDim.x > cap_f || gw4 < 1 || gw4 > 4))) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpc = fp + d.fp_start[0];
    const bool active = tid < d.nitems;
    const int64_t e = d.item_start + tid;
    // the thread's own edge: direct data, flag, local cells, colour
    T w[4] = {T(0), T(0), T(0), T(0)};
    int flag = 1, c1 = 0, c2 = 0, my_color = -1;
    if (active) {
        const ushort4 l = lmap[e];
        c1 = l.x;
        c2 = l.y;
        flag = eflag[e];
        if (INC == kIncColor) my_color = tcolor[e];
        space_disc_w<T, SOA>(ed, nedge, e, w);
    }
    for (int i = tid; i < nc; i += blockDim.x) {
        const int g = fpc[i];
        s_ia[i] = inv_area[g];
        s_gid[i] = g;
        if (INC == kIncGather) {
            const ushort4 *row = gat + (int64_t)(d.fp_start[0] + i) * gw4;
            for (int h = 0; h < gw4; ++h) s_ge[h * cap + i] = row[h];
        }
        mp_pdl_wait();  // res: written by the previous colour's launch
#pragma unroll
        for (int k = 0; k < 4; ++k) s_inc[k * cap + i] = *res_at<T, SOA>(res, ncell, g, k);
    }
    if constexpr (INC == kIncGather) {
        if (active) {
#pragma unroll
            for (int k = 0; k < 4; ++k) s_f[k * cap_f + tid] = w[k];
            s_flag[tid] = flag;
        }
        __syncthreads();
        // each cell: -w of the edges it is the first cell of, +w of the
        // interior edges it is the second cell of, over its inverse area
        for (int i = tid; i < nc; i += blockDim.x) {
            T a[4] = {T(0), T(0), T(0), T(0)};
            for (int h = 0; h < gw4; ++h) {
                const ushort4 e4 = s_ge[h * cap + i];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned en = es[j];
                    if (en == 0xFFFFu) continue;
                    const int t = (int)(en >> 4);
                    const bool second = (en & 15u) == 1u;
                    if (second && s_flag[t]) continue;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const T v = s_f[k * cap_f + t];
                        a[k] = second ? a[k] + v : a[k] - v;
                    }
                }
            }
            const T ia = s_ia[i];
            const int g = s_gid[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) *res_at<T, SOA>(res, ncell, g, k) = s_inc[k * cap + i] + ia * a[k];
        }
    } else {
        __syncthreads();
        for (int c = 0; c < d.ncolors; ++c) {
            if (my_color == c) {
                const T ia1 = s_ia[c1];
#pragma unroll
                for (int k = 0; k < 4; ++k) s_inc[k * cap + c1] -= ia1 * w[k];
                if (!flag) {
                    const T ia2 = s_ia[c2];
#pragma unroll
                    for (int k = 0; k < 4; ++k) s_inc[k * cap + c2] += ia2 * w[k];
                }
            }
            __syncthreads();
        }
        for (int i = tid; i < nc; i += blockDim.x) {
            const int g = s_gid[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) *res_at<T, SOA>(res, ncell, g, k) = s_inc[k * cap + i];
        }
    }
}

template <typename T, bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256) space_disc_direct(int e0, int e1, const int32_t *__restrict__ e2c,
                                                         const T *__restrict__ ed, const int32_t *__restrict__ eflag,
                                                         const T *__restrict__ inv_area, T *__restrict__ res,
                                                         int64_t nedge, int64_t ncell)
{
    mp_pdl_trigger();
    const int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    const int2 cc = reinterpret_cast<const int2 *>(e2c)[e];
    const int flag = eflag[e];
    T w[4];
    space_disc_w<T, SOA>(ed, nedge, e, w);
    const T ia1 = inv_area[cc.x], ia2 = inv_area[cc.y];
    if (!ATOMIC) mp_pdl_wait();  // res: read-add-written by the previous colour's launch
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T *p1 = res_at<T, SOA>(res, ncell, cc.x, k);
        if (ATOMIC)
            atomicAdd(p1, -ia1 * w[k]);
        else
            *p1 -= ia1 * w[k];
        if (!flag) {
            T *p2 = res_at<T, SOA>(res, ncell, cc.y, k);
            if (ATOMIC)
                atomicAdd(p2, ia2 * w[k]);
            else
                *p2 += ia2 * w[k];
        }
    }
}

// ------------------------------------------------------------------ getacc

template <typename T, bool SOA>
__device__ __forceinline__ void getacc_row(const T *__restrict__ cd, int64_t ncell, int64_t c, T v[17])
{
#pragma unroll
    for (int k = 0; k < 17; ++k) v[k] = SOA ? cd[k * ncell + c] : cd[17 * c + k];
}

// Shared memory for cap nodes and cap_f threads:
//   ushort4 ge[gw4][cap]   (gather only)
//   T inc[4][cap]          (nd prefetched, incremented)
//   T f[16][cap_f]         (gather only: node k, component a at 4 k + a)
//   int gid[cap]
template <typename T, bool SOA, int INC>
__global__ void __launch_bounds__(512) getacc_hier(const mp_block_desc *__restrict__ desc, int block0,
                                                   const ushort4 *__restrict__ lmap,
                                                   const uint8_t *__restrict__ tcolor,
                                                   const ushort4 *__restrict__ gat, int gw4,
                                                   const int32_t *__restrict__ fp, const T *__restrict__ cd,
                                                   T *__restrict__ nd, int64_t ncell, int64_t nnode, int cap,
                                                   int cap_f, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ushort4 *s_ge = reinterpret_cast<ushort4 *>(smem_raw);
    T *s_inc = reinterpret_cast<T *>(s_ge + (INC == kIncGather ? gw4 * cap : 0));
    T *s_f = s_inc + 4 * cap;
    int *s_gid = reinterpret_cast<int *>(s_f + (INC == kIncGather ? 16 * cap_f : 0));

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nn = d.fp_count[0];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gid + cap) - smem_raw) > dynamic_smem_bytes() || nn > cap ||
        d.nitems > (int)blockDim.x ||
        (INC == kIncGather && ((int)blockDim.x > cap_f || gw4 < 1 || gw4 > 4))) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpn = fp + d.fp_start[0];
    const bool active = tid < d.nitems;
    const int64_t c = d.item_start + tid;
    T v[17];
    ushort4 l = make_ushort4(0, 0, 0, 0);
    int my_color = -1;
    if (active) {
        l = lmap[c];
        if (INC == kIncColor) my_color = tcolor[c];
        getacc_row<T, SOA>(cd, ncell, c, v);
    }
    for (int i = tid; i < nn; i += blockDim.x) {
        const int g = fpn[i];
        s_gid[i] = g;
        if (INC == kIncGather) {
            const ushort4 *row = gat + (int64_t)(d.fp_start[0] + i) * gw4;
            for (int h = 0; h < gw4; ++h) s_ge[h * cap + i] = row[h];
        }
        mp_pdl_wait();  // nd: written by the previous colour's launch
#pragma unroll
        for (int k = 0; k < 4; ++k) s_inc[k * cap + i] = SOA ? nd[k * nnode + g] : nd[4 * (int64_t)g + k];
    }
    if constexpr (INC == kIncGather) {
        if (active) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s_f[(4 * k + 0) * cap_f + tid] = v[1 + k];
                s_f[(4 * k + 1) * cap_f + tid] = v[0] * v[5 + k];
                s_f[(4 * k + 2) * cap_f + tid] = v[9 + k];
                s_f[(4 * k + 3) * cap_f + tid] = v[13 + k];
            }
        }
        __syncthreads();
        for (int i = tid; i < nn; i += blockDim.x) {
            T a[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] = s_inc[k * cap + i];
            for (int h = 0; h < gw4; ++h) {
                const ushort4 e4 = s_ge[h * cap + i];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned en = es[j];
                    if (en == 0xFFFFu) continue;
                    const int t = (int)(en >> 4), k = (int)(en & 15u);
#pragma unroll
                    for (int comp = 0; comp < 4; ++comp) a[comp] += s_f[(4 * k + comp) * cap_f + t];
                }
            }
            const int64_t g = s_gid[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) (SOA ? nd[k * nnode + g] : nd[4 * g + k]) = a[k];
        }
    } else {
        __syncthreads();
        const int loc[4] = {l.x, l.y, l.z, l.w};
        for (int col = 0; col < d.ncolors; ++col) {
            if (my_color == col) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    s_inc[0 * cap + loc[k]] += v[1 + k];
                    s_inc[1 * cap + loc[k]] += v[0] * v[5 + k];
                    s_inc[2 * cap + loc[k]] += v[9 + k];
                    s_inc[3 * cap + loc[k]] += v[13 + k];
                }
            }
            __syncthreads();
        }
        for (int i = tid; i < nn; i += blockDim.x) {
            const int64_t g = s_gid[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) (SOA ? nd[k * nnode + g] : nd[4 * g + k]) = s_inc[k * cap + i];
        }
    }
}

template <typename T, bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256) getacc_direct(int c0, int c1, const int32_t *__restrict__ c2n,
                                                     const T *__restrict__ cd, T *__restrict__ nd, int64_t ncell,
                                                     int64_t nnode)
{
    mp_pdl_trigger();
    const int64_t c = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    const int4 n4 = reinterpret_cast<const int4 *>(c2n)[c];
    const int nk[4] = {n4.x, n4.y, n4.z, n4.w};
    T v[17];
    getacc_row<T, SOA>(cd, ncell, c, v);
    if (!ATOMIC) mp_pdl_wait();  // nd: read-add-written by the previous colour's launch
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T inc[4] = {v[1 + k], v[0] * v[5 + k], v[9 + k], v[13 + k]};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            T *p = SOA ? nd + a * nnode + nk[k] : nd + 4 * (int64_t)nk[k] + a;
            if (ATOMIC)
                atomicAdd(p, inc[a]);
            else
                *p += inc[a];
        }
    }
}

// ------------------------------------------------- owner-computes (TWOSTEP)
// The two-step method (Sec. 2.1) stores every increment in a temporary array
// and then gathers it per point through the inverse map.  The increments of
// these two loops are cheap functions of their iteration's direct data, so
// here each point recomputes them while it gathers: one launch over the
// written set, no temporary array, no atomics, fixed order (deterministic).

template <typename T, bool SOA>
__global__ void __launch_bounds__(256) space_disc_owner(const int32_t *__restrict__ inv_off,
                                                        const int32_t *__restrict__ inv_idx, const T *__restrict__ ed,
                                                        const int32_t *__restrict__ eflag,
                                                        const T *__restrict__ inv_area, T *__restrict__ res,
                                                        int64_t nedge, int64_t ncell)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int j = inv_off[c]; j < inv_off[c + 1]; ++j) {
        const int en = inv_idx[j];
        const int64_t e = en >> 1;
        const bool second = en & 1;
        if (second && eflag[e]) continue;
        T w[4];
        space_disc_w<T, SOA>(ed, nedge, e, w);
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = second ? a[k] + w[k] : a[k] - w[k];
    }
    const T ia = inv_area[c];
#pragma unroll
    for (int k = 0; k < 4; ++k) *res_at<T, SOA>(res, ncell, c, k) += ia * a[k];
}

template <typename T, bool SOA>
__global__ void __launch_bounds__(256) getacc_owner(const int32_t *__restrict__ inv_off,
                                                    const int32_t *__restrict__ inv_idx, const T *__restrict__ cd,
                                                    T *__restrict__ nd, int64_t ncell, int64_t nnode)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnode) return;
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int j = inv_off[p]; j < inv_off[p + 1]; ++j) {
        const int en = inv_idx[j];
        const int64_t c = en >> 2;
        const int k = en & 3;
        auto at = [&](int f) { return SOA ? cd[f * ncell + c] : cd[17 * c + f]; };
        a[0] += at(1 + k);
        a[1] += at(0) * at(5 + k);
        a[2] += at(9 + k);
        a[3] += at(13 + k);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) (SOA ? nd[k * nnode + p] : nd[4 * p + k]) += a[k];
}

// ----------------------------------------------------------------- drivers

template <typename T, bool SOA>
int space_disc_t(const mp_plan *P, const void *ed, const int32_t *eflag, const void *ia, void *res, cudaStream_t s)
{
    const int64_t nedge = P->from_size, ncell = P->maps[0].to_size;
    const int co = P->opts.coloring;
    if (co == MP_COLOR_HIER) {
        const int cap = P->stats.footprint_max[0];
        const bool gather = mp_staged(P, MP_STAGED_GATHER) == MP_STAGED_GATHER && mp_gather_ready(P);
        const int gw4 = gather ? P->gat_w / 4 : 0, cap_f = gather ? P->opts.block_size : 0;
        const int smem = cap * (int)(5 * sizeof(T) + 4) + gw4 * cap * 8 + cap_f * (int)(4 * sizeof(T) + 4);
        auto kern = gather ? space_disc_hier<T, SOA, kIncGather> : space_disc_hier<T, SOA, kIncColor>;
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
                                  reinterpret_cast<const ushort4 *>(P->dev.gat), gw4, P->dev.fp, (const T *)ed,
                                  eflag, (const T *)ia, (T *)res, nedge, ncell, cap, cap_f, err));
            overlap = true;
        }
        return MP_OK;
    }
    if (co == MP_COLOR_TWOSTEP) {
        MP_CUDA_TRY(mp_launch(space_disc_owner<T, SOA>, (int)((ncell + 255) / 256), 256, 0, s, false, P->dev.inv_off,
                              P->dev.inv_idx, (const T *)ed, eflag, (const T *)ia, (T *)res, nedge, ncell));
        return MP_OK;
    }
    if (co != MP_COLOR_GLOBAL && co != MP_COLOR_ATOMIC) return MP_EPLAN;
    const bool atomic = co == MP_COLOR_ATOMIC;
    bool overlap = false;
    for (int c = 0; c < P->ncolors; ++c) {
        const int e0 = P->color_offsets[c], e1 = P->color_offsets[c + 1];
        if (e1 <= e0) continue;
        auto kern = atomic ? space_disc_direct<T, SOA, true> : space_disc_direct<T, SOA, false>;
        MP_CUDA_TRY(mp_launch(kern, (e1 - e0 + 255) / 256, 256, 0, s, overlap && !atomic, e0, e1, P->dev.map[0],
                              (const T *)ed, eflag, (const T *)ia, (T *)res, nedge, ncell));
        overlap = true;
    }
    return MP_OK;
}

template <typename T, bool SOA>
int getacc_t(const mp_plan *P, const void *cd, void *nd, cudaStream_t s)
{
    const int64_t ncell = P->from_size, nnode = P->maps[0].to_size;
    const int co = P->opts.coloring;
    if (co == MP_COLOR_HIER) {
        if (P->opts.block_size > 512) return MP_EINVAL;
        const int cap = P->stats.footprint_max[0];
        const bool gather = mp_staged(P, MP_STAGED_GATHER) == MP_STAGED_GATHER && mp_gather_ready(P);
        const int gw4 = gather ? P->gat_w / 4 : 0, cap_f = gather ? P->opts.block_size : 0;
        const int smem = cap * (int)(4 * sizeof(T) + 4) + gw4 * cap * 8 + cap_f * 16 * (int)sizeof(T);
        auto kern = gather ? getacc_hier<T, SOA, kIncGather> : getacc_hier<T, SOA, kIncColor>;
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
                                  reinterpret_cast<const ushort4 *>(P->dev.gat), gw4, P->dev.fp, (const T *)cd,
                                  (T *)nd, ncell, nnode, cap, cap_f, err));
            overlap = true;
        }
        return MP_OK;
    }
    if (co == MP_COLOR_TWOSTEP) {
        MP_CUDA_TRY(mp_launch(getacc_owner<T, SOA>, (int)((nnode + 255) / 256), 256, 0, s, false, P->dev.inv_off,
                              P->dev.inv_idx, (const T *)cd, (T *)nd, ncell, nnode));
        return MP_OK;
    }
    if (co != MP_COLOR_GLOBAL && co != MP_COLOR_ATOMIC) return MP_EPLAN;
    const bool atomic = co == MP_COLOR_ATOMIC;
    bool overlap = false;
    for (int c = 0; c < P->ncolors; ++c) {
        const int c0 = P->color_offsets[c], c1 = P->color_offsets[c + 1];
        if (c1 <= c0) continue;
        auto kern = atomic ? getacc_direct<T, SOA, true> : getacc_direct<T, SOA, false>;
        MP_CUDA_TRY(mp_launch(kern, (c1 - c0 + 255) / 256, 256, 0, s, overlap && !atomic, c0, c1, P->dev.map[0],
                              (const T *)cd, (T *)nd, ncell, nnode));
        overlap = true;
    }
    return MP_OK;
}

bool ok_ptrs(std::initializer_list<const void *> ptrs)
{
    for (const void *p : ptrs)
        if (!p || !aligned16(p)) return false;
    return true;
}

}  // namespace

extern "C" int loop_space_disc(const mp_plan *P, int32_t dtype, const void *edata, const int32_t *eflag,
                               const void *inv_area, void *res, void *stream)
{
    if (!P || (dtype != MP_F64 && dtype != MP_F32)) return MP_EINVAL;
    if (P->nmaps != 1 || P->maps[0].arity != 2 || !P->maps[0].written) return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    if (!ok_ptrs({edata, eflag, inv_area, res})) return MP_EINVAL;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    cudaStream_t s = as_stream(stream);
    const bool soa = P->opts.layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64)
        rc = soa ? space_disc_t<double, true>(P, edata, eflag, inv_area, res, s)
                 : space_disc_t<double, false>(P, edata, eflag, inv_area, res, s);
    else
        rc = soa ? space_disc_t<float, true>(P, edata, eflag, inv_area, res, s)
                 : space_disc_t<float, false>(P, edata, eflag, inv_area, res, s);
    if (rc != MP_OK) return rc;
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

extern "C" int loop_getacc(const mp_plan *P, int32_t dtype, const void *cdata, void *nd, void *stream)
{
    if (!P || (dtype != MP_F64 && dtype != MP_F32)) return MP_EINVAL;
    if (P->nmaps != 1 || P->maps[0].arity != 4 || !P->maps[0].written) return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    if (!ok_ptrs({cdata, nd})) return MP_EINVAL;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    cudaStream_t s = as_stream(stream);
    const bool soa = P->opts.layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64)
        rc = soa ? getacc_t<double, true>(P, cdata, nd, s) : getacc_t<double, false>(P, cdata, nd, s);
    else
        rc = soa ? getacc_t<float, true>(P, cdata, nd, s) : getacc_t<float, false>(P, cdata, nd, s);
    if (rc != MP_OK) return rc;
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}
