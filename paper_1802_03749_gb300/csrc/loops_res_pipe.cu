// res_calc, two-layer staged kernel, pipelined and persistent.
//
// The staged kernel of Algorithm 1 spends most of its time waiting on a
// chain of dependent global loads per block (footprint ids, then the data
// they index).  Here each CTA processes several blocks of one colour and
// overlaps that chain with computation: while it computes block k from one
// shared-memory stage, asynchronous copies (cp.async) fill the other stage
// with block k+1's footprint data and a third id slot with block k+2's
// footprint ids.  Per block the work is Algorithm 1's: per-cell primitives,
// one edge flux per thread, thread-coloured increments in shared memory
// (onto res values prefetched with the footprint, legal because blocks of
// one colour share no cell), and one store per footprint cell.
//
// Shared-memory rows are array-of-structures so each footprint point is one
// or two 16-byte asynchronous copies (AoS data) and one vector access.
#include "common.cuh"
#include "dw.cuh"

namespace {

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async4(void *s, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void *s, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16(void *s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// copy n bytes (4, 8, 16 or 32) from global to shared memory asynchronously
template <int N>
__device__ __forceinline__ void cp_async_n(void *s, const void *g)
{
    if (N == 4) cp_async4(s, g);
    if (N == 8) cp_async8(s, g);
    if (N == 16) cp_async16(s, g);
    if (N == 32) {
        cp_async16(s, g);
        cp_async16(static_cast<char *>(s) + 16, static_cast<const char *>(g) + 16);
    }
}

__host__ __device__ constexpr int align16(int b) { return (b + 15) & ~15; }

constexpr int kMaxBlocksPerCta = 128;

// Byte layout of the dynamic shared memory; identical on host and device.
// E is the storage element (float or double).
//   2 stages:  q rows [cap_c][4], res rows [cap_c][4], adt [cap_c],
//              x rows [cap_n][2], local maps [S] (8 B), thread colours [S+16]
//   3 id slots: cell ids [cap_c], node ids [cap_n]
//   work:      per-cell rows [cap_c][WORK] (primitives, and for the
//              double-word variant also the converted state and increments)
//   descriptors of the CTA's blocks [kMaxBlocksPerCta]
struct pipe_layout {
    int cap_c, cap_n, S, esize, work_bytes;
    __host__ __device__ int q_off() const { return 0; }
    __host__ __device__ int res_off() const { return q_off() + align16(cap_c * 4 * esize); }
    __host__ __device__ int adt_off() const { return res_off() + align16(cap_c * 4 * esize); }
    __host__ __device__ int x_off() const { return adt_off() + align16(cap_c * esize); }
    __host__ __device__ int lm_off() const { return x_off() + align16(cap_n * 2 * esize); }
    __host__ __device__ int tc_off() const { return lm_off() + align16(S * 8); }
    __host__ __device__ int stage_bytes() const { return tc_off() + align16(S + 16); }
    __host__ __device__ int ids_bytes() const { return align16(cap_c * 4) + align16(cap_n * 4); }
    __host__ __device__ int ids_off(int slot) const { return 2 * stage_bytes() + slot * ids_bytes(); }
    __host__ __device__ int work_off() const { return ids_off(3); }
    __host__ __device__ int desc_off() const { return work_off() + align16(cap_c * work_bytes); }
    __host__ __device__ int total() const { return desc_off() + kMaxBlocksPerCta * (int)sizeof(mp_block_desc); }
};

// Issue the asynchronous copies of one block's footprint ids into an id slot.
__device__ __forceinline__ void issue_ids(const mp_block_desc &d, const int32_t *__restrict__ fp, int *gc, int *gn)
{
    for (int i = threadIdx.x; i < d.fp_count[1]; i += blockDim.x) cp_async4(gc + i, fp + d.fp_start[1] + i);
    for (int i = threadIdx.x; i < d.fp_count[0]; i += blockDim.x) cp_async4(gn + i, fp + d.fp_start[0] + i);
}

// Issue the asynchronous copies of one block's data (ids already in shared
// memory) into a stage: q, res, adt rows per cell, x rows per node, the
// block's local maps and its thread colours (4-byte words covering them).
template <typename E, bool SOA>
__device__ __forceinline__ void issue_data(const mp_block_desc &d, const pipe_layout &L, unsigned char *stage,
                                           const int *gc, const int *gn, const E *__restrict__ x,
                                           const E *__restrict__ q, const E *__restrict__ adt,
                                           const E *__restrict__ res, const uint2 *__restrict__ lmap,
                                           const uint8_t *__restrict__ tcolor, int64_t nnode, int64_t ncell)
{
    E *sq = reinterpret_cast<E *>(stage + L.q_off());
    E *sr = reinterpret_cast<E *>(stage + L.res_off());
    E *sa = reinterpret_cast<E *>(stage + L.adt_off());
    E *sx = reinterpret_cast<E *>(stage + L.x_off());
    uint2 *slm = reinterpret_cast<uint2 *>(stage + L.lm_off());
    uint32_t *stc = reinterpret_cast<uint32_t *>(stage + L.tc_off());
    for (int i = threadIdx.x; i < d.fp_count[1]; i += blockDim.x) {
        const int64_t g = gc[i];
        if (SOA) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                cp_async_n<sizeof(E)>(sq + 4 * i + k, q + k * ncell + g);
                cp_async_n<sizeof(E)>(sr + 4 * i + k, res + k * ncell + g);
            }
        } else {
            cp_async_n<4 * sizeof(E)>(sq + 4 * i, q + 4 * g);
            cp_async_n<4 * sizeof(E)>(sr + 4 * i, res + 4 * g);
        }
        cp_async_n<sizeof(E)>(sa + i, adt + g);
    }
    for (int i = threadIdx.x; i < d.fp_count[0]; i += blockDim.x) {
        const int64_t g = gn[i];
        if (SOA) {
            cp_async_n<sizeof(E)>(sx + 2 * i, x + g);
            cp_async_n<sizeof(E)>(sx + 2 * i + 1, x + nnode + g);
        } else {
            cp_async_n<2 * sizeof(E)>(sx + 2 * i, x + 2 * g);
        }
    }
    for (int t = threadIdx.x; t < d.nitems; t += blockDim.x) cp_async8(slm + t, lmap + d.item_start + t);
    const int w0 = d.item_start >> 2, w1 = (d.item_start + d.nitems + 3) >> 2;
    for (int w = w0 + (int)threadIdx.x; w < w1; w += blockDim.x)
        cp_async4(stc + (w - w0), reinterpret_cast<const uint32_t *>(tcolor) + w);
}

// Native arithmetic (E = T = float or double).
template <typename T>
struct native_ops {
    static constexpr int work_bytes = 4 * sizeof(T);  // u/2, v/2, p/2, H per cell (cell_prims_half)
};

template <typename T, bool SOA>
__global__ void __launch_bounds__(512) res_calc_pipe(const mp_block_desc *__restrict__ desc, int b0, int nb,
                                                     const uint2 *__restrict__ lmap,
                                                     const uint8_t *__restrict__ tcolor,
                                                     const int32_t *__restrict__ fp, const T *__restrict__ x,
                                                     const T *__restrict__ q, const T *__restrict__ adt,
                                                     T *__restrict__ res, int64_t nnode, int64_t ncell,
                                                     pipe_layout L, T gm1h, T half_eps, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int G = gridDim.x, me = blockIdx.x, tid = threadIdx.x;
    const int count = (nb - me + G - 1) / G;  // this CTA's blocks: me, me + G, ...
    if (count <= 0) return;
    __shared__ int bad;
    if (tid == 0) bad = (L.total() > (int)dynamic_smem_bytes() || count > kMaxBlocksPerCta || L.S > (int)blockDim.x);
    __syncthreads();
    if (bad) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    mp_block_desc *sd = reinterpret_cast<mp_block_desc *>(sm + L.desc_off());
    for (int k = tid; k < count; k += blockDim.x) {
        mp_block_desc d = desc[b0 + me + k * G];
        if (d.fp_count[1] > L.cap_c || d.fp_count[0] > L.cap_n || d.nitems > L.S) atomicOr(&bad, 1);
        sd[k] = d;
    }
    __syncthreads();
    if (bad) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    auto stage = [&](int k) { return sm + (k & 1) * L.stage_bytes(); };
    auto ids_c = [&](int k) { return reinterpret_cast<int *>(sm + L.ids_off(k % 3)); };
    auto ids_n = [&](int k) { return reinterpret_cast<int *>(sm + L.ids_off(k % 3) + align16(L.cap_c * 4)); };
    T *work = reinterpret_cast<T *>(sm + L.work_off());  // [cap_c][4]: u/2, v/2, p/2, H

    // prologue: ids of block 0, then its data and the ids of block 1
    issue_ids(sd[0], fp, ids_c(0), ids_n(0));
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    issue_data<T, SOA>(sd[0], L, stage(0), ids_c(0), ids_n(0), x, q, adt, res, lmap, tcolor, nnode, ncell);
    if (count > 1) issue_ids(sd[1], fp, ids_c(1), ids_n(1));
    cp_async_commit();

    for (int k = 0; k < count; ++k) {
        cp_async_wait_all();
        __syncthreads();  // block k's data and block k+1's ids are visible
        if (k + 1 < count)
            issue_data<T, SOA>(sd[k + 1], L, stage(k + 1), ids_c(k + 1), ids_n(k + 1), x, q, adt, res, lmap, tcolor,
                               nnode, ncell);
        if (k + 2 < count) issue_ids(sd[k + 2], fp, ids_c(k + 2), ids_n(k + 2));
        cp_async_commit();

        const mp_block_desc d = sd[k];
        unsigned char *st = stage(k);
        const T *sq = reinterpret_cast<const T *>(st + L.q_off());
        T *sr = reinterpret_cast<T *>(st + L.res_off());
        const T *sa = reinterpret_cast<const T *>(st + L.adt_off());
        const T *sx = reinterpret_cast<const T *>(st + L.x_off());
        const uint2 *slm = reinterpret_cast<const uint2 *>(st + L.lm_off());
        const uint8_t *stc = st + L.tc_off() + (d.item_start & 3);
        // per-cell primitives
        for (int i = tid; i < d.fp_count[1]; i += blockDim.x) {
            T u, v, p, H;
            cell_prims_half(sq[4 * i], sq[4 * i + 1], sq[4 * i + 2], sq[4 * i + 3], gm1h, u, v, p, H);
            work[4 * i] = u;
            work[4 * i + 1] = v;
            work[4 * i + 2] = p;
            work[4 * i + 3] = H;
        }
        __syncthreads();
        T f[4] = {T(0), T(0), T(0), T(0)};
        int c1 = 0, c2 = 0, my_color = -1;
        if (tid < d.nitems) {
            const uint2 lw = slm[tid];
            const int na = lw.x & 0xffff, nb_ = lw.x >> 16;
            c1 = lw.y & 0xffff;
            c2 = lw.y >> 16;
            my_color = stc[tid];
            const T nx = sx[2 * na + 1] - sx[2 * nb_ + 1];
            const T ny = sx[2 * nb_] - sx[2 * na];
            edge_flux(nx, ny, sq[4 * c1], sq[4 * c1 + 1], sq[4 * c1 + 2], sq[4 * c1 + 3], work[4 * c1],
                      work[4 * c1 + 1], work[4 * c1 + 2], work[4 * c1 + 3], sa[c1], sq[4 * c2], sq[4 * c2 + 1],
                      sq[4 * c2 + 2], sq[4 * c2 + 3], work[4 * c2], work[4 * c2 + 1], work[4 * c2 + 2],
                      work[4 * c2 + 3], sa[c2], half_eps, f);
        }
        for (int c = 0; c < d.ncolors; ++c) {
            if (my_color == c) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    sr[4 * c1 + j] += f[j];
                    sr[4 * c2 + j] -= f[j];
                }
            }
            __syncthreads();
        }
        const int *gc = ids_c(k);
        for (int i = tid; i < d.fp_count[1]; i += blockDim.x) {
            const int64_t g = gc[i];
            if (SOA) {
#pragma unroll
                for (int j = 0; j < 4; ++j) res[j * ncell + g] = sr[4 * i + j];
            } else if (sizeof(T) == 8) {
                double2 *r2 = reinterpret_cast<double2 *>(res) + 2 * g;
                r2[0] = make_double2((double)sr[4 * i], (double)sr[4 * i + 1]);
                r2[1] = make_double2((double)sr[4 * i + 2], (double)sr[4 * i + 3]);
            } else {
                reinterpret_cast<float4 *>(res)[g] =
                    make_float4((float)sr[4 * i], (float)sr[4 * i + 1], (float)sr[4 * i + 2], (float)sr[4 * i + 3]);
            }
        }
    }
    cp_async_wait_all();
}

// MP_EPLAN when the pipelined layout does not fit this plan (more than 512
// threads per block, or two stages of the largest footprint exceed shared
// memory): the caller then runs the one-block-per-CTA kernel.
template <typename T, bool SOA>
int res_calc_pipe_t(const mp_plan *P, const void *x, const void *q, const void *adt, void *res, double gam,
                    double eps, cudaStream_t s)
{
    pipe_layout L{P->stats.footprint_max[1], P->stats.footprint_max[0], P->opts.block_size, (int)sizeof(T),
                  native_ops<T>::work_bytes};
    const int smem = L.total();
    auto kern = res_calc_pipe<T, SOA>;
    if (P->opts.block_size > 512) return MP_EPLAN;
    int rc = mp_allow_smem(kern, smem);
    if (rc == MP_ESMEM) return MP_EPLAN;
    if (rc != MP_OK) return rc;
    int *err = nullptr;
    if ((rc = mp_device_error_word(&err)) != MP_OK) return rc;
    int dev = 0, sms = 0, occ = 0;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    MP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, P->opts.block_size, smem));
    if (occ < 1) return MP_ESMEM;
    for (int c = 0; c < P->ncolors; ++c) {
        const int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
        if (nb == 0) continue;
        int grid = std::min(nb, sms * occ);
        if ((nb + grid - 1) / grid > kMaxBlocksPerCta) grid = (nb + kMaxBlocksPerCta - 1) / kMaxBlocksPerCta;
        kern<<<grid, P->opts.block_size, smem, s>>>(P->dev.desc, b0, nb, reinterpret_cast<const uint2 *>(P->dev.lmap),
                                                    P->dev.tcolor, P->dev.fp, (const T *)x, (const T *)q,
                                                    (const T *)adt, (T *)res, P->maps[0].to_size, P->maps[1].to_size,
                                                    L, (T)(0.5 * (gam - 1.0)), (T)(0.5 * eps), err);
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int mp_res_calc_pipe(const mp_plan *P, int32_t dtype, const void *x, const void *q, const void *adt, void *res,
                     double gam, double eps, void *stream)
{
    if (P->opts.coloring != MP_COLOR_HIER || P->maps[0].slot != 0 || P->maps[1].slot != 1 || P->lmap_stride != 4)
        return MP_EPLAN;
    const bool soa = P->opts.layout == MP_LAYOUT_SOA;
    cudaStream_t s = as_stream(stream);
    if (dtype == MP_F64)
        return soa ? res_calc_pipe_t<double, true>(P, x, q, adt, res, gam, eps, s)
                   : res_calc_pipe_t<double, false>(P, x, q, adt, res, gam, eps, s);
    if (dtype == MP_F32)
        return soa ? res_calc_pipe_t<float, true>(P, x, q, adt, res, gam, eps, s)
                   : res_calc_pipe_t<float, false>(P, x, q, adt, res, gam, eps, s);
    return MP_EINVAL;
}
