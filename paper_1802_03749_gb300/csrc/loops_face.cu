// Face-flux loop with the access pattern of miniAero's compute_face_flux
// (Sec. 3.1.5): over the interior faces of a hex mesh, 12 values read
// directly per face, 28 read and 5 incremented on each of the 2 cells.
//
// Per face f between cells c1 and c2 (face data A[3] area normal from c1
// into c2, xf[3] face centre, nhat[3] = A/|A|, dx[3] = xc2 - xc1; cell data
// Q[5], gradients of the primitives (rho, u, v, w, p) at 5 + 3 v + d,
// limiters at 20 + v, centroid xc at 25):
//   V_face = V_cell + phi (G (xf - xc)) on each side;
//   F_inv = |A| ((F(V_1) + F(V_2))/2 - lambda (Q(V_2) - Q(V_1))/2), the
//           Rusanov flux, lambda = max |u.nhat| + c;
//   face gradients of u, v, w and T = p/rho: mean of the cell gradients
//           corrected along dx with the cell-centre difference;
//   F_v = (0, tau A, u_f.(tau A) + k grad T.A), tau Newtonian with mu,
//           k = mu gam / ((gam - 1) pr);
//   res[c1] += F_inv - F_v,  res[c2] -= F_inv - F_v.
//
// The 2 x 28 values a face reads per cell are what makes this loop heavy:
// on the paper's P100 staging them did not fit shared memory, and only the
// increments were cached.  Both forms are here: FULL stages the 28 values
// of every footprint cell in shared memory, INC_ONLY stages the increments
// (and the current res) only and reads the cell data through L1/L2.
#include "common.cuh"

namespace {

constexpr int kIncColor = 0, kIncGather = 2;
constexpr int kCell = 28, kFace = 12;

// cell data accessor: shared-memory SoA [k][stride] or global AoS / SoA
template <typename T>
struct cell_at {
    const T *p;
    int64_t stride;  // distance between consecutive values of one cell
    __device__ __forceinline__ T operator()(int k) const { return p[k * stride]; }
};

// What a face needs of a cell besides its raw gradients, limiters and
// centroid: the primitives V = (rho, u, v, w, p), T = p / rho and
// grad T = (grad p - T grad rho) / rho.  The fully staged kernels compute it
// once per staged cell (4 divides and ~20 operations a face would
// otherwise repeat for each of its 2 cells, the FP64 pipe being the bound).
template <typename T>
struct cell_prep {
    T V[5], Tc, gT[3];
};

template <typename T>
__device__ __forceinline__ void prepare_cell(const cell_at<T> &c, T gam, cell_prep<T> &s)
{
    const T rho = c(0), ri = T(1) / rho;
    s.V[0] = rho;
    s.V[1] = c(1) * ri;
    s.V[2] = c(2) * ri;
    s.V[3] = c(3) * ri;
    s.V[4] = (gam - T(1)) * (c(4) - T(0.5) * rho * (s.V[1] * s.V[1] + s.V[2] * s.V[2] + s.V[3] * s.V[3]));
    s.Tc = s.V[4] * ri;
#pragma unroll
    for (int d = 0; d < 3; ++d) s.gT[d] = (c(17 + d) - s.Tc * c(5 + d)) * ri;
}

// staged layout of a prepared cell: V at 0..4, raw gradients, limiters and
// centroid at their own slots 5..27, T at 28, grad T at 29..31
constexpr int kStaged = 32;

template <typename T>
__device__ __forceinline__ void load_prep(const cell_at<T> &c, cell_prep<T> &s)
{
#pragma unroll
    for (int v = 0; v < 5; ++v) s.V[v] = c(v);
    s.Tc = c(28);
#pragma unroll
    for (int d = 0; d < 3; ++d) s.gT[d] = c(29 + d);
}

template <typename T>
__device__ __forceinline__ void aero_side(const cell_at<T> &c, const cell_prep<T> &pc, const T xf[3], const T n[3],
                                          T gam, T Qs[5], T F[5], T &lam)
{
    const T r0 = xf[0] - c(25), r1 = xf[1] - c(26), r2 = xf[2] - c(27);
    T V[5];
#pragma unroll
    for (int v = 0; v < 5; ++v)
        V[v] = pc.V[v] + c(20 + v) * (c(5 + 3 * v) * r0 + c(6 + 3 * v) * r1 + c(7 + 3 * v) * r2);
    const T E = V[4] / (gam - T(1)) + T(0.5) * V[0] * (V[1] * V[1] + V[2] * V[2] + V[3] * V[3]);
    const T un = V[1] * n[0] + V[2] * n[1] + V[3] * n[2];
    lam = fabs(un) + sqrt(gam * V[4] / V[0]);
    Qs[0] = V[0];
    Qs[1] = V[0] * V[1];
    Qs[2] = V[0] * V[2];
    Qs[3] = V[0] * V[3];
    Qs[4] = E;
    F[0] = V[0] * un;
    F[1] = V[0] * V[1] * un + V[4] * n[0];
    F[2] = V[0] * V[2] * un + V[4] * n[1];
    F[3] = V[0] * V[3] * un + V[4] * n[2];
    F[4] = (E + V[4]) * un;
}

// F = F_inv - F_v of one face
template <typename T>
__device__ __forceinline__ void face_flux(const cell_at<T> &c1, const cell_at<T> &c2, const cell_prep<T> &p1,
                                          const cell_prep<T> &p2, const T fd[kFace], T gam, T mu, T kappa, T out[5])
{
    const T A[3] = {fd[0], fd[1], fd[2]}, xf[3] = {fd[3], fd[4], fd[5]}, n[3] = {fd[6], fd[7], fd[8]};
    const T dx[3] = {fd[9], fd[10], fd[11]};
    {
        T Q1[5], Q2[5], F1[5], F2[5], l1, l2;
        aero_side(c1, p1, xf, n, gam, Q1, F1, l1);
        aero_side(c2, p2, xf, n, gam, Q2, F2, l2);
        const T lam = l1 > l2 ? l1 : l2;
        const T area = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
#pragma unroll
        for (int k = 0; k < 5; ++k) out[k] = area * (T(0.5) * (F1[k] + F2[k]) - T(0.5) * lam * (Q2[k] - Q1[k]));
    }
    const T idd = T(1) / (dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
    T gu[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T gm[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) gm[d] = T(0.5) * (c1(5 + 3 * (1 + a) + d) + c2(5 + 3 * (1 + a) + d));
        const T corr = ((p2.V[1 + a] - p1.V[1 + a]) - (gm[0] * dx[0] + gm[1] * dx[1] + gm[2] * dx[2])) * idd;
#pragma unroll
        for (int d = 0; d < 3; ++d) gu[a][d] = gm[d] + corr * dx[d];
    }
    T gT[3];
    {
        T gm[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) gm[d] = T(0.5) * (p1.gT[d] + p2.gT[d]);
        const T corr = ((p2.Tc - p1.Tc) - (gm[0] * dx[0] + gm[1] * dx[1] + gm[2] * dx[2])) * idd;
#pragma unroll
        for (int d = 0; d < 3; ++d) gT[d] = gm[d] + corr * dx[d];
    }
    const T div = gu[0][0] + gu[1][1] + gu[2][2];
    T tA[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        tA[a] = T(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T tau = mu * (gu[a][b] + gu[b][a]) - (a == b ? T(2) / T(3) * mu * div : T(0));
            tA[a] += tau * A[b];
        }
    }
    const T uf0 = T(0.5) * (p1.V[1] + p2.V[1]), uf1 = T(0.5) * (p1.V[2] + p2.V[2]);
    const T uf2 = T(0.5) * (p1.V[3] + p2.V[3]);
    out[1] -= tA[0];
    out[2] -= tA[1];
    out[3] -= tA[2];
    out[4] -= uf0 * tA[0] + uf1 * tA[1] + uf2 * tA[2] + kappa * (gT[0] * A[0] + gT[1] * A[1] + gT[2] * A[2]);
}

// a face between two cells read from global memory (no staging)
template <typename T>
__device__ __forceinline__ void face_flux_global(const cell_at<T> &c1, const cell_at<T> &c2, const T fd[kFace], T gam,
                                                 T mu, T kappa, T out[5])
{
    cell_prep<T> p1, p2;
    prepare_cell(c1, gam, p1);
    prepare_cell(c2, gam, p2);
    face_flux(c1, c2, p1, p2, fd, gam, mu, kappa, out);
}

template <typename T, bool SOA>
__device__ __forceinline__ void load_face(const T *__restrict__ fdata, int64_t nface, int64_t f, T fd[kFace])
{
#pragma unroll
    for (int k = 0; k < kFace; ++k) fd[k] = SOA ? fdata[k * nface + f] : fdata[kFace * f + k];
}

template <typename T, bool SOA>
__device__ __forceinline__ cell_at<T> global_cell(const T *cdata, int64_t ncell, int64_t g)
{
    return SOA ? cell_at<T>{cdata + g, ncell} : cell_at<T>{cdata + kCell * g, 1};
}

template <typename T, bool SOA>
__device__ __forceinline__ T &res_at(T *res, int64_t ncell, int64_t c, int k)
{
    return SOA ? res[k * ncell + c] : res[5 * c + k];
}

// Shared memory (cap cells, cap_f threads):
//   ushort4 ge[gw4][cap]   gather only
//   T cd[32][cap]          FULL only: prepared cells (see cell_prep)
//   T inc[5][cap]          res prefetched, incremented
//   T f[5][cap_f]          gather only
//   int gid[cap]
template <typename T, bool SOA, bool FULL, int INC>
__global__ void __launch_bounds__(256) face_flux_hier(const mp_block_desc *__restrict__ desc, int block0,
                                                      const ushort4 *__restrict__ lmap,
                                                      const uint8_t *__restrict__ tcolor,
                                                      const ushort4 *__restrict__ gat, int gw4,
                                                      const int32_t *__restrict__ fp, const T *__restrict__ fdata,
                                                      const T *__restrict__ cdata, T *__restrict__ res,
                                                      int64_t nface, int64_t ncell, int cap, int cap_f, T gam,
                                                      T mu, T kappa, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ushort4 *s_ge = reinterpret_cast<ushort4 *>(smem_raw);
    T *s_cd = reinterpret_cast<T *>(s_ge + (INC == kIncGather ? gw4 * cap : 0));
    T *s_inc = s_cd + (FULL ? kStaged * cap : 0);
    T *s_f = s_inc + 5 * cap;
    int *s_gid = reinterpret_cast<int *>(s_f + (INC == kIncGather ? 5 * cap_f : 0));

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
    const int64_t f = d.item_start + tid;
    int c1 = 0, c2 = 0, my_color = -1;
    if (active) {
        const ushort4 l = lmap[f];
        c1 = l.x;
        c2 = l.y;
        if (INC == kIncColor) my_color = tcolor[f];
    }
    for (int i = tid; i < nc; i += blockDim.x) {
        const int g = fpc[i];
        s_gid[i] = g;
        if (FULL) {
            const cell_at<T> src = global_cell<T, SOA>(cdata, ncell, g);
#pragma unroll 4
            for (int k = 5; k < kCell; ++k) s_cd[k * cap + i] = src(k);
            cell_prep<T> pc;
            prepare_cell(src, gam, pc);
#pragma unroll
            for (int v = 0; v < 5; ++v) s_cd[v * cap + i] = pc.V[v];
            s_cd[28 * cap + i] = pc.Tc;
#pragma unroll
            for (int d = 0; d < 3; ++d) s_cd[(29 + d) * cap + i] = pc.gT[d];
        }
        if (INC == kIncGather) {
            const ushort4 *row = gat + (int64_t)(d.fp_start[0] + i) * gw4;
            for (int h = 0; h < gw4; ++h) s_ge[h * cap + i] = row[h];
        }
        mp_pdl_wait();  // res: written by the previous colour's launch
#pragma unroll
        for (int k = 0; k < 5; ++k) s_inc[k * cap + i] = res_at<T, SOA>(res, ncell, g, k);
    }
    __syncthreads();
    T F[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (active) {
        T fd[kFace];
        load_face<T, SOA>(fdata, nface, f, fd);
        if (FULL) {
            const cell_at<T> a1{s_cd + c1, cap}, a2{s_cd + c2, cap};
            cell_prep<T> p1, p2;
            load_prep(a1, p1);
            load_prep(a2, p2);
            face_flux(a1, a2, p1, p2, fd, gam, mu, kappa, F);
        } else {
            face_flux_global(global_cell<T, SOA>(cdata, ncell, s_gid[c1]),
                             global_cell<T, SOA>(cdata, ncell, s_gid[c2]), fd, gam, mu, kappa, F);
        }
    }
    if constexpr (INC == kIncGather) {
        if (active) {
#pragma unroll
            for (int k = 0; k < 5; ++k) s_f[k * cap_f + tid] = F[k];
        }
        __syncthreads();
        for (int i = tid; i < nc; i += blockDim.x) {
            T a[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) a[k] = s_inc[k * cap + i];
            for (int h = 0; h < gw4; ++h) {
                const ushort4 e4 = s_ge[h * cap + i];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned en = es[j];
                    if (en == 0xFFFFu) continue;
                    const int t = (int)(en >> 4);
                    const bool second = (en & 15u) == 1u;
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        const T v = s_f[k * cap_f + t];
                        a[k] = second ? a[k] - v : a[k] + v;
                    }
                }
            }
            const int g = s_gid[i];
#pragma unroll
            for (int k = 0; k < 5; ++k) res_at<T, SOA>(res, ncell, g, k) = a[k];
        }
    } else {
        for (int col = 0; col < d.ncolors; ++col) {
            if (my_color == col) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    s_inc[k * cap + c1] += F[k];
                    s_inc[k * cap + c2] -= F[k];
                }
            }
            __syncthreads();
        }
        for (int i = tid; i < nc; i += blockDim.x) {
            const int g = s_gid[i];
#pragma unroll
            for (int k = 0; k < 5; ++k) res_at<T, SOA>(res, ncell, g, k) = s_inc[k * cap + i];
        }
    }
}

// GLOBAL (plain read-add-write per colour), ATOMIC, or STEP1 of the
// temporary-array method (scratch[(2 f + slot) 5 + k] = +F / -F).
enum { kDirectColor = 0, kDirectAtomic = 1, kDirectStep1 = 2 };

template <typename T, bool SOA, int MODE>
__global__ void __launch_bounds__(256) face_flux_direct(int f0, int f1, const int32_t *__restrict__ f2c,
                                                        const T *__restrict__ fdata, const T *__restrict__ cdata,
                                                        T *__restrict__ out, int64_t nface, int64_t ncell, T gam,
                                                        T mu, T kappa)
{
    mp_pdl_trigger();
    const int64_t f = f0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= f1) return;
    const int2 cc = reinterpret_cast<const int2 *>(f2c)[f];
    T fd[kFace];
    load_face<T, SOA>(fdata, nface, f, fd);
    T F[5];
    face_flux_global(global_cell<T, SOA>(cdata, ncell, cc.x), global_cell<T, SOA>(cdata, ncell, cc.y), fd, gam, mu,
                     kappa, F);
    if (MODE == kDirectStep1) {
        T *o = out + 10 * f;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            o[k] = F[k];
            o[5 + k] = -F[k];
        }
        return;
    }
    if (MODE == kDirectColor) mp_pdl_wait();  // res: read-add-written by the previous colour's launch
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (MODE == kDirectAtomic) {
            atomicAdd(&res_at<T, SOA>(out, ncell, cc.x, k), F[k]);
            atomicAdd(&res_at<T, SOA>(out, ncell, cc.y, k), -F[k]);
        } else {
            res_at<T, SOA>(out, ncell, cc.x, k) += F[k];
            res_at<T, SOA>(out, ncell, cc.y, k) -= F[k];
        }
    }
}

template <typename T, bool SOA>
int face_flux_t(const mp_plan *P, const void *fdata, const void *cdata, void *res, double gam, double mu, double pr,
                cudaStream_t s)
{
    const int64_t nface = P->from_size, ncell = P->maps[0].to_size;
    const T g = (T)gam, m = (T)mu, k = (T)(mu * gam / ((gam - 1.0) * pr));
    const int co = P->opts.coloring;
    if (co == MP_COLOR_HIER) {
        if (P->opts.block_size > 256) return MP_EINVAL;
        const int cap = P->stats.footprint_max[0];
        // default: full staging with thread colours (measured fastest on
        // GB300, where the 28 values of a cell fit shared memory)
        const int variant = mp_staged(P, MP_STAGED_SIMPLE);
        const bool full = variant == MP_STAGED_SIMPLE || variant == MP_STAGED_GATHER;
        const bool gather =
            (variant == MP_STAGED_GATHER || variant == MP_STAGED_INC_ONLY_GATHER) && mp_gather_ready(P);
        const int gw4 = gather ? P->gat_w / 4 : 0, cap_f = gather ? P->opts.block_size : 0;
        const int smem = cap * (int)((full ? kStaged : 0) * sizeof(T) + 5 * sizeof(T) + 4) + gw4 * cap * 8 +
                         cap_f * 5 * (int)sizeof(T);
        auto kern = full ? (gather ? face_flux_hier<T, SOA, true, kIncGather> : face_flux_hier<T, SOA, true, kIncColor>)
                         : (gather ? face_flux_hier<T, SOA, false, kIncGather>
                                   : face_flux_hier<T, SOA, false, kIncColor>);
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
                                  reinterpret_cast<const ushort4 *>(P->dev.gat), gw4, P->dev.fp, (const T *)fdata,
                                  (const T *)cdata, (T *)res, nface, ncell, cap, cap_f, g, m, k, err));
            overlap = true;
        }
        return MP_OK;
    }
    if (co == MP_COLOR_TWOSTEP) {
        void *scratch = nullptr;
        int rc = mp_twostep_scratch(P, (size_t)nface * 10 * sizeof(T), &scratch);
        if (rc != MP_OK) return rc;
        MP_CUDA_TRY(mp_launch(face_flux_direct<T, SOA, kDirectStep1>, (int)((nface + 255) / 256), 256, 0, s, false, 0,
                              (int)nface, P->dev.map[0], (const T *)fdata, (const T *)cdata, (T *)scratch, nface,
                              ncell, g, m, k));
        return mp_twostep_gather(P, sizeof(T) == 8 ? MP_F64 : MP_F32, 5, scratch, res, s);
    }
    const bool atomic = co == MP_COLOR_ATOMIC;
    bool overlap = false;
    for (int c = 0; c < P->ncolors; ++c) {
        const int f0 = P->color_offsets[c], f1 = P->color_offsets[c + 1];
        if (f1 <= f0) continue;
        auto kern = atomic ? face_flux_direct<T, SOA, kDirectAtomic> : face_flux_direct<T, SOA, kDirectColor>;
        MP_CUDA_TRY(mp_launch(kern, (f1 - f0 + 255) / 256, 256, 0, s, overlap && !atomic, f0, f1, P->dev.map[0],
                              (const T *)fdata, (const T *)cdata, (T *)res, nface, ncell, g, m, k));
        overlap = true;
    }
    return MP_OK;
}

}  // namespace

extern "C" int loop_face_flux(const mp_plan *P, int32_t dtype, const void *fdata, const void *cdata, void *res,
                              double gam, double mu, double pr, void *stream)
{
    if (!P || (dtype != MP_F64 && dtype != MP_F32 && dtype != MP_F64_DW) || !(gam > 1.0) || !(mu >= 0.0) ||
        !(pr > 0.0))
        return MP_EINVAL;
    if (P->nmaps != 1 || P->maps[0].arity != 2 || !P->maps[0].written) return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    for (const void *p : {fdata, cdata, (const void *)res})
        if (!p || !aligned16(p)) return MP_EINVAL;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    if (dtype == MP_F64_DW) {
        rc = mp_face_flux_dw(P, fdata, cdata, res, gam, mu, pr, stream);
        if (rc != MP_OK) return rc;
        MP_CUDA_TRY(cudaGetLastError());
        return MP_OK;
    }
    cudaStream_t s = as_stream(stream);
    const bool soa = P->opts.layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64)
        rc = soa ? face_flux_t<double, true>(P, fdata, cdata, res, gam, mu, pr, s)
                 : face_flux_t<double, false>(P, fdata, cdata, res, gam, mu, pr, s);
    else
        rc = soa ? face_flux_t<float, true>(P, fdata, cdata, res, gam, mu, pr, s)
                 : face_flux_t<float, false>(P, fdata, cdata, res, gam, mu, pr, s);
    if (rc != MP_OK) return rc;
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}
