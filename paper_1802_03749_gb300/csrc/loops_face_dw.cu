// Face flux (loops_face.cu) with FP64 data and double-word arithmetic: the
// FP64 kernel keeps GB300's FP64 pipe 86 % busy; here every operation runs
// on the FP32 pipes as a pair of floats (dw.cuh), to FP64-level accuracy
// (a CPU emulation of this exact sequence gave 2.8e-14 rel-L2 against the
// FP64 oracle at 64^3; the parity tests hold it to 1e-12).
//
// Two-layer staged form: the block's cells are prepared once at staging
// (primitives V, temperature T and grad T in double-word, the 15 gradients
// and 5 limiters split to double-word, the centroid kept in FP64), each
// thread computes one face from shared memory, increments accumulate in
// double-word one thread colour at a time, and each cell's res is written
// once (FP64 res + double-word sum, two FP64 additions).
//
// Square roots: one Newton (Heron) step in double-word on the FP32 square
// root, s = s0 + (x - s0^2) / (2 s0) with s0^2 formed exactly (Karp and
// Markstein, "High-precision division and square root", ACM TOMS 23(4),
// 1997).  Divisions: a double-word reciprocal (Newton step) times the
// dividend.
#include "common.cuh"
#include "dw.cuh"

namespace {

constexpr int kFace = 12, kCell = 28;
// staged double-word values per cell: V[5], T, gT[3], G[15], phi[5]
constexpr int kDwStaged = 29;
constexpr int kSlotT = 5, kSlotGT = 6, kSlotG = 9, kSlotPhi = 24;

__device__ __forceinline__ dw dw_sqrt(dw x)
{
    const float s0 = __fsqrt_rn(x.hi);
    if (s0 == 0.0f) return {0.0f, 0.0f};
    const dw p = dw_two_prod(s0, s0);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
    return dw_fast_two_sum(s0, __fdiv_rn(d, __fmul_rn(2.0f, s0)));
}

__device__ __forceinline__ dw dw_abs(dw x) { return x.hi < 0.0f ? dw_neg(x) : x; }

__device__ __forceinline__ dw dw_max(dw x, dw y)
{
    return (x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo)) ? x : y;
}

__device__ __forceinline__ dw dw3(const dw a[3], const dw b[3])
{
    dw_acc A = dw_dot_begin(a[0], b[0]);
    dw_dot_add(A, a[1], b[1]);
    dw_dot_add(A, a[2], b[2]);
    return dw_dot_end(A);
}

__device__ __forceinline__ dw ld2(const float2 *a, int i)
{
    const float2 v = a[i];
    return {v.x, v.y};
}
__device__ __forceinline__ void st2(float2 *a, int i, dw v) { a[i] = make_float2(v.hi, v.lo); }

struct dw_consts {
    dw gm1, igm1, gam, mu, kappa, two3;
};

// One side of a face: reconstruct to the face centre, then the conserved
// state, the normal Euler flux and |u.n| + c.
__device__ __forceinline__ void dw_side(const float2 *s, int cap, int c, const double *xc, const double xf[3],
                                        const dw n[3], const dw_consts &K, dw Q[5], dw F[5], dw &lam)
{
    dw r[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) r[d] = dw_from_double_int(xf[d] - xc[d * cap + c]);
    dw V[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        dw_acc A = dw_dot_begin(ld2(s, (kSlotG + 3 * v) * cap + c), r[0]);
        dw_dot_add(A, ld2(s, (kSlotG + 3 * v + 1) * cap + c), r[1]);
        dw_dot_add(A, ld2(s, (kSlotG + 3 * v + 2) * cap + c), r[2]);
        V[v] = dw_add_fast(ld2(s, v * cap + c), dw_mul(ld2(s, (kSlotPhi + v) * cap + c), dw_dot_end(A)));
    }
    Q[0] = V[0];
    Q[1] = dw_mul(V[0], V[1]);
    Q[2] = dw_mul(V[0], V[2]);
    Q[3] = dw_mul(V[0], V[3]);
    const dw kin = dw_scale2(dw_add_fast(dw_add_fast(dw_mul(Q[1], V[1]), dw_mul(Q[2], V[2])), dw_mul(Q[3], V[3])), 0.5f);
    Q[4] = dw_add_fast(dw_mul(V[4], K.igm1), kin);
    const dw un = dw3(&V[1], n);
    const dw c_s = dw_sqrt(dw_mul(dw_mul(K.gam, V[4]), dw_recip_fast(V[0])));
    lam = dw_add_fast(dw_abs(un), c_s);
    F[0] = dw_mul(V[0], un);
#pragma unroll
    for (int a = 0; a < 3; ++a) F[1 + a] = dw_add_fast(dw_mul(Q[1 + a], un), dw_mul(V[4], n[a]));
    F[4] = dw_mul(dw_add_fast(Q[4], V[4]), un);
}

// Shared memory (cap cells):
//   double xc[3][cap], res[5][cap]      (FP64 first, 8-byte aligned)
//   float2 staged[29][cap], inc[5][cap]
//   int    gid[cap]
template <bool SOA>
__global__ void __launch_bounds__(128, 5) face_flux_hier_dw(const mp_block_desc *__restrict__ desc, int block0,
                                                         const ushort4 *__restrict__ lmap,
                                                         const uint8_t *__restrict__ tcolor,
                                                         const int32_t *__restrict__ fp,
                                                         const double *__restrict__ fdata,
                                                         const double *__restrict__ cdata, double *__restrict__ res,
                                                         int64_t nface, int64_t ncell, int cap, dw_consts K,
                                                         int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *s_xc = reinterpret_cast<double *>(smem_raw);
    double *s_res = s_xc + 3 * cap;
    float2 *s_st = reinterpret_cast<float2 *>(s_res + 5 * cap);
    float2 *s_inc = s_st + kDwStaged * cap;
    int *s_gid = reinterpret_cast<int *>(s_inc + 5 * cap);

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nc = d.fp_count[0];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gid + cap) - smem_raw) > dynamic_smem_bytes() || nc > cap ||
        d.nitems > (int)blockDim.x) {
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
        my_color = tcolor[f];
    }
    for (int i = tid; i < nc; i += blockDim.x) {
        const int64_t g = fpc[i];
        auto at = [&](int k) { return SOA ? cdata[k * ncell + g] : cdata[kCell * g + k]; };
        // prepared cell: V, T, grad T in double-word
        dw Q[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) Q[k] = dw_from_double_int(at(k));
        const dw ri = dw_recip_fast(Q[0]);
        const dw u = dw_mul(Q[1], ri), v = dw_mul(Q[2], ri), w = dw_mul(Q[3], ri);
        const dw kin = dw_scale2(dw_add_fast(dw_add_fast(dw_mul(Q[1], u), dw_mul(Q[2], v)), dw_mul(Q[3], w)), 0.5f);
        const dw p = dw_mul(K.gm1, dw_add(Q[4], dw_neg(kin)));
        const dw T = dw_mul(p, ri);
        st2(s_st, 0 * cap + i, Q[0]);
        st2(s_st, 1 * cap + i, u);
        st2(s_st, 2 * cap + i, v);
        st2(s_st, 3 * cap + i, w);
        st2(s_st, 4 * cap + i, p);
        st2(s_st, kSlotT * cap + i, T);
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
            const dw grho = dw_from_double_int(at(5 + dd)), gp = dw_from_double_int(at(17 + dd));
            st2(s_st, (kSlotGT + dd) * cap + i, dw_mul(dw_add(gp, dw_neg(dw_mul(T, grho))), ri));
        }
#pragma unroll 5
        for (int k = 0; k < 15; ++k) st2(s_st, (kSlotG + k) * cap + i, dw_from_double_int(at(5 + k)));
#pragma unroll
        for (int k = 0; k < 5; ++k) st2(s_st, (kSlotPhi + k) * cap + i, dw_from_double_int(at(20 + k)));
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) s_xc[dd * cap + i] = at(25 + dd);
#pragma unroll
        for (int k = 0; k < 5; ++k) s_inc[k * cap + i] = make_float2(0.0f, 0.0f);
        s_gid[i] = (int)g;
        mp_pdl_wait();  // res: written by the previous colour's launch
#pragma unroll
        for (int k = 0; k < 5; ++k) s_res[k * cap + i] = SOA ? res[k * ncell + g] : res[5 * g + k];
    }
    __syncthreads();

    dw out[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (active) {
        double fd[kFace];
#pragma unroll
        for (int k = 0; k < kFace; ++k) fd[k] = SOA ? fdata[k * nface + f] : fdata[kFace * f + k];
        const double xf[3] = {fd[3], fd[4], fd[5]};
        dw A[3], n[3], dx[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            A[k] = dw_from_double_int(fd[k]);
            n[k] = dw_from_double_int(fd[6 + k]);
            dx[k] = dw_from_double_int(fd[9 + k]);
        }
        {
            dw Q1[5], F1[5], l1, Q2[5], F2[5], l2;
            dw_side(s_st, cap, c1, s_xc, xf, n, K, Q1, F1, l1);
            dw_side(s_st, cap, c2, s_xc, xf, n, K, Q2, F2, l2);
            const dw lam = dw_max(l1, l2);
            const dw area = dw_sqrt(dw3(A, A));
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const dw diss = dw_scale2(dw_mul(lam, dw_add_fast(Q2[k], dw_neg(Q1[k]))), 0.5f);
                out[k] = dw_mul(area, dw_add_fast(dw_scale2(dw_add_fast(F1[k], F2[k]), 0.5f), dw_neg(diss)));
            }
        }
        // viscous and heat flux from the corrected face gradients
        const dw idd = dw_recip_fast(dw3(dx, dx));
        dw gu[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dw gm[3];
#pragma unroll
            for (int dd = 0; dd < 3; ++dd)
                gm[dd] = dw_scale2(dw_add_fast(ld2(s_st, (kSlotG + 3 * (1 + a) + dd) * cap + c1),
                                               ld2(s_st, (kSlotG + 3 * (1 + a) + dd) * cap + c2)),
                                   0.5f);
            const dw dv = dw_add_fast(ld2(s_st, (1 + a) * cap + c2), dw_neg(ld2(s_st, (1 + a) * cap + c1)));
            const dw corr = dw_mul(dw_add_fast(dv, dw_neg(dw3(gm, dx))), idd);
#pragma unroll
            for (int dd = 0; dd < 3; ++dd) gu[a][dd] = dw_add_fast(gm[dd], dw_mul(corr, dx[dd]));
        }
        dw gT[3];
        {
            dw gm[3];
#pragma unroll
            for (int dd = 0; dd < 3; ++dd)
                gm[dd] = dw_scale2(
                    dw_add_fast(ld2(s_st, (kSlotGT + dd) * cap + c1), ld2(s_st, (kSlotGT + dd) * cap + c2)), 0.5f);
            const dw dT = dw_add_fast(ld2(s_st, kSlotT * cap + c2), dw_neg(ld2(s_st, kSlotT * cap + c1)));
            const dw corr = dw_mul(dw_add_fast(dT, dw_neg(dw3(gm, dx))), idd);
#pragma unroll
            for (int dd = 0; dd < 3; ++dd) gT[dd] = dw_add_fast(gm[dd], dw_mul(corr, dx[dd]));
        }
        const dw div23 = dw_mul(K.two3, dw_add_fast(dw_add_fast(gu[0][0], gu[1][1]), gu[2][2]));
        dw tA[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dw_acc S = dw_dot_begin(dw_add_fast(gu[a][0], gu[0][a]), A[0]);
            dw_dot_add(S, dw_add_fast(gu[a][1], gu[1][a]), A[1]);
            dw_dot_add(S, dw_add_fast(gu[a][2], gu[2][a]), A[2]);
            dw_dot_add(S, dw_neg(div23), A[a]);
            tA[a] = dw_mul(K.mu, dw_dot_end(S));
        }
        dw uf[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            uf[a] = dw_scale2(dw_add_fast(ld2(s_st, (1 + a) * cap + c1), ld2(s_st, (1 + a) * cap + c2)), 0.5f);
        dw_acc S = dw_dot_begin(uf[0], tA[0]);
        dw_dot_add(S, uf[1], tA[1]);
        dw_dot_add(S, uf[2], tA[2]);
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) dw_dot_add(S, dw_mul(K.kappa, gT[dd]), A[dd]);
#pragma unroll
        for (int a = 0; a < 3; ++a) out[1 + a] = dw_add_fast(out[1 + a], dw_neg(tA[a]));
        out[4] = dw_add_fast(out[4], dw_neg(dw_dot_end(S)));
    }
    for (int col = 0; col < d.ncolors; ++col) {
        if (my_color == col) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                st2(s_inc, k * cap + c1, dw_add_fast(ld2(s_inc, k * cap + c1), out[k]));
                st2(s_inc, k * cap + c2, dw_add_fast(ld2(s_inc, k * cap + c2), dw_neg(out[k])));
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < nc; i += blockDim.x) {
        const int64_t g = s_gid[i];
#pragma unroll
        for (int k = 0; k < 5; ++k)
            (SOA ? res[k * ncell + g] : res[5 * g + k]) = f64_add_dw(s_res[k * cap + i], ld2(s_inc, k * cap + i));
    }
}

dw dw_const(double c)
{
    const float h = (float)c;
    return {h, (float)(c - (double)h)};
}

template <bool SOA>
int face_flux_dw_t(const mp_plan *P, const void *fdata, const void *cdata, void *res, double gam, double mu, double pr,
                   cudaStream_t s)
{
    if (P->opts.block_size > 128) return MP_EINVAL;
    const int64_t nface = P->from_size, ncell = P->maps[0].to_size;
    const int cap = P->stats.footprint_max[0];
    const int smem = cap * (3 * 8 + 5 * 8 + kDwStaged * 8 + 5 * 8 + 4);
    auto kern = face_flux_hier_dw<SOA>;
    int rc = mp_allow_smem(kern, smem);
    if (rc != MP_OK) return rc;
    int *err = nullptr;
    if ((rc = mp_device_error_word(&err)) != MP_OK) return rc;
    const dw_consts K{dw_const(gam - 1.0), dw_const(1.0 / (gam - 1.0)), dw_const(gam), dw_const(mu),
                      dw_const(mu * gam / ((gam - 1.0) * pr)), dw_const(2.0 / 3.0)};
    bool overlap = false;
    for (int c = 0; c < P->ncolors; ++c) {
        const int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
        if (nb == 0) continue;
        MP_CUDA_TRY(mp_launch(kern, nb, P->opts.block_size, smem, s, overlap, P->dev.desc, b0,
                              reinterpret_cast<const ushort4 *>(P->dev.lmap), P->dev.tcolor, P->dev.fp,
                              (const double *)fdata, (const double *)cdata, (double *)res, nface, ncell, cap, K, err));
        overlap = true;
    }
    return MP_OK;
}

}  // namespace

int mp_face_flux_dw(const mp_plan *P, const void *fdata, const void *cdata, void *res, double gam, double mu,
                    double pr, void *stream)
{
    if (P->opts.coloring != MP_COLOR_HIER) return MP_EPLAN;
    return P->opts.layout == MP_LAYOUT_SOA ? face_flux_dw_t<true>(P, fdata, cdata, res, gam, mu, pr, as_stream(stream))
                                           : face_flux_dw_t<false>(P, fdata, cdata, res, gam, mu, pr, as_stream(stream));
}
