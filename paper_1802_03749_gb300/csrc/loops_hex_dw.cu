// Hex assembly with FP64 data and double-word (FP32 pair) arithmetic: the
// FP64-accurate variant for GB300, where about 550 FP64 operations per
// element would otherwise run on the FP64 pipe (2 per clock per SM).
//
// Staged two-layer structure as hex_hier: the block's node footprint (x, v
// converted to double-word, and the current f in FP64) is staged in shared
// memory; each thread computes one element's forces in double-word
// arithmetic; the 24 increments either go to a shared force buffer that
// each node then sums through the plan's gather rows (the default), or
// accumulate in shared memory one thread colour at a time (MP_STAGED_SIMPLE);
// each footprint node's f is written back once
// (FP64 + double-word, two FP64 additions).  Element volumes are written
// directly.  The formulas are those of the FP64 kernel (loops_hex.cu).
// GLOBAL and ATOMIC plans run the baselines of Sec. 2.1 in the same
// arithmetic (hex_direct_dw).
#include "common.cuh"
#include "dw.cuh"

namespace {

__device__ __forceinline__ constexpr int sx(int i) { return (i == 1 || i == 2 || i == 5 || i == 6) ? 1 : -1; }
__device__ __forceinline__ constexpr int sy(int i) { return (i == 2 || i == 3 || i == 6 || i == 7) ? 1 : -1; }
__device__ __forceinline__ constexpr int sz(int i) { return i >= 4 ? 1 : -1; }

__device__ __forceinline__ dw ld2(const float2 *a, int i)
{
    float2 v = a[i];
    return {v.x, v.y};
}
__device__ __forceinline__ void st2(float2 *a, int i, dw v) { a[i] = make_float2(v.hi, v.lo); }
__device__ __forceinline__ dw sgn(dw x, int s) { return s > 0 ? x : dw_neg(x); }

// a*b - c*d as one compensated sum
__device__ __forceinline__ dw dw_det2(dw a, dw b, dw c, dw d)
{
    dw_acc A = dw_dot_begin(a, b);
    dw_dot_add(A, dw_neg(c), d);
    return dw_dot_end(A);
}

// smem per footprint node: x[3], v[3], increments[3] (coloured form) as
// double-word, f[3] prefetched in FP64 (24 B), global id (4 B); the gather
// form has no increments but one row of gather entries (gw4 x 8 B) per node
// and a force buffer of 24 double-words per thread
constexpr int kHexDwNodeBytes = 9 * 8 + 24 + 4;

// force of element corner i: stress sum_b xi_i[b] t[a][b] minus the hourglass
// sum_k g_{k,i} q_k[a]
__device__ __forceinline__ void corner_force(int i, const dw t[3][3], const dw w[4][3], const dw qk[4][3], dw iV,
                                             dw fa[3])
{
    dw gi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int Gk = k == 0 ? sy(i) * sz(i) : (k == 1 ? sx(i) * sz(i) : (k == 2 ? sx(i) * sy(i) : sx(i) * sy(i) * sz(i)));
        const dw xb = dw_add_fast(dw_add_fast(sgn(w[k][0], sx(i)), sgn(w[k][1], sy(i))), sgn(w[k][2], sz(i)));
        gi[k] = dw_add_fast(dw{(float)Gk, 0.f}, dw_neg(dw_mul(xb, iV)));
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const dw st = dw_add_fast(dw_add_fast(sgn(t[a][0], sx(i)), sgn(t[a][1], sy(i))), sgn(t[a][2], sz(i)));
        dw_acc H = dw_dot_begin(gi[0], qk[0][a]);
        dw_dot_add(H, gi[1], qk[1][a]);
        dw_dot_add(H, gi[2], qk[2][a]);
        dw_dot_add(H, gi[3], qk[3][a]);
        fa[a] = dw_add_fast(st, dw_neg(dw_dot_end(H)));
    }
}

// The element quantities that the corner forces need, in double-word
// arithmetic, from accessors X(a, i), Vel(a, i) (component a of corner i's
// coordinates and velocity) and Sig(a) (the element's stress component a);
// Vol(V) receives the volume V = 8 det J as soon as it is known.
// With C = cof(J) and B_i = C xi_i:
//   stress   f_i[a] = -s_a B_i[a] = sum_b xi_i[b] t[a][b],  t[a][b] = -s_a C[a][b]
//   hourglass g_{k,i} = Gamma_{k,i} - (xi_i . w_k) / V,    w_k[b] = sum_a h_k[a] C[a][b]
//            q_k = kappa sum_j g_{k,j} v_j,  f_i -= sum_k g_{k,i} q_k
// so only t, w and q (not the 8 B_i) are kept between the two phases;
// iV = 1/V.
template <typename FX, typename FV, typename FS, typename FW>
__device__ __forceinline__ void hex_terms_dw(FX X, FV Vel, FS Sig, FW Vol, dw kappa, dw t[3][3], dw w[4][3],
                                             dw qk[4][3], dw &iV)
{
    // J = 1/8 sum_i x_i xi_i^T
    dw J[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const dw x0 = X(a, 0);
        dw j0 = sgn(x0, sx(0)), j1 = sgn(x0, sy(0)), j2 = sgn(x0, sz(0));
#pragma unroll
        for (int i = 1; i < 8; ++i) {
            const dw xi = X(a, i);
            j0 = dw_add_fast(j0, sgn(xi, sx(i)));
            j1 = dw_add_fast(j1, sgn(xi, sy(i)));
            j2 = dw_add_fast(j2, sgn(xi, sz(i)));
        }
        J[a][0] = dw_scale2(j0, 0.125f);
        J[a][1] = dw_scale2(j1, 0.125f);
        J[a][2] = dw_scale2(j2, 0.125f);
    }
    dw C[3][3];
    C[0][0] = dw_det2(J[1][1], J[2][2], J[1][2], J[2][1]);
    C[0][1] = dw_det2(J[1][2], J[2][0], J[1][0], J[2][2]);
    C[0][2] = dw_det2(J[1][0], J[2][1], J[1][1], J[2][0]);
    C[1][0] = dw_det2(J[0][2], J[2][1], J[0][1], J[2][2]);
    C[1][1] = dw_det2(J[0][0], J[2][2], J[0][2], J[2][0]);
    C[1][2] = dw_det2(J[0][1], J[2][0], J[0][0], J[2][1]);
    C[2][0] = dw_det2(J[0][1], J[1][2], J[0][2], J[1][1]);
    C[2][1] = dw_det2(J[0][2], J[1][0], J[0][0], J[1][2]);
    C[2][2] = dw_det2(J[0][0], J[1][1], J[0][1], J[1][0]);
    dw_acc A = dw_dot_begin(J[0][0], C[0][0]);
    dw_dot_add(A, J[0][1], C[0][1]);
    dw_dot_add(A, J[0][2], C[0][2]);
    const dw V = dw_scale2(dw_dot_end(A), 8.0f);
    Vol(V);
    iV = dw_recip(V);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const dw sa = Sig(a);
#pragma unroll
        for (int b = 0; b < 3; ++b) t[a][b] = dw_neg(dw_mul(sa, C[a][b]));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int G[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            G[j] = k == 0 ? sy(j) * sz(j) : (k == 1 ? sx(j) * sz(j) : (k == 2 ? sx(j) * sy(j) : sx(j) * sy(j) * sz(j)));
        dw h[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            h[a] = sgn(X(a, 0), G[0]);
#pragma unroll
            for (int j = 1; j < 8; ++j) h[a] = dw_add_fast(h[a], sgn(X(a, j), G[j]));
        }
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            dw_acc P = dw_dot_begin(h[0], C[0][b]);
            dw_dot_add(P, h[1], C[1][b]);
            dw_dot_add(P, h[2], C[2][b]);
            w[k][b] = dw_dot_end(P);
        }
        dw_acc Q[3];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const dw xb = dw_add_fast(dw_add_fast(sgn(w[k][0], sx(j)), sgn(w[k][1], sy(j))), sgn(w[k][2], sz(j)));
            const dw gj = dw_add_fast(dw{(float)G[j], 0.f}, dw_neg(dw_mul(xb, iV)));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const dw vj = Vel(a, j);
                if (j == 0)
                    Q[a] = dw_dot_begin(gj, vj);
                else
                    dw_dot_add(Q[a], gj, vj);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) qk[k][a] = dw_mul(dw_dot_end(Q[a]), kappa);
    }
}

template <bool SOA, bool GATHER>
__global__ void __launch_bounds__(256, 2) hex_hier_dw(const mp_block_desc *__restrict__ desc, int block0,
                                                   const uint4 *__restrict__ lmap, const uint8_t *__restrict__ tcolor,
                                                   const ushort4 *__restrict__ gat, int gw4,
                                                   const int32_t *__restrict__ fp, const double *__restrict__ x,
                                                   const double *__restrict__ v, const double *__restrict__ sig,
                                                   double *__restrict__ f, double *__restrict__ vol, int64_t nnode,
                                                   int64_t nelem, int cap, int cap_f, dw kappa,
                                                   int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *s_f = reinterpret_cast<double *>(smem_raw);    // [3][cap] FP64
    float2 *s_x = reinterpret_cast<float2 *>(s_f + 3 * cap);  // [3][cap]
    float2 *s_v = s_x + 3 * cap;                           // [3][cap]
    float2 *s_i = s_v + 3 * cap;                           // coloured: [3][cap] increments
    float2 *s_fb = s_i + (GATHER ? 0 : 3 * cap);           // gather: [24][cap_f] corner forces
    ushort4 *s_ge = reinterpret_cast<ushort4 *>(s_fb + (GATHER ? 24 * cap_f : 0));  // gather: [gw4][cap]
    int *s_gid = reinterpret_cast<int *>(s_ge + (GATHER ? gw4 * cap : 0));

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nn = d.fp_count[0];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gid + cap) - smem_raw) > dynamic_smem_bytes() || nn > cap ||
        d.nitems > (int)blockDim.x || (GATHER && ((int)blockDim.x > cap_f || gw4 < 1 || gw4 > 4))) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpn = fp + d.fp_start[0];
    const bool active = tid < d.nitems;
    uint4 l = make_uint4(0, 0, 0, 0);
    int my_color = -1;
    if (active) {
        l = lmap[d.item_start + tid];
        if (!GATHER) my_color = tcolor[d.item_start + tid];
    }
    // nodes, two per thread and pass: both nodes' index and coordinate loads
    // are issued before either is converted, so a block's footprint (often
    // between one and two nodes per thread) costs one chain of dependent
    // loads instead of two
    auto stage_node = [&](int i, int64_t g, const double (&xv)[6]) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            st2(s_x, a * cap + i, dw_from_double_int(xv[a]));
            st2(s_v, a * cap + i, dw_from_double_int(xv[3 + a]));
        }
        if (GATHER) {
            const ushort4 *row = gat + (int64_t)(d.fp_start[0] + i) * gw4;
            for (int h = 0; h < gw4; ++h) s_ge[h * cap + i] = row[h];
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) s_i[a * cap + i] = make_float2(0.f, 0.f);
        }
        s_gid[i] = (int)g;
    };
    auto load_xv = [&](int64_t g, double (&xv)[6]) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int64_t j = SOA ? a * nnode + g : 3 * g + a;
            xv[a] = x[j];
            xv[3 + a] = v[j];
        }
    };
    auto load_f = [&](int i, int64_t g) {  // f: written by the previous colour's launch
#pragma unroll
        for (int a = 0; a < 3; ++a) s_f[a * cap + i] = f[SOA ? a * nnode + g : 3 * g + a];
    };
    for (int i0 = tid; i0 < nn; i0 += 2 * (int)blockDim.x) {
        const int i1 = i0 + (int)blockDim.x;
        const bool two = i1 < nn;
        const int64_t g0 = fpn[i0], g1 = two ? fpn[i1] : g0;
        double xv0[6], xv1[6];
        load_xv(g0, xv0);
        if (two) load_xv(g1, xv1);
        stage_node(i0, g0, xv0);
        if (two) stage_node(i1, g1, xv1);
        mp_pdl_wait();
        load_f(i0, g0);
        if (two) load_f(i1, g1);
    }
    __syncthreads();
    // the element's force terms from the staged nodes
    int loc[8];
    dw t[3][3], w[4][3], qk[4][3], iV;
    if (active) {
        const int e = d.item_start + tid;
        loc[0] = l.x & 0xffff;
        loc[1] = l.x >> 16;
        loc[2] = l.y & 0xffff;
        loc[3] = l.y >> 16;
        loc[4] = l.z & 0xffff;
        loc[5] = l.z >> 16;
        loc[6] = l.w & 0xffff;
        loc[7] = l.w >> 16;
        hex_terms_dw([&](int a, int i) { return ld2(s_x, a * cap + loc[i]); },
                     [&](int a, int i) { return ld2(s_v, a * cap + loc[i]); },
                     [&](int a) { return dw_from_double_int(SOA ? sig[a * nelem + e] : sig[3 * (int64_t)e + a]); },
                     [&](dw V) { vol[e] = dw_to_double(V); }, kappa, t, w, qk, iV);
    }
    if constexpr (GATHER) {
        // every thread writes its 24 corner forces at once, then each node
        // sums the forces of its elements in the block (plan's gather rows)
        if (active) {
            // one corner at a time (not unrolled: unrolling spills registers)
#pragma unroll 1
            for (int i = 0; i < 8; ++i) {
                dw fa[3];
                corner_force(i, t, w, qk, iV, fa);
#pragma unroll
                for (int a = 0; a < 3; ++a) st2(s_fb, (3 * i + a) * cap_f + tid, fa[a]);
            }
        }
        __syncthreads();
        // compensated double-word sums, branch-free: a padding entry adds 0
        // times corner 0 of thread 0 (computed in every block)
        for (int i = tid; i < nn; i += blockDim.x) {
            dw_acc S[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            for (int h = 0; h < gw4; ++h) {
                const ushort4 e4 = s_ge[h * cap + i];
                const unsigned short es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned en = es[j];
                    const bool valid = en != 0xFFFFu;
                    const int te = valid ? (int)(en >> 4) : 0, corner = valid ? (int)(en & 15u) : 0;
                    const float sg = valid ? 1.0f : 0.0f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) dw_sum_add(S[a], ld2(s_fb, (3 * corner + a) * cap_f + te), sg);
                }
            }
            const int64_t g = s_gid[i];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                f[SOA ? a * nnode + g : 3 * g + a] = f64_add_dw(s_f[a * cap + i], dw_sum_end(S[a]));
        }
    } else {
        for (int c = 0; c < d.ncolors; ++c) {
            if (my_color == c) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    dw fa[3];
                    corner_force(i, t, w, qk, iV, fa);
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        st2(s_i, a * cap + loc[i], dw_add_fast(ld2(s_i, a * cap + loc[i]), fa[a]));
                }
            }
            __syncthreads();
        }
        for (int i = tid; i < nn; i += blockDim.x) {
            const int64_t g = s_gid[i];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                f[SOA ? a * nnode + g : 3 * g + a] = f64_add_dw(s_f[a * cap + i], ld2(s_i, a * cap + i));
        }
    }
}

// The baselines of Sec. 2.1 in the same double-word arithmetic, so that the
// strategies compare at equal arithmetic: one thread per element of
// [e0, e1) gathers its 8 nodes' x and v from global memory (FP64), converts
// them into its own slice of shared memory (private scratch: no thread reads
// another's), computes the element as the staged kernel does, writes vol and
// adds its 24 corner forces to f:
//   GLOBAL (elements of one colour share no node): f = f + fa in FP64 (two
//          FP64 additions, as the staged write-back);
//   ATOMIC: atomicAdd of the nearest double of fa (hi + lo, one FP64
//          addition).
constexpr int kHexDirectDwBlock = 128;
constexpr int kHexDirectDwSmem = 48 * 8 * kHexDirectDwBlock;  // x, v of 8 corners as double-words

template <bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(kHexDirectDwBlock) hex_direct_dw(int e0, int e1, const int32_t *__restrict__ e2n,
                                                                  const double *__restrict__ x,
                                                                  const double *__restrict__ v,
                                                                  const double *__restrict__ sig,
                                                                  double *__restrict__ f, double *__restrict__ vol,
                                                                  int64_t nnode, int64_t nelem, dw kappa)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *s_xv = reinterpret_cast<float2 *>(smem_raw);  // [48][blockDim]: x, then v, component-major
    mp_pdl_trigger();
    const int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;  // no barrier below: threads past the end leave
    const int nt = blockDim.x, tid = threadIdx.x;
    const int4 na = reinterpret_cast<const int4 *>(e2n)[2 * (int64_t)e];
    const int4 nb = reinterpret_cast<const int4 *>(e2n)[2 * (int64_t)e + 1];
    const int nd[8] = {na.x, na.y, na.z, na.w, nb.x, nb.y, nb.z, nb.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int64_t j = SOA ? a * nnode + nd[i] : 3 * (int64_t)nd[i] + a;
            st2(s_xv, (a * 8 + i) * nt + tid, dw_from_double_int(x[j]));
            st2(s_xv, (24 + a * 8 + i) * nt + tid, dw_from_double_int(v[j]));
        }
    }
    dw t[3][3], w[4][3], qk[4][3], iV;
    hex_terms_dw([&](int a, int i) { return ld2(s_xv, (a * 8 + i) * nt + tid); },
                 [&](int a, int i) { return ld2(s_xv, (24 + a * 8 + i) * nt + tid); },
                 [&](int a) { return dw_from_double_int(SOA ? sig[a * nelem + e] : sig[3 * (int64_t)e + a]); },
                 [&](dw V) { vol[e] = dw_to_double(V); }, kappa, t, w, qk, iV);
    if (!ATOMIC) mp_pdl_wait();  // f: read-add-written by the previous colour's launch
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
        dw fa[3];
        corner_force(i, t, w, qk, iV, fa);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int64_t j = SOA ? a * nnode + nd[i] : 3 * (int64_t)nd[i] + a;
            if (ATOMIC)
                atomicAdd(f + j, f32_to_f64_int(fa[a].hi) + f32_to_f64_int(fa[a].lo));
            else
                f[j] = f64_add_dw(f[j], fa[a]);
        }
    }
}

template <bool SOA>
int hex_direct_dw_t(const mp_plan *P, const void *x, const void *v, const void *sig, void *f, void *vol, dw kap,
                    cudaStream_t s)
{
    const bool atomic = P->opts.coloring == MP_COLOR_ATOMIC;
    auto kern = atomic ? hex_direct_dw<SOA, true> : hex_direct_dw<SOA, false>;
    int rc = mp_allow_smem(kern, kHexDirectDwSmem);
    if (rc != MP_OK) return rc;
    bool overlap = false;
    for (int c = 0; c < P->ncolors; ++c) {
        const int e0 = P->color_offsets[c], e1 = P->color_offsets[c + 1];
        if (e1 <= e0) continue;
        MP_CUDA_TRY(mp_launch(kern, (e1 - e0 + kHexDirectDwBlock - 1) / kHexDirectDwBlock, kHexDirectDwBlock,
                              kHexDirectDwSmem, s, overlap && !atomic, e0, e1, P->dev.map[0], (const double *)x,
                              (const double *)v, (const double *)sig, (double *)f, (double *)vol, P->maps[0].to_size,
                              P->from_size, kap));
        overlap = true;
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

template <bool SOA>
int hex_dw_t(const mp_plan *P, const void *x, const void *v, const void *sig, void *f, void *vol, double kappa,
             cudaStream_t s)
{
    if (P->opts.block_size > 256) return MP_EINVAL;
    const int cap = P->stats.footprint_max[0];
    const bool gather = mp_staged(P, MP_STAGED_GATHER) == MP_STAGED_GATHER && mp_gather_ready(P);
    const int gw4 = gather ? P->gat_w / 4 : 0, cap_f = gather ? P->opts.block_size : 0;
    const int smem = cap * (gather ? kHexDwNodeBytes - 24 : kHexDwNodeBytes) + 24 * 8 * cap_f + 8 * gw4 * cap;
    auto kern = gather ? hex_hier_dw<SOA, true> : hex_hier_dw<SOA, false>;
    int rc = mp_allow_smem(kern, smem);
    if (rc != MP_OK) return rc;
    int *err = nullptr;
    if ((rc = mp_device_error_word(&err)) != MP_OK) return rc;
    const float kh = (float)kappa;
    const dw kap{kh, (float)(kappa - (double)kh)};
    bool overlap = false;
    for (int c = 0; c < P->ncolors; ++c) {
        const int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
        if (nb == 0) continue;
        MP_CUDA_TRY(mp_launch(kern, nb, P->opts.block_size, smem, s, overlap, P->dev.desc, b0,
                              reinterpret_cast<const uint4 *>(P->dev.lmap), P->dev.tcolor,
                              reinterpret_cast<const ushort4 *>(P->dev.gat), gw4, P->dev.fp, (const double *)x,
                              (const double *)v, (const double *)sig, (double *)f, (double *)vol, P->maps[0].to_size,
                              P->from_size, cap, cap_f, kap, err));
        overlap = true;
    }
    return MP_OK;
}

}  // namespace

int mp_hex_dw(const mp_plan *P, const void *x, const void *v, const void *sig, void *f, void *vol, double kappa,
              void *stream)
{
    const bool soa = P->opts.layout == MP_LAYOUT_SOA;
    if (P->opts.coloring == MP_COLOR_GLOBAL || P->opts.coloring == MP_COLOR_ATOMIC) {
        const float kh = (float)kappa;
        const dw kap{kh, (float)(kappa - (double)kh)};
        return soa ? hex_direct_dw_t<true>(P, x, v, sig, f, vol, kap, as_stream(stream))
                   : hex_direct_dw_t<false>(P, x, v, sig, f, vol, kap, as_stream(stream));
    }
    if (P->opts.coloring != MP_COLOR_HIER) return MP_EPLAN;
    return soa ? hex_dw_t<true>(P, x, v, sig, f, vol, kappa, as_stream(stream))
               : hex_dw_t<false>(P, x, v, sig, f, vol, kappa, as_stream(stream));
}
