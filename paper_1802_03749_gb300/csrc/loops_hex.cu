// Hex assembly (the access pattern of IntegrateStressForElems, Sec. 3.1.4):
// per hex8 element gather x and v on 8 nodes, read sig directly, compute the
// one-point stress force and Flanagan-Belytschko hourglass force, write the
// element volume directly and increment the nodal force on 8 nodes.
//
// Variants (plan colouring): HIER stages the block's node footprint (x, v)
// in shared memory and applies the 24 increments per element one thread
// colour at a time (hex_hier), with shared-memory atomics (hex_hier_c, the
// compact element terms) or warp-aggregated atomics, then writes each
// footprint node back once; GLOBAL runs one launch per element colour with
// direct global read-add-writes and ATOMIC uses atomicAdd on f (both
// hex_direct_c); TWOSTEP writes per-corner forces for a gather.
#include "common.cuh"

namespace {

// Corner signs of the reference element in the elem->node order:
// (-,-,-),(+,-,-),(+,+,-),(-,+,-),(-,-,+),(+,-,+),(+,+,+),(-,+,+).
__device__ __forceinline__ constexpr int sx(int i) { return (i == 1 || i == 2 || i == 5 || i == 6) ? 1 : -1; }
__device__ __forceinline__ constexpr int sy(int i) { return (i == 2 || i == 3 || i == 6 || i == 7) ? 1 : -1; }
__device__ __forceinline__ constexpr int sz(int i) { return i >= 4 ? 1 : -1; }

// Element forces fe[i][a] (i = corner, a = component) and volume for corner
// coordinates xe and velocities ve:
//   J = 1/8 sum_i x_i xi_i^T, V = 8 det J, B_i = cof(J) xi_i,
//   f_i = -diag(sig) B_i - kappa sum_k g_{k,i} sum_j g_{k,j} v_j,
//   g_{k,i} = Gamma_{k,i} - (sum_j Gamma_{k,j} x_j) . B_i / V.
template <typename T>
__device__ __forceinline__ void hex_element(const T xe[8][3], const T ve[8][3], T s0, T s1, T s2, T kappa,
                                            T fe[8][3], T &vol)
{
    T J[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T j0 = T(0), j1 = T(0), j2 = T(0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            j0 += sx(i) > 0 ? xe[i][a] : -xe[i][a];
            j1 += sy(i) > 0 ? xe[i][a] : -xe[i][a];
            j2 += sz(i) > 0 ? xe[i][a] : -xe[i][a];
        }
        J[a][0] = T(0.125) * j0;
        J[a][1] = T(0.125) * j1;
        J[a][2] = T(0.125) * j2;
    }
    T C[3][3];
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    T det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    T V = T(8) * det;
    vol = V;
    T B[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            B[i][a] = (sx(i) > 0 ? C[a][0] : -C[a][0]) + (sy(i) > 0 ? C[a][1] : -C[a][1]) +
                      (sz(i) > 0 ? C[a][2] : -C[a][2]);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        fe[i][0] = -s0 * B[i][0];
        fe[i][1] = -s1 * B[i][1];
        fe[i][2] = -s2 * B[i][2];
    }
    const T iV = T(1) / V;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // Gamma_k: eta zeta, xi zeta, xi eta, xi eta zeta
        T h[3] = {T(0), T(0), T(0)};
        int G[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            G[j] = k == 0 ? sy(j) * sz(j) : (k == 1 ? sx(j) * sz(j) : (k == 2 ? sx(j) * sy(j) : sx(j) * sy(j) * sz(j)));
#pragma unroll
            for (int a = 0; a < 3; ++a) h[a] += G[j] > 0 ? xe[j][a] : -xe[j][a];
        }
        T g[8];
        T qk[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            g[i] = T(G[i]) - (h[0] * B[i][0] + h[1] * B[i][1] + h[2] * B[i][2]) * iV;
#pragma unroll
            for (int a = 0; a < 3; ++a) qk[a] += g[i] * ve[i][a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) qk[a] *= kappa;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int a = 0; a < 3; ++a) fe[i][a] -= g[i] * qk[a];
    }
}

template <typename T, bool SOA>
__device__ __forceinline__ void load3(const T *__restrict__ p, int64_t n, int64_t i, T &a, T &b, T &c)
{
    if (SOA) {
        a = p[i];
        b = p[n + i];
        c = p[2 * n + i];
    } else {
        a = p[3 * i];
        b = p[3 * i + 1];
        c = p[3 * i + 2];
    }
}

// smem per footprint node: one record of 8 values (x, y, z, - | vx, vy, vz,
// -), read with one vector load per position or velocity; f (prefetched,
// incremented)[3] and the global id
template <typename T>
__host__ __device__ constexpr int hex_smem_per_node()
{
    return 11 * (int)sizeof(T) + 4;
}

// A node record of 8 values in shared memory (16-byte aligned).
template <typename T>
__device__ __forceinline__ void st_node_rec(T *rec, int i, const T xv[6])
{
    if (sizeof(T) == 8) {
        double2 *p = reinterpret_cast<double2 *>(rec) + 4 * i;
        p[0] = make_double2((double)xv[0], (double)xv[1]);
        p[1] = make_double2((double)xv[2], 0.0);
        p[2] = make_double2((double)xv[3], (double)xv[4]);
        p[3] = make_double2((double)xv[5], 0.0);
    } else {
        float4 *p = reinterpret_cast<float4 *>(rec) + 2 * i;
        p[0] = make_float4((float)xv[0], (float)xv[1], (float)xv[2], 0.f);
        p[1] = make_float4((float)xv[3], (float)xv[4], (float)xv[5], 0.f);
    }
}
// half h of record i: 0 the position, 1 the velocity
template <typename T>
__device__ __forceinline__ void ld_node_half(const T *rec, int i, int h, T o[3])
{
    if (sizeof(T) == 8) {
        const double2 *p = reinterpret_cast<const double2 *>(rec) + 4 * i + 2 * h;
        const double2 a = p[0], b = p[1];
        o[0] = (T)a.x;
        o[1] = (T)a.y;
        o[2] = (T)b.x;
    } else {
        const float4 a = reinterpret_cast<const float4 *>(rec)[2 * i + h];
        o[0] = (T)a.x;
        o[1] = (T)a.y;
        o[2] = (T)a.z;
    }
}
template <typename T>
__device__ __forceinline__ void ld_node_rec(const T *rec, int i, T xe[3], T ve[3])
{
    ld_node_half(rec, i, 0, xe);
    ld_node_half(rec, i, 1, ve);
}

// The element quantities the corner forces need, in the compact form that
// keeps few values alive (the same algebra as hex_element): with C =
// cof(J) and B_i = C xi_i,
//   stress   f_i[a] = -s_a B_i[a] = sum_b xi_i[b] t[a][b],  t[a][b] = -s_a C[a][b]
//   hourglass g_{k,i} = Gamma_{k,i} - (xi_i . w_k) / V,    w_k[b] = sum_a h_k[a] C[a][b],
//            h_k = sum_j Gamma_{k,j} x_j,  q_k = kappa sum_j g_{k,j} v_j,
//   f_i -= sum_k g_{k,i} q_k.
// Vel(j, v) gives corner j's velocity.  Returns V = 8 det J; iV = 1/V.
template <typename T, typename FV>
__device__ __forceinline__ T hex_terms(const T xe[8][3], FV Vel, T s0, T s1, T s2, T kappa, T t[3][3], T w[4][3],
                                       T qk[4][3], T &iV)
{
    T J[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T j0 = T(0), j1 = T(0), j2 = T(0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            j0 += sx(i) > 0 ? xe[i][a] : -xe[i][a];
            j1 += sy(i) > 0 ? xe[i][a] : -xe[i][a];
            j2 += sz(i) > 0 ? xe[i][a] : -xe[i][a];
        }
        J[a][0] = T(0.125) * j0;
        J[a][1] = T(0.125) * j1;
        J[a][2] = T(0.125) * j2;
    }
    T C[3][3];
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const T V = T(8) * (J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2]);
    iV = T(1) / V;
    const T sg[3] = {s0, s1, s2};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) t[a][b] = -sg[a] * C[a][b];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int G[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            G[j] = k == 0 ? sy(j) * sz(j) : (k == 1 ? sx(j) * sz(j) : (k == 2 ? sx(j) * sy(j) : sx(j) * sy(j) * sz(j)));
        T h[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a) h[a] += G[j] > 0 ? xe[j][a] : -xe[j][a];
#pragma unroll
        for (int b = 0; b < 3; ++b) w[k][b] = h[0] * C[0][b] + h[1] * C[1][b] + h[2] * C[2][b];
        T Q[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const T xb = (sx(j) > 0 ? w[k][0] : -w[k][0]) + (sy(j) > 0 ? w[k][1] : -w[k][1]) +
                         (sz(j) > 0 ? w[k][2] : -w[k][2]);
            const T gj = T(G[j]) - xb * iV;
            T vj[3];
            Vel(j, vj);
#pragma unroll
            for (int a = 0; a < 3; ++a) Q[a] += gj * vj[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) qk[k][a] = kappa * Q[a];
    }
    return V;
}

// Force on corner i from the compact terms.
template <typename T>
__device__ __forceinline__ void hex_corner(int i, const T t[3][3], const T w[4][3], const T qk[4][3], T iV, T fa[3])
{
    T gi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int Gk = k == 0 ? sy(i) * sz(i) : (k == 1 ? sx(i) * sz(i) : (k == 2 ? sx(i) * sy(i) : sx(i) * sy(i) * sz(i)));
        const T xb = (sx(i) > 0 ? w[k][0] : -w[k][0]) + (sy(i) > 0 ? w[k][1] : -w[k][1]) +
                     (sz(i) > 0 ? w[k][2] : -w[k][2]);
        gi[k] = T(Gk) - xb * iV;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T st = (sx(i) > 0 ? t[a][0] : -t[a][0]) + (sy(i) > 0 ? t[a][1] : -t[a][1]) +
                     (sz(i) > 0 ? t[a][2] : -t[a][2]);
        fa[a] = st - (gi[0] * qk[0][a] + gi[1] * qk[1][a] + gi[2] * qk[2][a] + gi[3] * qk[3][a]);
    }
}

// increments: 0 thread colours, 1 shared-memory atomics, 3 warp-aggregated
// shared-memory atomics
template <typename T, bool SOA, int INC>
__global__ void __launch_bounds__(512) hex_hier(const mp_block_desc *__restrict__ desc, int block0,
                                                const uint4 *__restrict__ lmap, const uint8_t *__restrict__ tcolor,
                                                const int32_t *__restrict__ fp, const T *__restrict__ x,
                                                const T *__restrict__ v, const T *__restrict__ sig,
                                                T *__restrict__ f, T *__restrict__ vol, int64_t nnode,
                                                int64_t nelem, int cap, T kappa, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_xv = reinterpret_cast<T *>(smem_raw);  // [cap][8] node records
    T *s_f = s_xv + 8 * cap;                    // [3][cap]
    int *s_gid = reinterpret_cast<int *>(s_f + 3 * cap);

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nn = d.fp_count[0];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gid + cap) - smem_raw) > dynamic_smem_bytes() || nn > cap ||
        d.nitems > (int)blockDim.x) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpn = fp + d.fp_start[0];
    const bool active = tid < d.nitems;
    uint4 l = make_uint4(0, 0, 0, 0);
    int my_color = -1;
    if (active) {  // independent of the staging: issued first
        l = lmap[d.item_start + tid];
        my_color = tcolor[d.item_start + tid];
    }
    // stage x, v and the current f (increments accumulate onto it; blocks of
    // one colour share no node, so the write-back is a plain store)
    // nodes, two per thread and pass: both nodes' index and data loads are
    // issued before either is stored, so a footprint of one to two nodes per
    // thread costs one chain of dependent loads instead of two
    auto stage3 = [&](T *dst, int i, T a, T b, T c) {
        dst[i] = a;
        dst[cap + i] = b;
        dst[2 * cap + i] = c;
    };
    for (int i0 = tid; i0 < nn; i0 += 2 * (int)blockDim.x) {
        const int i1 = i0 + (int)blockDim.x;
        const bool two = i1 < nn;
        const int g0 = fpn[i0], g1 = two ? fpn[i1] : g0;
        T xv0[6], xv1[6];
        load3<T, SOA>(x, nnode, g0, xv0[0], xv0[1], xv0[2]);
        load3<T, SOA>(v, nnode, g0, xv0[3], xv0[4], xv0[5]);
        if (two) {
            load3<T, SOA>(x, nnode, g1, xv1[0], xv1[1], xv1[2]);
            load3<T, SOA>(v, nnode, g1, xv1[3], xv1[4], xv1[5]);
        }
        st_node_rec(s_xv, i0, xv0);
        s_gid[i0] = g0;
        if (two) {
            st_node_rec(s_xv, i1, xv1);
            s_gid[i1] = g1;
        }
        mp_pdl_wait();  // f: written by the previous colour's launch
        T f0[3], f1[3];
        load3<T, SOA>(f, nnode, g0, f0[0], f0[1], f0[2]);
        if (two) load3<T, SOA>(f, nnode, g1, f1[0], f1[1], f1[2]);
        stage3(s_f, i0, f0[0], f0[1], f0[2]);
        if (two) stage3(s_f, i1, f1[0], f1[1], f1[2]);
    }
    __syncthreads();
    T fe[8][3];
    int loc[8];
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
        T xe[8][3], ve[8][3];
#pragma unroll
        for (int i = 0; i < 8; ++i) ld_node_rec(s_xv, loc[i], xe[i], ve[i]);
        T s0, s1, s2, V;
        load3<T, SOA>(sig, nelem, e, s0, s1, s2);
        hex_element(xe, ve, s0, s1, s2, kappa, fe, V);
        vol[e] = V;
    }
    if (INC == 3) {  // warp-aggregated shared-memory atomics
        const unsigned act = __ballot_sync(0xffffffffu, active);
        if (active) {
#pragma unroll
            for (int i = 0; i < 8; ++i) warp_aggregated_add<T, 3>(act, loc[i], fe[i], s_f, cap);
        }
        __syncthreads();
    } else if (INC == 1) {  // shared-memory atomics instead of thread colours
        if (active) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int a = 0; a < 3; ++a) atomicAdd(s_f + a * cap + loc[i], fe[i][a]);
        }
        __syncthreads();
    } else {
        for (int c = 0; c < d.ncolors; ++c) {
            if (my_color == c) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int a = 0; a < 3; ++a) s_f[a * cap + loc[i]] += fe[i][a];
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < nn; i += blockDim.x) {
        int64_t g = s_gid[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int64_t j = SOA ? a * nnode + g : 3 * g + a;
            f[j] = s_f[a * cap + i];
        }
    }
}

// Step 1 of the temporary-array method (Sec. 2.1): element e's force on
// its corner i goes to scratch[(8e + i) * 3 + a]; vol is written directly.
template <typename T, bool SOA>
__global__ void __launch_bounds__(256) hex_step1(int n, const int32_t *__restrict__ e2n, const T *__restrict__ x,
                                                 const T *__restrict__ v, const T *__restrict__ sig,
                                                 T *__restrict__ scratch, T *__restrict__ vol, int64_t nnode,
                                                 int64_t nelem, T kappa)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int4 *row = reinterpret_cast<const int4 *>(e2n) + 2 * (int64_t)e;
    int4 r0 = row[0], r1 = row[1];
    const int nd[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    T xe[8][3], ve[8][3], fe[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        load3<T, SOA>(x, nnode, nd[i], xe[i][0], xe[i][1], xe[i][2]);
        load3<T, SOA>(v, nnode, nd[i], ve[i][0], ve[i][1], ve[i][2]);
    }
    T s0, s1, s2, V;
    load3<T, SOA>(sig, nelem, e, s0, s1, s2);
    hex_element(xe, ve, s0, s1, s2, kappa, fe, V);
    vol[e] = V;
    T *o = scratch + 24 * (int64_t)e;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) o[3 * i + a] = fe[i][a];
}

// Staged two-layer kernel with the compact element terms and shared-memory
// atomic increments (blocks of at most 256 elements): per element the
// positions are held in registers, the velocities read from the node
// records as the hourglass rates need them, and the 24 corner forces formed
// one corner at a time from the terms; fewer registers than hex_hier (85
// against 128 in FP32: 3 CTAs of 256 per SM instead of 2, measured faster
// than 4 with spills; in FP64 the same 128 without hex_hier's ~1 KB of
// spills).
template <typename T, bool SOA>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) hex_hier_c(
    const mp_block_desc *__restrict__ desc, int block0, const uint4 *__restrict__ lmap,
    const uint8_t *__restrict__ /* thread colours: not used */, const int32_t *__restrict__ fp,
    const T *__restrict__ x, const T *__restrict__ v, const T *__restrict__ sig, T *__restrict__ f,
    T *__restrict__ vol, int64_t nnode, int64_t nelem, int cap, T kappa, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_xv = reinterpret_cast<T *>(smem_raw);  // [cap][8] node records
    T *s_f = s_xv + 8 * cap;                    // [3][cap]
    int *s_gid = reinterpret_cast<int *>(s_f + 3 * cap);

    mp_pdl_trigger();
    const mp_block_desc d = desc[block0 + blockIdx.x];
    const int tid = threadIdx.x;
    const int nn = d.fp_count[0];
    if ((unsigned)(reinterpret_cast<unsigned char *>(s_gid + cap) - smem_raw) > dynamic_smem_bytes() || nn > cap ||
        d.nitems > (int)blockDim.x) {
        if (tid == 0) atomicExch(err, MP_DEVERR_SMEM);
        return;
    }
    const int32_t *fpn = fp + d.fp_start[0];
    const bool active = tid < d.nitems;
    uint4 l = make_uint4(0, 0, 0, 0);
    if (active) l = lmap[d.item_start + tid];
    // nodes, two per thread and pass, both nodes' loads in flight together;
    // f (written by the previous colour's launch) after the dependent wait
    for (int i0 = tid; i0 < nn; i0 += 2 * (int)blockDim.x) {
        const int i1 = i0 + (int)blockDim.x;
        const bool two = i1 < nn;
        const int g0 = fpn[i0], g1 = two ? fpn[i1] : g0;
        T xv0[6], xv1[6];
        load3<T, SOA>(x, nnode, g0, xv0[0], xv0[1], xv0[2]);
        load3<T, SOA>(v, nnode, g0, xv0[3], xv0[4], xv0[5]);
        if (two) {
            load3<T, SOA>(x, nnode, g1, xv1[0], xv1[1], xv1[2]);
            load3<T, SOA>(v, nnode, g1, xv1[3], xv1[4], xv1[5]);
        }
        st_node_rec(s_xv, i0, xv0);
        s_gid[i0] = g0;
        if (two) {
            st_node_rec(s_xv, i1, xv1);
            s_gid[i1] = g1;
        }
        mp_pdl_wait();
        T f0[3], f1[3];
        load3<T, SOA>(f, nnode, g0, f0[0], f0[1], f0[2]);
        if (two) load3<T, SOA>(f, nnode, g1, f1[0], f1[1], f1[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s_f[a * cap + i0] = f0[a];
            if (two) s_f[a * cap + i1] = f1[a];
        }
    }
    __syncthreads();
    if (active) {
        const int e = d.item_start + tid;
        const int loc[8] = {(int)(l.x & 0xffff), (int)(l.x >> 16), (int)(l.y & 0xffff), (int)(l.y >> 16),
                            (int)(l.z & 0xffff), (int)(l.z >> 16), (int)(l.w & 0xffff), (int)(l.w >> 16)};
        T xe[8][3];
#pragma unroll
        for (int i = 0; i < 8; ++i) ld_node_half(s_xv, loc[i], 0, xe[i]);
        T s0, s1, s2;
        load3<T, SOA>(sig, nelem, e, s0, s1, s2);
        T t[3][3], w[4][3], qk[4][3], iV;
        vol[e] = hex_terms(xe, [&](int j, T vj[3]) { ld_node_half(s_xv, loc[j], 1, vj); }, s0, s1, s2, kappa, t, w,
                           qk, iV);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            T fa[3];
            hex_corner(i, t, w, qk, iV, fa);
#pragma unroll
            for (int a = 0; a < 3; ++a) atomicAdd(s_f + a * cap + loc[i], fa[a]);
        }
    }
    __syncthreads();
    for (int i = tid; i < nn; i += blockDim.x) {
        const int64_t g = s_gid[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) f[SOA ? a * nnode + g : 3 * g + a] = s_f[a * cap + i];
    }
}

// The global-colour / atomics baselines with the same compact element terms
// (positions and velocities of the 8 corners in registers).
template <typename T, bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) hex_direct_c(
    int e0, int e1, const int32_t *__restrict__ e2n, const T *__restrict__ x, const T *__restrict__ v,
    const T *__restrict__ sig, T *__restrict__ f, T *__restrict__ vol, int64_t nnode, int64_t nelem, T kappa)
{
    mp_pdl_trigger();
    const int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    const int4 *row = reinterpret_cast<const int4 *>(e2n) + 2 * (int64_t)e;
    const int4 r0 = row[0], r1 = row[1];
    const int nd[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    T xe[8][3], ve[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        load3<T, SOA>(x, nnode, nd[i], xe[i][0], xe[i][1], xe[i][2]);
        load3<T, SOA>(v, nnode, nd[i], ve[i][0], ve[i][1], ve[i][2]);
    }
    T s0, s1, s2;
    load3<T, SOA>(sig, nelem, e, s0, s1, s2);
    T t[3][3], w[4][3], qk[4][3], iV;
    vol[e] = hex_terms(xe, [&](int j, T vj[3]) {
        vj[0] = ve[j][0];
        vj[1] = ve[j][1];
        vj[2] = ve[j][2];
    }, s0, s1, s2, kappa, t, w, qk, iV);
    if (!ATOMIC) mp_pdl_wait();  // f: read-add-written by the previous colour's launch
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        T fa[3];
        hex_corner(i, t, w, qk, iV, fa);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int64_t j = SOA ? a * nnode + nd[i] : 3 * (int64_t)nd[i] + a;
            if (ATOMIC)
                atomicAdd(f + j, fa[a]);
            else
                f[j] += fa[a];
        }
    }
}

template <typename T, bool SOA>
int elem_assemble_t(const mp_plan *P, const void *x, const void *v, const void *sig, void *f, void *vol,
                    double kappa, cudaStream_t s)
{
    const int64_t nnode = P->maps[0].to_size, nelem = P->from_size;
    if (P->opts.coloring == MP_COLOR_HIER) {
        const int cap = P->stats.footprint_max[0];
        const int smem = cap * hex_smem_per_node<T>();
        // default increments: shared-memory atomics with the compact element
        // terms (measured fastest in both precisions: FP64 2.04 ms against
        // 2.16 warp-aggregated and 2.37 thread-coloured at 120^3)
        const int variant = mp_staged(P, MP_STAGED_SMEM_ATOMIC);
        // shared-memory atomics with the compact element terms for blocks of
        // at most 256 elements (the register budget of its launch bounds)
        auto kern = variant == MP_STAGED_SMEM_ATOMIC
                        ? (P->opts.block_size <= 256 ? hex_hier_c<T, SOA> : hex_hier<T, SOA, 1>)
                    : variant == MP_STAGED_WARP_AGG ? hex_hier<T, SOA, 3>
                                                    : hex_hier<T, SOA, 0>;
        int rc = mp_allow_smem(kern, smem);
        if (rc != MP_OK) return rc;
        int *err = nullptr;
        if ((rc = mp_device_error_word(&err)) != MP_OK) return rc;
        if (P->opts.block_size > 512) return MP_EINVAL;
        bool overlap = false;
        for (int c = 0; c < P->ncolors; ++c) {
            int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
            if (nb == 0) continue;
            MP_CUDA_TRY(mp_launch(kern, nb, P->opts.block_size, smem, s, overlap, P->dev.desc, b0,
                                  reinterpret_cast<const uint4 *>(P->dev.lmap), P->dev.tcolor, P->dev.fp,
                                  (const T *)x, (const T *)v, (const T *)sig, (T *)f, (T *)vol, nnode, nelem, cap,
                                  (T)kappa, err));
            overlap = true;
        }
    } else if (P->opts.coloring == MP_COLOR_TWOSTEP) {
        void *scratch = nullptr;
        int rc = mp_twostep_scratch(P, (size_t)nelem * 24 * sizeof(T), &scratch);
        if (rc != MP_OK) return rc;
        const int n = (int)nelem;
        hex_step1<T, SOA><<<(n + 255) / 256, 256, 0, s>>>(n, P->dev.map[0], (const T *)x, (const T *)v, (const T *)sig,
                                                           (T *)scratch, (T *)vol, nnode, nelem, (T)kappa);
        MP_CUDA_TRY(cudaGetLastError());
        return mp_twostep_gather(P, sizeof(T) == 8 ? MP_F64 : MP_F32, 3, scratch, f, s);
    } else {
        const bool atomic = P->opts.coloring == MP_COLOR_ATOMIC;
        bool overlap = false;
        for (int c = 0; c < P->ncolors; ++c) {
            int e0 = P->color_offsets[c], e1 = P->color_offsets[c + 1];
            if (e1 <= e0) continue;
            auto kern = atomic ? hex_direct_c<T, SOA, true> : hex_direct_c<T, SOA, false>;
            MP_CUDA_TRY(mp_launch(kern, (e1 - e0 + 255) / 256, 256, 0, s, overlap && !atomic, e0, e1, P->dev.map[0],
                                  (const T *)x, (const T *)v, (const T *)sig, (T *)f, (T *)vol, nnode, nelem,
                                  (T)kappa));
            overlap = true;
        }
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

extern "C" int loop_elem_assemble(const mp_plan *P, int32_t dtype, const void *x, const void *v, const void *sig,
                                  void *f, void *vol, double kappa, void *stream)
{
    if (!P || (dtype != MP_F64 && dtype != MP_F32 && dtype != MP_F64_DW)) return MP_EINVAL;
    if (P->nmaps != 1 || P->maps[0].arity != 8 || !P->maps[0].written) return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    for (const void *p : {x, v, sig, (const void *)f, (const void *)vol})
        if (!p || !aligned16(p)) return MP_EINVAL;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    if (dtype == MP_F64_DW) return mp_hex_dw(P, x, v, sig, f, vol, kappa, stream);
    cudaStream_t s = as_stream(stream);
    bool soa = P->opts.layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64)
        return soa ? elem_assemble_t<double, true>(P, x, v, sig, f, vol, kappa, s)
                   : elem_assemble_t<double, false>(P, x, v, sig, f, vol, kappa, s);
    return soa ? elem_assemble_t<float, true>(P, x, v, sig, f, vol, kappa, s)
               : elem_assemble_t<float, false>(P, x, v, sig, f, vol, kappa, s);
}
