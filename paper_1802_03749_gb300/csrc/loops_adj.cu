// Adjoint of res_calc with x, q, adt held fixed (adt not differentiated):
//   q_bar += (d res / d q)^T res_bar,   x_bar += (d res / d x)^T res_bar.
// Every edge increments q_bar on its 2 cells and x_bar on its 2 nodes, so
// the plan is coloured on both maps.  HIER stages q, adt, res_bar and the
// per-cell primitives of the block's cells and x of its nodes in shared
// memory, applies both increment sets one thread colour at a time and writes
// each footprint cell and node back once; GLOBAL / ATOMIC read global memory.
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

namespace {

template <typename T>
__device__ __forceinline__ void flux_rev(T r, T ru, T rv, T u, T v, T p, T H, T ri, T nx, T ny, T gm1, const T h[4],
                                         T qb[4], T &nbx, T &nby)
{
    T V = u * nx + v * ny;
    T Vb = h[0] * r + h[1] * ru + h[2] * rv + h[3] * H;
    T pb = h[1] * nx + h[2] * ny + h[3] * V;
    T Wb = Vb * ri;
    T gpb = gm1 * pb;
    qb[0] = h[0] * V - Wb * V + gpb * T(0.5) * (u * u + v * v);
    qb[1] = h[1] * V + Wb * nx - gpb * u;
    qb[2] = h[2] * V + Wb * ny - gpb * v;
    qb[3] = h[3] * V + gpb;
    nbx += h[1] * p + Wb * ru;
    nby += h[2] * p + Wb * rv;
}

// smem per cell: q[4], adt, u, v, p, H, ri, rb[4], inc[4] (18 T) + gid;
// per node: x[2], inc[2] (4 T) + gid
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
                                                     int cap_n, T gm1, T half_eps, int *__restrict__ err)
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
        T ri = T(1) / qq[0];
        T u = qq[1] * ri, v = qq[2] * ri;
        T p = gm1 * (qq[3] - T(0.5) * (qq[1] * u + qq[2] * v));
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
        T fb[4], h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            fb[k] = s_rb[k * cap_c + c1] - s_rb[k * cap_c + c2];
            h[k] = T(0.5) * fb[k];
        }
        flux_rev(s_q[c1], s_q[cap_c + c1], s_q[2 * cap_c + c1], s_u[c1], s_v[c1], s_p[c1], s_H[c1], s_ri[c1], nx,
                 ny, gm1, h, qb1, nbx, nby);
        flux_rev(s_q[c2], s_q[cap_c + c2], s_q[2 * cap_c + c2], s_u[c2], s_v[c2], s_p[c2], s_H[c2], s_ri[c2], nx,
                 ny, gm1, h, qb2, nbx, nby);
        T mu = (s_adt[c1] + s_adt[c2]) * half_eps;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qb1[k] += mu * fb[k];
            qb2[k] -= mu * fb[k];
        }
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

template <typename T, bool SOA, bool ATOMIC>
__global__ void __launch_bounds__(256) adjoint_direct(int e0, int e1, const int32_t *__restrict__ e2n,
                                                      const int32_t *__restrict__ e2c, const T *__restrict__ x,
                                                      const T *__restrict__ q, const T *__restrict__ adt,
                                                      const T *__restrict__ rbar, T *__restrict__ qbar,
                                                      T *__restrict__ xbar, int64_t nnode, int64_t ncell, T gm1,
                                                      T half_eps)
{
    int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    int2 nab = reinterpret_cast<const int2 *>(e2n)[e];
    int2 cc = reinterpret_cast<const int2 *>(e2c)[e];
    auto X = [&](int64_t g, int k) { return SOA ? x[k * nnode + g] : x[2 * g + k]; };
    T nx = X(nab.x, 1) - X(nab.y, 1);
    T ny = X(nab.y, 0) - X(nab.x, 0);
    T q1[4], q2[4], fb[4], h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int64_t j1 = SOA ? k * ncell + cc.x : 4 * (int64_t)cc.x + k;
        int64_t j2 = SOA ? k * ncell + cc.y : 4 * (int64_t)cc.y + k;
        q1[k] = q[j1];
        q2[k] = q[j2];
        fb[k] = rbar[j1] - rbar[j2];
        h[k] = T(0.5) * fb[k];
    }
    T qb1[4], qb2[4], nbx = T(0), nby = T(0);
    {
        T ri = T(1) / q1[0], u = q1[1] * ri, v = q1[2] * ri;
        T p = gm1 * (q1[3] - T(0.5) * (q1[1] * u + q1[2] * v));
        flux_rev(q1[0], q1[1], q1[2], u, v, p, q1[3] + p, ri, nx, ny, gm1, h, qb1, nbx, nby);
    }
    {
        T ri = T(1) / q2[0], u = q2[1] * ri, v = q2[2] * ri;
        T p = gm1 * (q2[3] - T(0.5) * (q2[1] * u + q2[2] * v));
        flux_rev(q2[0], q2[1], q2[2], u, v, p, q2[3] + p, ri, nx, ny, gm1, h, qb2, nbx, nby);
    }
    T mu = (adt[cc.x] + adt[cc.y]) * half_eps;
    T xa0 = -nby, xb0 = nby, xa1 = nbx, xb1 = -nbx;
    int64_t ja0 = SOA ? nab.x : 2 * (int64_t)nab.x, ja1 = SOA ? nnode + nab.x : 2 * (int64_t)nab.x + 1;
    int64_t jb0 = SOA ? nab.y : 2 * (int64_t)nab.y, jb1 = SOA ? nnode + nab.y : 2 * (int64_t)nab.y + 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int64_t j1 = SOA ? k * ncell + cc.x : 4 * (int64_t)cc.x + k;
        int64_t j2 = SOA ? k * ncell + cc.y : 4 * (int64_t)cc.y + k;
        T a = qb1[k] + mu * fb[k], b = qb2[k] - mu * fb[k];
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
    const T gm1 = (T)(gam - 1.0), half_eps = (T)(0.5 * eps);
    if (P->opts.coloring == MP_COLOR_HIER) {
        if (P->maps[0].slot != 0 || P->maps[1].slot != 1) return MP_EPLAN;
        const int cap_n = P->stats.footprint_max[0], cap_c = P->stats.footprint_max[1];
        const int smem = cap_c * adj_smem_per_cell<T>() + cap_n * adj_smem_per_node<T>();
        auto kern = adjoint_hier<T, SOA>;
        int rc = mp_allow_smem(kern, smem);
        if (rc != MP_OK) return rc;
        int *err = nullptr;
        if ((rc = mp_device_error_word(&err)) != MP_OK) return rc;
        bool overlap = false;
        for (int c = 0; c < P->ncolors; ++c) {
            int b0 = P->color_offsets[c], nb = P->color_offsets[c + 1] - b0;
            if (nb == 0) continue;
            MP_CUDA_TRY(mp_launch(kern, nb, P->opts.block_size, smem, s, overlap, P->dev.desc, b0,
                                  reinterpret_cast<const ushort4 *>(P->dev.lmap), P->dev.tcolor, P->dev.fp,
                                  (const T *)x, (const T *)q, (const T *)adt, (const T *)rbar, (T *)qbar, (T *)xbar,
                                  nnode, ncell, cap_c, cap_n, gm1, half_eps, err));
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
                                                       (T *)xbar, nnode, ncell, gm1, half_eps);
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
