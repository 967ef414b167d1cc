// Device-side helpers shared by the loop kernels.  Internal.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "plan_internal.h"

#define MP_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return MP_ECUDA;             \
    } while (0)

// Largest dynamic shared memory a CTA may opt into on sm_103a (227 KB).
constexpr int MP_SMEM_LIMIT = 227 * 1024;

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// True when p is 16-byte aligned (vector loads of double2 / float4 rows).
inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Programmatic dependent launch between the colour launches of one loop.
// A launch made with overlap = true may start while the previous kernel of
// the stream is finishing: its CTAs fill the SMs that the previous launch's
// last CTAs free, and stage everything that launch does not write (plan
// tables, read-only dats) before mp_pdl_wait(), which returns once the
// previous grid has completed and its writes are visible.  Every kernel
// calls mp_pdl_trigger() first: dependents may then launch as soon as all
// of its CTAs are resident.  Without the launch attribute both are no-ops.
// The environment variable MESHLOOP_NO_PDL (any value) turns the overlap
// off for the process (plain stream order everywhere).
inline bool mp_pdl_enabled()
{
    static const bool on = std::getenv("MESHLOOP_NO_PDL") == nullptr;
    return on;
}
__device__ __forceinline__ void mp_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void mp_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Warp-aggregated increment: the lanes of a warp that target the same
// point (found with match.any) sum their values by a segmented shuffle
// tree in rank order and the lowest of them adds the sum with one
// shared-memory atomic.  All lanes of `act` must call it (uniform trip
// count: the largest group decides the tree depth).
template <typename T, int N>
__device__ __forceinline__ void warp_aggregated_add(unsigned act, int target, T v[N], T *base, int stride)
{
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(act, target);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const unsigned widest = __reduce_max_sync(act, (unsigned)__popc(peers));
    for (unsigned off = 1; off < widest; off <<= 1) {
        const unsigned src = __fns(peers, lane, off + 1);  // the peer off ranks above
        const bool take = (rank % (2 * off)) == 0 && src != 0xffffffffu;
        const int from = src != 0xffffffffu ? (int)src : lane;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T y = __shfl_sync(act, v[k], from);
            if (take) v[k] += y;
        }
    }
    if (rank == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) atomicAdd(base + k * stride + target, v[k]);
    }
}

template <typename... KArgs, typename... Args>
cudaError_t mp_launch(void (*kern)(KArgs...), int grid, int block, int smem, cudaStream_t s, bool overlap,
                      Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = overlap && mp_pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Data accessor for a dat of DIM components per point in AoS ([n][DIM]) or
// SoA ([DIM][n]) layout.
template <typename T, int DIM, bool SOA>
struct dat {
    T *p;
    int64_t n;
    __device__ __forceinline__ T &at(int64_t i, int k) const { return SOA ? p[k * n + i] : p[i * DIM + k]; }
};

// Size of the dynamic shared memory this CTA was launched with.
__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// Device error word codes (read by mp_check_device_status).
enum { MP_DEVERR_NONE = 0, MP_DEVERR_TIMEOUT = 1, MP_DEVERR_SMEM = 2 };

// Limit of a device-side wait (ns of %globaltimer) in the library's
// persistent kernels: a wait that runs out records MP_DEVERR_TIMEOUT and
// the kernel returns instead of waiting on.
constexpr unsigned long long MP_GRID_WAIT_NS = 1000000000ull;

__device__ __forceinline__ unsigned long long mp_globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned mp_ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch (every CTA resident) with a
// bounded wait: each CTA's thread 0 publishes the CTA's writes (fence) and
// arrives on a counter that the launch starts at 0, then waits until
// `target` arrivals are visible (acquire) or wait_ns has passed.  Returns
// false when the wait gave up: MP_DEVERR_TIMEOUT is then in the error word
// and the caller must return (its results are invalid).  Uniform per CTA.
__device__ __forceinline__ bool mp_grid_barrier(unsigned *count, unsigned target, unsigned long long wait_ns,
                                                int *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned long long t0 = mp_globaltimer_ns();
        int ok = 1;
        while (mp_ld_acquire(count) < target) {
            if (mp_globaltimer_ns() - t0 > wait_ns) {
                atomicExch(err, MP_DEVERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(256);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Library-owned device error word of the current device.
int mp_device_error_word(int **word);

// Uploads the plan's tables to the current device if not done yet.
int mp_plan_ensure_device(const mp_plan *plan);
// releases what loop_res_calc_host keeps on the plan (host_io.cu)
void mp_host_io_free(void *io);

// Pipelined persistent two-layer res_calc (FP64 / FP32).
int mp_res_calc_pipe(const mp_plan *P, int32_t dtype, const void *x, const void *q, const void *adt, void *res,
                     double gam, double eps, void *stream);
// Staged implementation of a HIER plan: opts.staged, or the loop default.
inline int mp_staged(const mp_plan *P, int loop_default) { return P->opts.staged < 0 ? loop_default : P->opts.staged; }
// the plan carries (and has uploaded) a gather table of at most 16 entries
// per footprint point; plans without one run the thread-coloured form
inline bool mp_gather_ready(const mp_plan *P)
{
    return P->gat_w >= 4 && P->gat_w <= 16 && P->dev.gat != nullptr;
}

// Two-layer res_calc with FP64 data and double-word arithmetic.
int mp_res_calc_dw(const mp_plan *P, const void *x, const void *q, const void *adt, void *res, double gam, double eps,
                   void *stream);

// Two-layer hex assembly with FP64 data and double-word arithmetic.
int mp_face_flux_dw(const mp_plan *P, const void *fdata, const void *cdata, void *res, double gam, double mu,
                    double pr, void *stream);
int mp_hex_dw(const mp_plan *P, const void *x, const void *v, const void *sig, void *f, void *vol, double kappa,
              void *stream);

// Two-layer res_calc adjoint with FP64 data and double-word arithmetic.
int mp_adjoint_dw(const mp_plan *P, const void *x, const void *q, const void *adt, const void *rbar, void *qbar,
                  void *xbar, double gam, double eps, void *stream);

// TWOSTEP plans: the per-(item, slot) increment scratch (allocated on first
// use, kept with the plan) and the gather of step 2 into out (+=).
int mp_twostep_scratch(const mp_plan *P, size_t bytes, void **out);
int mp_twostep_gather(const mp_plan *P, int32_t dtype, int dim, const void *scratch, void *out, void *stream);

// Library-owned device scratch for deterministic reductions (per device).
int mp_reduce_scratch(double **partials, int *nparts);

// Lets a kernel use `bytes` of dynamic shared memory: the opt-in limit
// (227 KB per CTA) minus the kernel's static shared memory.
template <typename K>
inline int mp_allow_smem(K kernel, int bytes)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return MP_ECUDA;
    const int limit = MP_SMEM_LIMIT - (int)fa.sharedSizeBytes;
    if (bytes > limit) return MP_ESMEM;
    if (bytes > 48 * 1024 && fa.maxDynamicSharedSizeBytes < bytes) {
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess)
            return MP_ECUDA;
    }
    return MP_OK;
}

// ------------------------------------------------------------ 2D Euler flux
// Per-cell primitives: velocity (u, v), pressure p = (gam-1)(E - rho |u|^2 / 2)
// and total enthalpy density H = E + p.  The 1/2 of the kinetic energy is
// folded into gam-1 (exact scaling): p = (gam-1) E - ((gam-1)/2)(ru u + rv v).
// Used where the full values are needed (the far-field boundary flux).
template <typename T>
__device__ __forceinline__ void cell_prims(T rho, T ru, T rv, T E, T gm1, T &u, T &v, T &p, T &H)
{
    T ri = T(1) / rho;
    u = ru * ri;
    v = rv * ri;
    p = gm1 * E - (T(0.5) * gm1) * (ru * u + rv * v);
    H = E + p;
}

// Reciprocals of the flux kernels, rcp(x) = 1 / x and rcp_half(x) = 1 / (2 x).
// FP32: the IEEE quotients.  FP64, whose pipe bounds the flux kernels on
// GB300: Newton-Raphson iteration for the reciprocal from an FP32 seed, in
// its third-order form y = y0 (1 + e + e^2), e = 1 - x y0 (the series of
// 1/(1 - e); e.g. Muller et al., Handbook of Floating-Point Arithmetic, 2nd
// ed., Sec. 11.2 and 11.3).  The seed is rcp.approx.f32 of x's significand
// cut to its leading 20 bits, rebuilt as a double with x's negated exponent
// by integer operations, so no FP64 conversion is issued: |e| < 2^-19, hence
// |e|^3 < 2^-57, below FP64 rounding, and the result is the product
// y0 (1 + (e + e^2)) (or y0 / 2 times it) with one rounding: 3 FP64
// operations instead of an IEEE division.  x whose exponent field lies
// outside [1, 2040] (zero, subnormal, above 2^1017, infinite, NaN) takes the
// IEEE division, so those give the IEEE results.
// The seed y0 of 1/x and y0/2; false when x is outside the seed's range.
__device__ __forceinline__ bool rcp_seed(double x, double &y0, double &y0h)
{
    const int hi = __double2hiint(x);
    const unsigned ex = ((unsigned)hi >> 20) & 0x7ffu;
    if (ex - 1u >= 2040u) return false;
    // leading 20 bits of the significand as a float in [1, 2)
    const float m = __int_as_float(0x3f800000 | ((hi & 0x000fffff) << 3));
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(m));  // in (1/2, 1]
    const int rb = __float_as_int(r);
    // r 2^(1023 - ex): exponent field (rb >> 23) - 127 + 1023 - (ex - 1023),
    // the 23 significand bits of r split over the two words
    const int yhi = (hi & (int)0x80000000) | (((rb >> 23) + 1919 - (int)ex) << 20) | ((rb & 0x7fffff) >> 3);
    const int ylo = rb << 29;
    y0 = __hiloint2double(yhi, ylo);
    y0h = __hiloint2double(yhi - (1 << 20), ylo);  // y0 / 2: exponent - 1
    return true;
}
template <typename T>
__device__ __forceinline__ T rcp_half(T x)
{
    return T(0.5) / x;
}
template <>
__device__ __forceinline__ double rcp_half<double>(double x)
{
    double y0, y0h;
    if (!rcp_seed(x, y0, y0h)) return 0.5 / x;
    const double e = fma(-x, y0, 1.0);
    return fma(y0h, fma(e, e, e), y0h);
}
template <typename T>
__device__ __forceinline__ T rcp(T x)
{
    return T(1) / x;
}
template <>
__device__ __forceinline__ double rcp<double>(double x)
{
    double y0, y0h;
    if (!rcp_seed(x, y0, y0h)) return 1.0 / x;
    const double e = fma(-x, y0, 1.0);
    return fma(y0, fma(e, e, e), y0);
}

// x / 2, exact.  FP64: by decrementing the exponent field when x is normal
// with exponent field at least 2 (integer operations, off the FP64 pipe),
// else (zero, smallest normals, subnormals, infinities, NaN) x * 0.5.
template <typename T>
__device__ __forceinline__ T half_of(T x)
{
    return T(0.5) * x;
}
template <>
__device__ __forceinline__ double half_of<double>(double x)
{
    const int hi = __double2hiint(x);
    const unsigned ex = ((unsigned)hi >> 20) & 0x7ffu;
    return ex - 2u < 2045u ? __hiloint2double(hi - (1 << 20), __double2loint(x)) : 0.5 * x;
}

// Per-cell primitives with the 1/2 of the central flux average folded in:
// uh = u / 2, vh = v / 2, ph = p / 2 and H = E + p, from ri = 1 / (2 rho) and
// gm1h = (gam-1)/2:  ph = gm1h (E - (ru uh + rv vh)), H = E + 2 ph.  With
// these the edge flux takes the full normal n = (dy, -dx): u . n / 2 =
// uh . n and p n / 2 = ph n, so the nodes need no scaling.
template <typename T>
__device__ __forceinline__ void cell_prims_half(T rho, T ru, T rv, T E, T gm1h, T &uh, T &vh, T &ph, T &H)
{
    const T ri = rcp_half(rho);
    uh = ru * ri;
    vh = rv * ri;
    ph = gm1h * (E - (ru * uh + rv * vh));
    H = fma(T(2), ph, E);
}

// Edge flux from two cells' conserved states and the half primitives of
// cell_prims_half with the full normal (nx, ny) = (y1 - y2, x2 - x1):
//   f = (F(q1).n + F(q2).n)/2 + mu (q1 - q2),  F.n = (rho V, rho u V + p n_x,
//   rho v V + p n_y, H V),  V = u . n,  mu = eps (adt1 + adt2) / 2,
// evaluated with the half normal velocities V1 = uh1 . n = u1 . n / 2.
// With W1 = V1 + mu and W2 = V2 - mu the dissipation of the first three
// components folds into the normal velocities (rho1 V1 + mu rho1 =
// rho1 W1, ...): 22 operations per edge instead of 26.
template <typename T>
__device__ __forceinline__ void edge_flux(T nx, T ny, T r1, T ru1, T rv1, T E1, T uh1, T vh1, T ph1, T H1, T a1,
                                          T r2, T ru2, T rv2, T E2, T uh2, T vh2, T ph2, T H2, T a2, T half_eps,
                                          T f[4])
{
    T V1 = uh1 * nx + vh1 * ny;
    T V2 = uh2 * nx + vh2 * ny;
    T ps = ph1 + ph2;
    T mu = (a1 + a2) * half_eps;
    T W1 = V1 + mu, W2 = V2 - mu;
    f[0] = r1 * W1 + r2 * W2;
    f[1] = ru1 * W1 + ru2 * W2 + ps * nx;
    f[2] = rv1 * W1 + rv2 * W2 + ps * ny;
    f[3] = H1 * V1 + H2 * V2 + mu * (E1 - E2);
}
