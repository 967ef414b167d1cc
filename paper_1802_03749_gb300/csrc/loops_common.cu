// Plan upload, library scratch and the direct loops of the time step
// (save_soln, update with the FP64 residual sum).
#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace {

template <typename T>
int upload(T **dst, const T *src, size_t n, int64_t &bytes)
{
    if (n == 0) return MP_OK;
    MP_CUDA_TRY(cudaMalloc(reinterpret_cast<void **>(dst), n * sizeof(T)));
    MP_CUDA_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    bytes += (int64_t)(n * sizeof(T));
    return MP_OK;
}

std::mutex g_upload_mu;

}  // namespace

void mp_plan_free_device(mp_plan *P)
{
    mp_device_tables &d = P->dev;
    if (d.device < 0) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != d.device) cudaSetDevice(d.device);
    cudaFree(d.desc);
    cudaFree(d.lmap);
    cudaFree(d.fp);
    cudaFree(d.tcolor);
    cudaFree(d.gat);
    cudaFree(d.color_off);
    cudaFree(d.bar);
    for (auto &m : d.map) cudaFree(m);
    cudaFree(d.inv_off);
    cudaFree(d.inv_idx);
    cudaFree(d.scratch);
    mp_host_io_free(d.host_io);
    if (cur >= 0 && cur != d.device) cudaSetDevice(cur);
    d = mp_device_tables{};
}

int mp_plan_ensure_device(const mp_plan *cplan)
{
    mp_plan *P = const_cast<mp_plan *>(cplan);
    std::lock_guard<std::mutex> lk(g_upload_mu);
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    if (P->dev.device == dev) return MP_OK;
    if (P->dev.device >= 0) mp_plan_free_device(P);
    mp_device_tables &d = P->dev;
    int rc = MP_OK;
    int64_t bytes = 0;
    if (P->opts.coloring == MP_COLOR_HIER) {
        if ((rc = upload(&d.desc, P->desc.data(), P->desc.size(), bytes)) != MP_OK) goto fail;
        if ((rc = upload(&d.lmap, P->lmap.data(), P->lmap.size(), bytes)) != MP_OK) goto fail;
        {
            // padded to whole 16-byte words: the pipelined kernels copy the
            // colours of a block as 4-byte words that may run past the end
            std::vector<uint8_t> tc(P->thread_color);
            tc.resize(((tc.size() + 4) + 15) / 16 * 16, 0);
            if ((rc = upload(&d.tcolor, tc.data(), tc.size(), bytes)) != MP_OK) goto fail;
        }
        {
            std::vector<int32_t> all;
            for (int s = 0; s < P->ntosets; ++s) all.insert(all.end(), P->fp_ids[s].begin(), P->fp_ids[s].end());
            if ((rc = upload(&d.fp, all.data(), all.size(), bytes)) != MP_OK) goto fail;
        }
        if (!P->gat_tab.empty() &&
            (rc = upload(&d.gat, P->gat_tab.data(), P->gat_tab.size(), bytes)) != MP_OK)
            goto fail;
        if ((rc = upload(&d.color_off, P->color_offsets.data(), P->color_offsets.size(), bytes)) != MP_OK)
            goto fail;
        {
            // grid-barrier arrivals and one block counter per colour
            const std::vector<unsigned> zeros((size_t)P->ncolors + 1, 0u);
            if ((rc = upload(&d.bar, zeros.data(), zeros.size(), bytes)) != MP_OK) goto fail;
        }
    } else {
        for (int m = 0; m < P->nmaps; ++m)
            if ((rc = upload(&d.map[m], P->maps[m].idx.data(), P->maps[m].idx.size(), bytes)) != MP_OK) goto fail;
        if (P->opts.coloring == MP_COLOR_TWOSTEP) {
            if ((rc = upload(&d.inv_off, P->inv_off.data(), P->inv_off.size(), bytes)) != MP_OK) goto fail;
            if ((rc = upload(&d.inv_idx, P->inv_idx.data(), P->inv_idx.size(), bytes)) != MP_OK) goto fail;
        }
    }
    d.device = dev;
    d.bytes = bytes;
    return MP_OK;
fail:
    d.device = dev;
    mp_plan_free_device(P);
    return rc;
}

extern "C" int mesh_plan_upload(mp_plan *plan)
{
    if (!plan) return MP_EINVAL;
    return mp_plan_ensure_device(plan);
}

// ------------------------------------------------------------- scratch

namespace {
constexpr int kReduceParts = 152 * 4;  // one partial per CTA of the update grid
std::mutex g_scratch_mu;
double *g_partials[64] = {nullptr};
int *g_error_word[64] = {nullptr};
}  // namespace

int mp_reduce_scratch(double **partials, int *nparts)
{
    int dev = 0;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MP_EINVAL;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_partials[dev]) MP_CUDA_TRY(cudaMalloc(&g_partials[dev], kReduceParts * sizeof(double)));
    *partials = g_partials[dev];
    *nparts = kReduceParts;
    return MP_OK;
}

int mp_device_error_word(int **word)
{
    int dev = 0;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MP_EINVAL;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_error_word[dev]) {
        MP_CUDA_TRY(cudaMalloc(&g_error_word[dev], sizeof(int)));
        MP_CUDA_TRY(cudaMemset(g_error_word[dev], 0, sizeof(int)));
    }
    *word = g_error_word[dev];
    return MP_OK;
}

extern "C" int mp_check_device_status(void *stream)
{
    int *w = nullptr;
    int rc = mp_device_error_word(&w);
    if (rc != MP_OK) return rc;
    int h = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, as_stream(stream)));
    MP_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    if (h != MP_DEVERR_NONE) {
        MP_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(int), as_stream(stream)));
        MP_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
        return h == MP_DEVERR_SMEM ? MP_ESMEM : MP_ETIMEOUT;
    }
    return MP_OK;
}

// ------------------------------------------------- bounded grid-wide wait

namespace {
unsigned *g_wait_count[64] = {nullptr};

// Every CTA arrives once on the counter and waits for `target` arrivals:
// with target above the grid size the wait can only run out.
__global__ void grid_wait_probe(unsigned *count, unsigned target, unsigned long long wait_ns, int *err)
{
    mp_grid_barrier(count, target, wait_ns, err);
}
}  // namespace

extern "C" int mp_grid_wait_test(int32_t nctas, int64_t wait_ns, int32_t missing, void *stream)
{
    if (nctas < 1 || missing < 0 || wait_ns < 0 || wait_ns > (int64_t)MP_GRID_WAIT_NS) return MP_EINVAL;
    int dev = 0, sms = 0;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    MP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 0 || dev >= 64 || nctas > sms) return MP_EINVAL;  // one CTA per SM at most: all resident
    int *err = nullptr;
    int rc = mp_device_error_word(&err);
    if (rc != MP_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_wait_count[dev]) MP_CUDA_TRY(cudaMalloc(&g_wait_count[dev], sizeof(unsigned)));
    }
    cudaStream_t s = as_stream(stream);
    MP_CUDA_TRY(cudaMemsetAsync(g_wait_count[dev], 0, sizeof(unsigned), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nctas);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    MP_CUDA_TRY(cudaLaunchKernelEx(&cfg, grid_wait_probe, g_wait_count[dev], (unsigned)(nctas + missing),
                                   (unsigned long long)wait_ns, err));
    return MP_OK;
}

// ------------------------------------------------ flux kernels' reciprocals

namespace {
__global__ void recip_probe(const double *__restrict__ x, double *__restrict__ y, int64_t n, int mode)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = mode == 0 ? rcp(x[i]) : mode == 1 ? rcp_half(x[i]) : half_of(x[i]);
}
}  // namespace

extern "C" int mp_recip_test(const double *x, double *y, int64_t n, int32_t mode, void *stream)
{
    if (n < 0 || (n > 0 && (!x || !y)) || mode < 0 || mode > 2) return MP_EINVAL;
    if (n == 0) return MP_OK;
    for (const void *p : {(const void *)x, (const void *)y}) {  // device memory only
        cudaPointerAttributes a;
        MP_CUDA_TRY(cudaPointerGetAttributes(&a, p));
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return MP_EINVAL;
    }
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    recip_probe<<<grid, 256, 0, as_stream(stream)>>>(x, y, n, mode);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

// ------------------------------------------------------------ direct loops

namespace {

template <typename T>
__global__ void save_soln_kernel(const T *__restrict__ q, T *__restrict__ qold, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        qold[i] = q[i];
}

// update (Airfoil's direct cell loop): d = res/adt in FP64, q = qold - d,
// res = 0, and a fixed-order sum of d^2: thread-strided partial sums, a
// fixed tree per CTA, one partial per CTA in scratch.
template <typename T, bool SOA>
__global__ void __launch_bounds__(256) update_kernel(const T *__restrict__ qold, T *__restrict__ q,
                                                     T *__restrict__ res, const T *__restrict__ adt,
                                                     int64_t ncell, double *__restrict__ partials)
{
    double s = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        double ai = 1.0 / (double)adt[c];
        for (int k = 0; k < 4; ++k) {
            int64_t j = SOA ? k * ncell + c : 4 * c + k;
            double d = (double)res[j] * ai;
            q[j] = (T)((double)qold[j] - d);
            res[j] = T(0);
            s += d * d;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) sum_partials_kernel(const double *__restrict__ partials, int n,
                                                          double *__restrict__ out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += partials[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out += red[0];
}

}  // namespace

extern "C" int loop_save_soln(int64_t ncell, int32_t dtype, int32_t layout, const void *q, void *qold, void *stream)
{
    (void)layout;  // a plain copy of all 4*ncell values, layout-independent
    if (ncell < 0 || (dtype != MP_F64 && dtype != MP_F32)) return MP_EINVAL;
    if (ncell == 0) return MP_OK;
    if (!q || !qold) return MP_EINVAL;
    int64_t n = 4 * ncell;
    int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    if (dtype == MP_F64)
        save_soln_kernel<double><<<grid, 256, 0, as_stream(stream)>>>((const double *)q, (double *)qold, n);
    else
        save_soln_kernel<float><<<grid, 256, 0, as_stream(stream)>>>((const float *)q, (float *)qold, n);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

extern "C" int loop_update(int64_t ncell, int32_t dtype, int32_t layout, const void *qold, void *q, void *res,
                           const void *adt, double *rms_dev, void *stream)
{
    if (ncell < 0 || (dtype != MP_F64 && dtype != MP_F32) || (layout != MP_LAYOUT_AOS && layout != MP_LAYOUT_SOA))
        return MP_EINVAL;
    if (ncell == 0) return MP_OK;
    if (!qold || !q || !res || !adt || !rms_dev) return MP_EINVAL;
    double *parts = nullptr;
    int nparts = 0;
    int rc = mp_reduce_scratch(&parts, &nparts);
    if (rc != MP_OK) return rc;
    cudaStream_t s = as_stream(stream);
    bool soa = layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64) {
        auto k = soa ? update_kernel<double, true> : update_kernel<double, false>;
        k<<<nparts, 256, 0, s>>>((const double *)qold, (double *)q, (double *)res, (const double *)adt, ncell, parts);
    } else {
        auto k = soa ? update_kernel<float, true> : update_kernel<float, false>;
        k<<<nparts, 256, 0, s>>>((const float *)qold, (float *)q, (float *)res, (const float *)adt, ncell, parts);
    }
    sum_partials_kernel<<<1, 256, 0, s>>>(parts, nparts, rms_dev);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

// ------------------------------------------------- allocation-free update

namespace {
// Static scratch of loop_update_noalloc: one partial sum per CTA.  In host
// code this name is only a stand-in; kernels get its device address.
static __device__ __align__(256) double g_noalloc_partials[MP_NOALLOC_MAX_PARTIALS];
std::mutex g_noalloc_mu;
double *g_noalloc_addr[64] = {nullptr};

// Device address of the static scratch on the current device, looked up
// once per device with that device current.
int noalloc_scratch(double **out)
{
    int dev = 0;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MP_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        double *p = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_partials) != cudaSuccess || !p)
            return MP_ECUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return MP_OK;
}
}  // namespace

extern "C" int loop_update_noalloc(int64_t ncell, int32_t dtype, int32_t layout, const void *qold, void *q,
                                   void *res, const void *adt, double *rms_dev, void *stream)
{
    if (ncell < 0 || (dtype != MP_F64 && dtype != MP_F32) || (layout != MP_LAYOUT_AOS && layout != MP_LAYOUT_SOA))
        return MP_EINVAL;
    if (ncell > MP_NOALLOC_MAX_CELLS) return MP_ETOOBIG;
    if (ncell == 0) return MP_OK;
    if (!qold || !q || !res || !adt || !rms_dev) return MP_EINVAL;
    double *parts = nullptr;
    int rc = noalloc_scratch(&parts);
    if (rc != MP_OK) return rc;
    // one CTA per MP_NOALLOC_CELLS_PER_PARTIAL cells: at most
    // MP_NOALLOC_MAX_PARTIALS partials, each written before it is summed
    const int nparts = (int)((ncell + MP_NOALLOC_CELLS_PER_PARTIAL - 1) / MP_NOALLOC_CELLS_PER_PARTIAL);
    cudaStream_t s = as_stream(stream);
    bool soa = layout == MP_LAYOUT_SOA;
    if (dtype == MP_F64) {
        auto k = soa ? update_kernel<double, true> : update_kernel<double, false>;
        k<<<nparts, 256, 0, s>>>((const double *)qold, (double *)q, (double *)res, (const double *)adt, ncell, parts);
    } else {
        auto k = soa ? update_kernel<float, true> : update_kernel<float, false>;
        k<<<nparts, 256, 0, s>>>((const float *)qold, (float *)q, (float *)res, (const float *)adt, ncell, parts);
    }
    sum_partials_kernel<<<1, 256, 0, s>>>(parts, nparts, rms_dev);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

// ----------------------------------------------------- two-step gather

int mp_twostep_scratch(const mp_plan *cplan, size_t bytes, void **out)
{
    mp_plan *P = const_cast<mp_plan *>(cplan);
    mp_device_tables &d = P->dev;
    if (d.scratch_bytes < bytes) {
        if (d.scratch) MP_CUDA_TRY(cudaFree(d.scratch));
        d.scratch = nullptr;
        d.scratch_bytes = 0;
        MP_CUDA_TRY(cudaMalloc(&d.scratch, bytes));
        d.scratch_bytes = bytes;
    }
    *out = d.scratch;
    return MP_OK;
}

namespace {

// Step 2 of the temporary-array method: each point of the written to-set
// sums its (item, slot) increments in inverse-map order and adds them once.
template <typename T, int DIM, bool SOA>
__global__ void __launch_bounds__(256) twostep_gather(const int32_t *__restrict__ inv_off,
                                                      const int32_t *__restrict__ inv_idx,
                                                      const T *__restrict__ scratch, T *__restrict__ out, int64_t n)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    T acc[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) acc[k] = T(0);
    for (int j = inv_off[p]; j < inv_off[p + 1]; ++j) {
        const int64_t base = (int64_t)inv_idx[j] * DIM;
#pragma unroll
        for (int k = 0; k < DIM; ++k) acc[k] += scratch[base + k];
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) out[SOA ? k * n + p : p * DIM + k] += acc[k];
}

template <typename T, int DIM>
void launch_gather(const mp_plan *P, const void *scratch, void *out, cudaStream_t s)
{
    const int64_t n = P->maps[P->inv_map].to_size;
    const int grid = (int)((n + 255) / 256);
    if (P->opts.layout == MP_LAYOUT_SOA)
        twostep_gather<T, DIM, true><<<grid, 256, 0, s>>>(P->dev.inv_off, P->dev.inv_idx, (const T *)scratch, (T *)out, n);
    else
        twostep_gather<T, DIM, false><<<grid, 256, 0, s>>>(P->dev.inv_off, P->dev.inv_idx, (const T *)scratch, (T *)out,
                                                           n);
}

}  // namespace

int mp_twostep_gather(const mp_plan *P, int32_t dtype, int dim, const void *scratch, void *out, void *stream)
{
    cudaStream_t s = as_stream(stream);
    if (dim == 4)
        dtype == MP_F64 ? launch_gather<double, 4>(P, scratch, out, s) : launch_gather<float, 4>(P, scratch, out, s);
    else if (dim == 3)
        dtype == MP_F64 ? launch_gather<double, 3>(P, scratch, out, s) : launch_gather<float, 3>(P, scratch, out, s);
    else if (dim == 5)
        dtype == MP_F64 ? launch_gather<double, 5>(P, scratch, out, s) : launch_gather<float, 5>(P, scratch, out, s);
    else
        return MP_EINVAL;
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}
