// res_calc with host buffers: the C-ABI call an application makes when its
// mesh data live in (pinned) host memory.  Per call, on the caller's stream:
// the four inputs are copied into library-owned device buffers in chunks of
// at most 16 MB spread over four copy-in streams forked from the caller's
// stream (several copy engines at once), the loop runs, and res is copied
// back in chunks over two copy-out streams joined back into the caller's
// stream.
//
// Two buffer slots alternate between calls, so a caller that issues
// consecutive steps on two streams overlaps one step's copies with the
// other's loop and read-back; a slot is reused only after the read-back of
// its previous call (an event on that call's stream).
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kIn = 4, kOut = 2;
constexpr size_t kChunk = 16u << 20;

struct host_io {
    int device = -1;
    size_t slot_bytes = 0;
    void *buf[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    int next = 0;
    cudaStream_t in[kIn] = {}, out[kOut] = {};
    cudaEvent_t start = nullptr, computed = nullptr;
    cudaEvent_t copied[kIn] = {}, returned[kOut] = {};
    cudaEvent_t freed[2] = {nullptr, nullptr};
    std::mutex mu;
};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

int create(host_io *io, size_t slot_bytes, int device)
{
    io->device = device;
    io->slot_bytes = slot_bytes;
    for (int b = 0; b < 2; ++b) MP_CUDA_TRY(cudaMalloc(&io->buf[b], slot_bytes));
    for (int j = 0; j < kIn; ++j) {
        MP_CUDA_TRY(cudaStreamCreateWithFlags(&io->in[j], cudaStreamNonBlocking));
        MP_CUDA_TRY(cudaEventCreateWithFlags(&io->copied[j], cudaEventDisableTiming));
    }
    for (int j = 0; j < kOut; ++j) {
        MP_CUDA_TRY(cudaStreamCreateWithFlags(&io->out[j], cudaStreamNonBlocking));
        MP_CUDA_TRY(cudaEventCreateWithFlags(&io->returned[j], cudaEventDisableTiming));
    }
    for (int b = 0; b < 2; ++b) MP_CUDA_TRY(cudaEventCreateWithFlags(&io->freed[b], cudaEventDisableTiming));
    MP_CUDA_TRY(cudaEventCreateWithFlags(&io->start, cudaEventDisableTiming));
    MP_CUDA_TRY(cudaEventCreateWithFlags(&io->computed, cudaEventDisableTiming));
    return MP_OK;
}

void destroy(host_io *io)
{
    if (!io) return;
    if (io->device >= 0) {
        for (int j = 0; j < kIn; ++j)
            if (io->in[j]) cudaStreamSynchronize(io->in[j]);
        for (int j = 0; j < kOut; ++j)
            if (io->out[j]) cudaStreamSynchronize(io->out[j]);
        for (int b = 0; b < 2; ++b)
            if (io->freed[b] && io->used[b]) cudaEventSynchronize(io->freed[b]);
        for (int b = 0; b < 2; ++b) cudaFree(io->buf[b]);
        for (int j = 0; j < kIn; ++j) {
            if (io->in[j]) cudaStreamDestroy(io->in[j]);
            if (io->copied[j]) cudaEventDestroy(io->copied[j]);
        }
        for (int j = 0; j < kOut; ++j) {
            if (io->out[j]) cudaStreamDestroy(io->out[j]);
            if (io->returned[j]) cudaEventDestroy(io->returned[j]);
        }
        for (int b = 0; b < 2; ++b)
            if (io->freed[b]) cudaEventDestroy(io->freed[b]);
        if (io->start) cudaEventDestroy(io->start);
        if (io->computed) cudaEventDestroy(io->computed);
    }
    delete io;
}

std::mutex g_io_mu;

}  // namespace

void mp_host_io_free(void *io) { destroy(static_cast<host_io *>(io)); }

extern "C" int loop_res_calc_host(const mp_plan *cplan, int32_t dtype, const void *x, const void *q, const void *adt,
                                  void *res, double gam, double eps, void *stream)
{
    if (!cplan || !x || !q || !adt || !res || (dtype != MP_F64 && dtype != MP_F32 && dtype != MP_F64_DW))
        return MP_EINVAL;
    mp_plan *P = const_cast<mp_plan *>(cplan);
    if (P->nmaps != 2) return MP_EPLAN;
    if (P->from_size == 0) return MP_OK;
    int rc = mp_plan_ensure_device(P);
    if (rc != MP_OK) return rc;
    const size_t elt = dtype == MP_F32 ? 4 : 8;
    const int64_t nnode = P->maps[0].to_size, ncell = P->maps[1].to_size;
    const size_t bx = (size_t)(2 * nnode) * elt, bq = (size_t)(4 * ncell) * elt, ba = (size_t)ncell * elt;
    const size_t off_q = round256(bx), off_a = off_q + round256(bq), off_r = off_a + round256(ba);
    const size_t slot_bytes = off_r + round256(bq);
    host_io *io;
    {
        std::lock_guard<std::mutex> lk(g_io_mu);
        io = static_cast<host_io *>(P->dev.host_io);
        if (io && io->slot_bytes < slot_bytes) {  // a larger dtype than before: start over
            destroy(io);
            P->dev.host_io = io = nullptr;
        }
        if (!io) {
            io = new host_io();
            if ((rc = create(io, slot_bytes, P->dev.device)) != MP_OK) {
                destroy(io);
                return rc;
            }
            P->dev.host_io = io;
        }
    }
    std::lock_guard<std::mutex> lk(io->mu);
    cudaStream_t s = as_stream(stream);
    const int b = io->next;
    io->next ^= 1;
    unsigned char *base = static_cast<unsigned char *>(io->buf[b]);
    void *dx = base, *dq = base + off_q, *da = base + off_a, *dr = base + off_r;
    // the copies follow the caller's earlier work and the slot's last read-back
    MP_CUDA_TRY(cudaEventRecord(io->start, s));
    for (int j = 0; j < kIn; ++j) {
        MP_CUDA_TRY(cudaStreamWaitEvent(io->in[j], io->start, 0));
        if (io->used[b]) MP_CUDA_TRY(cudaStreamWaitEvent(io->in[j], io->freed[b], 0));
    }
    int turn = 0;
    auto chunked = [&](void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t *ss, int ns) {
        for (size_t o = 0; o < bytes; o += kChunk) {
            const size_t n = bytes - o < kChunk ? bytes - o : kChunk;
            const cudaError_t e = cudaMemcpyAsync(static_cast<unsigned char *>(dst) + o,
                                                  static_cast<const unsigned char *>(src) + o, n, kind,
                                                  ss[turn++ % ns]);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    MP_CUDA_TRY(chunked(dq, q, bq, cudaMemcpyHostToDevice, io->in, kIn));
    MP_CUDA_TRY(chunked(dr, res, bq, cudaMemcpyHostToDevice, io->in, kIn));
    MP_CUDA_TRY(chunked(dx, x, bx, cudaMemcpyHostToDevice, io->in, kIn));
    MP_CUDA_TRY(chunked(da, adt, ba, cudaMemcpyHostToDevice, io->in, kIn));
    for (int j = 0; j < kIn; ++j) {
        MP_CUDA_TRY(cudaEventRecord(io->copied[j], io->in[j]));
        MP_CUDA_TRY(cudaStreamWaitEvent(s, io->copied[j], 0));
    }
    if ((rc = loop_res_calc(P, dtype, dx, dq, da, dr, gam, eps, stream)) != MP_OK) return rc;
    MP_CUDA_TRY(cudaEventRecord(io->computed, s));
    for (int j = 0; j < kOut; ++j) MP_CUDA_TRY(cudaStreamWaitEvent(io->out[j], io->computed, 0));
    turn = 0;
    MP_CUDA_TRY(chunked(res, dr, bq, cudaMemcpyDeviceToHost, io->out, kOut));
    for (int j = 0; j < kOut; ++j) {
        MP_CUDA_TRY(cudaEventRecord(io->returned[j], io->out[j]));
        MP_CUDA_TRY(cudaStreamWaitEvent(s, io->returned[j], 0));
    }
    MP_CUDA_TRY(cudaEventRecord(io->freed[b], s));
    io->used[b] = true;
    return MP_OK;
}
