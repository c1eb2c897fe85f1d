// qldpc_decode_host_noalloc: the host-buffer decode staged through a static device array instead
// of device memory allocated at run time (for callers that cannot call cudaMalloc once running;
// see include/qldpc.h).  The decode itself is the regular qldpc_decode_ex launch.
#include "qldpc.h"

#include <cstddef>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "graph.h"

namespace {

// The scratch every call shares: prior, syndromes, e_hat, iterations and ok of one batch.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QLDPC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned char *g_addr[kMaxDevices] = {};

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch on the current device, resolved once per device.  The first
// resolution loads this file's module onto the device (lazy module loading), which is when the
// driver places the array in device memory.
int scratch_address(unsigned char **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return QLDPC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return QLDPC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return QLDPC_ERR_CUDA;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return QLDPC_OK;
}

}  // namespace

extern "C" QLDPC_API size_t qldpc_noalloc_scratch_bytes(void) { return sizeof(g_noalloc_scratch); }

extern "C" QLDPC_API int qldpc_decode_host_noalloc(const qldpc_graph *g, const uint8_t *h_syndromes,
                                                   int32_t batch, const float *h_prior,
                                                   int32_t max_iter, float alpha, uint8_t *h_err,
                                                   int32_t *h_iters, uint8_t *h_ok,
                                                   int32_t precision, uint32_t flags, void *stream)
{
    if (!g || batch < 0) return QLDPC_ERR_INVALID_ARG;
    if (batch > 0 && (!h_syndromes || !h_prior || !h_err || !h_iters || !h_ok))
        return QLDPC_ERR_INVALID_ARG;
    // Every argument check and the launch plan of this batch, before anything is enqueued.
    int rc = qldpc::detail::decode_plan(g, batch, max_iter, alpha, precision, flags);
    if (rc != QLDPC_OK) return rc;
    const size_t prior_b = round256(size_t(g->n) * sizeof(float));
    const size_t syn_b = round256(size_t(batch) * size_t(g->m));
    const size_t err_b = round256(size_t(batch) * size_t(g->n));
    const size_t it_b = round256(size_t(batch) * sizeof(int32_t));
    const size_t ok_b = round256(size_t(batch));
    if (prior_b + syn_b + err_b + it_b + ok_b > sizeof(g_noalloc_scratch)) return QLDPC_ERR_UNSUPPORTED;
    // Resolved even for an empty batch, so that a zero-shot call at start-up is the warm-up.
    unsigned char *base = nullptr;
    rc = scratch_address(&base);
    if (rc != QLDPC_OK || batch == 0) return rc;
    float *d_prior = reinterpret_cast<float *>(base);
    uint8_t *d_syn = base + prior_b;
    uint8_t *d_err = d_syn + syn_b;
    int32_t *d_iters = reinterpret_cast<int32_t *>(d_err + err_b);
    uint8_t *d_ok = reinterpret_cast<uint8_t *>(d_err + err_b + it_b);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(d_prior, h_prior, size_t(g->n) * sizeof(float),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_syn, h_syndromes, size_t(batch) * size_t(g->m), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        return QLDPC_ERR_CUDA;
    }
    rc = qldpc_decode_ex(g, d_syn, batch, d_prior, max_iter, alpha, d_err, d_iters, d_ok, nullptr,
                         precision, flags, stream);
    if (rc != QLDPC_OK) {
        cudaStreamSynchronize(st);
        return rc;
    }
    e = cudaMemcpyAsync(h_err, d_err, size_t(batch) * size_t(g->n), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_iters, d_iters, size_t(batch) * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_ok, d_ok, size_t(batch), cudaMemcpyDeviceToHost, st);
    const cudaError_t se = cudaStreamSynchronize(st);
    if (e != cudaSuccess || se != cudaSuccess) return QLDPC_ERR_CUDA;
    return QLDPC_OK;
}
