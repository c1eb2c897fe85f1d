// Host side of the persistent decoding server (include/qldpc.h: qldpc_server_*).
//
// The server owns, per code, a ring of request slots in page-locked host memory mapped into the
// device address space and the device copy of the code's prior (and learned weights), plus one
// arrival-ordered queue of request entries (also mapped) and its device-side claim counter; one
// persistent kernel (server_kernel.cuh, or the layered workers of msa_layered.cu) runs all worker
// blocks on a private stream.  The host publishes a request by writing its syndrome into a free slot
// of its code's ring and then the request's entry into the queue with a release store; any free
// worker claims the oldest entry, whatever its code.  Completion is the slot's done word (acquire
// load).  Relaunching after the workers left (idle) is safe: workers only leave with every
// published request claimed and finished, and the counters survive in memory.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "graph.h"
#include "msa_launch.h"
#include "qldpc.h"

using namespace qldpc;
using namespace qldpc::detail;

struct qldpc_server {
    int device = 0;
    int precision = QLDPC_FP32;
    bool layered = false;                   // QLDPC_LAYERED: layered-schedule workers
    int ncodes = 0;
    const qldpc_graph *graphs[kServerMaxCodes] = {};
    int32_t m[kServerMaxCodes] = {}, n[kServerMaxCodes] = {};
    int32_t capacity = 0;                   // slots per code ring
    ServerParams sp{};
    KernelChoice kc{};
    int blocks = 0, threads = 0;
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    unsigned char *host_block = nullptr;    // queue + rings + stop (page-locked, mapped)
    unsigned long long *queue = nullptr;    // [queue_cap] entries
    uint32_t queue_cap = 0;
    unsigned char *ring[kServerMaxCodes] = {};
    uint32_t *stop = nullptr;
    void *dev_block = nullptr;              // head + status + priors + weights
    uint32_t *head = nullptr;
    uint32_t *status = nullptr;
    uint64_t next_global = 0;               // arrival number of the next request
    uint64_t next[kServerMaxCodes] = {};    // next ticket (sequence number) per code
    // per slot: holds a request whose result is uncollected, and that request's completion word
    std::vector<uint8_t> busy[kServerMaxCodes];
    std::vector<uint32_t> done_word[kServerMaxCodes];
    bool launched = false;
    std::mutex mu;
};

namespace {

int launch_server(qldpc_server *s)
{
    cudaError_t e = s->layered ? launch_server_layered(s->precision, s->sp, s->kc, s->blocks, s->threads, s->smem, s->stream)
                    : s->precision == QLDPC_INT16 ? launch_server_i16(s->sp, s->kc, s->blocks, s->threads, s->smem, s->stream)
                    : s->precision == QLDPC_INT8  ? launch_server_i8(s->sp, s->kc, s->blocks, s->threads, s->smem, s->stream)
                                                  : launch_server_f32(s->sp, s->kc, s->blocks, s->threads, s->smem, s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    s->launched = true;
    return QLDPC_OK;
}

// Relaunch the workers if they left (idle timeout) while requests may be waiting.
int ensure_running(qldpc_server *s)
{
    if (s->launched) {
        const cudaError_t q = cudaStreamQuery(s->stream);
        if (q == cudaErrorNotReady) return QLDPC_OK;
        if (q != cudaSuccess) return cuda_status(q);
        s->launched = false;
    }
    return launch_server(s);
}

unsigned char *slot_ptr(qldpc_server *s, int code, uint64_t seq)
{
    return s->ring[code] + size_t(seq & uint64_t(s->capacity - 1)) * size_t(s->sp.code[code].slot_bytes);
}

int submit_locked(qldpc_server *s, int32_t code, const uint8_t *syndrome, uint64_t *ticket)
{
    const uint64_t seq = s->next[code];
    const size_t idx = size_t(seq & uint64_t(s->capacity - 1));
    if (s->busy[code][idx]) return QLDPC_BUSY;
    unsigned char *slot = slot_ptr(s, code, seq);
    std::memcpy(slot + s->sp.code[code].syn_off, syndrome, size_t(s->m[code]));
    // The queue holds at most every ring slot's request at once (its capacity covers them all), so
    // the entry about to be overwritten was claimed long ago.
    const uint64_t g = s->next_global++;
    const uint32_t done = uint32_t(g + 1);
    __atomic_store_n(reinterpret_cast<uint32_t *>(slot), done - 1u, __ATOMIC_RELAXED);   // not done
    s->busy[code][idx] = 1;
    s->done_word[code][idx] = done;
    s->next[code] = seq + 1;
    const unsigned long long entry = (static_cast<unsigned long long>(done) << 32) |
                                     (static_cast<unsigned long long>(code) << kQueueCodeShift) | idx;
    __atomic_store_n(s->queue + (g & (s->queue_cap - 1)), entry, __ATOMIC_RELEASE);   // publish
    if (int rc = ensure_running(s)) return rc;
    *ticket = seq;
    return QLDPC_OK;
}

// QLDPC_OK with the outputs copied (and the slot released) once the request is done.
int poll_locked(qldpc_server *s, int32_t code, uint64_t ticket, uint8_t *err, int32_t *iters, uint8_t *ok,
                int32_t *worker)
{
    if (ticket >= s->next[code] || ticket + uint64_t(s->capacity) < s->next[code]) return QLDPC_ERR_INVALID_ARG;
    const size_t idx = size_t(ticket & uint64_t(s->capacity - 1));
    if (!s->busy[code][idx]) return QLDPC_ERR_INVALID_ARG;     // already collected
    unsigned char *slot = slot_ptr(s, code, ticket);
    const uint32_t done = __atomic_load_n(reinterpret_cast<uint32_t *>(slot), __ATOMIC_ACQUIRE);
    if (done != s->done_word[code][idx]) {
        if (int rc = ensure_running(s)) return rc;
        return QLDPC_PENDING;
    }
    if (err) std::memcpy(err, slot + s->sp.code[code].err_off, size_t(s->n[code]));
    if (iters) std::memcpy(iters, slot + 4, 4);
    if (ok) *ok = slot[8];
    if (worker) {
        uint16_t w;
        std::memcpy(&w, slot + 10, 2);
        *worker = int32_t(w);
    }
    s->busy[code][idx] = 0;
    return QLDPC_OK;
}

void free_server(qldpc_server *s)
{
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->host_block) cudaFreeHost(s->host_block);
    if (s->dev_block) cudaFree(s->dev_block);
    delete s;
}

}  // namespace

extern "C" {

int qldpc_server_create(const qldpc_graph *const *graphs, const float *const *priors, int32_t ncodes,
                        const qldpc_server_config *cfg, qldpc_server **out)
{
    if (!out) return QLDPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!graphs || !priors || !cfg || ncodes < 1 || ncodes > QLDPC_SERVER_MAX_CODES) return QLDPC_ERR_INVALID_ARG;
    if (cfg->precision != QLDPC_FP32 && cfg->precision != QLDPC_INT16 && cfg->precision != QLDPC_INT8)
        return QLDPC_ERR_INVALID_ARG;
    if ((cfg->flags & ~uint32_t(QLDPC_NO_EARLY_STOP | QLDPC_LEARNED | QLDPC_LAYERED)) != 0 || cfg->max_iter < 0)
        return QLDPC_ERR_INVALID_ARG;
    const bool learned = (cfg->flags & QLDPC_LEARNED) != 0;
    const bool layered = (cfg->flags & QLDPC_LAYERED) != 0;
    if (learned && layered) return QLDPC_ERR_INVALID_ARG;
    if (learned && (cfg->precision != QLDPC_FP32 || (cfg->flags & QLDPC_NO_EARLY_STOP))) return QLDPC_ERR_INVALID_ARG;
    if (!std::isfinite(cfg->alpha) || cfg->alpha <= 0.0f) return QLDPC_ERR_INVALID_ARG;
    const int aq = cfg->precision == QLDPC_FP32 ? 0 : alpha_fixed(cfg->alpha);
    if (aq < 0) return QLDPC_ERR_INVALID_ARG;
    const int32_t cap = cfg->ring_capacity ? cfg->ring_capacity : 256;
    if (cap < 2 || cap > (1 << 20) || (cap & (cap - 1))) return QLDPC_ERR_INVALID_ARG;
    for (int c = 0; c < ncodes; ++c) {
        if (!graphs[c] || !priors[c] || cfg->blocks[c] < 0) return QLDPC_ERR_INVALID_ARG;
        for (int32_t v = 0; v < graphs[c]->n; ++v)
            if (!std::isfinite(priors[c][v])) return QLDPC_ERR_INVALID_ARG;
        if (graphs[c]->device != graphs[0]->device) return QLDPC_ERR_INVALID_ARG;
    }
    if (int rc = check_device(graphs[0])) return rc;

    qldpc_server *s = new (std::nothrow) qldpc_server();
    if (!s) return QLDPC_ERR_OOM;
    s->device = graphs[0]->device;
    s->precision = cfg->precision;
    s->layered = layered;
    s->ncodes = ncodes;
    s->capacity = cap;

    // One footprint for every worker, the largest any code needs (kernel variant of the largest
    // degrees, threads, shared memory), so that every worker can decode every code.
    int dc = 0, dv = 0, want = 32;
    bool uniform = true;
    size_t smem = 0;
    for (int c = 0; c < ncodes; ++c) {
        const qldpc_graph *g = graphs[c];
        s->graphs[c] = g;
        s->m[c] = g->m;
        s->n[c] = g->n;
        dc = std::max(dc, g->dc_max);
        dv = std::max(dv, g->dv_max);
        uniform = uniform && g->uniform_rows && g->dc_max == graphs[0]->dc_max;
        const int one = (std::max(g->m, g->nv) + 31) / 32 * 32;
        const int two = (std::max((g->m + 1) / 2, (g->nv + 1) / 2) + 31) / 32 * 32;
        want = std::max(want, one <= kLatencyMaxThreads ? one : two);
        smem = std::max(smem, latency_layout(g->m, g->dc_max, msg_bytes(cfg->precision)).total);
    }
    s->kc = kernel_variant(dc, dv, uniform, true, false);
    for (int c = 0; c < ncodes; ++c) s->kc.learned = s->kc.learned || (learned && graphs[c]->d_weights);
    bool fits;
    int layered_reg[kServerMaxCodes] = {};
    if (layered) {
        // a thread per check of the widest layer; a code of at most 8 layers keeps one check per
        // layer per thread in registers, one with more layers its messages in shared memory
        int widest = 32;
        smem = 0;
        fits = dc <= 8;
        for (int c = 0; c < ncodes; ++c) {
            const qldpc_graph *g = graphs[c];
            widest = std::max(widest, (g->dg.max_layer + 31) / 32 * 32);
            layered_reg[c] = g->dg.nlayers <= kLayeredServerMaxLayers && g->n <= 65536;
            smem = std::max(smem, layered_reg[c] ? align16(size_t(g->n) * 4)
                                                 : layered_layout(g->m, g->n, g->dc_max, msg_bytes(cfg->precision)).total);
        }
        s->kc = kernel_variant(dc, dv, uniform, false, false);
        s->kc.layered = true;
        s->threads = cfg->threads_per_block ? cfg->threads_per_block : widest;
        fits = fits && s->threads >= widest && s->threads <= kLayeredServerMaxThreads && s->threads % 32 == 0;
    } else {
        s->threads = cfg->threads_per_block ? cfg->threads_per_block : std::min(want, kLatencyMaxThreads);
        fits = s->threads >= 32 && s->threads <= kLatencyMaxThreads && s->threads % 32 == 0;
        for (int c = 0; c < ncodes; ++c)
            fits = fits && graphs[c]->m <= kLatencyCnPerThread * s->threads &&
                   graphs[c]->nv <= kLatencyVnPerThread * s->threads;
    }
    s->smem = smem;
    const void *k = !fits                            ? nullptr
                    : layered                        ? server_kernel_layered(cfg->precision, s->kc)
                    : cfg->precision == QLDPC_INT16 ? server_kernel_i16(s->kc)
                    : cfg->precision == QLDPC_INT8  ? server_kernel_i8(s->kc)
                                                    : server_kernel_f32(s->kc);
    if (!k) {
        delete s;
        return QLDPC_ERR_UNSUPPORTED;
    }
    if (int rc = ensure_kernel_attrs(k, smem, graphs[0]->smem_optin)) {
        delete s;
        return rc;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, s->threads, smem) != cudaSuccess || per_sm < 1) {
        delete s;
        return QLDPC_ERR_UNSUPPORTED;
    }
    // A worker reloads a code's graph arrays through L1 when it switches codes: ask for the smallest
    // shared-memory carve-out that still holds the resident workers, which leaves the rest of each
    // SM's 256 KB to L1 (a hint the driver rounds up to a supported size).  Kept only if the
    // residency stays the same.
    {
        const size_t need = size_t(per_sm) * (smem + 2048);
        const int pct = int(std::min<size_t>(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024)));
        int again = 0;
        if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&again, k, s->threads, smem) != cudaSuccess || again != per_sm) {
            cudaGetLastError();
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, -1);
            cudaGetLastError();
        }
    }
    // Worker pool: the sum of cfg->blocks when given, else every worker that fits on the GPU at
    // this footprint.  All of them must be resident at once (a worker that never starts would never
    // take a request).
    const int resident = per_sm * graphs[0]->sm_count;
    int total = 0;
    for (int c = 0; c < ncodes; ++c) total += cfg->blocks[c];
    if (total == 0) total = resident;
    if (total > resident || total > 65535) {
        delete s;
        return QLDPC_ERR_UNSUPPORTED;
    }
    s->blocks = total;

    // page-locked, mapped host memory: the queue (one entry per ring slot of every code, rounded up
    // to a power of two), the rings, the stop flag
    uint32_t qcap = 1;
    while (qcap < uint32_t(ncodes) * uint32_t(cap)) qcap <<= 1;
    s->queue_cap = qcap;
    size_t host_bytes = size_t(qcap) * sizeof(unsigned long long);
    size_t ring_off[kServerMaxCodes];
    for (int c = 0; c < ncodes; ++c) {
        ring_off[c] = host_bytes;
        host_bytes += size_t(cap) * size_t(server_slot_bytes(s->m[c], s->n[c]));
    }
    const size_t stop_off = align16(host_bytes);
    host_bytes = stop_off + 64;
    void *hb = nullptr;
    cudaError_t e = cudaHostAlloc(&hb, host_bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) {
        delete s;
        return cuda_status(e);
    }
    std::memset(hb, 0, host_bytes);
    s->host_block = static_cast<unsigned char *>(hb);
    s->queue = reinterpret_cast<unsigned long long *>(s->host_block);
    s->stop = reinterpret_cast<uint32_t *>(s->host_block + stop_off);
    void *hb_dev = nullptr;
    if (cudaHostGetDevicePointer(&hb_dev, hb, 0) != cudaSuccess) {
        free_server(s);
        return QLDPC_ERR_CUDA;
    }
    unsigned char *hd = static_cast<unsigned char *>(hb_dev);

    // device memory: claim counter, status, priors, and a private copy of each code's learned
    // weights (QLDPC_LEARNED; a code without weights decodes plainly)
    size_t dev_bytes = 256;
    size_t prior_off[kServerMaxCodes], w_off[kServerMaxCodes], w_bytes[kServerMaxCodes];
    for (int c = 0; c < ncodes; ++c) {
        prior_off[c] = dev_bytes;
        dev_bytes += align16(size_t(s->n[c]) * sizeof(float));
        const qldpc_graph *g = graphs[c];
        w_bytes[c] = (learned && g->d_weights) ? size_t(g->learned_T) * g->dc_max * g->m * sizeof(float) : 0;
        w_off[c] = dev_bytes;
        dev_bytes += align16(w_bytes[c]);
    }
    e = cudaMalloc(&s->dev_block, dev_bytes);
    if (e == cudaSuccess) e = cudaMemset(s->dev_block, 0, 256);
    for (int c = 0; c < ncodes && e == cudaSuccess; ++c) {
        e = cudaMemcpy(static_cast<char *>(s->dev_block) + prior_off[c], priors[c], size_t(s->n[c]) * sizeof(float),
                       cudaMemcpyHostToDevice);
        if (e == cudaSuccess && w_bytes[c])
            e = cudaMemcpy(static_cast<char *>(s->dev_block) + w_off[c], graphs[c]->d_weights, w_bytes[c],
                           cudaMemcpyDeviceToDevice);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_server(s);
        return cuda_status(e);
    }
    s->head = static_cast<uint32_t *>(s->dev_block);
    s->status = static_cast<uint32_t *>(s->dev_block) + 32;

    ServerParams &sp = s->sp;
    sp.ncodes = ncodes;
    sp.queue = reinterpret_cast<const unsigned long long *>(hd);
    sp.queue_mask = qcap - 1;
    sp.head = s->head;
    sp.max_iter = cfg->max_iter;
    sp.alpha = cfg->alpha;
    sp.alpha_q = aq;
    sp.flags = cfg->flags & QLDPC_NO_EARLY_STOP;
    sp.stop = reinterpret_cast<const uint32_t *>(hd + stop_off);
    sp.status = s->status;
    sp.idle_ns = uint64_t(cfg->idle_timeout_ns > 0 ? cfg->idle_timeout_ns : 500000000LL);
    sp.max_runtime_ns = uint64_t(cfg->max_runtime_ns > 0 ? cfg->max_runtime_ns : 600000000000LL);
    for (int c = 0; c < ncodes; ++c) {
        ServerCode &sc = sp.code[c];
        sc.g = graphs[c]->dg;
        sc.prior = reinterpret_cast<const float *>(static_cast<char *>(s->dev_block) + prior_off[c]);
        sc.weights = w_bytes[c] ? reinterpret_cast<const float *>(static_cast<char *>(s->dev_block) + w_off[c]) : nullptr;
        sc.learned_iters = w_bytes[c] ? graphs[c]->learned_T : 0;
        sc.ring = hd + ring_off[c];
        sc.slot_bytes = server_slot_bytes(s->m[c], s->n[c]);
        sc.syn_off = 16;
        sc.err_off = int32_t(align16(16 + size_t(s->m[c])));
        sc.layered_reg = layered_reg[c];
        sc.udc = (graphs[c]->uniform_rows && graphs[c]->dc_max >= 6 && graphs[c]->dc_max <= 9) ? graphs[c]->dc_max : 0;
        s->ring[c] = s->host_block + ring_off[c];
        s->busy[c].assign(size_t(cap), 0);
        s->done_word[c].assign(size_t(cap), 0);
    }
    *out = s;
    return QLDPC_OK;
}

int qldpc_server_submit(qldpc_server *s, int32_t code, const uint8_t *syndrome, uint64_t *ticket)
{
    if (!s || !syndrome || !ticket || code < 0 || code >= s->ncodes) return QLDPC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    return submit_locked(s, code, syndrome, ticket);
}

int qldpc_server_poll(qldpc_server *s, int32_t code, uint64_t ticket, uint8_t *err, int32_t *iters, uint8_t *ok)
{
    if (!s || code < 0 || code >= s->ncodes) return QLDPC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    return poll_locked(s, code, ticket, err, iters, ok, nullptr);
}

int qldpc_server_replay(qldpc_server *s, int32_t nreq, const int32_t *codes, const uint8_t *syndromes,
                        const int64_t *syn_offsets, const int64_t *arrival_ns, uint8_t *errs,
                        const int64_t *err_offsets, int32_t *iters, uint8_t *oks, int64_t *latency_ns,
                        int32_t *workers, int64_t timeout_ns)
{
    if (!s || nreq < 0) return QLDPC_ERR_INVALID_ARG;
    if (nreq == 0) return QLDPC_OK;
    if (!codes || !syndromes || !syn_offsets || !arrival_ns || !errs || !err_offsets || !iters || !oks || !latency_ns)
        return QLDPC_ERR_INVALID_ARG;
    for (int32_t i = 0; i < nreq; ++i)
        if (codes[i] < 0 || codes[i] >= s->ncodes || (i && arrival_ns[i] < arrival_ns[i - 1])) return QLDPC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    using clock = std::chrono::steady_clock;
    std::vector<int32_t> inflight;
    std::vector<uint64_t> tickets(size_t(nreq), 0);
    inflight.reserve(1024);
    const auto t0 = clock::now();
    const int64_t deadline = arrival_ns[nreq - 1] + (timeout_ns > 0 ? timeout_ns : 10000000000LL);
    int32_t next = 0, completed = 0;
    while (completed < nreq) {
        const int64_t now = std::chrono::duration_cast<std::chrono::nanoseconds>(clock::now() - t0).count();
        if (now > deadline) return QLDPC_ERR_TIMEOUT;
        while (next < nreq && arrival_ns[next] <= now) {
            const int rc = submit_locked(s, codes[next], syndromes + syn_offsets[next], &tickets[size_t(next)]);
            if (rc == QLDPC_BUSY) break;            // ring full: serve completions first
            if (rc) return rc;
            inflight.push_back(next++);
        }
        for (size_t j = 0; j < inflight.size();) {
            const int32_t i = inflight[j];
            const int rc = poll_locked(s, codes[i], tickets[size_t(i)], errs + err_offsets[i], iters + i, oks + i,
                                       workers ? workers + i : nullptr);
            if (rc == QLDPC_OK) {
                const int64_t t = std::chrono::duration_cast<std::chrono::nanoseconds>(clock::now() - t0).count();
                latency_ns[i] = t - arrival_ns[i];
                ++completed;
                inflight[j] = inflight.back();
                inflight.pop_back();
            } else if (rc == QLDPC_PENDING) {
                ++j;
            } else {
                return rc;
            }
        }
    }
    return QLDPC_OK;
}

int qldpc_server_info(const qldpc_server *s, int32_t *workers, int32_t *threads_per_block, size_t *smem_per_block)
{
    if (!s) return QLDPC_ERR_INVALID_ARG;
    if (workers) *workers = s->blocks;
    if (threads_per_block) *threads_per_block = s->threads;
    if (smem_per_block) *smem_per_block = s->smem;
    return QLDPC_OK;
}

int qldpc_server_status(qldpc_server *s, uint32_t *status)
{
    if (!s || !status) return QLDPC_ERR_INVALID_ARG;
    return cuda_status(cudaMemcpy(status, s->status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
}

void qldpc_server_destroy(qldpc_server *s)
{
    if (!s) return;
    __atomic_store_n(s->stop, 1u, __ATOMIC_RELEASE);
    if (s->stream) cudaStreamSynchronize(s->stream);   // workers leave at the stop flag
    free_server(s);
}

}  // extern "C"
