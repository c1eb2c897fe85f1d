// The opaque qldpc_graph of the C ABI and the host helpers shared by the library's translation
// units (qldpc_host.cpp: graphs and decodes; qldpc_server.cpp: the persistent server).  Internal.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "msa_launch.h"
#include "qldpc.h"

struct qldpc_graph {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;      // max dynamic shared memory per block (opt-in)
    int32_t m = 0, n = 0, nnz = 0, dc_max = 0, dv_max = 0;
    int32_t nv = 0;             // variable lanes of the kernels: n plus idle lanes (bank packing)
    bool uniform_rows = false;  // every row has degree dc_max
    void *d_block = nullptr;    // one device allocation for all graph arrays
    int32_t *d_counters = nullptr;              // [kShotCounterSlots][2] shot counters (inside d_block)
    mutable std::atomic<uint32_t> counter_seq{0};
    qldpc::DeviceGraph dg{};
    // launch overrides (0 = automatic)
    int user_kernel = QLDPC_KERNEL_AUTO, user_threads = 0, user_blocks_per_sm = 0;
    // staging for qldpc_decode_host
    std::mutex host_mu;
    int32_t cap = 0;
    void *d_stage = nullptr;
    uint8_t *d_syn = nullptr, *d_err = nullptr, *d_ok = nullptr;
    int32_t *d_iters = nullptr;
    float *d_prior = nullptr;
    uint8_t *h_stage = nullptr;     // page-locked copy-back buffer for small batches
    size_t h_stage_bytes = 0;
    std::vector<float> prior_cache;
    bool prior_valid = false;
    // learned decoding: [learned_T][dc_max * m] slot-layout weights (qldpc_graph_set_weights)
    float *d_weights = nullptr;
    int32_t learned_T = 0;
    // last training launch plan (qldpc_learned.cpp), keyed by (batch, T)
    std::mutex train_mu;
    int32_t train_batch = 0, train_T = 0;
    unsigned char train_plan[256];
};

namespace qldpc {

int dc_bucket(int d);   // row-degree bucket 8 / 16 / 32, -1 above
int dv_bucket(int d);   // column-degree bucket 4 / 8 / 16, -1 above
// Compiled kernel variant for graphs of largest row degree dc and column degree dv: the exact
// degree when every row has degree dc in 6..9 (uniform), else the buckets.
KernelChoice kernel_variant(int dc, int dv, bool uniform, bool latency, bool learned);

namespace detail {

int cuda_status(cudaError_t e);                                             // cudaError -> qldpc_status
int ensure_kernel_attrs(const void *k, size_t smem, size_t smem_optin);     // >48 KB dynamic smem opt-in
int check_device(const qldpc_graph *g);                                     // graph belongs to the current device
int alpha_fixed(float alpha);                                               // round(alpha*2^15), -1 outside (0,1]
// Every argument check and the launch plan of a qldpc_decode_ex call on g with this batch, without
// enqueuing anything: QLDPC_OK when such a call would launch.
int decode_plan(const qldpc_graph *g, int32_t batch, int32_t max_iter, float alpha, int32_t precision,
                uint32_t flags);

}  // namespace detail
}  // namespace qldpc
