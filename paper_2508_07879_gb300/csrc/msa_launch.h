// Internal interface between the C-ABI host code (qldpc_host.cpp) and the sm_103a kernels
// (msa_f32.cu, msa_i16.cu).  Not installed; the public ABI is include/qldpc.h.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "qldpc.h"

namespace qldpc {

// Tanner graph in the kernels' layout.  Messages of check i live in shared-memory "slots"
// j*m + i (j = position of the edge in row i), so a warp working on 32 consecutive checks touches
// 32 consecutive slots; the check side needs no index at all.  Variables occupy nv >= n lanes:
// grouped by descending degree and packed so that the k-th slots of a warp's 32 variables fall in
// distinct shared-memory banks where possible, with idle lanes (vperm = n) closing a warp early.
// Lane u holds the caller's variable vperm[u]; the k-th edge of lane u (ascending check order) is
// the slot vslot[k*nv + u] = j*m + i, and i = slot mod m (m_magic, m_shift; the two-shots-per-block
// kernel reads it from vchk16) when a decision flips.  An idle lane has its warp's degree and every edge on a scratch slot dc_max*m + b
// (b < kScratch) in a bank its warp leaves free, so it runs its warp's path without divergence;
// its prior is 0 and its scratch slots hold 0, so its decision never flips.
constexpr int kMaxDegClasses = QLDPC_MAX_COL_DEGREE + 1;   // column degrees 0..16

struct DeviceGraph {
    const uint32_t *vslot;   // [dv_max * nv] slot j*m + i of lane u's k-th edge
    const uint8_t *vdeg;     // [nv] column degree of lane u (idle: its warp's degree)
    const uint8_t *rdeg;     // [m] row degrees
    const uint32_t *vperm;   // [nv] caller's index of the variable in lane u (n: idle lane)
    const uint32_t *ecol;    // [dc_max * m] original variable of slot j*m + i (0xffffffff: no edge)
    const int32_t *slot_edge;// [dc_max * m] CSR edge index of slot j*m + i (-1: no edge)
    const uint32_t *eslot;   // [nnz] slot j*m + i of CSR edge e
    const int32_t *layer_ptr;// [nlayers + 1] layered schedule: checks of layer l are
    const uint32_t *layer_chk;//   layer_chk[layer_ptr[l] .. layer_ptr[l+1]) (ascending)
    int32_t nlayers, max_layer;
    int32_t m, n, nnz;
    int32_t nv;              // variable lanes (n <= nv)
    uint32_t m_magic;        // floor(slot / m) = umulhi(slot, m_magic) >> m_shift for every slot
    int32_t m_shift;
    int32_t dc_max, dv_max;  // largest row / column degree
    // The same slot lists as 16-bit indices (nullptr when a slot index exceeds 65535), and the lanes'
    // degree classes: lanes [cls_end[c-1], cls_end[c]) (cls_end[-1] = 0) all have degree cls_deg[c],
    // c < ncls.  The two-shots-per-block kernel walks the classes with the degree known at compile
    // time instead of reading vdeg per lane.
    const uint16_t *vslot16;
    const uint32_t *vlane;   // [n] lane of each variable (the inverse of vperm on the real lanes)
    const uint16_t *vchk16;  // [dv_max * nv] the check of each vslot16 entry (slot mod m), with vslot16
    int32_t ncls;
    int32_t cls_end[kMaxDegClasses];
    int32_t cls_deg[kMaxDegClasses];
};

// One decoding problem: a graph and the caller's buffers for one batch.
struct Problem {
    DeviceGraph g;
    const uint8_t *syn;      // [batch * m]
    const float *prior;      // [n]
    uint8_t *err;            // [batch * n]
    int32_t *iters;          // [batch]
    uint8_t *ok;             // [batch]
    float *post;             // [batch * n] or nullptr
    const float *weights;    // learned decoding: [learned_iters][dc_max * m] slot-layout weights
    int32_t learned_iters;   // learned iterations before the plain fallback (learned kernels only)
};

struct LaunchParams {
    Problem prob[2];         // prob[blockIdx.y]; two for the X+Z pair decode
    int32_t nprob;
    int32_t batch;
    int32_t max_iter;
    float alpha;             // FP32 scale
    int32_t alpha_q;         // fixed-point scale, round(alpha * 2^15)
    uint32_t flags;
    int32_t *next_shot;      // batch and layered kernels: zeroed per-launch shot counters
                             // [blockIdx.y], claimed with atomicAdd; nullptr: shots b = blockIdx.x + k*gridDim.x
};

// Counters for dynamic shot claiming: a ring per graph, one pair per launch, zeroed in-stream
// before the launch, so launches in flight on different streams use different pairs.
constexpr int kShotCounterSlots = 1024;

constexpr uint32_t kFlagNoEarlyStop = 1u;

// Idle variable lanes (see DeviceGraph) read and write one of kScratch words past the last slot,
// which no check step reads.
constexpr int kScratch = 32;

// Shared-memory layout of one shot in the batch kernel (identical on host and device);
// n = variable lanes.
struct SmemLayout {
    size_t q_off, g_off, par_off, slot_off, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SmemLayout smem_layout(int m, int n, int dc_max, int msg_bytes)
{
    SmemLayout s;
    s.q_off = 0;                                                       // a-posteriori Q_n [n] (4 B)
    s.g_off = align16(s.q_off + size_t(n) * 4);                        // prior gamma_n    [n] (4 B)
    s.par_off = align16(s.g_off + size_t(n) * 4);                      // parity words     [m] (4 B)
    s.slot_off = align16(s.par_off + size_t(m) * 4);                   // messages [dc_max*m + scratch]
    s.total = align16(s.slot_off + (size_t(dc_max) * m + kScratch) * msg_bytes);
    return s;
}

// Latency kernel: parity words and messages only (everything else lives in registers).
struct LatencyLayout {
    size_t par_off, slot_off, total;
};

__host__ __device__ inline LatencyLayout latency_layout(int m, int dc_max, int msg_bytes)
{
    LatencyLayout s;
    s.par_off = 0;
    s.slot_off = align16(size_t(m) * 4);
    s.total = align16(s.slot_off + (size_t(dc_max) * m + kScratch) * msg_bytes);
    return s;
}

enum Precision { kFP32 = 0, kINT16 = 1, kINT8 = 2 };

// Bytes per edge message: FP32 4, INT16 2, INT8 1.
inline int msg_bytes(int precision) { return precision == kINT16 ? 2 : precision == kINT8 ? 1 : 4; }

// Which compiled variant runs a launch.
struct KernelChoice {
    bool latency;    // msa_latency_kernel (else msa_batch_kernel)
    int dc;          // exact row degree (uniform) or row-degree bucket 8/16/32
    bool uniform;    // every row has exactly dc edges
    int dvb;         // column-degree bucket 4/8/16
    bool learned = false;   // learned weights first, then plain fallback (FP32 only)
    bool layered = false;   // msa_layered_kernel (row-serial schedule)
    bool packed = false;    // msa_packed_kernel: two fixed-point shots per message word (INT16 / INT8)
};

// Latency kernel limits: checks M <= 2 * threads, variables N <= 2 * threads, threads <= 640
// (a block of at most 640 threads leaves each thread about 100 registers).
constexpr int kLatencyCnPerThread = 2;
constexpr int kLatencyVnPerThread = 2;
constexpr int kLatencyMaxThreads = 640;

// ---------------------------------------------------------------------------------------------
// Persistent server (server_kernel.cuh): worker blocks that take requests of any code from one
// arrival-ordered queue.
// ---------------------------------------------------------------------------------------------
constexpr int kServerMaxCodes = 4;

// Status bits a server kernel leaves in ServerParams::status.
constexpr uint32_t kServerIdleExit = 1u;     // a worker left after idle_ns without a request
constexpr uint32_t kServerTimeLimit = 2u;    // a worker left at max_runtime_ns
constexpr uint32_t kServerSpinLimit = 4u;    // a worker left at the spin-count safety cap
constexpr uint32_t kServerStopped = 8u;      // a worker left on the host's stop flag

// Queue entry (64 bits, page-locked host memory mapped into the device address space), written by
// the host with a release store when it publishes request number g (counting from 0):
//   [32, 64)  g + 1 (mod 2^32): the entry is published for the worker whose head count is g;
//             also the completion word the worker writes into the slot
//   [20, 24)  code      [0, 20)  slot index in the code's ring
// Bits [24, 32) are zero in every entry, so an all-ones value can stand for "no request".
constexpr int kQueueCodeShift = 20;
constexpr int kQueueCodeMask = 0xf;
constexpr uint32_t kQueueSlotMask = (1u << 20) - 1u;
constexpr unsigned long long kQueueLeave = ~0ull;

// Request slot in a code's ring (page-locked host memory mapped into the device address space):
//   [0, 4)   done: the entry's arrival number + 1, written by the device last (release)
//   [4, 8)   iterations run          [8] ok          [10, 12) index of the worker block
//   [syn_off, syn_off + m)  syndrome bits, written by the host before it publishes the request
//   [err_off, err_off + n)  e_hat, written by the device
struct ServerCode {
    DeviceGraph g;
    const float *prior;         // device [n]
    const float *weights;       // FP32 learned decoding: [learned_iters][dc_max * m], or nullptr
    int32_t learned_iters;
    unsigned char *ring;        // ring_capacity slots of slot_bytes
    int32_t slot_bytes, syn_off, err_off;
    int32_t layered_reg;        // layered workers: 1 = register-resident checks (<= 8 layers), 0 = shared memory
    int32_t udc;                // every row has this degree (6..9), else 0: the check step's compiled degree
};

struct ServerParams {
    ServerCode code[kServerMaxCodes];
    int32_t ncodes;
    const unsigned long long *queue;   // [queue_mask + 1] entries (host-written)
    uint32_t queue_mask;        // capacity - 1, capacity a power of two >= every ring slot together
    uint32_t *head;             // device count of claimed entries
    int32_t max_iter;
    float alpha;
    int32_t alpha_q;
    uint32_t flags;
    const uint32_t *stop;       // host-written stop flag
    uint32_t *status;           // device status bits
    uint64_t idle_ns, max_runtime_ns;
};

inline int server_slot_bytes(int m, int n) { return int(align16(16 + size_t(m)) + align16(size_t(n))); }

const void *server_kernel_f32(const KernelChoice &kc);
const void *server_kernel_i16(const KernelChoice &kc);
const void *server_kernel_i8(const KernelChoice &kc);
cudaError_t launch_server_f32(const ServerParams &p, const KernelChoice &kc, int blocks, int threads,
                              size_t smem, cudaStream_t stream);
cudaError_t launch_server_i16(const ServerParams &p, const KernelChoice &kc, int blocks, int threads,
                              size_t smem, cudaStream_t stream);
cudaError_t launch_server_i8(const ServerParams &p, const KernelChoice &kc, int blocks, int threads,
                             size_t smem, cudaStream_t stream);
// Server workers on the layered schedule (msa_layered.cu): rows of degree <= 8 and at most
// kLayeredServerMaxThreads checks per layer.  A code of at most kLayeredServerMaxLayers layers keeps
// its checks in registers; one with more layers keeps its messages in shared memory.
constexpr int kLayeredServerMaxLayers = 8;
constexpr int kLayeredServerMaxThreads = 256;
const void *server_kernel_layered(int precision, const KernelChoice &kc);
cudaError_t launch_server_layered(int precision, const ServerParams &p, const KernelChoice &kc, int blocks,
                                  int threads, size_t smem, cudaStream_t stream);

// Per-precision instantiation tables (one translation unit each).
const void *msa_kernel_f32(const KernelChoice &kc);
const void *msa_kernel_i16(const KernelChoice &kc);
cudaError_t launch_msa_f32(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                           size_t smem, cudaStream_t stream);
cudaError_t launch_msa_i16(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                           size_t smem, cudaStream_t stream);
const void *msa_kernel_i8(const KernelChoice &kc);
cudaError_t launch_msa_i8(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                          size_t smem, cudaStream_t stream);
// Two-shots-per-word fixed-point throughput kernels, msa_i16x2.cu / msa_i8x2.cu (msa_packed.cuh).
const void *msa_kernel_i16x2(const KernelChoice &kc);
const void *msa_kernel_i8x2(const KernelChoice &kc);
const void *msa_kernel_f32x2(const KernelChoice &kc);
cudaError_t launch_msa_f32x2(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                             size_t smem, cudaStream_t stream);
cudaError_t launch_msa_i16x2(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                             size_t smem, cudaStream_t stream);
cudaError_t launch_msa_i8x2(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                            size_t smem, cudaStream_t stream);

// Threads per block of the packed kernel at most (its register budget, up to 128 per thread, assumes no
// more).  A tighter register cap (63 for 7 blocks per SM) made the compiler recompute values: 19 %
// more instructions and a slower kernel, although twice as many warps were resident.
constexpr int kPackedMaxThreads = 512;

// Shared memory of one block of the packed kernel (two shots): gamma [nv] (4 B), Q [nv] (two lanes,
// 8 B), parity words [m], paired message slots [dc_max*m + scratch] of word_bytes (4: two 16-bit
// fixed-point lanes; 8: two FP32 lanes).
struct PackedLayout {
    size_t g_off, q_off, par_off, slot_off, total;
};

__host__ __device__ inline PackedLayout packed_layout(int m, int nv, int dc_max, int word_bytes)
{
    PackedLayout l;
    l.g_off = 0;
    l.q_off = align16(size_t(nv) * 4);
    l.par_off = align16(l.q_off + size_t(nv) * 8);
    l.slot_off = align16(l.par_off + size_t(m) * 4);
    l.total = align16(l.slot_off + (size_t(dc_max) * m + kScratch) * size_t(word_bytes));
    return l;
}

// Layered-schedule kernels, msa_layered.cu.
const void *msa_kernel_layered(int precision, const KernelChoice &kc);
cudaError_t launch_msa_layered(int precision, const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                               size_t smem, cudaStream_t stream);

// Shared memory of one shot in the layered kernel: Q [n] (4 B), r slots [dc_max*m], syndrome bits [m].
struct LayeredLayout {
    size_t q_off, slot_off, s_off, total;
};

__host__ __device__ inline LayeredLayout layered_layout(int m, int n, int dc_max, int msg_bytes)
{
    LayeredLayout l;
    l.q_off = 0;
    l.slot_off = align16(size_t(n) * 4);
    l.s_off = align16(l.slot_off + size_t(dc_max) * m * msg_bytes);
    l.total = align16(l.s_off + size_t(m));
    return l;
}

// Learned (FP32) decoder kernels, msa_learned.cu.
const void *msa_kernel_learned(const KernelChoice &kc);
cudaError_t launch_msa_learned(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                               size_t smem, cudaStream_t stream);

// ---------------------------------------------------------------------------------------------
// Training of the learned decoder and its helpers (nms_train.cu).
// ---------------------------------------------------------------------------------------------
// Recorded check-node state of one iteration: 4 words per check, word f of check i at f*m + i:
//   0: min1 (FP32 bits)  1: min2 (FP32 bits)  2: sign bits, bit j = [q_j < 0]
//   3: idx1 | idx2 << 8 | negall << 16   (negall = s_i XOR parity of all sign bits)
constexpr int kStateWords = 4;
constexpr int kTrainThreads = 128;   // threads per training block (one shot per block)

struct TrainParams {
    DeviceGraph g;
    const uint8_t *syn;         // [batch * m]
    const uint8_t *target;      // [batch * n] true error bits, caller's variable order
    const float *prior;         // [n]
    const float *w;             // [T][dc_max * m] slot-layout weights
    uint32_t *state;            // [batch][T][kStateWords * m]
    float *loss;                // [batch]
    float *post;                // [batch * n] a-posteriori LLR of iteration T, or nullptr
    const float *grad_loss;     // [batch]
    const float *loss_w;        // [T] per-iteration loss weights lambda_t, or nullptr for 1/T each
    float *partial;             // [T][dc_max * m] slot-layout weight gradient, zeroed before the backward
    int32_t T, batch;
    int32_t loss_kind;          // kLossError or kLossSyndrome
};

constexpr int kLossError = 0;      // BCE of sigma(-Q) against the sampled error, mean over variables
constexpr int kLossSyndrome = 1;   // BCE of the soft syndrome against s, mean over checks

struct TrainChoice {
    int dc;          // exact uniform row degree 6..8, else bucket 8/16/32
    bool uniform;
    int dvb;         // column-degree bucket 4/8/16
};

const void *nms_forward_kernel_ptr(const TrainChoice &tc, int loss_kind);
const void *nms_backward_kernel_ptr(const TrainChoice &tc, int loss_kind);
cudaError_t launch_nms_forward(const TrainParams &p, const TrainChoice &tc, int grid, int threads, size_t smem,
                               cudaStream_t stream);
cudaError_t launch_nms_backward(const TrainParams &p, const TrainChoice &tc, int grid, int threads, size_t smem,
                                cudaStream_t stream);
cudaError_t launch_permute_weights(const float *w_csr, const uint32_t *eslot, int32_t T, int32_t nnz, int32_t S,
                                   float *w_slot, cudaStream_t stream);
cudaError_t launch_gather_grad(const float *grad_slot, const uint32_t *eslot, int32_t T, int32_t S, int32_t nnz,
                               float *grad, cudaStream_t stream);
cudaError_t launch_adam(float *param, const float *grad, float *m1, float *m2, int64_t count, int32_t step,
                        float lr, float beta1, float beta2, float eps, cudaStream_t stream);
cudaError_t launch_sample(const DeviceGraph &g, uint64_t seed, int64_t first_shot, int32_t batch, double p_lo,
                          double p_hi, uint8_t *err, uint8_t *syn, int grid, cudaStream_t stream);
cudaError_t launch_logical(const uint8_t *logicals, int32_t k, int32_t n, const uint8_t *err, const uint8_t *dec,
                           const uint8_t *ok, int32_t batch, uint8_t *fail, int grid, cudaStream_t stream);

// Shared memory of one training shot (forward: q slots, gamma, targets, syndrome; backward adds
// the recomputed r slots and the recorded state of two iterations).  The syndrome loss adds the
// per-edge codes to the forward and Q per lane to the backward, whose codes overwrite r in place.
struct TrainLayout {
    size_t slot_off, r_off, c_off, t_off, g_off, y_off, s_off, total;
};

__host__ __device__ inline TrainLayout train_layout(int m, int n, int dc_max, bool backward, bool syndrome = false)
{
    TrainLayout t;
    const size_t S = size_t(dc_max) * m + kScratch;
    t.slot_off = 0;                                                          // q / gradient slots [S] f32
    t.r_off = align16(S * 4);                                                // r slots [S] f32 (backward)
    t.c_off = backward ? align16(t.r_off + S * 4) : t.r_off;                 // state [2][4m] u32 (backward)
    t.t_off = backward ? align16(t.c_off + 2 * size_t(kStateWords) * m * 4) : t.c_off;   // syndrome loss:
    const size_t g0 = syndrome ? align16(t.t_off + (backward ? size_t(n) : S) * 4) : t.t_off; // codes [S] / Q [n]
    t.g_off = g0;                                                                        // gamma [n] f32
    t.y_off = align16(t.g_off + size_t(n) * 4);                              // targets [n] u8
    t.s_off = align16(t.y_off + size_t(n));                                  // syndrome bits [m] u8
    t.total = align16(t.s_off + size_t(m));
    return t;
}

}  // namespace qldpc
