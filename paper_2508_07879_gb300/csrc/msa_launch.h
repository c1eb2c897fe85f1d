// Internal interface between the C-ABI host code (qldpc_host.cpp) and the sm_103a kernels
// (msa_f32.cu, msa_i16.cu).  Not installed; the public ABI is include/qldpc.h.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace qldpc {

// Tanner graph in the kernels' layout.  Messages of check i live in shared-memory "slots"
// j*m + i (j = position of the edge in row i), so a warp working on 32 consecutive checks touches
// 32 consecutive slots.  Variable v finds its edges through vslot[k*n + v] (k-th edge of v in
// ascending check order); the check side needs no index at all.
struct DeviceGraph {
    const uint32_t *vslot;   // [dv_max * n] slot of variable v's k-th edge
    const uint8_t *vdeg;     // [n] column degrees
    const uint8_t *rdeg;     // [m] row degrees
    int32_t m, n;
    int32_t dc_max, dv_max;  // largest row / column degree
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
};

struct LaunchParams {
    Problem prob[2];         // prob[blockIdx.y]; two for the X+Z pair decode
    int32_t nprob;
    int32_t batch;
    int32_t max_iter;
    float alpha;             // FP32 scale
    int32_t alpha_q;         // INT16 scale, round(alpha * 2^15)
    uint32_t flags;
};

constexpr uint32_t kFlagNoEarlyStop = 1u;

// Shared-memory layout of one shot (identical on host and device).
struct SmemLayout {
    size_t q_off, g_off, msg_off, dec_off, syn_off, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SmemLayout smem_layout(int m, int n, int dc_max, int msg_bytes)
{
    SmemLayout s;
    s.q_off = 0;                                                     // a-posteriori Q_n  [n] (4 B)
    s.g_off = align16(s.q_off + size_t(n) * 4);                      // prior gamma_n     [n] (4 B)
    s.msg_off = align16(s.g_off + size_t(n) * 4);                    // edge messages     [dc_max*m]
    s.dec_off = align16(s.msg_off + size_t(dc_max) * m * msg_bytes); // decision per slot [dc_max*m]
    s.syn_off = align16(s.dec_off + size_t(dc_max) * m);             // syndrome          [m]
    s.total = align16(s.syn_off + size_t(m));
    return s;
}

enum Precision { kFP32 = 0, kINT16 = 1 };

inline int msg_bytes(int precision) { return precision == kINT16 ? 2 : 4; }

// Kernel variant buckets: compile-time maxima the degrees are rounded up to.
int dc_bucket(int dc_max);   // 8, 16, 32 or -1
int dv_bucket(int dv_max);   // 4, 8, 16 or -1

// Kernel entry for (precision, dc bucket, dv bucket), for attributes and occupancy queries.
const void *msa_kernel(int precision, int dcb, int dvb);

// Launch the flooding decoder: grid (grid_x, nprob), `threads` per block, `smem` dynamic bytes.
cudaError_t launch_msa(const LaunchParams &p, int precision, int dcb, int dvb, int threads,
                       int grid_x, size_t smem, cudaStream_t stream);

// Per-precision instantiation tables (one translation unit each).
const void *msa_kernel_f32(int dcb, int dvb);
const void *msa_kernel_i16(int dcb, int dvb);
cudaError_t launch_msa_f32(const LaunchParams &p, int dcb, int dvb, dim3 grid, int threads,
                           size_t smem, cudaStream_t stream);
cudaError_t launch_msa_i16(const LaunchParams &p, int dcb, int dvb, dim3 grid, int threads,
                           size_t smem, cudaStream_t stream);

}  // namespace qldpc
