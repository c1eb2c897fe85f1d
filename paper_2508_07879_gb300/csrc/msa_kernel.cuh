// Flooding normalized min-sum decoder driven by a syndrome -- Algorithm 1 ("MSA for
// syndrome-based LDPC decoding"), Sec. 2 of arXiv 2508.07879 -- for sm_103a.
//
// Mapping (a GB300 design, not the paper's per-iteration launches over global memory):
//   * one thread block per shot, persistent over shots (block b takes shots b, b + gridDim.x, ...);
//     gridDim.y selects the X or Z problem of a pair decode (the paper's concatenated X+Z kernel);
//   * all edge messages of the shot live in shared memory, in place: the check step overwrites
//     q_{m,n} with r_{m,n}, the variable step overwrites r with the next q.  Slots are check-major
//     (slot j*M + m), so the check step reads and writes 32 consecutive words per warp;
//   * the variable step also stores its decision e_n into every slot of its edges, so the stop
//     test H e^T = s is folded into the next check step (each check XORs the decisions of its
//     slots) and decided by one __syncthreads_and.  An iteration costs two block barriers instead of
//     the paper's four (Fig. 2 caption);
//   * the graph is read through the read-only path (L1-resident: one copy per SM for all blocks).
//
// Arithmetic is operation-for-operation that of the CPU oracle:
//   r = sign * (alpha * min_{j != n} |q_j|)        min_{j != n} taken as min1 or min2 of the row
//   q_{m,n} = gamma_n + sum_{i != m} r_{i,n}        ascending check order, prefix/suffix reuse
//   Q_n = gamma_n + sum_i r_{i,n}                   ascending check order
// so FP32 results are bit-identical (every add/multiply is an explicit round-to-nearest intrinsic,
// nothing is fused or reassociated) and INT16 results are exact integer arithmetic.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "msa_launch.h"

namespace qldpc {
namespace kern {

// ---------------------------------------------------------------------------------------------
// Precision policies
// ---------------------------------------------------------------------------------------------
struct F32 {
    using msg_t = float;    // a message stored in a slot
    using acc_t = float;    // variable-node sums, Q_n
    using mag_t = float;    // |q| and scaled minima
    static __device__ __forceinline__ acc_t quantize(float g) { return g; }
    static __device__ __forceinline__ acc_t add(acc_t a, msg_t b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ msg_t to_msg(acc_t a) { return a; }
    static __device__ __forceinline__ bool neg(float x) { return x < 0.0f; }
    static __device__ __forceinline__ mag_t mag(msg_t x) { return fabsf(x); }
    static __device__ __forceinline__ mag_t mag_init() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ mag_t mag_min(mag_t a, mag_t b) { return fminf(a, b); }
    static __device__ __forceinline__ mag_t scale(mag_t m, const LaunchParams &p)
    {
        return __fmul_rn(p.alpha, m);
    }
    static __device__ __forceinline__ msg_t with_sign(mag_t m, uint32_t negative)
    {
        return negative ? -m : m;
    }
    static __device__ __forceinline__ float post(acc_t a) { return a; }
};

struct I16 {
    using msg_t = int16_t;
    using acc_t = int32_t;
    using mag_t = int32_t;
    // gamma_q = clamp(round_half_away(gamma * 2^8), -32767, 32767); gamma*256 is exact in binary32
    static __device__ __forceinline__ acc_t quantize(float g)
    {
        float t = roundf(g * 256.0f);
        t = fminf(fmaxf(t, -32767.0f), 32767.0f);
        return static_cast<int32_t>(t);
    }
    static __device__ __forceinline__ acc_t add(acc_t a, msg_t b) { return a + int32_t(b); }
    static __device__ __forceinline__ msg_t to_msg(acc_t a)
    {
        return static_cast<int16_t>(max(-32767, min(32767, a)));
    }
    static __device__ __forceinline__ bool neg(int32_t x) { return x < 0; }
    static __device__ __forceinline__ mag_t mag(msg_t x) { return abs(int32_t(x)); }
    static __device__ __forceinline__ mag_t mag_init() { return 0x7fffffff; }
    static __device__ __forceinline__ mag_t mag_min(mag_t a, mag_t b) { return min(a, b); }
    // |r| = floor(min * alpha_q / 2^15); min <= 32767 and alpha_q <= 2^15 keep it in 31 bits
    static __device__ __forceinline__ mag_t scale(mag_t m, const LaunchParams &p)
    {
        return (m * p.alpha_q) >> 15;
    }
    static __device__ __forceinline__ msg_t with_sign(mag_t m, uint32_t negative)
    {
        return static_cast<int16_t>(negative ? -m : m);
    }
    static __device__ __forceinline__ float post(acc_t a) { return float(a) * 0.00390625f; }
};

// ---------------------------------------------------------------------------------------------
// Check-node step (Alg. 1, CN processing) fused with the stop test of the previous decisions.
// Returns 1 iff the decisions stored in this check's slots satisfy s_m.
// ---------------------------------------------------------------------------------------------
template <class P, int DC>
__device__ __forceinline__ int check_step(int c, int M, int deg, uint32_t s, bool update,
                                          typename P::msg_t *__restrict__ msg,
                                          const uint8_t *__restrict__ dec,
                                          const LaunchParams &p)
{
    using msg_t = typename P::msg_t;
    using mag_t = typename P::mag_t;
    msg_t q[DC];
    uint32_t par = s;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (j < deg) {
            q[j] = msg[j * M + c];
            par ^= dec[j * M + c];
        }
    }
    if (update) {
        uint32_t mask = 0, negall = s;
        mag_t m1 = P::mag_init(), m2 = P::mag_init();
        int idx = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (j < deg) {
                const uint32_t sg = P::neg(q[j]) ? 1u : 0u;
                mask |= sg << j;
                negall ^= sg;
                const mag_t a = P::mag(q[j]);
                if (a < m1) {           // strict: a tie keeps the lower slot as the argmin
                    m2 = m1;
                    m1 = a;
                    idx = j;
                } else {
                    m2 = P::mag_min(m2, a);
                }
            }
        }
        const mag_t r1 = P::scale(m1, p);   // alpha * min over the other slots, j != idx
        const mag_t r2 = P::scale(m2, p);   // alpha * min over the other slots, j == idx
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (j < deg) msg[j * M + c] = P::with_sign(j == idx ? r2 : r1, (negall ^ (mask >> j)) & 1u);
        }
    }
    return (par & 1u) == 0;
}

// ---------------------------------------------------------------------------------------------
// Variable-node step (Alg. 1, VN processing + a-posteriori LLR + tentative decision) for a
// variable of degree exactly D.  q_k = gamma + sum_{i != k} r_i in ascending order:
// q_k = ((pre_k + r_{k+1}) + r_{k+2}) + ...  with pre_k = ((gamma + r_0) + r_1) + ... + r_{k-1}.
// ---------------------------------------------------------------------------------------------
template <class P, int D>
__device__ __forceinline__ void var_step_exact(int v, int N, const uint32_t *__restrict__ vslot,
                                               typename P::acc_t gamma,
                                               typename P::msg_t *__restrict__ msg,
                                               uint8_t *__restrict__ dec,
                                               typename P::acc_t *__restrict__ Qs)
{
    using acc_t = typename P::acc_t;
    using msg_t = typename P::msg_t;
    if constexpr (D == 0) {
        Qs[v] = gamma;
    } else {
        uint32_t sl[D];
        msg_t r[D];
#pragma unroll
        for (int k = 0; k < D; ++k) sl[k] = __ldg(vslot + size_t(k) * N + v);
#pragma unroll
        for (int k = 0; k < D; ++k) r[k] = msg[sl[k]];
        acc_t pre[D + 1];
        pre[0] = gamma;
#pragma unroll
        for (int k = 0; k < D; ++k) pre[k + 1] = P::add(pre[k], r[k]);
        const acc_t Q = pre[D];
        const uint8_t d = P::neg(Q) ? 1 : 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            acc_t q = pre[k];
#pragma unroll
            for (int i = k + 1; i < D; ++i) q = P::add(q, r[i]);
            msg[sl[k]] = P::to_msg(q);
            dec[sl[k]] = d;
        }
        Qs[v] = Q;
    }
}

template <class P, int D, int DV>
__device__ __forceinline__ void var_step_dispatch(int deg, int v, int N, const uint32_t *vslot,
                                                  typename P::acc_t gamma, typename P::msg_t *msg,
                                                  uint8_t *dec, typename P::acc_t *Qs)
{
    if constexpr (D <= DV) {
        if (deg == D) {
            var_step_exact<P, D>(v, N, vslot, gamma, msg, dec, Qs);
        } else {
            var_step_dispatch<P, D + 1, DV>(deg, v, N, vslot, gamma, msg, dec, Qs);
        }
    }
}

// Initialization (Alg. 1): q^(0)_{m,n} = gamma_n on every edge, decisions from the prior.
template <class P>
__device__ __forceinline__ void var_init(int v, int N, int deg, const uint32_t *__restrict__ vslot,
                                         typename P::acc_t gamma, typename P::msg_t *msg,
                                         uint8_t *dec, typename P::acc_t *Qs)
{
    const typename P::msg_t g = P::to_msg(gamma);
    const uint8_t d = P::neg(gamma) ? 1 : 0;
    for (int k = 0; k < deg; ++k) {
        const uint32_t s = __ldg(vslot + size_t(k) * N + v);
        msg[s] = g;
        dec[s] = d;
    }
    Qs[v] = gamma;
}

// ---------------------------------------------------------------------------------------------
// The decoder kernel.
// ---------------------------------------------------------------------------------------------
template <class P, int DC, int DV>
__global__ void __launch_bounds__(1024) msa_flood_kernel(const LaunchParams p)
{
    using msg_t = typename P::msg_t;
    using acc_t = typename P::acc_t;

    const Problem pr = blockIdx.y == 0 ? p.prob[0] : p.prob[1];
    const int M = pr.g.m, N = pr.g.n;
    const int T = blockDim.x, tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(M, N, pr.g.dc_max, int(sizeof(msg_t)));
    acc_t *Qs = reinterpret_cast<acc_t *>(smem + L.q_off);
    acc_t *gam = reinterpret_cast<acc_t *>(smem + L.g_off);
    msg_t *msg = reinterpret_cast<msg_t *>(smem + L.msg_off);
    uint8_t *dec = smem + L.dec_off;
    uint8_t *syn = smem + L.syn_off;

    // Prior LLRs: loaded once per block, shared by all its shots.
    int bad = 0;
    for (int v = tid; v < N; v += T) {
        const float g = pr.prior[v];
        bad |= !isfinite(g);
        gam[v] = P::quantize(g);
    }
    bad = __syncthreads_or(bad);

    const bool early = (p.flags & kFlagNoEarlyStop) == 0;
    for (int b = blockIdx.x; b < p.batch; b += gridDim.x) {
        uint8_t *err = pr.err + size_t(b) * N;
        if (bad) {   // non-finite prior: report the shot as not decoded
            for (int v = tid; v < N; v += T) {
                err[v] = 0;
                if (pr.post) pr.post[size_t(b) * N + v] = __int_as_float(0x7fc00000);
            }
            if (tid == 0) {
                pr.iters[b] = -1;
                pr.ok[b] = 0;
            }
            continue;
        }
        const uint8_t *s = pr.syn + size_t(b) * M;
        for (int c = tid; c < M; c += T) syn[c] = s[c] & 1;
        for (int v = tid; v < N; v += T) var_init<P>(v, N, pr.g.vdeg[v], pr.g.vslot, gam[v], msg, dec, Qs);
        __syncthreads();

        int k = 0, all = 0;
        for (;; ++k) {
            const bool last = k >= p.max_iter;
            int ok = 1;
            for (int c = tid; c < M; c += T)
                ok &= check_step<P, DC>(c, M, __ldg(pr.g.rdeg + c), syn[c], !last, msg, dec, p);
            all = __syncthreads_and(ok);
            if (last || (early && all)) break;
            for (int v = tid; v < N; v += T)
                var_step_dispatch<P, 0, DV>(__ldg(pr.g.vdeg + v), v, N, pr.g.vslot, gam[v], msg, dec, Qs);
            __syncthreads();
        }

        for (int v = tid; v < N; v += T) {
            const acc_t q = Qs[v];
            err[v] = P::neg(q) ? 1 : 0;
            if (pr.post) pr.post[size_t(b) * N + v] = P::post(q);
        }
        if (tid == 0) {
            pr.iters[b] = k;
            pr.ok[b] = all ? 1 : 0;
        }
        __syncthreads();   // the next shot reuses shared memory
    }
}

}  // namespace kern

// Instantiation table for one precision policy.
template <class P>
const void *kernel_table(int dcb, int dvb)
{
#define QLDPC_K(DCV, DVV)                                                                       \
    if (dcb == DCV && dvb == DVV)                                                               \
        return reinterpret_cast<const void *>(&kern::msa_flood_kernel<P, DCV, DVV>);
    QLDPC_K(8, 4) QLDPC_K(8, 8) QLDPC_K(8, 16)
    QLDPC_K(16, 4) QLDPC_K(16, 8) QLDPC_K(16, 16)
    QLDPC_K(32, 4) QLDPC_K(32, 8) QLDPC_K(32, 16)
#undef QLDPC_K
    return nullptr;
}

template <class P>
cudaError_t launch_table(const LaunchParams &p, int dcb, int dvb, dim3 grid, int threads,
                         size_t smem, cudaStream_t stream)
{
#define QLDPC_L(DCV, DVV)                                                                       \
    if (dcb == DCV && dvb == DVV) {                                                             \
        kern::msa_flood_kernel<P, DCV, DVV><<<grid, threads, smem, stream>>>(p);                \
        return cudaGetLastError();                                                              \
    }
    QLDPC_L(8, 4) QLDPC_L(8, 8) QLDPC_L(8, 16)
    QLDPC_L(16, 4) QLDPC_L(16, 8) QLDPC_L(16, 16)
    QLDPC_L(32, 4) QLDPC_L(32, 8) QLDPC_L(32, 16)
#undef QLDPC_L
    return cudaErrorInvalidValue;
}

}  // namespace qldpc
