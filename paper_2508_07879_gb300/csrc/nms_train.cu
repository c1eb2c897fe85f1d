// Training of the neural normalized min-sum decoder on sm_103a: Algorithm 1 (Sec. 2 of
// arXiv 2508.07879) with the scale alpha replaced by a learned weight w[t][e] per iteration and
// edge, unrolled over T iterations, trained on the BCE of the soft outputs sigma(-Q).
//
//   nms_forward_kernel   one block per shot, persistent over the batch.  T iterations of the learned
//                        check step and the exact variable step of the decoder kernels (so FP32
//                        messages are bit-identical to the learned decoder's), the per-shot loss
//                        sum_t lambda_t / N sum_n BCE(sigma(-Q^t_n), y_n) (lambda_t = 1/T unless
//                        given), and, per iteration and check, the
//                        compressed check state: min1, min2, the positions attaining them (lowest on
//                        ties), the sign bits of the inputs and the syndrome-flipped total sign.
//   nms_backward_kernel  the reverse sweep.  It stores no message: every r^(t) is recomputed from
//                        the recorded state (r_{m,n} = sign * (w * (n == idx1 ? min2 : min1))),
//                        Q^(t) from those r, and the gradient flows
//                          dL/dr_{m,n}   = dL/dQ_n + sum_{i != m} dL/dq_{i,n}      (variable step)
//                          dL/dw_{m,n}   = dL/dr_{m,n} * sign * min_{j != n}|q_j|
//                          dL/dq_{m,idx1} = sum_{n != idx1} dL/dr_{m,n} w sign * sign(q_idx1)
//                          dL/dq_{m,idx2} = dL/dr_{m,idx1} w sign * sign(q_idx2)     (all other q: 0)
//                        Two block barriers per iteration; the next iteration's recorded state
//                        streams into shared memory (cp.async) while the variable side runs.  Weight
//                        gradients are added into one L2-resident [T][slots] buffer with global
//                        reductions, so the order of the sum over shots follows the schedule: the
//                        gradient is deterministic only up to the order of its FP32 additions
//                        (last-bit differences between calls).
//   helpers              CSR <-> slot-layout weight permutation, an Adam step, a counter-based
//                        SplitMix64 error sampler with syndromes, and the logical-failure test.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "msa_kernel.cuh"
#include "msa_launch.h"

namespace qldpc {
namespace kern {

__device__ __forceinline__ float softplus(float x) { return fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x))); }
__device__ __forceinline__ float sigmoid(float x) { return 1.0f / (1.0f + expf(-x)); }

// Sum over the block (deterministic order); every thread gets the total.
__device__ __forceinline__ float block_sum(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.0f;
    for (int i = 0; i < nw; ++i) t += red[i];
    return t;
}

// Learned check step of the training forward for check c: r = sign * (w * min over the others),
// written in place of q, and the compressed state of this iteration.
template <int DC, bool UNIFORM>
__device__ __forceinline__ void train_check_fwd(int c, int M, int deg, uint32_t s_bit, float *__restrict__ slots,
                                                const float *__restrict__ w, uint32_t *__restrict__ st)
{
    float q[DC];
    uint32_t signs = 0;
    float m1 = __int_as_float(0x7f800000), m2 = m1;
    int i1 = 0, i2 = 0;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            q[j] = slots[j * M + c];
            signs |= (__float_as_uint(q[j]) >> 31) << j;
            const float a = fabsf(q[j]);
            if (a < m1) {
                m2 = m1;
                i2 = i1;
                m1 = a;
                i1 = j;
            } else if (a < m2) {
                m2 = a;
                i2 = j;
            }
        }
    }
    const uint32_t negall = (s_bit ^ uint32_t(__popc(signs))) & 1u;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            const float r = __fmul_rn(__ldg(w + j * M + c), j == i1 ? m2 : m1);
            slots[j * M + c] = F32::signed_like(r, q[j], negall);
        }
    }
    st[c] = __float_as_uint(m1);
    st[M + c] = __float_as_uint(m2);
    st[2 * M + c] = signs;
    st[3 * M + c] = uint32_t(i1) | (uint32_t(i2) << 8) | (negall << 16);
}

// Per-lane inputs: the prior and the target of the variable in lane u; idle lanes get prior 0
// and the marker kIdleLane (they have no edges and add nothing to the loss).
constexpr uint8_t kIdleLane = 2;
__device__ __forceinline__ float lane_prior(const DeviceGraph &g, const float *prior, int u, int N)
{
    const uint32_t v = __ldg(g.vperm + u);
    return v < uint32_t(N) ? prior[v] : 0.0f;
}
__device__ __forceinline__ uint8_t lane_target(const DeviceGraph &g, const uint8_t *tg, int u, int N)
{
    const uint32_t v = __ldg(g.vperm + u);
    return v < uint32_t(N) ? (tg ? uint8_t(tg[v] & 1u) : uint8_t(0)) : kIdleLane;
}

// Syndrome loss.  With t_v = tanh(Q_v / 2), P_c = (1 + (-1)^s prod_{v in c} t_v) / 2 is the
// probability that row c's parity under independent bits sigma(-Q) equals s.  Each variable
// stores, on its edge slots, its log-magnitude code
//   lm_v = sign(Q_v) * (-log |t_v|),  -log |t_v| = log1p(e^-|Q_v|) - log1p(-e^-|Q_v|)  (+inf at Q = 0),
// computed once per variable.  A check then has prod |t| = exp(A), A = -sum |lm|, and a violated,
// confident check gets P = -expm1(A) / 2 without the cancellation of 1 - prod (|t| rounds to 1
// long before 1 - |t| is negligible).
constexpr float kSynLossFloor = 1e-7f;

// The sign travels in the sign bit (also on a magnitude of 0, where |Q| is so large that |t| = 1).
__device__ __forceinline__ float log_magnitude_code(float Q)
{
    const float x = expf(-fabsf(Q));
    const float mag = log1pf(x) - log1pf(-x);   // -log |tanh(Q/2)| >= 0
    return __uint_as_float(__float_as_uint(mag) | (Q < 0.0f ? 0x80000000u : 0u));
}

// P_c from the codes in check c's slots; optionally t_j = sign * exp(-|lm_j|) for the caller.
template <int DC, bool UNIFORM, bool WANT_T>
__device__ __forceinline__ float parity_match_prob(int c, int M, int deg, uint32_t s_bit, const float *__restrict__ ls,
                                                   float *t)
{
    float A = 0.0f;
    uint32_t neg = s_bit & 1u;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            const float lm = ls[j * M + c];
            const bool nj = (__float_as_uint(lm) >> 31) != 0u;
            A -= fabsf(lm);
            neg ^= nj ? 1u : 0u;
            if (WANT_T) {
                const float at = expf(-fabsf(lm));
                t[j] = nj ? -at : at;
            }
        } else if (WANT_T) {
            t[j] = 1.0f;
        }
    }
    return neg ? -0.5f * expm1f(A) : 0.5f * (1.0f + expf(A));
}

template <int DC, bool UNIFORM>
__device__ __forceinline__ float syndrome_term(int c, int M, int deg, uint32_t s_bit, const float *__restrict__ ls)
{
    const float P = parity_match_prob<DC, UNIFORM, false>(c, M, deg, s_bit, ls, nullptr);
    return -logf(fmaxf(P, kSynLossFloor));
}

// d(syndrome term)/d t_j = -(1 / P) (-1)^s / 2 prod_{i != j} t_i (0 at the floor), written over the
// codes of check c.
template <int DC, bool UNIFORM>
__device__ __forceinline__ void syndrome_term_grad(int c, int M, int deg, uint32_t s_bit, float *__restrict__ ls)
{
    float t[DC], pre[DC];
    const float P = parity_match_prob<DC, UNIFORM, true>(c, M, deg, s_bit, ls, t);
    const float sg = s_bit ? -1.0f : 1.0f;
    const float coef = P > kSynLossFloor ? -0.5f * sg / P : 0.0f;
    float prod = 1.0f;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        pre[j] = prod;                       // t_0 ... t_{j-1}
        prod *= t[j];
    }
    float suf = 1.0f;                        // t_{j+1} ... t_{deg-1}
#pragma unroll
    for (int j = DC - 1; j >= 0; --j) {
        if (UNIFORM || j < deg) {
            ls[j * M + c] = coef * (pre[j] * suf);
            suf *= t[j];
        }
    }
}

// d tanh(Q/2) / dQ = sech^2(Q/2) / 2 (no cancellation for large |Q|)
__device__ __forceinline__ float half_sech2_half(float Q)
{
    const float ch = coshf(0.5f * Q);
    return 0.5f / (ch * ch);
}

// The weights of check c's edges in one iteration, all loads issued before any is used.
template <int DC, bool UNIFORM>
__device__ __forceinline__ void load_check_weights(int c, int M, int deg, const float *__restrict__ w, float (&wv)[DC])
{
#pragma unroll
    for (int j = 0; j < DC; ++j) wv[j] = (UNIFORM || j < deg) ? __ldg(w + j * M + c) : 0.0f;
}

// r of check c recomputed from its recorded state and its edges' weights (bit-identical to the
// forward's r).
template <int DC, bool UNIFORM>
__device__ __forceinline__ void recompute_r(int c, int M, int deg, uint32_t m1b, uint32_t m2b, uint32_t signs,
                                            uint32_t iw, const float (&wv)[DC], float *__restrict__ rs)
{
    const int i1 = int(iw & 0xffu);
    const uint32_t negall = (iw >> 16) & 1u;
    const float m1 = __uint_as_float(m1b), m2 = __uint_as_float(m2b);
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            const float r = __fmul_rn(wv[j], j == i1 ? m2 : m1);
            rs[j * M + c] = __uint_as_float(__float_as_uint(r) ^ ((((signs >> j) & 1u) ^ negall) << 31));
        }
    }
}

// SYN: the syndrome loss (compiled separately, so the error-loss kernels carry none of its code).
template <int DC, bool UNIFORM, int DV, bool SYN>
__global__ void __launch_bounds__(kTrainThreads, 4) nms_forward_kernel(const TrainParams p)
{
    const int M = p.g.m, N = p.g.n, NV = p.g.nv, T = blockDim.x, tid = threadIdx.x;
    const size_t S = size_t(p.g.dc_max) * M;
    constexpr bool syn_loss = SYN;
    extern __shared__ __align__(16) unsigned char smem[];
    const TrainLayout L = train_layout(M, NV, p.g.dc_max, false, syn_loss);
    float *slots = reinterpret_cast<float *>(smem + L.slot_off);
    float *ts = reinterpret_cast<float *>(smem + L.t_off);        // syndrome loss: each edge's variable's code
    float *gam = reinterpret_cast<float *>(smem + L.g_off);
    uint8_t *y = smem + L.y_off;
    uint8_t *sb = smem + L.s_off;
    __shared__ float red[32];

    for (int u = tid; u < NV; u += T) gam[u] = F32::quantize(lane_prior(p.g, p.prior, u, N));
    // uniform lambda: sum the terms and scale once by 1/(T K); else weight each iteration's terms
    // (K = N variables for the error loss, M checks for the syndrome loss)
    const float K = float(syn_loss ? M : N);
    const float inv = p.loss_w ? 1.0f / K : 1.0f / (float(p.T) * K);
    for (int b = blockIdx.x; b < p.batch; b += gridDim.x) {
        const uint8_t *s = p.syn + size_t(b) * M;
        const uint8_t *tg = syn_loss ? nullptr : p.target + size_t(b) * N;
        for (int c = tid; c < M; c += T) sb[c] = s[c] & 1u;
        __syncthreads();   // gam (first shot) and the previous shot's last reads are done
        for (int u = tid; u < NV; u += T) {
            y[u] = lane_target(p.g, tg, u, N);
            const int deg = __ldg(p.g.vdeg + u);
            for (int k = 0; k < deg; ++k) slots[__ldg(p.g.vslot + size_t(k) * NV + u)] = gam[u];
        }
        __syncthreads();
        float acc = 0.0f;
        for (int k = 0; k < p.T; ++k) {
            const float *wk = p.w + size_t(k) * S;
            uint32_t *st = p.state + (size_t(b) * p.T + k) * size_t(kStateWords) * M;
            // syndrome loss of iteration k-1 (its code slots are complete) beside the check step of k
            const float lw_prev = (syn_loss && k > 0) ? (p.loss_w ? __ldg(p.loss_w + k - 1) : 1.0f) : 0.0f;
            for (int c = tid; c < M; c += T) {
                const int deg = UNIFORM ? DC : int(__ldg(p.g.rdeg + c));
                if (syn_loss && k > 0) acc += lw_prev * syndrome_term<DC, UNIFORM>(c, M, deg, sb[c], ts);
                train_check_fwd<DC, UNIFORM>(c, M, deg, sb[c], slots, wk, st);
            }
            __syncthreads();
            const bool lastk = k + 1 == p.T;
            const float lw = p.loss_w ? __ldg(p.loss_w + k) : 1.0f;
            for (int u = tid; u < NV; u += T) {
                const int deg = __ldg(p.g.vdeg + u);
                const float Q = var_step_batch<F32, DV, false>(deg, u, NV, CheckOf(p.g), p.g.vslot, gam[u], false,
                                                               slots, nullptr);
                if (y[u] == kIdleLane) continue;
                if (syn_loss) {
                    const float lm = log_magnitude_code(Q);
                    for (int i = 0; i < deg; ++i) ts[__ldg(p.g.vslot + size_t(i) * NV + u)] = lm;
                } else {
                    acc += lw * (y[u] ? softplus(Q) : softplus(-Q));
                }
                if (lastk && p.post) p.post[size_t(b) * N + __ldg(p.g.vperm + u)] = Q;
            }
            __syncthreads();
        }
        if (syn_loss) {   // the last iteration's syndrome loss
            const float lw = p.loss_w ? __ldg(p.loss_w + p.T - 1) : 1.0f;
            for (int c = tid; c < M; c += T) {
                const int deg = UNIFORM ? DC : int(__ldg(p.g.rdeg + c));
                acc += lw * syndrome_term<DC, UNIFORM>(c, M, deg, sb[c], ts);
            }
        }
        const float total = block_sum(acc, red);
        if (tid == 0) p.loss[b] = total * inv;
    }
}

// Start an asynchronous copy of one iteration's recorded state (kStateWords * M words, a
// contiguous, 16-byte aligned slice) into shared memory; cp_async_wait() completes it.
__device__ __forceinline__ void prefetch_state(uint32_t *dst, const uint32_t *src, int M)
{
    const uint32_t base = uint32_t(__cvta_generic_to_shared(dst));
    for (int i = threadIdx.x; i < M; i += blockDim.x)   // kStateWords * M * 4 bytes = M chunks of 16
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + 16u * uint32_t(i)),
                     "l"(src + 4 * size_t(i))
                     : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int DC, bool UNIFORM, int DV, bool SYN>
__global__ void __launch_bounds__(kTrainThreads, 4) nms_backward_kernel(const TrainParams p)
{
    const int M = p.g.m, N = p.g.n, NV = p.g.nv, T = blockDim.x, tid = threadIdx.x;
    const size_t S = size_t(p.g.dc_max) * M;
    const size_t SW = size_t(kStateWords) * M;                    // state words of one iteration
    constexpr bool syn_loss = SYN;
    extern __shared__ __align__(16) unsigned char smem[];
    const TrainLayout L = train_layout(M, NV, p.g.dc_max, true, syn_loss);
    float *gs = reinterpret_cast<float *>(smem + L.slot_off);     // dL/dq (next iteration), then dL/dr
    float *rs = reinterpret_cast<float *>(smem + L.r_off);        // recomputed r of the current iteration
    uint32_t *scb = reinterpret_cast<uint32_t *>(smem + L.c_off); // recorded state, two iterations
    // Syndrome loss: once Q^(k) is formed, each variable overwrites its own r slots with its code
    // (no other thread reads them), and each check then replaces the codes with d(term)/d(code).
    float *ts = rs;
    float *qlane = reinterpret_cast<float *>(smem + L.t_off);     // syndrome loss: Q^(k) per lane
    float *gam = reinterpret_cast<float *>(smem + L.g_off);
    uint8_t *y = smem + L.y_off;
    uint8_t *sb = smem + L.s_off;

    for (int u = tid; u < NV; u += T) gam[u] = F32::quantize(lane_prior(p.g, p.prior, u, N));
    const float inv = 1.0f / float(syn_loss ? M : N);
    for (int b = blockIdx.x; b < p.batch; b += gridDim.x) {
        const uint8_t *tg = syn_loss ? nullptr : p.target + size_t(b) * N;
        const float gscale = p.grad_loss[b] * inv;
        const uint32_t *stb = p.state + size_t(b) * p.T * SW;
        __syncthreads();   // gam (first shot) and the previous shot's last reads are done
        prefetch_state(scb, stb + size_t(p.T - 1) * SW, M);
        for (int u = tid; u < NV; u += T) y[u] = lane_target(p.g, tg, u, N);
        if (syn_loss)
            for (int c = tid; c < M; c += T) sb[c] = p.syn[size_t(b) * M + c] & 1u;
        cp_async_wait();
        __syncthreads();
        // iteration T: recompute r; dL/dq of iteration T+1 is zero
        {
            const float *wk = p.w + size_t(p.T - 1) * S;
            for (int c = tid; c < M; c += T) {
                const int deg = UNIFORM ? DC : int(__ldg(p.g.rdeg + c));
                float wv[DC];
                load_check_weights<DC, UNIFORM>(c, M, deg, wk, wv);
                recompute_r<DC, UNIFORM>(c, M, deg, scb[c], scb[M + c], scb[2 * M + c], scb[3 * M + c], wv, rs);
#pragma unroll
                for (int j = 0; j < DC; ++j)
                    if (UNIFORM || j < deg) gs[j * M + c] = 0.0f;
            }
        }
        __syncthreads();
        for (int k = p.T - 1; k >= 0; --k) {
            const uint32_t *sc = scb + size_t((p.T - 1 - k) & 1) * SW;    // state of iteration k
            uint32_t *sn = scb + size_t(((p.T - 1 - k) & 1) ^ 1) * SW;    // state of iteration k-1
            if (k > 0) prefetch_state(sn, stb + size_t(k - 1) * SW, M);  // overlaps the variable side
            const float gk = gscale * (p.loss_w ? __ldg(p.loss_w + k) : 1.0f / float(p.T));
            if (syn_loss) {
                // the code of Q^(k) on every edge slot, then each check's d(loss term)/d t in its place
                for (int u = tid; u < NV; u += T) {
                    const int deg = __ldg(p.g.vdeg + u);
                    uint32_t sl[DV];
                    float Q = gam[u];
#pragma unroll
                    for (int i = 0; i < DV; ++i) {
                        if (i < deg) {
                            sl[i] = __ldg(p.g.vslot + size_t(i) * NV + u);
                            Q = __fadd_rn(Q, rs[sl[i]]);
                        }
                    }
                    qlane[u] = Q;
                    const float lm = log_magnitude_code(Q);
#pragma unroll
                    for (int i = 0; i < DV; ++i)
                        if (i < deg) ts[sl[i]] = lm;
                }
                __syncthreads();
                for (int c = tid; c < M; c += T) {
                    const int deg = UNIFORM ? DC : int(__ldg(p.g.rdeg + c));
                    syndrome_term_grad<DC, UNIFORM>(c, M, deg, sb[c], ts);
                }
                __syncthreads();
            }
            // variable side: Q^(k) from the recomputed r, dL/dQ, and dL/dr for every edge
            for (int u = tid; u < NV; u += T) {
                const int deg = __ldg(p.g.vdeg + u);   // idle lanes: their warp's degree, scratch slots
                uint32_t sl[DV];
                float Q = syn_loss ? qlane[u] : gam[u], G = 0.0f, H = 0.0f;
#pragma unroll
                for (int i = 0; i < DV; ++i) {
                    if (i < deg) {
                        sl[i] = __ldg(p.g.vslot + size_t(i) * NV + u);
                        if (syn_loss)
                            H += ts[sl[i]];
                        else
                            Q = __fadd_rn(Q, rs[sl[i]]);
                        G += gs[sl[i]];
                    }
                }
                const float gQ = syn_loss ? gk * half_sech2_half(Q) * H : gk * (float(y[u]) - sigmoid(-Q));
#pragma unroll
                for (int i = 0; i < DV; ++i)
                    if (i < deg) gs[sl[i]] = gQ + (G - gs[sl[i]]);
            }
            cp_async_wait();
            __syncthreads();
            // check side: weight gradient, dL/dq of iteration k, and r of iteration k-1
            const float *wk = p.w + size_t(k) * S;
            float *gk_out = p.partial + size_t(k) * S;
            for (int c = tid; c < M; c += T) {
                const int deg = UNIFORM ? DC : int(__ldg(p.g.rdeg + c));
                float wv[DC], wp[DC];   // this iteration's weights and the previous one's, loaded together
                load_check_weights<DC, UNIFORM>(c, M, deg, wk, wv);
                if (k > 0) load_check_weights<DC, UNIFORM>(c, M, deg, wk - S, wp);
                const float m1 = __uint_as_float(sc[c]), m2 = __uint_as_float(sc[M + c]);
                const uint32_t signs = sc[2 * M + c], iw = sc[3 * M + c];
                const int i1 = int(iw & 0xffu), i2 = int((iw >> 8) & 0xffu);
                const uint32_t negall = (iw >> 16) & 1u;
                float acc1 = 0.0f, t1 = 0.0f;
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    if (UNIFORM || j < deg) {
                        const float gr = gs[j * M + c];
                        const float sgn = (((signs >> j) & 1u) ^ negall) ? -1.0f : 1.0f;
                        const float mu = j == i1 ? m2 : m1;
                        atomicAdd(gk_out + j * M + c, gr * sgn * mu);   // result unused: a reduction
                        const float t = gr * wv[j] * sgn;
                        if (j == i1)
                            t1 = t;
                        else
                            acc1 += t;
                    }
                }
                const float gq1 = ((signs >> i1) & 1u) ? -acc1 : acc1;
                const float gq2 = ((signs >> i2) & 1u) ? -t1 : t1;
#pragma unroll
                for (int j = 0; j < DC; ++j)
                    if (UNIFORM || j < deg) gs[j * M + c] = j == i1 ? gq1 : (j == i2 ? gq2 : 0.0f);
                if (k > 0) recompute_r<DC, UNIFORM>(c, M, deg, sn[c], sn[M + c], sn[2 * M + c], sn[3 * M + c], wp, rs);
            }
            __syncthreads();
        }
    }
}

// w_slot[t][eslot[e]] = w_csr[t][e]; padding slots are never read.
__global__ void permute_weights_kernel(const float *__restrict__ w_csr, const uint32_t *__restrict__ eslot, int32_t T,
                                       int32_t nnz, int32_t S, float *__restrict__ w_slot)
{
    const int64_t total = int64_t(T) * nnz;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = i / nnz, e = i - t * nnz;
        w_slot[t * S + __ldg(eslot + e)] = w_csr[i];
    }
}

// grad[t][e] = grad_slot[t][eslot[e]]: the slot-layout gradient in CSR edge order.
__global__ void gather_grad_kernel(const float *__restrict__ grad_slot, const uint32_t *__restrict__ eslot, int32_t T,
                                   int32_t S, int32_t nnz, float *__restrict__ grad)
{
    const int64_t total = int64_t(T) * nnz;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = i / nnz, e = i - t * nnz;
        grad[i] = grad_slot[t * S + __ldg(eslot + e)];
    }
}

// One Adam step (Kingma and Ba, 2015) in the form of PyTorch's single-tensor implementation:
//   m = m + (1 - b1) (g - m);  v = b2 v + (1 - b2) g^2;
//   p = p - (lr / (1 - b1^t)) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)
__global__ void adam_kernel(float *__restrict__ param, const float *__restrict__ grad, float *__restrict__ m1,
                            float *__restrict__ m2, int64_t count, float beta1, float beta2, float eps,
                            float step_size, float bc2_sqrt)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
        const float g = grad[i];
        const float a = m1[i] + (1.0f - beta1) * (g - m1[i]);
        const float v = beta2 * m2[i] + (1.0f - beta2) * g * g;
        m1[i] = a;
        m2[i] = v;
        param[i] = param[i] - step_size * (a / (sqrtf(v) / bc2_sqrt + eps));
    }
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output of one step from state x.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Errors at a per-shot rate and their syndromes, one block per shot.  Counter-based keying
// (seed, shot, qubit): u = top 53 bits of mix(mix(mix(seed) + shot) + qubit) / 2^53;
// p_shot = p_lo + p_span * u(qubit n); e_q = [u(q) < p_shot]; s_i = XOR of e over row i.
__global__ void sample_kernel(const DeviceGraph g, uint64_t seed, int64_t first_shot, int32_t batch, double p_lo,
                              double p_span, uint8_t *__restrict__ err, uint8_t *__restrict__ syn)
{
    extern __shared__ __align__(16) unsigned char es[];
    const int M = g.m, N = g.n, T = blockDim.x, tid = threadIdx.x;
    const uint64_t k_seed = splitmix64(seed);
    for (int b = blockIdx.x; b < batch; b += gridDim.x) {
        const uint64_t k_shot = splitmix64(k_seed + uint64_t(first_shot + b));
        const double un = double(splitmix64(k_shot + uint64_t(N)) >> 11) * 1.1102230246251565e-16;   // 2^-53
        const double thr = __dmul_rn(__dadd_rn(p_lo, __dmul_rn(p_span, un)), 9007199254740992.0);     // p * 2^53
        for (int q = tid; q < N; q += T) {
            const uint8_t e = double(splitmix64(k_shot + uint64_t(q)) >> 11) < thr ? 1 : 0;
            es[q] = e;
            err[size_t(b) * N + q] = e;
        }
        __syncthreads();
        for (int c = tid; c < M; c += T) {
            const int deg = __ldg(g.rdeg + c);
            uint32_t par = 0;
            for (int j = 0; j < deg; ++j) par ^= es[__ldg(g.ecol + size_t(j) * M + c)];
            syn[size_t(b) * M + c] = uint8_t(par);
        }
        __syncthreads();
    }
}

// fail_b = !ok_b OR some logical operator l has odd overlap with the residual e_b XOR e_hat_b.
__global__ void logical_kernel(const uint8_t *__restrict__ logicals, int32_t K, int32_t N, const uint8_t *__restrict__ err,
                               const uint8_t *__restrict__ dec, const uint8_t *__restrict__ ok, int32_t batch,
                               uint8_t *__restrict__ fail)
{
    extern __shared__ __align__(16) uint32_t lw[];
    const int W = (N + 31) / 32, T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarp = (T + 31) / 32;
    uint32_t *rw = lw + size_t(K) * W;
    for (int idx = warp; idx < K * W; idx += nwarp) {   // pack L row by row, 32 qubits per word
        const int l = idx / W, wd = idx - l * W, q = wd * 32 + lane;
        const uint32_t bits = __ballot_sync(0xffffffffu, q < N && logicals[size_t(l) * N + q]);
        if (lane == 0) lw[idx] = bits;
    }
    for (int b = blockIdx.x; b < batch; b += gridDim.x) {
        __syncthreads();
        for (int wd = warp; wd < W; wd += nwarp) {
            const int q = wd * 32 + lane;
            const bool r = q < N && ((err[size_t(b) * N + q] ^ dec[size_t(b) * N + q]) & 1u);
            const uint32_t bits = __ballot_sync(0xffffffffu, r);
            if (lane == 0) rw[wd] = bits;
        }
        __syncthreads();
        int odd = 0;
        for (int l = tid; l < K; l += T) {
            uint32_t par = 0;
            for (int wd = 0; wd < W; ++wd) par ^= uint32_t(__popc(lw[l * W + wd] & rw[wd]));
            odd |= int(par & 1u);
        }
        odd = __syncthreads_or(odd);
        if (tid == 0) fail[b] = (ok[b] == 0 || odd) ? 1 : 0;
    }
}

}  // namespace kern

// Compiled training variants: uniform row degree 6..8 with column-degree bucket 4 or 8, else a
// row-degree bucket 8/16/32 with column-degree bucket 8 or 16.
#define QLDPC_TRAIN_VARIANTS(X)                                                                 \
    X(6, true, 4) X(6, true, 8) X(7, true, 4) X(7, true, 8) X(8, true, 4) X(8, true, 8)        \
    X(8, false, 8) X(8, false, 16) X(16, false, 8) X(16, false, 16) X(32, false, 8) X(32, false, 16)

const void *nms_forward_kernel_ptr(const TrainChoice &tc, int loss_kind)
{
    const bool syn = loss_kind == kLossSyndrome;
#define QLDPC_K(DCV, UNI, DVV)                                                                  \
    if (tc.dc == DCV && tc.uniform == UNI && tc.dvb == DVV)                                     \
        return syn ? reinterpret_cast<const void *>(&kern::nms_forward_kernel<DCV, UNI, DVV, true>) \
                   : reinterpret_cast<const void *>(&kern::nms_forward_kernel<DCV, UNI, DVV, false>);
    QLDPC_TRAIN_VARIANTS(QLDPC_K)
#undef QLDPC_K
    return nullptr;
}

const void *nms_backward_kernel_ptr(const TrainChoice &tc, int loss_kind)
{
    const bool syn = loss_kind == kLossSyndrome;
#define QLDPC_K(DCV, UNI, DVV)                                                                  \
    if (tc.dc == DCV && tc.uniform == UNI && tc.dvb == DVV)                                     \
        return syn ? reinterpret_cast<const void *>(&kern::nms_backward_kernel<DCV, UNI, DVV, true>) \
                   : reinterpret_cast<const void *>(&kern::nms_backward_kernel<DCV, UNI, DVV, false>);
    QLDPC_TRAIN_VARIANTS(QLDPC_K)
#undef QLDPC_K
    return nullptr;
}

cudaError_t launch_nms_forward(const TrainParams &p, const TrainChoice &tc, int grid, int threads, size_t smem,
                               cudaStream_t stream)
{
    const bool syn = p.loss_kind == kLossSyndrome;
#define QLDPC_L(DCV, UNI, DVV)                                                                  \
    if (tc.dc == DCV && tc.uniform == UNI && tc.dvb == DVV) {                                   \
        if (syn)                                                                                \
            kern::nms_forward_kernel<DCV, UNI, DVV, true><<<grid, threads, smem, stream>>>(p);  \
        else                                                                                    \
            kern::nms_forward_kernel<DCV, UNI, DVV, false><<<grid, threads, smem, stream>>>(p); \
        return cudaGetLastError();                                                              \
    }
    QLDPC_TRAIN_VARIANTS(QLDPC_L)
#undef QLDPC_L
    return cudaErrorInvalidValue;
}

cudaError_t launch_nms_backward(const TrainParams &p, const TrainChoice &tc, int grid, int threads, size_t smem,
                                cudaStream_t stream)
{
    const bool syn = p.loss_kind == kLossSyndrome;
#define QLDPC_L(DCV, UNI, DVV)                                                                  \
    if (tc.dc == DCV && tc.uniform == UNI && tc.dvb == DVV) {                                   \
        if (syn)                                                                                \
            kern::nms_backward_kernel<DCV, UNI, DVV, true><<<grid, threads, smem, stream>>>(p); \
        else                                                                                    \
            kern::nms_backward_kernel<DCV, UNI, DVV, false><<<grid, threads, smem, stream>>>(p); \
        return cudaGetLastError();                                                              \
    }
    QLDPC_TRAIN_VARIANTS(QLDPC_L)
#undef QLDPC_L
    return cudaErrorInvalidValue;
}

namespace {
int elementwise_grid(int64_t count)
{
    return int(std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 4096)));
}
}  // namespace

cudaError_t launch_permute_weights(const float *w_csr, const uint32_t *eslot, int32_t T, int32_t nnz, int32_t S,
                                   float *w_slot, cudaStream_t stream)
{
    kern::permute_weights_kernel<<<elementwise_grid(int64_t(T) * nnz), 256, 0, stream>>>(w_csr, eslot, T, nnz, S,
                                                                                         w_slot);
    return cudaGetLastError();
}

cudaError_t launch_gather_grad(const float *grad_slot, const uint32_t *eslot, int32_t T, int32_t S, int32_t nnz,
                               float *grad, cudaStream_t stream)
{
    kern::gather_grad_kernel<<<elementwise_grid(int64_t(T) * nnz), 256, 0, stream>>>(grad_slot, eslot, T, S, nnz, grad);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *param, const float *grad, float *m1, float *m2, int64_t count, int32_t step,
                        float lr, float beta1, float beta2, float eps, cudaStream_t stream)
{
    const double bc1 = 1.0 - std::pow(double(beta1), double(step));
    const double bc2 = 1.0 - std::pow(double(beta2), double(step));
    kern::adam_kernel<<<elementwise_grid(count), 256, 0, stream>>>(param, grad, m1, m2, count, beta1, beta2, eps,
                                                                   float(double(lr) / bc1), float(std::sqrt(bc2)));
    return cudaGetLastError();
}

cudaError_t launch_sample(const DeviceGraph &g, uint64_t seed, int64_t first_shot, int32_t batch, double p_lo,
                          double p_hi, uint8_t *err, uint8_t *syn, int grid, cudaStream_t stream)
{
    kern::sample_kernel<<<grid, 256, size_t(g.n), stream>>>(g, seed, first_shot, batch, p_lo, p_hi - p_lo, err, syn);
    return cudaGetLastError();
}

cudaError_t launch_logical(const uint8_t *logicals, int32_t k, int32_t n, const uint8_t *err, const uint8_t *dec,
                           const uint8_t *ok, int32_t batch, uint8_t *fail, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t(k) + 1) * size_t((n + 31) / 32) * 4;
    kern::logical_kernel<<<grid, 128, smem, stream>>>(logicals, k, n, err, dec, ok, batch, fail);
    return cudaGetLastError();
}

}  // namespace qldpc
