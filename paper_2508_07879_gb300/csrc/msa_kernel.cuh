// Flooding normalized min-sum decoder driven by a syndrome -- Algorithm 1 ("MSA for
// syndrome-based LDPC decoding"), Sec. 2 of arXiv 2508.07879 -- for sm_103a.
//
// Two kernels share the arithmetic below and one shared-memory layout:
//
//   msa_batch_kernel    throughput: one block per shot, persistent over the batch, one thread per
//                       check in the check step and one thread per variable in the variable step;
//                       edge lists are read through the read-only path (L1-resident).
//   msa_latency_kernel  single-shot latency: the same steps, but every thread keeps its edge
//                       lists, degrees, priors and a-posteriori LLRs in registers for the whole
//                       decode, so an iteration touches only shared memory.
//
// Layout (a GB300 design, not the paper's per-iteration launches over global memory):
//   * every edge message of a shot lives in shared memory, in place: the check step overwrites
//     q_{m,n} with r_{m,n}, the variable step overwrites r with the next q.  Slots are check-major
//     (slot j*M + m, 4 bytes FP32 / 2 bytes INT16), so 32 consecutive checks touch 32 consecutive
//     slots;
//   * the stop test H e^T = s is kept incrementally: check m owns a parity word
//     (bit 1 = s_m, bit 0 = s_m XOR the decisions of its variables); a variable whose decision
//     flips XORs bit 0 of its checks' words (shared-memory atomics, exact).  The next check step
//     reads one word per check and the block settles the test with one __syncthreads_and, so an
//     iteration costs two block barriers (the paper's kernel: four);
//   * the check step keeps no argmin: min over S_v(m)\n is min2 where |q_n| equals min1 and min1
//     elsewhere (min2 = min1 when the minimum is shared), which is exact.
//
// Arithmetic is operation-for-operation that of the CPU oracle:
//   r = sign * (alpha * min_{j != n} |q_j|)
//   q_{m,n} = gamma_n + sum_{i != m} r_{i,n}        ascending check order, prefixes reused
//   Q_n = gamma_n + sum_i r_{i,n}                   ascending check order
// so FP32 results are bit-identical (every add/multiply is an explicit round-to-nearest intrinsic,
// nothing is fused or reassociated) and INT16 results are exact integer arithmetic.
// (A lane-per-edge check step with warp-shuffle reductions, a two-lanes-per-check step and a
// thread-block-cluster split of one shot over several SMs were all measured slower on GB300.)
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "msa_launch.h"

namespace qldpc {
namespace kern {

// ---------------------------------------------------------------------------------------------
// Precision policies: arithmetic and the slot format
// ---------------------------------------------------------------------------------------------
struct F32 {
    using acc_t = float;    // variable-node sums, Q_n
    using mag_t = float;    // |q| and scaled minima
    using msg_t = float;    // a slot
    // g + 0 is g except that -0 becomes +0; with no -0 prior no message is ever -0 (a rounded sum
    // is -0 only when every term is), so the sign bit of a message equals [message < 0].
    static __device__ __forceinline__ acc_t quantize(float g) { return __fadd_rn(g, 0.0f); }
    static __device__ __forceinline__ acc_t add(acc_t a, acc_t b) { return __fadd_rn(a, b); }
    // layered schedule: Q - r_old, and the check's input clamped to the message range (none here)
    static __device__ __forceinline__ acc_t sub(acc_t Q, acc_t r) { return __fsub_rn(Q, r); }
    static __device__ __forceinline__ acc_t clampq(acc_t x) { return x; }
    static __device__ __forceinline__ bool neg(float x) { return x < 0.0f; }
    static __device__ __forceinline__ mag_t mag(acc_t x) { return fabsf(x); }
    static __device__ __forceinline__ mag_t mag_init() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ mag_t mn(mag_t a, mag_t b) { return fminf(a, b); }
    static __device__ __forceinline__ mag_t mx(mag_t a, mag_t b) { return fmaxf(a, b); }
    // three-input minimum (sm_100 and later)
    static __device__ __forceinline__ mag_t mn3(mag_t a, mag_t b, mag_t c)
    {
        float r;
        asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
        return r;
    }
    static __device__ __forceinline__ mag_t scale(mag_t m, const LaunchParams &p)
    {
        return __fmul_rn(p.alpha, m);
    }
    // bit 31 = [x < 0] (valid because no message is -0)
    static __device__ __forceinline__ uint32_t sign_word(acc_t x) { return __float_as_uint(x); }
    // sign * m with sign = (-1)^{negall} * sign(x): the sign bit flipped, one logic operation
    // (-m is exact, also -0 for m = 0 as in the oracle)
    static __device__ __forceinline__ acc_t signed_like(mag_t m, acc_t x, uint32_t negall)
    {
        return __uint_as_float(__float_as_uint(m) ^ (__float_as_uint(x) & 0x80000000u) ^ (negall << 31));
    }
    // the same in two steps: the check's factor on a magnitude once, then each edge's own sign
    static __device__ __forceinline__ mag_t presign(mag_t m, uint32_t negall)
    {
        return __uint_as_float(__float_as_uint(m) ^ (negall << 31));
    }
    static __device__ __forceinline__ acc_t apply_sign(mag_t pm, acc_t x)
    {
        return __uint_as_float(__float_as_uint(pm) ^ (__float_as_uint(x) & 0x80000000u));
    }
    static __device__ __forceinline__ float post(acc_t a) { return a; }
    static __device__ __forceinline__ msg_t to_msg(acc_t q) { return q; }
};

// Fixed point with 32-bit accumulation: LLR * 2^FRAC, messages clamped to +-LIM.
//   I16: 8 fractional bits, +-32767;  I8: 2 fractional bits, +-127.
template <class MSG, int FRAC, int LIM>
struct IFix {
    static constexpr int kFrac = FRAC, kLim = LIM;
    using acc_t = int32_t;
    using mag_t = int32_t;
    using msg_t = MSG;
    // gamma_q = clamp(round_half_away(gamma * 2^FRAC), -LIM, LIM); the scaling is exact in binary32
    static __device__ __forceinline__ acc_t quantize(float g)
    {
        float t = roundf(g * float(1 << FRAC));
        t = fminf(fmaxf(t, -float(LIM)), float(LIM));
        return static_cast<int32_t>(t);
    }
    static __device__ __forceinline__ acc_t add(acc_t a, acc_t b) { return a + b; }
    // layered schedule: Q - r_old exactly in 32 bits, and the check's input q = clamp(Q - r_old)
    static __device__ __forceinline__ acc_t sub(acc_t Q, acc_t r) { return Q - r; }
    static __device__ __forceinline__ acc_t clampq(acc_t x) { return max(-LIM, min(LIM, x)); }
    static __device__ __forceinline__ bool neg(int32_t x) { return x < 0; }
    static __device__ __forceinline__ mag_t mag(acc_t x) { return abs(x); }
    static __device__ __forceinline__ mag_t mag_init() { return 0x7fffffff; }
    static __device__ __forceinline__ mag_t mn(mag_t a, mag_t b) { return min(a, b); }
    static __device__ __forceinline__ mag_t mx(mag_t a, mag_t b) { return max(a, b); }
    static __device__ __forceinline__ mag_t mn3(mag_t a, mag_t b, mag_t c) { return __vimin3_s32(a, b, c); }
    // |r| = floor(min * alpha_q / 2^15); min <= 32767 and alpha_q <= 2^15 keep it in 31 bits
    static __device__ __forceinline__ mag_t scale(mag_t m, const LaunchParams &p)
    {
        return (m * p.alpha_q) >> 15;
    }
    static __device__ __forceinline__ uint32_t sign_word(acc_t x) { return uint32_t(x); }
    static __device__ __forceinline__ acc_t signed_like(mag_t m, acc_t x, uint32_t negall)
    {
        const int32_t neg = int32_t(negall ^ (uint32_t(x) >> 31));   // 0 or 1
        return (m ^ -neg) + neg;
    }
    static __device__ __forceinline__ mag_t presign(mag_t m, uint32_t negall) { return negall ? -m : m; }
    static __device__ __forceinline__ acc_t apply_sign(mag_t pm, acc_t x) { return x < 0 ? -pm : pm; }
    static __device__ __forceinline__ float post(acc_t a) { return float(a) * (1.0f / float(1 << FRAC)); }
    static __device__ __forceinline__ msg_t to_msg(acc_t q) { return msg_t(max(-LIM, min(LIM, q))); }
};
using I16 = IFix<int16_t, 8, 32767>;
using I8 = IFix<int8_t, 2, 127>;

template <class P>
__device__ __forceinline__ typename P::acc_t load_msg(const typename P::msg_t *s, uint32_t i)
{
    return typename P::acc_t(s[i]);
}

// Flip the decision bit of one check's parity word (exact: integer XOR in shared memory).
__device__ __forceinline__ void flip_check(uint32_t *parity, uint32_t m) { atomicXor(parity + m, 1u); }

// Edge-list entries are slot indices j*M + m; the check of a slot is needed only when a decision
// flips: m = slot - M * floor(slot / M), the quotient by a multiply-high with a magic number the
// host verified for every slot (Granlund and Montgomery, PLDI 1994).
struct CheckOf {
    uint32_t M, magic, shift;
    __device__ __forceinline__ CheckOf() : M(1u), magic(0u), shift(0u) {}
    __device__ __forceinline__ explicit CheckOf(const DeviceGraph &g)
        : M(uint32_t(g.m)), magic(g.m_magic), shift(uint32_t(g.m_shift)) {}
    __device__ __forceinline__ uint32_t operator()(uint32_t slot) const
    {
        return M == 1u ? 0u : slot - M * (__umulhi(slot, magic) >> shift);
    }
};

// The two smallest of a[LO .. LO+N), with multiplicity, as a balanced tree: the two smallest of
// {x1 <= x2} and {y1 <= y2} together are min(x1, y1) and min(max(x1, y1), x2, y2).  Every step is
// an exact minimum or maximum, so any grouping gives the same pair; the tree only shortens the
// chain of dependent operations (depth 5 for eight magnitudes against 7 for a running pair).
// Ops supplies mn, mx and mn3 (three-input minimum) on magnitudes of type M.
template <class Ops, int LO, int N, class M>
__device__ __forceinline__ void min2_tree(const M *a, M &m1, M &m2)
{
    static_assert(N >= 2, "two magnitudes at least");
    if constexpr (N == 2) {
        m1 = Ops::mn(a[LO], a[LO + 1]);
        m2 = Ops::mx(a[LO], a[LO + 1]);
    } else if constexpr (N == 3) {
        const M lo = Ops::mn(a[LO + 1], a[LO + 2]), hi = Ops::mx(a[LO + 1], a[LO + 2]);
        m1 = Ops::mn(a[LO], lo);
        m2 = Ops::mn(Ops::mx(a[LO], lo), hi);
    } else {
        constexpr int H = (N / 2) % 2 == 0 || N == 5 ? N / 2 : N / 2 + 1;   // halves of >= 2
        M x1, x2, y1, y2;
        min2_tree<Ops, LO, H>(a, x1, x2);
        min2_tree<Ops, LO + H, N - H>(a, y1, y2);
        m1 = Ops::mn(x1, y1);
        m2 = Ops::mn3(Ops::mx(x1, y1), x2, y2);
    }
}

// The two smallest magnitudes of a row, with multiplicity (m2 = m1 when the minimum is shared).
// Rows of exact degree take the magnitudes in pairs (lo, hi): the second smallest of {m1 <= m2}
// and {lo <= hi} is min(max(m1, lo), m2, hi), one three-input minimum (an odd degree starts from
// m1 = the first magnitude, m2 = +inf); rows of varying degree stream them one at a time.  Either
// way the result is the exact pair of minima.  (A balanced tree, min2_tree, shortens the chain but
// keeps every magnitude live at once: in the FP32 kernels that cost a resident block per SM.)
template <class P, int DC, bool UNIFORM>
__device__ __forceinline__ void two_smallest(const typename P::acc_t *q, int deg, typename P::mag_t &m1,
                                             typename P::mag_t &m2)
{
    using mag_t = typename P::mag_t;
    if constexpr (UNIFORM && DC >= 2) {
        constexpr int j0 = DC % 2 == 0 ? 2 : 1;
        if constexpr (DC % 2 == 0) {
            m1 = P::mn(P::mag(q[0]), P::mag(q[1]));
            m2 = P::mx(P::mag(q[0]), P::mag(q[1]));
        } else {
            m1 = P::mag(q[0]);
            m2 = P::mag_init();
        }
#pragma unroll
        for (int j = j0; j < DC; j += 2) {
            const mag_t a = P::mag(q[j]), b = P::mag(q[j + 1]);
            const mag_t lo = P::mn(a, b), hi = P::mx(a, b);
            m2 = P::mn3(P::mx(m1, lo), m2, hi);
            m1 = P::mn(m1, lo);
        }
    } else {
        m1 = P::mag_init();
        m2 = P::mag_init();
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (UNIFORM || j < deg) {
                const mag_t a = P::mag(q[j]);
                m2 = P::mn(m2, P::mx(m1, a));
                m1 = P::mn(m1, a);
            }
        }
    }
}

// min(|a|, |b|) carrying the sign sign(a) xor sign(b) (sm_86 and later)
__device__ __forceinline__ float min_xorsign_abs(float a, float b)
{
    float d;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// The two smallest FP32 magnitudes of a row of exactly DC messages, two at a time, with the parity of
// the signs riding on the smallest: |m1s| = min |q|, the sign bit of m1s = xor of every sign bit; m2
// the second smallest magnitude (with multiplicity).  The same pairs of minima and maxima as
// two_smallest, so the same values.
template <int DC>
__device__ __forceinline__ void two_smallest_signed(const float *q, float &m1s, float &m2)
{
    constexpr int j0 = DC % 2 == 0 ? 2 : 1;
    if constexpr (DC % 2 == 0) {
        m1s = min_xorsign_abs(q[0], q[1]);
        m2 = fmaxf(fabsf(q[0]), fabsf(q[1]));
    } else {
        m1s = q[0];
        m2 = F32::mag_init();
    }
#pragma unroll
    for (int j = j0; j < DC; j += 2) {
        const float lo = min_xorsign_abs(q[j], q[j + 1]);
        const float hi = fmaxf(fabsf(q[j]), fabsf(q[j + 1]));
        m2 = F32::mn3(fmaxf(fabsf(m1s), fabsf(lo)), m2, hi);
        m1s = min_xorsign_abs(m1s, lo);
    }
}

// The check update's reductions of one row: its two smallest magnitudes m1 <= m2 (with multiplicity)
// and the parity of its messages' sign bits (bit 31 of sx).  FP32 rows of exact degree take the parity
// with the smallest magnitude (one instruction per pair of messages fewer); the others xor the signs.
template <class P, int DC, bool UNIFORM>
__device__ __forceinline__ void row_minima(const typename P::acc_t *q, int deg, typename P::mag_t &m1,
                                           typename P::mag_t &m2, uint32_t &sx)
{
    if constexpr (std::is_same<P, F32>::value && UNIFORM && DC >= 2) {
        float m1s;
        two_smallest_signed<DC>(q, m1s, m2);
        m1 = fabsf(m1s);
        sx = __float_as_uint(m1s);
    } else {
        sx = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j)
            if (UNIFORM || j < deg) sx ^= P::sign_word(q[j]);
        two_smallest<P, DC, UNIFORM>(q, deg, m1, m2);
    }
}

// ---------------------------------------------------------------------------------------------
// Check-node step (Alg. 1, CN processing) of one check, fused with the stop test of the previous
// decisions.  Returns 1 iff the check's parity word says s_m is satisfied.
// UNIFORM: every row has exactly DC edges; otherwise deg <= DC.
// ---------------------------------------------------------------------------------------------
// LEARNED (FP32 only): when w is non-null the scale is the learned weight of each edge,
// r = sign * (w_{m,n} * min_{j != n} |q_j|), w = this iteration's slot-layout weights.
template <class P, int DC, bool UNIFORM, bool LEARNED = false>
__device__ __forceinline__ int check_step(int c, int M, int deg, uint32_t pw, bool update,
                                          typename P::msg_t *__restrict__ slots, const LaunchParams &p,
                                          const float *__restrict__ w = nullptr)
{
    using acc_t = typename P::acc_t;
    using mag_t = typename P::mag_t;
    if (update) {
        acc_t q[DC];
#pragma unroll
        for (int j = 0; j < DC; ++j)
            if (UNIFORM || j < deg) q[j] = load_msg<P>(slots, uint32_t(j * M + c));
        mag_t m1, m2;
        uint32_t sx;                               // bit 31: parity of the signs
        row_minima<P, DC, UNIFORM>(q, deg, m1, m2, sx);
        const uint32_t negall = ((pw >> 1) ^ (sx >> 31)) & 1u;   // (-1)^{s_m} * prod of all signs
        if constexpr (LEARNED) {
            if (w) {
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    if (UNIFORM || j < deg) {
                        const mag_t mu = P::mag(q[j]) == m1 ? m2 : m1;   // min over the others
                        const mag_t r = __fmul_rn(__ldg(w + j * M + c), mu);
                        slots[j * M + c] = typename P::msg_t(P::signed_like(r, q[j], negall));
                    }
                }
                return (pw & 1u) == 0;
            }
        }
        // alpha * min over the others (r2 where |q_j| is the minimum), with the check's sign factor
        const mag_t r1 = P::presign(P::scale(m1, p), negall);
        const mag_t r2 = P::presign(P::scale(m2, p), negall);
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (UNIFORM || j < deg)
                slots[j * M + c] = typename P::msg_t(P::apply_sign(P::mag(q[j]) == m1 ? r2 : r1, q[j]));
        }
    }
    return (pw & 1u) == 0;
}

// ---------------------------------------------------------------------------------------------
// Variable-node step (Alg. 1, VN processing + a-posteriori LLR + tentative decision) of a
// variable of degree exactly D whose edges are e[0..D).  q_k = gamma + sum_{i != k} r_i in
// ascending order: q_k = ((pre_k + r_{k+1}) + r_{k+2}) + ...  with pre_k = ((gamma + r_0) + r_1)
// + ... + r_{k-1}.  Stores every q_k, flips the parity bit of its checks when the decision
// [Q < 0] differs from `prev`, and returns Q.
// ---------------------------------------------------------------------------------------------
// TRACK = false (training forward): no decision tracking, parity may be null.
template <class P, int D, bool TRACK = true>
__device__ __forceinline__ typename P::acc_t var_step_exact(const uint32_t *sl, const CheckOf &ck, typename P::acc_t gamma,
                                                            bool prev, typename P::msg_t *__restrict__ slots,
                                                            uint32_t *__restrict__ parity)
{
    using acc_t = typename P::acc_t;
    if constexpr (D == 0) {
        return gamma;
    } else {
        acc_t r[D];
#pragma unroll
        for (int k = 0; k < D; ++k) r[k] = load_msg<P>(slots, sl[k]);
        acc_t pre[D + 1];
        pre[0] = gamma;
#pragma unroll
        for (int k = 0; k < D; ++k) pre[k + 1] = P::add(pre[k], r[k]);
        const acc_t Q = pre[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            acc_t q = pre[k];
#pragma unroll
            for (int i = k + 1; i < D; ++i) q = P::add(q, r[i]);
            slots[sl[k]] = P::to_msg(q);
        }
        if (TRACK && P::neg(Q) != prev) {
#pragma unroll
            for (int k = 0; k < D; ++k) flip_check(parity, ck(sl[k]));
        }
        return Q;
    }
}

#define QLDPC_DEG_CASES(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

// Batch variant: the edge list comes from global memory (L1-resident).
template <class P, int D, bool TRACK = true>
__device__ __forceinline__ typename P::acc_t var_step_global(int v, int N, const CheckOf &ck, const uint32_t *__restrict__ vslot,
                                                             typename P::acc_t gamma, bool prev,
                                                             typename P::msg_t *slots, uint32_t *parity)
{
    uint32_t e[D > 0 ? D : 1];
#pragma unroll
    for (int k = 0; k < D; ++k) e[k] = __ldg(vslot + size_t(k) * N + v);
    return var_step_exact<P, D, TRACK>(e, ck, gamma, prev, slots, parity);
}

// Variable step of the batch kernel for one variable: dispatch on its degree (internal variables
// are sorted by degree, so the lanes of a warp almost always take the same case).
template <class P, int DV, bool TRACK = true>
__device__ __forceinline__ typename P::acc_t var_step_batch(int deg, int u, int N, const CheckOf &ck, const uint32_t *vslot,
                                                            typename P::acc_t gamma, bool prev,
                                                            typename P::msg_t *slots, uint32_t *parity)
{
    switch (deg) {
#define QLDPC_CASE(D)                                                                           \
    case D:                                                                                     \
        if constexpr (D <= DV) return var_step_global<P, D, TRACK>(u, N, ck, vslot, gamma, prev, slots, parity); \
        break;
        QLDPC_DEG_CASES(QLDPC_CASE)
#undef QLDPC_CASE
    default: break;
    }
    return gamma;
}

// ---------------------------------------------------------------------------------------------
// Throughput kernel
// ---------------------------------------------------------------------------------------------
// Initialization (Alg. 1) of one shot: q^(0) = gamma on every edge; the parity words start at s_m
// and take the decisions of the prior.  Ends with a barrier.  N = variable lanes.
template <class P>
__device__ __forceinline__ void batch_init_shot(const Problem &pr, const uint8_t *s, int M, int N, int tid, int T,
                                                const typename P::acc_t *gam, typename P::acc_t *Qs,
                                                uint32_t *parity, typename P::msg_t *slots)
{
    for (int c = tid; c < M; c += T) parity[c] = (s[c] & 1u) * 3u;
    __syncthreads();
    const CheckOf ck(pr.g);
    for (int u = tid; u < N; u += T) {
        const typename P::acc_t g = gam[u];
        const int deg = __ldg(pr.g.vdeg + u);
        const bool d = P::neg(g);
        for (int k = 0; k < deg; ++k) {
            const uint32_t e = __ldg(pr.g.vslot + size_t(k) * N + u);
            slots[e] = P::to_msg(g);
            if (d) flip_check(parity, ck(e));
        }
        Qs[u] = g;
    }
    __syncthreads();
}

// LEARNED: iterations 1..learned_iters use the learned weights; a shot whose syndrome is still not
// met then restarts from its prior with plain min-sum (alpha) for up to max_iter iterations, and
// reports learned_iters + the plain iterations.  Learned launches always stop early.
template <class P, int DC, bool UNIFORM, int DV, bool LEARNED = false>
__global__ void __launch_bounds__(1024, 1) msa_batch_kernel(const LaunchParams p)
{
    using acc_t = typename P::acc_t;
    using msg_t = typename P::msg_t;

    const Problem pr = blockIdx.y == 0 ? p.prob[0] : p.prob[1];
    const int M = pr.g.m, N = pr.g.n, NV = pr.g.nv;   // checks, variables, variable lanes
    const int T = blockDim.x, tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(M, NV, pr.g.dc_max, int(sizeof(msg_t)));
    acc_t *Qs = reinterpret_cast<acc_t *>(smem + L.q_off);
    acc_t *gam = reinterpret_cast<acc_t *>(smem + L.g_off);
    uint32_t *parity = reinterpret_cast<uint32_t *>(smem + L.par_off);
    msg_t *slots = reinterpret_cast<msg_t *>(smem + L.slot_off);

    // Prior LLRs: loaded once per block, shared by all its shots (idle lanes: 0, no edges).
    int bad = 0;
    for (int u = tid; u < NV; u += T) {
        const uint32_t v = __ldg(pr.g.vperm + u);
        const float g = v < uint32_t(N) ? pr.prior[v] : 0.0f;
        bad |= !isfinite(g);
        gam[u] = P::quantize(g);
    }
    bad = __syncthreads_or(bad);

    const bool early = LEARNED || (p.flags & kFlagNoEarlyStop) == 0;
    const size_t wstride = size_t(pr.g.dc_max) * M;   // learned weights of one iteration
    // Shots are claimed one at a time from a per-launch counter, so blocks that draw slowly
    // converging shots take fewer of them (or taken statically when no counter is given).
    // (Two claim words alternate: a thread reads word k&1 after claim k's barrier, and the word is
    // rewritten only after claim k+1's barrier, which every thread reaches after its read.)
    __shared__ int s_shot[2];
    int claim = 0;
    for (int b = blockIdx.x;; b += gridDim.x) {
        if (p.next_shot) {
            if (tid == 0) s_shot[claim] = atomicAdd(p.next_shot + blockIdx.y, 1);
            __syncthreads();
            b = s_shot[claim];
            claim ^= 1;
        }
        if (b >= p.batch) break;
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
        batch_init_shot<P>(pr, s, M, NV, tid, T, gam, Qs, parity, slots);

        int k = 0, all = 0;
        bool learned = LEARNED;
        int end = LEARNED ? pr.learned_iters : p.max_iter;   // k at which the current phase ends
        for (;;) {
            const bool last = k >= end;
            const float *wk = nullptr;
            if constexpr (LEARNED) wk = (learned && !last) ? pr.weights + size_t(k) * wstride : nullptr;
            int ok = 1;
            for (int c = tid; c < M; c += T) {
                const int deg = UNIFORM ? DC : int(__ldg(pr.g.rdeg + c));
                ok &= check_step<P, DC, UNIFORM, LEARNED>(c, M, deg, parity[c], !last, slots, p, wk);
            }
            all = __syncthreads_and(ok);
            if (early && all) break;
            if (last) {
                if (!LEARNED || !learned) break;
                learned = false;                  // fallback: plain min-sum from the prior
                end = k + p.max_iter;
                batch_init_shot<P>(pr, s, M, NV, tid, T, gam, Qs, parity, slots);
                continue;
            }
            for (int u = tid; u < NV; u += T)
                Qs[u] = var_step_batch<P, DV>(__ldg(pr.g.vdeg + u), u, NV, CheckOf(pr.g), pr.g.vslot, gam[u],
                                              P::neg(Qs[u]), slots, parity);
            __syncthreads();
            ++k;
        }

        for (int u = tid; u < NV; u += T) {
            const acc_t q = Qs[u];
            const uint32_t v = __ldg(pr.g.vperm + u);
            if (v < uint32_t(N)) {
                err[v] = P::neg(q) ? 1 : 0;
                if (pr.post) pr.post[size_t(b) * N + v] = P::post(q);
            }
        }
        if (tid == 0) {
            pr.iters[b] = k;
            pr.ok[b] = all ? 1 : 0;
        }
        __syncthreads();   // the next shot reuses shared memory
    }
}

// ---------------------------------------------------------------------------------------------
// Latency kernel: one block per shot, everything a thread needs across iterations in registers.
// ---------------------------------------------------------------------------------------------
constexpr int kLatCnPerThread = kLatencyCnPerThread;   // checks per thread: M <= 2*blockDim
constexpr int kLatVnPerThread = kLatencyVnPerThread;   // variables per thread: N <= 2*blockDim

template <class P, int DV>
__device__ __forceinline__ typename P::acc_t var_step_regs(int deg, const uint32_t *e, const CheckOf &ck,
                                                           typename P::acc_t gamma, bool prev,
                                                           typename P::msg_t *slots, uint32_t *parity)
{
    switch (deg) {
#define QLDPC_CASE(D)                                                                           \
    case D:                                                                                     \
        if constexpr (D <= DV) return var_step_exact<P, D>(e, ck, gamma, prev, slots, parity); \
        break;
        QLDPC_DEG_CASES(QLDPC_CASE)
#undef QLDPC_CASE
    default: break;
    }
    return gamma;
}

template <class P, int DC, bool UNIFORM, int DV, bool LEARNED = false>
__global__ void __launch_bounds__(kLatencyMaxThreads, 1) msa_latency_kernel(const LaunchParams p)
{
    using acc_t = typename P::acc_t;
    using msg_t = typename P::msg_t;

    const Problem pr = blockIdx.y == 0 ? p.prob[0] : p.prob[1];
    const int M = pr.g.m, N = pr.g.n, NV = pr.g.nv;
    const int T = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem[];
    const LatencyLayout L = latency_layout(M, pr.g.dc_max, int(sizeof(msg_t)));
    uint32_t *parity = reinterpret_cast<uint32_t *>(smem + L.par_off);
    msg_t *slots = reinterpret_cast<msg_t *>(smem + L.slot_off);

    // Checks c = tid + i*T: degree in registers.
    int cdeg[kLatCnPerThread];
#pragma unroll
    for (int i = 0; i < kLatCnPerThread; ++i) {
        const int c = tid + i * T;
        cdeg[i] = c < M ? (UNIFORM ? DC : int(__ldg(pr.g.rdeg + c))) : -1;
    }
    // Variable lanes u = tid + i*T (heaviest first, so the few second-pass variables are the
    // lightest): edge lists, degree and prior in registers; vid = original index for the outputs.
    uint32_t ev[kLatVnPerThread][DV];
    int vdeg[kLatVnPerThread], vid[kLatVnPerThread];
    acc_t gam[kLatVnPerThread];
    int bad = 0;
#pragma unroll
    for (int i = 0; i < kLatVnPerThread; ++i) {
        const int u = tid + i * T;
        const int v = u < NV ? int(__ldg(pr.g.vperm + u)) : N;   // N: idle lane
        vid[i] = v;
        vdeg[i] = u < NV ? int(__ldg(pr.g.vdeg + u)) : -1;
#pragma unroll
        for (int k = 0; k < DV; ++k)
            ev[i][k] = (k < vdeg[i]) ? __ldg(pr.g.vslot + size_t(k) * NV + u) : 0u;
        const float g = v < N ? pr.prior[v] : 0.0f;
        bad |= !isfinite(g);
        gam[i] = P::quantize(g);
    }
    bad = __syncthreads_or(bad);

    const bool early = LEARNED || (p.flags & kFlagNoEarlyStop) == 0;
    const size_t wstride = size_t(pr.g.dc_max) * M;
    for (int b = blockIdx.x; b < p.batch; b += gridDim.x) {
        uint8_t *err = pr.err + size_t(b) * N;
        if (bad) {
#pragma unroll
            for (int i = 0; i < kLatVnPerThread; ++i) {
                const int v = vid[i];
                if (v < N) {
                    err[v] = 0;
                    if (pr.post) pr.post[size_t(b) * N + v] = __int_as_float(0x7fc00000);
                }
            }
            if (tid == 0) {
                pr.iters[b] = -1;
                pr.ok[b] = 0;
            }
            continue;
        }
        const uint8_t *s = pr.syn + size_t(b) * M;
        acc_t Q[kLatVnPerThread];
        // Initialization (Alg. 1), also the restart of the plain fallback; ends with a barrier.
        auto init_shot = [&]() {
#pragma unroll
            for (int i = 0; i < kLatCnPerThread; ++i)
                if (cdeg[i] >= 0) parity[tid + i * T] = (s[tid + i * T] & 1u) * 3u;
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kLatVnPerThread; ++i) {
                Q[i] = gam[i];
                const bool d = P::neg(gam[i]);
#pragma unroll
                for (int k = 0; k < DV; ++k) {
                    if (k < vdeg[i]) {
                        slots[ev[i][k]] = P::to_msg(gam[i]);
                        if (d) flip_check(parity, CheckOf(pr.g)(ev[i][k]));
                    }
                }
            }
            __syncthreads();
        };
        init_shot();

        int k = 0, all = 0;
        bool learned = LEARNED;
        int end = LEARNED ? pr.learned_iters : p.max_iter;
        for (;;) {
            const bool last = k >= end;
            const float *wk = nullptr;
            if constexpr (LEARNED) wk = (learned && !last) ? pr.weights + size_t(k) * wstride : nullptr;
            int ok = 1;
#pragma unroll
            for (int i = 0; i < kLatCnPerThread; ++i)
                if (cdeg[i] >= 0)
                    ok &= check_step<P, DC, UNIFORM, LEARNED>(tid + i * T, M, cdeg[i], parity[tid + i * T], !last,
                                                              slots, p, wk);
            all = __syncthreads_and(ok);
            if (early && all) break;
            if (last) {
                if (!LEARNED || !learned) break;
                learned = false;                  // fallback: plain min-sum from the prior
                end = k + p.max_iter;
                init_shot();
                continue;
            }
#pragma unroll
            for (int i = 0; i < kLatVnPerThread; ++i)
                if (vdeg[i] >= 0)
                    Q[i] = var_step_regs<P, DV>(vdeg[i], ev[i], CheckOf(pr.g), gam[i], P::neg(Q[i]), slots, parity);
            __syncthreads();
            ++k;
        }

#pragma unroll
        for (int i = 0; i < kLatVnPerThread; ++i) {
            const int v = vid[i];
            if (v < N) {
                err[v] = P::neg(Q[i]) ? 1 : 0;
                if (pr.post) pr.post[size_t(b) * N + v] = P::post(Q[i]);
            }
        }
        if (tid == 0) {
            pr.iters[b] = k;
            pr.ok[b] = all ? 1 : 0;
        }
        __syncthreads();   // the next shot reuses shared memory
    }
}

}  // namespace kern

// ---------------------------------------------------------------------------------------------
// Instantiation tables for one precision policy: uniform row degree 6, 7, 8, 9 (exact; 9 is a
// degree-8 code's row on the data-syndrome graph [H | I]) or any degree up to 8, 16, 32;
// column-degree bucket 4, 8, 16; for each, the batch and the latency kernel.
// ---------------------------------------------------------------------------------------------
#define QLDPC_DV_LIST(X, A, B) X(A, B, 4) X(A, B, 8) X(A, B, 16)
#define QLDPC_VARIANTS(X)                                                                       \
    QLDPC_DV_LIST(X, 6, true) QLDPC_DV_LIST(X, 7, true) QLDPC_DV_LIST(X, 8, true)               \
    QLDPC_DV_LIST(X, 9, true) QLDPC_DV_LIST(X, 8, false) QLDPC_DV_LIST(X, 16, false) QLDPC_DV_LIST(X, 32, false)

template <class P, bool LEARNED = false>
const void *kernel_table(const KernelChoice &kc)
{
#define QLDPC_K(DCV, UNI, DVV)                                                                  \
    if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == DVV)                                     \
        return kc.latency ? reinterpret_cast<const void *>(&kern::msa_latency_kernel<P, DCV, UNI, DVV, LEARNED>) \
                          : reinterpret_cast<const void *>(&kern::msa_batch_kernel<P, DCV, UNI, DVV, LEARNED>);
    QLDPC_VARIANTS(QLDPC_K)
#undef QLDPC_K
    return nullptr;
}

template <class P, bool LEARNED = false>
cudaError_t launch_table(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                         size_t smem, cudaStream_t stream)
{
#define QLDPC_L(DCV, UNI, DVV)                                                                  \
    if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == DVV) {                                   \
        if (kc.latency)                                                                         \
            kern::msa_latency_kernel<P, DCV, UNI, DVV, LEARNED><<<grid, threads, smem, stream>>>(p); \
        else                                                                                    \
            kern::msa_batch_kernel<P, DCV, UNI, DVV, LEARNED><<<grid, threads, smem, stream>>>(p); \
        return cudaGetLastError();                                                              \
    }
    QLDPC_VARIANTS(QLDPC_L)
#undef QLDPC_L
    return cudaErrorInvalidValue;
}

}  // namespace qldpc
