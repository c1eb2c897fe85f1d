// Two shots per block, their messages paired in one slot per edge: the throughput kernel of every
// precision.
//
// Algorithm 1 (Sec. 2 of arXiv 2508.07879) with the arithmetic of the precision policies of
// msa_kernel.cuh, but every shared-memory slot holds the same edge's message of two shots: lane 0
// and lane 1 of a float2 (FP32), of a 32-bit word of two 16-bit two's-complement lanes (INT16, and
// INT8 above column degree 8, within +-127), or of a half2 (INT8 up to column degree 8: the integers
// as FP16 numbers, exact).  One block decodes two shots at a time:
//   * check step: one thread per check handles both shots, one load and one store per edge for both
//     (paired-lane instructions in the 16-bit forms: min/max, lane-wise add, byte permutes);
//   * variable step: one thread per variable loads each slot once for both shots, forms each lane's
//     sums exactly (Q_n = gamma_n + sum r, q = the literal sum over the other checks, clamped in the
//     integer forms) and writes the pair back; the edge list, degree and prior are read once for both;
//   * stop test: the parity word of a check carries both shots (bit 0: lane 0's s_m xor decisions,
//     bit 15: lane 0's s_m, bit 16 and bit 31 the same for lane 1), so one block OR settles both.
// Each lane stops at its own iteration (the scalar kernel's rule) and is refilled with the next
// shot of the batch in the same variable step, so a lane never waits for its partner: the block
// takes shots from the launch's counter one lane at a time.
//
// A refill writes the prior into the lane's half of every slot and Q, and flips the lane's parity
// bit of a check where the variable's decision changes from the old shot's to the prior's; the next
// check step replaces the old syndrome bit by the new one (bit 0 and bit 15 both take s_old xor
// s_new), which leaves exactly the initial state of the new shot.
#pragma once

#include <type_traits>

#include <cuda_fp16.h>

#include "msa_kernel.cuh"

namespace qldpc {
namespace kern {

// A hint to bring the cache line holding p into L2 (generic address; no data is returned).
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.L2 [%0];" ::"l"(p)); }

// An output store (decisions, a-posteriori LLRs): written once, read by the caller after the launch.
template <class T>
__device__ __forceinline__ void store_out(T *p, T v) { *p = v; }

// ---------------------------------------------------------------------------------------------
// Paired-lane helpers (lane 0 = bits 0..15, lane 1 = bits 16..31)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t max_s16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t min_s16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// lane-wise sum modulo 2^16 (no carry between the lanes)
__device__ __forceinline__ uint32_t add_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("add.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// each lane's sign bit (bit 15 / bit 31) replicated over its 16 bits: a byte permute whose
// selector nibbles 0x9 / 0xB take the sign of byte 1 / byte 3
__device__ __forceinline__ uint32_t signmask16x2(uint32_t x)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(d) : "r"(x));
    return d;
}
// lane-wise negation (two's complement; -0 = 0 without a carry into the other lane)
__device__ __forceinline__ uint32_t neg16x2(uint32_t x) { return add_u16x2(~x, 0x00010001u); }
// lane-wise |x| for lanes in [-32767, 32767]
__device__ __forceinline__ uint32_t abs16x2(uint32_t x) { return max_s16x2(x, neg16x2(x)); }
// a where the lane of m is all ones, else b
__device__ __forceinline__ uint32_t select16x2(uint32_t m, uint32_t a, uint32_t b) { return (a & m) | (b & ~m); }
__device__ __forceinline__ int32_t lane0(uint32_t w) { return int32_t(int16_t(uint16_t(w & 0xffffu))); }
__device__ __forceinline__ int32_t lane1(uint32_t w) { return int32_t(w) >> 16; }
// Saturate two 32-bit sums to [-32768, 32767] and pack them (lane 0 = x0, lane 1 = x1).
// cvt.pack.sat.s16.s32 d, a, b puts a in the upper and b in the lower half.
__device__ __forceinline__ uint32_t pack_sat16x2(int32_t x0, int32_t x1)
{
    uint32_t d;
    asm("cvt.pack.sat.s16.s32 %0, %1, %2;" : "=r"(d) : "r"(x1), "r"(x0));
    return d;
}

// Lane-wise minima and maxima of 16-bit magnitudes, the operations min2_tree takes.
struct U16x2Ops {
    static __device__ __forceinline__ uint32_t mn(uint32_t a, uint32_t b) { return min_u16x2(a, b); }
    static __device__ __forceinline__ uint32_t mx(uint32_t a, uint32_t b) { return max_u16x2(a, b); }
    static __device__ __forceinline__ uint32_t mn3(uint32_t a, uint32_t b, uint32_t c) { return min_u16x2(min_u16x2(a, b), c); }
};

// The message clamp of a fixed-point policy on a packed pair: [-LIM, LIM] in each lane.
template <class P>
__device__ __forceinline__ uint32_t clamp_pair(int32_t x0, int32_t x1)
{
    constexpr uint32_t lim = uint32_t(P::kLim) | (uint32_t(P::kLim) << 16);
    constexpr uint32_t nlim = (uint32_t(-P::kLim) & 0xffffu) | ((uint32_t(-P::kLim) & 0xffffu) << 16);
    const uint32_t w = pack_sat16x2(x0, x1);        // [-32768, 32767]
    if constexpr (P::kLim == 32767) return max_s16x2(w, nlim);
    else return max_s16x2(min_s16x2(w, lim), nlim);
}

// |r| = floor(min * alpha_q / 2^15) in each lane (min <= 32767, alpha_q <= 2^15: 30-bit products)
__device__ __forceinline__ uint32_t scale16x2(uint32_t m, int32_t alpha_q)
{
    const uint32_t lo = (uint32_t(m & 0xffffu) * uint32_t(alpha_q)) >> 15;
    const uint32_t hi = ((m >> 16) * uint32_t(alpha_q)) >> 15;
    return lo | (hi << 16);
}

// ---------------------------------------------------------------------------------------------
// Check step of one check for both lanes (Alg. 1, CN processing).  pw: the check's parity word
// (bits 15 / 31: s_m of lane 0 / 1).  Writes r over q in place.
// ---------------------------------------------------------------------------------------------
template <class P, int DC, bool UNIFORM>
__device__ __forceinline__ void check_step_x2(int c, int M, int deg, uint32_t pw, uint32_t *__restrict__ slots,
                                              int32_t alpha_q)
{
    uint32_t q[DC], a[DC];
    uint32_t sx = 0;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            q[j] = slots[j * M + c];
            sx ^= q[j];                                 // bits 15 / 31: parity of the signs
            a[j] = abs16x2(q[j]);
        }
    }
    // the two smallest magnitudes of each lane, with multiplicity (rows of exact degree: a tree)
    uint32_t m1 = 0x7fff7fffu, m2 = 0x7fff7fffu;
    if constexpr (UNIFORM && DC >= 2) {
        min2_tree<U16x2Ops, 0, DC>(a, m1, m2);
    } else {
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (UNIFORM || j < deg) {
                m2 = min_u16x2(m2, max_u16x2(m1, a[j]));
                m1 = min_u16x2(m1, a[j]);
            }
        }
    }
    // (-1)^{s_m} prod of all signs, per lane, replicated over the lane
    const uint32_t negm = signmask16x2(pw ^ sx);
    const uint32_t s1 = scale16x2(m1, alpha_q), s2 = scale16x2(m2, alpha_q);
    const uint32_t n1 = neg16x2(s1), n2 = neg16x2(s2);
    // alpha * min over the others with the check's factor applied (r1: |q| above the minimum, r2: at
    // it), and the same negated for an edge whose own sign is negative
    const uint32_t rp1 = select16x2(negm, n1, s1), rp2 = select16x2(negm, n2, s2);
    const uint32_t rn1 = select16x2(negm, s1, n1), rn2 = select16x2(negm, s2, n2);
    // per lane 0x7fff - m1: |q| + (0x7fff - m1) has bit 15 set iff |q| > m1, and stays below 0x10000
    // (|q|, m1 <= 32767), so one 32-bit add serves both lanes without a carry between them
    const uint32_t k1 = 0x7fff7fffu - m1;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            const uint32_t gt = signmask16x2(a[j] + k1);
            const uint32_t pos = select16x2(gt, rp1, rp2), neg = select16x2(gt, rn1, rn2);
            slots[j * M + c] = select16x2(signmask16x2(q[j]), neg, pos);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Variable step of one variable of degree exactly D for both lanes (Alg. 1, VN processing,
// a-posteriori LLR and decision).  keep: per lane 0xffff where the lane updates (its r is used),
// 0 where the lane restarts from the prior (r taken as 0: Q = gamma, q = gamma).  Returns the new
// (Q0, Q1); flips the lane's parity bit of every check of the variable whose decision changed.
// ---------------------------------------------------------------------------------------------
// MASK = false: both lanes update (keep = all ones), the messages are used as loaded.
template <class P, int D, bool MASK>
__device__ __forceinline__ int2 var_step_x2(int u, int NV, const uint16_t *__restrict__ vchk, const uint16_t *__restrict__ vslot,
                                            int32_t gamma, int2 Qold, uint32_t keep, uint32_t *__restrict__ slots,
                                            uint32_t *__restrict__ parity)
{
    if constexpr (D == 0) {
        return make_int2(gamma, gamma);
    } else {
        uint32_t e[D], r[D];
#pragma unroll
        for (int k = 0; k < D; ++k) e[k] = __ldg(vslot + k * NV + u);
#pragma unroll
        for (int k = 0; k < D; ++k) r[k] = MASK ? slots[e[k]] & keep : slots[e[k]];
        int32_t Q0 = gamma, Q1 = gamma;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            Q0 += lane0(r[k]);
            Q1 += lane1(r[k]);
        }
#pragma unroll
        for (int k = 0; k < D; ++k) slots[e[k]] = clamp_pair<P>(Q0 - lane0(r[k]), Q1 - lane1(r[k]));
        const uint32_t flip = (uint32_t(Q0 ^ Qold.x) >> 31) | ((uint32_t(Q1 ^ Qold.y) >> 31) << 16);
        if (flip) {
#pragma unroll
            for (int k = 0; k < D; ++k) atomicXor(parity + __ldg(vchk + k * NV + u), flip);
        }
        return make_int2(Q0, Q1);
    }
}

// ---------------------------------------------------------------------------------------------
// Two FP32 shots per block: the slots hold float2 pairs (lane 0 in .x, lane 1 in .y).  The check
// step runs the FP32 arithmetic of check_step on each lane (one 8-byte load and store per edge
// for both); the variable step forms both lanes' literal prefix and exclusive sums with one
// add.rn.f32x2 per addition (each lane rounded to nearest on its own, so both are bit-identical to
// var_step_exact).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 add2_rn(float2 a, float2 b)
{
    unsigned long long x, y, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

template <int DC, bool UNIFORM>
__device__ __forceinline__ void check_step_f32x2(int c, int M, int deg, uint32_t pw, float2 *__restrict__ slots,
                                                 float alpha)
{
    using P = F32;
    float q0[DC], q1[DC];
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            const float2 v = slots[j * M + c];
            q0[j] = v.x;
            q1[j] = v.y;
        }
    }
    float a1, a2, b1, b2;
    uint32_t sx0, sx1;
    row_minima<P, DC, UNIFORM>(q0, deg, a1, a2, sx0);
    row_minima<P, DC, UNIFORM>(q1, deg, b1, b2, sx1);
    // the check's factor (-1)^{s_m} prod of the signs as a sign bit per lane (pw bit 15 / 31: s_m)
    const uint32_t na = (sx0 ^ (pw << 16)) & 0x80000000u, nb = (sx1 ^ pw) & 0x80000000u;
    const float ra1 = __uint_as_float(__float_as_uint(__fmul_rn(alpha, a1)) ^ na);
    const float ra2 = __uint_as_float(__float_as_uint(__fmul_rn(alpha, a2)) ^ na);
    const float rb1 = __uint_as_float(__float_as_uint(__fmul_rn(alpha, b1)) ^ nb);
    const float rb2 = __uint_as_float(__float_as_uint(__fmul_rn(alpha, b2)) ^ nb);
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg)
            slots[j * M + c] = make_float2(P::apply_sign(fabsf(q0[j]) == a1 ? ra2 : ra1, q0[j]),
                                           P::apply_sign(fabsf(q1[j]) == b1 ? rb2 : rb1, q1[j]));
    }
}

template <int D, bool MASK>
__device__ __forceinline__ float2 var_step_f32x2(int u, int NV, const CheckOf &ck, const uint16_t *__restrict__ vslot,
                                                 float gamma, float2 Qold, uint32_t act, float2 *__restrict__ slots,
                                                 uint32_t *__restrict__ parity)
{
    if constexpr (D == 0) {
        return make_float2(gamma, gamma);
    } else {
        const uint32_t k0 = (act & 1u) ? 0xffffffffu : 0u, k1 = (act & 2u) ? 0xffffffffu : 0u;
        uint32_t e[D];
        float2 r[D];
#pragma unroll
        for (int k = 0; k < D; ++k) e[k] = __ldg(vslot + k * NV + u);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float2 v = slots[e[k]];        // a lane that restarts takes r = +0: Q = q = gamma
            r[k] = MASK ? make_float2(__uint_as_float(__float_as_uint(v.x) & k0), __uint_as_float(__float_as_uint(v.y) & k1))
                        : v;
        }
        float2 pre[D + 1];
        pre[0] = make_float2(gamma, gamma);
#pragma unroll
        for (int k = 0; k < D; ++k) pre[k + 1] = add2_rn(pre[k], r[k]);
        const float2 Q = pre[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            float2 q = pre[k];
#pragma unroll
            for (int i = k + 1; i < D; ++i) q = add2_rn(q, r[i]);
            slots[e[k]] = q;
        }
        // the lanes whose decision [Q < 0] changed: the sign bits differ (no Q is -0, and the only NaN
        // the arithmetic can form, inf - inf, is the positive canonical one)
        const uint32_t flip = ((__float_as_uint(Q.x) ^ __float_as_uint(Qold.x)) >> 31) |
                              (((__float_as_uint(Q.y) ^ __float_as_uint(Qold.y)) >> 15) & 0x00010000u);
        if (flip) {
#pragma unroll
            for (int k = 0; k < D; ++k) atomicXor(parity + ck(e[k]), flip);
        }
        return Q;
    }
}

// ---------------------------------------------------------------------------------------------
// Lane-pair policies: what the kernel below needs of each precision.
// ---------------------------------------------------------------------------------------------
template <class P>   // I16 or I8: two 16-bit two's-complement lanes per 32-bit word
struct Pair16 {
    using word_t = uint32_t;
    using gam_t = int32_t;
    using pair_t = int2;
    static __device__ __forceinline__ gam_t quantize(float g) { return P::quantize(g); }
    static __device__ __forceinline__ pair_t both(gam_t g) { return make_int2(g, g); }
    static __device__ __forceinline__ gam_t lane(pair_t x, int l) { return l ? x.y : x.x; }
    static __device__ __forceinline__ bool neg(gam_t x) { return x < 0; }
    static __device__ __forceinline__ float post(gam_t x) { return P::post(x); }
    static __device__ __forceinline__ void setup(int, int, const LaunchParams &) {}
    template <int DC, bool UNIFORM>
    static __device__ __forceinline__ void check(int c, int M, int deg, uint32_t pw, word_t *slots, const LaunchParams &p)
    {
        check_step_x2<P, DC, UNIFORM>(c, M, deg, pw, slots, p.alpha_q);
    }
    template <int D, bool MASK>
    static __device__ __forceinline__ pair_t var(int u, int NV, const CheckOf &ck, const uint16_t *vchk, const uint16_t *vslot,
                                                 gam_t gamma,
                                                 pair_t Qold, uint32_t act, word_t *slots, uint32_t *parity)
    {
        const uint32_t keep = ((act & 1u) ? 0x0000ffffu : 0u) | ((act & 2u) ? 0xffff0000u : 0u);
        (void)ck;
        return var_step_x2<P, D, MASK>(u, NV, vchk, vslot, gamma, Qold, keep, slots, parity);
    }
};

struct PairF32 {     // two FP32 lanes per 8-byte slot
    using word_t = float2;
    using gam_t = float;
    using pair_t = float2;
    static __device__ __forceinline__ gam_t quantize(float g) { return F32::quantize(g); }
    static __device__ __forceinline__ pair_t both(gam_t g) { return make_float2(g, g); }
    static __device__ __forceinline__ gam_t lane(pair_t x, int l) { return l ? x.y : x.x; }
    static __device__ __forceinline__ bool neg(gam_t x) { return x < 0.0f; }
    static __device__ __forceinline__ float post(gam_t x) { return x; }
    static __device__ __forceinline__ void setup(int, int, const LaunchParams &) {}
    template <int DC, bool UNIFORM>
    static __device__ __forceinline__ void check(int c, int M, int deg, uint32_t pw, word_t *slots, const LaunchParams &p)
    {
        check_step_f32x2<DC, UNIFORM>(c, M, deg, pw, slots, p.alpha);
    }
    template <int D, bool MASK>
    static __device__ __forceinline__ pair_t var(int u, int NV, const CheckOf &ck, const uint16_t *vchk, const uint16_t *vslot,
                                                 gam_t gamma,
                                                 pair_t Qold, uint32_t act, word_t *slots, uint32_t *parity)
    {
        (void)vchk;   // FP32 pairs decode the check from the slot: a second 16-bit list costs them L1 room
        return var_step_f32x2<D, MASK>(u, NV, ck, vslot, gamma, Qold, act, slots, parity);
    }
};

// ---------------------------------------------------------------------------------------------
// INT8 messages in half-precision lanes: the same integers as I8 (quarter-LLR units), each lane an
// FP16 number.  Every value the decoder forms is an integer of magnitude at most 127 (a message) or
// 127 (1 + d_v) (a sum over a variable: 1143 for column degrees up to 8), and FP16 represents every
// integer up to 2048 exactly, so each FP16 addition, minimum and comparison below is the exact
// integer operation of I8 and the results are bit-identical to it.  The paired FP16 instructions
// give what the 16-bit integer lanes lack: |x| as part of the minimum (min.xorsign.abs, which also
// carries the product of the signs on the smallest magnitude), a lane-wise equality mask (set.eq) and
// lane-wise additions.  Zero: a message is never -0 (every sum starts from the prior, +0 or a nonzero
// integer, and a rounded sum is -0 only when every term is), so a lane's sign bit is [x < 0]; an
// output r = -0 (a zero magnitude with a negative sign) only ever enters such sums.
// The scale |r| = floor(min * alpha_q / 2^15) comes from a 128-entry table per block (exact integers).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t h2_minxs(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.xorsign.abs.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2_maxxs(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.xorsign.abs.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2_min(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2_max(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2_add(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// 0xffff in each lane where a == b, else 0
__device__ __forceinline__ uint32_t h2_eq_mask(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("set.eq.u32.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// The magnitudes (signs ignored) of the minimum and maximum, for min2_tree; mn keeps the xor of the
// signs, so the smallest of a tree carries the parity of all its leaves' signs.
struct H2XsOps {
    static __device__ __forceinline__ uint32_t mn(uint32_t a, uint32_t b) { return h2_minxs(a, b); }
    static __device__ __forceinline__ uint32_t mx(uint32_t a, uint32_t b) { return h2_maxxs(a, b); }
    static __device__ __forceinline__ uint32_t mn3(uint32_t a, uint32_t b, uint32_t c) { return h2_minxs(h2_minxs(a, b), c); }
};
constexpr uint32_t kH2Sign = 0x80008000u, kH2Mag = 0x7fff7fffu;
constexpr uint32_t kH2Lim = 0x57f057f0u;    // +127.0 in both lanes
constexpr uint32_t kH2NegLim = 0xd7f0d7f0u; // -127.0
constexpr uint32_t kH2K1024 = 0x64006400u;  // +1024.0: adding it leaves an integer m < 1024 in the mantissa

template <int DC, bool UNIFORM>
__device__ __forceinline__ void check_step_h8(int c, int M, int deg, uint32_t pw, uint32_t *__restrict__ slots,
                                              const uint16_t *__restrict__ tab)
{
    uint32_t q[DC];
#pragma unroll
    for (int j = 0; j < DC; ++j)
        if (UNIFORM || j < deg) q[j] = slots[j * M + c];
    // two smallest magnitudes per lane (m2's sign is meaningless); m1's sign bits: the sign parity
    uint32_t m1, m2;
    if constexpr (UNIFORM && DC >= 2) {
        min2_tree<H2XsOps, 0, DC>(q, m1, m2);
    } else {
        m1 = m2 = 0x7c007c00u;   // +inf
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (UNIFORM || j < deg) {
                m2 = h2_minxs(m2, h2_maxxs(m1, q[j]));
                m1 = h2_minxs(m1, q[j]);
            }
        }
    }
    const uint32_t negb = (m1 ^ pw) & kH2Sign;   // per lane (-1)^{s_m} prod of the signs (pw bits 15 / 31: s_m)
    const uint32_t a1 = m1 & kH2Mag, a2 = m2 & kH2Mag;
    // |r| = floor(|m| alpha_q / 2^15) from the table, both lanes: 1024 + |m| puts |m| in the low bits
    const uint32_t t1 = h2_add(a1, kH2K1024), t2 = h2_add(a2, kH2K1024);
    const uint32_t r1 = (uint32_t(tab[t1 & 0x7fu]) | (uint32_t(tab[(t1 >> 16) & 0x7fu]) << 16)) ^ negb;
    const uint32_t r2 = (uint32_t(tab[t2 & 0x7fu]) | (uint32_t(tab[(t2 >> 16) & 0x7fu]) << 16)) ^ negb;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            const uint32_t at = h2_eq_mask(q[j] & kH2Mag, a1);   // the lane's |q| is the minimum: r2
            slots[j * M + c] = ((at & r2) | (~at & r1)) ^ (q[j] & kH2Sign);
        }
    }
}

template <int D, bool MASK>
__device__ __forceinline__ uint32_t var_step_h8(int u, int NV, const uint16_t *__restrict__ vchk, const uint16_t *__restrict__ vslot,
                                                uint32_t gamma, uint32_t Qold, uint32_t keep, uint32_t *__restrict__ slots,
                                                uint32_t *__restrict__ parity)
{
    if constexpr (D == 0) {
        return gamma;
    } else {
        uint32_t e[D], r[D];
#pragma unroll
        for (int k = 0; k < D; ++k) e[k] = __ldg(vslot + k * NV + u);
#pragma unroll
        for (int k = 0; k < D; ++k) r[k] = MASK ? slots[e[k]] & keep : slots[e[k]];   // restart: r = +0
        uint32_t pre[D + 1];
        pre[0] = gamma;
#pragma unroll
        for (int k = 0; k < D; ++k) pre[k + 1] = h2_add(pre[k], r[k]);
        const uint32_t Q = pre[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            uint32_t q = pre[k];
#pragma unroll
            for (int i = k + 1; i < D; ++i) q = h2_add(q, r[i]);
            slots[e[k]] = h2_max(h2_min(q, kH2Lim), kH2NegLim);
        }
        const uint32_t flip = ((Q ^ Qold) >> 15) & 0x00010001u;   // lane decisions that changed (bits 0 / 16)
        if (flip) {
#pragma unroll
            for (int k = 0; k < D; ++k) atomicXor(parity + __ldg(vchk + k * NV + u), flip);
        }
        return Q;
    }
}

struct PairH8 {      // two INT8 messages in half-precision lanes per 32-bit slot
    using word_t = uint32_t;
    using gam_t = uint32_t;   // FP16 bits: the prior in both lanes (quantize), or one lane's value (lane)
    using pair_t = uint32_t;
    static __device__ __forceinline__ gam_t quantize(float g)
    {
        const uint32_t h = __half_as_ushort(__int2half_rn(I8::quantize(g)));   // an integer in [-127, 127]: exact
        return h | (h << 16);
    }
    static __device__ __forceinline__ pair_t both(gam_t g) { return g; }
    static __device__ __forceinline__ gam_t lane(pair_t x, int l) { return l ? x >> 16 : x & 0xffffu; }
    static __device__ __forceinline__ bool neg(gam_t x) { return (x & 0x8000u) != 0u; }
    static __device__ __forceinline__ float post(gam_t x)
    {
        return __half2float(__ushort_as_half(uint16_t(x))) * 0.25f;   // the I8 value / 4, exact
    }
    static __device__ __forceinline__ uint16_t *table()
    {
        __shared__ uint16_t t[128];
        return t;
    }
    // the scale table: FP16 bits of floor(m alpha_q / 2^15), m = 0..127
    static __device__ __forceinline__ void setup(int tid, int T, const LaunchParams &p)
    {
        for (int m = tid; m < 128; m += T)
            table()[m] = __half_as_ushort(__int2half_rn(int((uint32_t(m) * uint32_t(p.alpha_q)) >> 15)));
    }
    template <int DC, bool UNIFORM>
    static __device__ __forceinline__ void check(int c, int M, int deg, uint32_t pw, word_t *slots, const LaunchParams &)
    {
        check_step_h8<DC, UNIFORM>(c, M, deg, pw, slots, table());
    }
    template <int D, bool MASK>
    static __device__ __forceinline__ pair_t var(int u, int NV, const CheckOf &ck, const uint16_t *vchk, const uint16_t *vslot,
                                                 gam_t gamma,
                                                 pair_t Qold, uint32_t act, word_t *slots, uint32_t *parity)
    {
        const uint32_t keep = ((act & 1u) ? 0x0000ffffu : 0u) | ((act & 2u) ? 0xffff0000u : 0u);
        (void)ck;
        return var_step_h8<D, MASK>(u, NV, vchk, vslot, gamma, Qold, keep, slots, parity);
    }
};

template <class PP, int DC, bool UNIFORM, int DV>
__global__ void __launch_bounds__(kPackedMaxThreads, 1) msa_packed_kernel(const __grid_constant__ LaunchParams p)
{
    const Problem pr = blockIdx.y == 0 ? p.prob[0] : p.prob[1];
    const DeviceGraph &G = p.prob[blockIdx.y].g;   // read in place (the class tables are indexed at run time)
    const int M = pr.g.m, N = pr.g.n, NV = pr.g.nv;
    const int T = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem[];
    using word_t = typename PP::word_t;
    using gam_t = typename PP::gam_t;
    using pair_t = typename PP::pair_t;
    const PackedLayout L = packed_layout(M, NV, pr.g.dc_max, int(sizeof(word_t)));
    gam_t *gam = reinterpret_cast<gam_t *>(smem + L.g_off);
    pair_t *Qs = reinterpret_cast<pair_t *>(smem + L.q_off);
    uint32_t *parity = reinterpret_cast<uint32_t *>(smem + L.par_off);
    word_t *slots = reinterpret_cast<word_t *>(smem + L.slot_off);
    __shared__ int s_claim[2];
    __shared__ uint32_t s_any[2];   // OR of the parity words' lane bits (alternating per iteration)

    int bad = 0;
    for (int u = tid; u < NV; u += T) {
        const uint32_t v = __ldg(pr.g.vperm + u);
        const float g = v < uint32_t(N) ? pr.prior[v] : 0.0f;
        bad |= !isfinite(g);
        gam[u] = PP::quantize(g);
        Qs[u] = PP::both(gam_t(0));     // the decisions a refill compares against: none set
    }
    for (int c = tid; c < M; c += T) parity[c] = 0u;
    if (tid < 2) s_any[tid] = 0u;
    PP::setup(tid, T, p);
    bad = __syncthreads_or(bad);
    if (bad) {   // non-finite prior: every shot of the launch is reported as not decoded
        for (;;) {
            if (tid == 0) s_claim[0] = atomicAdd(p.next_shot + blockIdx.y, 1);
            __syncthreads();
            const int b = s_claim[0];
            __syncthreads();
            if (b >= p.batch) return;
            for (int v = tid; v < N; v += T) {
                pr.err[size_t(b) * N + v] = 0;
                if (pr.post) pr.post[size_t(b) * N + v] = __int_as_float(0x7fc00000);
            }
            if (tid == 0) {
                pr.iters[b] = -1;
                pr.ok[b] = 0;
            }
        }
    }

    const bool early = (p.flags & kFlagNoEarlyStop) == 0;
    const CheckOf ck(pr.g);
    // Block-uniform lane state: shot of each lane (-1: idle), iterations run, the lanes whose var
    // step updates (act), the lanes that take a new shot in the next var step (refill), the lanes
    // whose finished shot the next var step writes out (out), and the lanes filled by the last var
    // step (fresh: the next check step installs their syndrome bits).
    int shot[2] = {-1, -1}, k[2] = {0, 0}, okl[2] = {0, 0};
    uint32_t act = 0u, refill = 3u, out = 0u, fresh = 0u, ph = 0u;
    // Shots are claimed one ahead: thread 0 holds each lane's next shot (pend), claimed when the
    // lane took its current one, and prefetches that shot's syndrome into L2 at the next variable
    // step, so neither the claim's round trip nor the syndrome's first read from DRAM stalls the
    // block at a refill.  (A lane's queue is one shot deep, so the order in which shots finish
    // changes, never a result.)
    int pend[2] = {0, 0};
    uint32_t pf = 0u;   // thread 0: lanes whose pending shot is still to be prefetched
    if (tid == 0) {
        pend[0] = atomicAdd(p.next_shot + blockIdx.y, 1);
        pend[1] = atomicAdd(p.next_shot + blockIdx.y, 1);
    }
    for (;;) {
        // ---- variable step: updates, outputs of finished shots, refills ----
        if (tid == 0 && pf) {
#pragma unroll
            for (int l = 0; l < 2; ++l)
                if ((pf & (1u << l)) && pend[l] < p.batch) {
                    const uint8_t *sp = pr.syn + size_t(pend[l]) * M;
                    for (int i = 0; i < M; i += 128) prefetch_l2(sp + i);
                    prefetch_l2(sp + M - 1);
                }
            pf = 0u;
        }
        // Finished shots are written out in variable order (consecutive threads, consecutive
        // variables: each warp store covers 32 adjacent bytes of e_hat), before the variable step
        // below overwrites Q.
        if (out) {
#pragma unroll 1
            for (int v = tid; v < N; v += T) {
                const pair_t Qo = Qs[__ldg(pr.g.vlane + v)];
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    if (out & (1u << l)) {
                        const gam_t q = PP::lane(Qo, l);
                        store_out(pr.err + size_t(shot[l]) * N + v, uint8_t(PP::neg(q) ? 1 : 0));
                        if (pr.post) store_out(pr.post + size_t(shot[l]) * N + v, PP::post(q));
                    }
                }
            }
            __syncthreads();
        }
        // Lanes come in classes of one degree (cls_end / cls_deg), walked in order along this
        // thread's lanes u = tid, tid + T, ...; within a class the degree is a compile-time constant.
        // Both lanes updating (no refill, no restart mask) is the common case.
        auto var_pass = [&](auto mask_tag) {
            constexpr bool MASK = decltype(mask_tag)::value;
            int u = tid;
            for (int cl = 0; cl < pr.g.ncls && u < NV; ++cl) {
                const int u1 = G.cls_end[cl];
                auto run = [&](auto deg_tag) {
                    constexpr int D = decltype(deg_tag)::value;
#pragma unroll 1
                    for (; u < u1; u += T)
                        Qs[u] = PP::template var<D, MASK>(u, NV, ck, pr.g.vchk16, pr.g.vslot16, gam[u], Qs[u], act, slots, parity);
                };
                switch (G.cls_deg[cl]) {
#define QLDPC_CASE(DD)                                                                          \
    case DD:                                                                                    \
        if constexpr (DD <= DV) run(std::integral_constant<int, DD>{});                         \
        break;
                    QLDPC_DEG_CASES(QLDPC_CASE)
#undef QLDPC_CASE
                default:   // a degree above the variant's bucket (the host never launches one)
                    while (u < u1) u += T;
                    break;
                }
            }
        };
        if (act == 3u)
            var_pass(std::false_type{});
        else
            var_pass(std::true_type{});
        if (tid == 0) {
            s_any[ph] = 0u;                           // the word the next check step reduces into
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                if (out & (1u << l)) {
                    pr.iters[shot[l]] = k[l];
                    pr.ok[shot[l]] = okl[l] ? 1 : 0;
                }
                if (refill & (1u << l)) {
                    s_claim[l] = pend[l];
                    pend[l] = atomicAdd(p.next_shot + blockIdx.y, 1);
                    pf |= 1u << l;
                }
            }
        }
        __syncthreads();
        fresh = 0u;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            if (refill & (1u << l)) {
                const int b = s_claim[l];
                shot[l] = b < p.batch ? b : -1;
                k[l] = 0;
                if (shot[l] >= 0) fresh |= 1u << l;
            } else if (act & (1u << l)) {
                ++k[l];
            }
        }
        if (shot[0] < 0 && shot[1] < 0) break;

        // ---- check step and stop test of both lanes ----
        const uint8_t *s0 = (fresh & 1u) ? pr.syn + size_t(shot[0]) * M : nullptr;
        const uint8_t *s1 = (fresh & 2u) ? pr.syn + size_t(shot[1]) * M : nullptr;
        // a new shot's syndrome bits of this thread's checks (check tid + i*T at bit i, i < 32), read
        // up front so that their loads overlap
        uint32_t sb0 = 0u, sb1 = 0u;
        if (fresh) {
#pragma unroll 4
            for (int c = tid, i = 0; c < M && i < 32; c += T, ++i) {
                if (s0) sb0 |= (uint32_t(s0[c]) & 1u) << i;
                if (s1) sb1 |= (uint32_t(s1[c]) & 1u) << i;
            }
        }
        uint32_t unsat = 0u;
        for (int c = tid, i = 0; c < M; c += T, ++i) {
            uint32_t pw = parity[c];
            if (fresh) {   // the new shots' syndrome bits replace the old ones (bit 0 and bit 15 / 16 and 31)
                if (s0) pw ^= (((pw >> 15) ^ (i < 32 ? sb0 >> i : uint32_t(s0[c]))) & 1u) * 0x00008001u;
                if (s1) pw ^= (((pw >> 31) ^ (i < 32 ? sb1 >> i : uint32_t(s1[c]))) & 1u) * 0x80010000u;
                parity[c] = pw;
            }
            unsat |= pw;
            PP::template check<DC, UNIFORM>(c, M, UNIFORM ? DC : int(__ldg(pr.g.rdeg + c)), pw, slots, p);
        }
        // block OR of both lanes' unsatisfied bits (bit 0 and bit 16): warp OR, one shared OR per warp
        const uint32_t wv = __reduce_or_sync(0xffffffffu, unsat & 0x00010001u);
        if ((tid & 31) == 0 && wv) atomicOr(&s_any[ph], wv);
        __syncthreads();
        const uint32_t any = s_any[ph];
        ph ^= 1u;
        out = refill = act = 0u;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            if (shot[l] < 0) continue;                // idle lane: keeps restarting from the prior
            const int met = ((any >> (16 * l)) & 1u) == 0u;
            if ((early && met) || k[l] >= p.max_iter) {
                okl[l] = met;
                out |= 1u << l;
                refill |= 1u << l;
            } else {
                act |= 1u << l;
            }
        }
    }
}

}  // namespace kern

// Instantiation tables of the packed kernel for one fixed-point policy (same variants as the other
// flooding kernels).
// DVLO..DVHI: the column-degree buckets instantiated for this policy (the others return nothing).
template <class PP, int DVLO = 0, int DVHI = 16>
const void *packed_table(const KernelChoice &kc)
{
#define QLDPC_K(DCV, UNI, DVV)                                                                  \
    if constexpr (DVV >= DVLO && DVV <= DVHI)                                                   \
        if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == DVV)                                 \
            return reinterpret_cast<const void *>(&kern::msa_packed_kernel<PP, DCV, UNI, DVV>);
    QLDPC_VARIANTS(QLDPC_K)
#undef QLDPC_K
    return nullptr;
}

template <class PP, int DVLO = 0, int DVHI = 16>
cudaError_t packed_launch(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads, size_t smem,
                          cudaStream_t stream)
{
#define QLDPC_L(DCV, UNI, DVV)                                                                  \
    if constexpr (DVV >= DVLO && DVV <= DVHI)                                                   \
        if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == DVV) {                               \
            kern::msa_packed_kernel<PP, DCV, UNI, DVV><<<grid, threads, smem, stream>>>(p);     \
            return cudaGetLastError();                                                          \
        }
    QLDPC_VARIANTS(QLDPC_L)
#undef QLDPC_L
    return cudaErrorInvalidValue;
}

}  // namespace qldpc
