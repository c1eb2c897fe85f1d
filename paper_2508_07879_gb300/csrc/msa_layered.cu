// Layered (row-serial) schedule of the normalized min-sum decoder, FP32, INT16 and INT8, for sm_103a.
//
// Algorithm 1 (Sec. 2 of arXiv 2508.07879) updates all checks from the previous iteration's
// messages (flooding).  The layered schedule applies the same check update to one check after
// another, each reading the a-posteriori LLRs already refreshed by the checks before it:
//   q_{m,n} = Q_n - r_{m,n};  r_{m,n} = (-1)^{s_m} prod_{j != n} sign(q_{m,j}) alpha min_{j != n} |q_{m,j}|;
//   Q_n = q_{m,n} + r_{m,n}        (checks in ascending index; then decisions and the stop test)
// Two checks that share no variable commute, so the host groups the checks into layers (a check's
// layer is one more than the largest layer of an earlier check it shares a variable with): the
// checks of a layer run in parallel, the layers in order, and every result is bit-identical to the
// strictly serial order.  One block per shot, persistent over the batch; per shot in shared memory:
// Q [n] (FP32, or INT32 for the fixed-point modes), the messages r in check-major slots (j*m + i),
// the syndrome bits.
// One barrier per layer, then a stop-test pass over all checks (block AND).
#include <cstdint>

#include <cuda_runtime.h>

#include "msa_kernel.cuh"

namespace qldpc {
namespace kern {

// One check of the layered schedule: q = Q - r_old, the min-sum update, Q = q + r_new.
template <class P, int DC, bool UNIFORM>
__device__ __forceinline__ void layered_check(int c, int M, int deg, uint32_t s_bit, typename P::acc_t *__restrict__ Q,
                                              typename P::msg_t *__restrict__ slots, const uint32_t *__restrict__ ecol,
                                              const LaunchParams &p)
{
    using acc_t = typename P::acc_t;
    using mag_t = typename P::mag_t;
    acc_t q[DC];
    uint32_t v[DC];
    uint32_t sx = 0;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            v[j] = __ldg(ecol + size_t(j) * M + c);
            q[j] = P::sub_q(Q[v[j]], load_msg<P>(slots, uint32_t(j * M + c)));
            sx ^= P::sign_word(q[j]);
        }
    }
    mag_t m1, m2;
    two_smallest<P, DC, UNIFORM>(q, deg, m1, m2);
    const uint32_t negall = (s_bit ^ (sx >> 31)) & 1u;
    const mag_t r1 = P::presign(P::scale(m1, p), negall), r2 = P::presign(P::scale(m2, p), negall);
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            const acc_t r = P::apply_sign(P::mag(q[j]) == m1 ? r2 : r1, q[j]);
            Q[v[j]] = P::add(q[j], r);
            slots[j * M + c] = P::to_msg(r);
        }
    }
}

// 1 iff the decisions [Q < 0] of check c's variables meet s_c.
template <class P, int DC, bool UNIFORM>
__device__ __forceinline__ int check_met(int c, int M, int deg, uint32_t s_bit, const typename P::acc_t *__restrict__ Q,
                                         const uint32_t *__restrict__ ecol)
{
    uint32_t par = s_bit;
#pragma unroll
    for (int j = 0; j < DC; ++j)
        if (UNIFORM || j < deg) par ^= P::neg(Q[__ldg(ecol + size_t(j) * M + c)]) ? 1u : 0u;
    return par == 0;
}

template <class P, int DC, bool UNIFORM>
__global__ void __launch_bounds__(1024, 1) msa_layered_kernel(const LaunchParams p)
{
    using acc_t = typename P::acc_t;
    using msg_t = typename P::msg_t;
    const Problem pr = blockIdx.y == 0 ? p.prob[0] : p.prob[1];
    const int M = pr.g.m, N = pr.g.n, L = pr.g.nlayers;
    const int T = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem[];
    const LayeredLayout lay = layered_layout(M, N, pr.g.dc_max, int(sizeof(msg_t)));
    acc_t *Q = reinterpret_cast<acc_t *>(smem + lay.q_off);
    msg_t *slots = reinterpret_cast<msg_t *>(smem + lay.slot_off);
    uint8_t *sb = smem + lay.s_off;

    int bad = 0;
    for (int v = tid; v < N; v += T) bad |= !isfinite(pr.prior[v]);
    bad = __syncthreads_or(bad);
    const bool early = (p.flags & kFlagNoEarlyStop) == 0;
    __shared__ int s_shot[2];   // alternating claim words, as in the batch kernel
    int claim = 0;
    for (int b = blockIdx.x;; b += gridDim.x) {
        if (p.next_shot) {   // dynamic claiming from a per-launch counter
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
        // Q = gamma, r = 0, syndrome bits
        for (int v = tid; v < N; v += T) Q[v] = P::quantize(pr.prior[v]);
        for (int c = tid; c < M; c += T) {
            sb[c] = s[c] & 1u;
            const int deg = UNIFORM ? DC : int(__ldg(pr.g.rdeg + c));
            for (int j = 0; j < deg; ++j) slots[j * M + c] = msg_t(0);
        }
        __syncthreads();
        int ok = 1;
        for (int c = tid; c < M; c += T)
            ok &= check_met<P, DC, UNIFORM>(c, M, UNIFORM ? DC : int(__ldg(pr.g.rdeg + c)), sb[c], Q, pr.g.ecol);
        int all = __syncthreads_and(ok);
        int k = 0;
        if (!(early && all)) {
            for (k = 1; k <= p.max_iter; ++k) {
                for (int l = 0; l < L; ++l) {
                    const int lo = __ldg(pr.g.layer_ptr + l), hi = __ldg(pr.g.layer_ptr + l + 1);
                    for (int i = lo + tid; i < hi; i += T) {
                        const int c = int(__ldg(pr.g.layer_chk + i));
                        layered_check<P, DC, UNIFORM>(c, M, UNIFORM ? DC : int(__ldg(pr.g.rdeg + c)), sb[c], Q, slots,
                                                      pr.g.ecol, p);
                    }
                    __syncthreads();
                }
                ok = 1;
                for (int c = tid; c < M; c += T)
                    ok &= check_met<P, DC, UNIFORM>(c, M, UNIFORM ? DC : int(__ldg(pr.g.rdeg + c)), sb[c], Q,
                                                    pr.g.ecol);
                all = __syncthreads_and(ok);
                if (early && all) break;
            }
            if (k > p.max_iter) k = p.max_iter;
        }
        for (int v = tid; v < N; v += T) {
            err[v] = P::neg(Q[v]) ? 1 : 0;
            if (pr.post) pr.post[size_t(b) * N + v] = P::post(Q[v]);
        }
        if (tid == 0) {
            pr.iters[b] = k;
            pr.ok[b] = all ? 1 : 0;
        }
        __syncthreads();   // the next shot reuses shared memory
    }
}

// Register-resident variant for graphs with at most MAXL layers and rows of degree <= DC: thread t
// owns check t of every layer (at most one per layer), and keeps that check's variable indices and
// messages in registers across iterations, so an iteration touches shared memory only for Q.
// Arithmetic and order are those of msa_layered_kernel.
template <class P, int DC, bool UNIFORM, int MAXL>
__global__ void __launch_bounds__(256, 1) msa_layered_reg_kernel(const LaunchParams p)
{
    using acc_t = typename P::acc_t;
    using mag_t = typename P::mag_t;
    const Problem pr = blockIdx.y == 0 ? p.prob[0] : p.prob[1];
    const int M = pr.g.m, N = pr.g.n, L = pr.g.nlayers;
    const int T = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem[];
    acc_t *Q = reinterpret_cast<acc_t *>(smem);

    // ownership: check myc[l] of layer l (or -1), its degree and variables (two 16-bit indices per word)
    int myc[MAXL], mdeg[MAXL];
    uint32_t ev[MAXL][(DC + 1) / 2];
    acc_t r[MAXL][DC];
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        myc[l] = -1;
        mdeg[l] = 0;
        if (l < L) {
            const int i = __ldg(pr.g.layer_ptr + l) + tid;
            if (i < __ldg(pr.g.layer_ptr + l + 1)) {
                myc[l] = int(__ldg(pr.g.layer_chk + i));
                mdeg[l] = UNIFORM ? DC : int(__ldg(pr.g.rdeg + myc[l]));
            }
        }
#pragma unroll
        for (int j = 0; j < DC; j += 2) {
            uint32_t lo = 0, hi = 0;
            if (j < mdeg[l]) lo = __ldg(pr.g.ecol + size_t(j) * M + myc[l]);
            if (j + 1 < DC && j + 1 < mdeg[l]) hi = __ldg(pr.g.ecol + size_t(j + 1) * M + myc[l]);
            ev[l][j / 2] = lo | (hi << 16);
        }
    }

    int bad = 0;
    for (int v = tid; v < N; v += T) bad |= !isfinite(pr.prior[v]);
    bad = __syncthreads_or(bad);
    const bool early = (p.flags & kFlagNoEarlyStop) == 0;
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
        if (bad) {
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
        uint32_t sbits = 0;
#pragma unroll
        for (int l = 0; l < MAXL; ++l) {
            if (myc[l] >= 0) sbits |= uint32_t(s[myc[l]] & 1u) << l;
#pragma unroll
            for (int j = 0; j < DC; ++j) r[l][j] = acc_t(0);
        }
        for (int v = tid; v < N; v += T) Q[v] = P::quantize(pr.prior[v]);
        __syncthreads();
        // stop test over the thread's own checks
        auto met = [&]() {
            int ok = 1;
#pragma unroll
            for (int l = 0; l < MAXL; ++l) {
                if (myc[l] >= 0) {
                    uint32_t par = (sbits >> l) & 1u;
#pragma unroll
                    for (int j = 0; j < DC; ++j)
                        if (UNIFORM || j < mdeg[l]) par ^= P::neg(Q[(ev[l][j / 2] >> (16 * (j & 1))) & 0xffffu]) ? 1u : 0u;
                    ok &= par == 0;
                }
            }
            return ok;
        };
        int all = __syncthreads_and(met());
        int k = 0;
        if (!(early && all)) {
            for (k = 1; k <= p.max_iter; ++k) {
#pragma unroll
                for (int l = 0; l < MAXL; ++l) {
                    if (l < L) {
                        if (myc[l] >= 0) {
                            acc_t q[DC];
                            uint32_t v[DC];
                            uint32_t sx = 0;
#pragma unroll
                            for (int j = 0; j < DC; ++j) {
                                if (UNIFORM || j < mdeg[l]) {
                                    v[j] = (ev[l][j / 2] >> (16 * (j & 1))) & 0xffffu;
                                    q[j] = P::sub_q(Q[v[j]], r[l][j]);
                                    sx ^= P::sign_word(q[j]);
                                }
                            }
                            mag_t m1, m2;
                            two_smallest<P, DC, UNIFORM>(q, mdeg[l], m1, m2);
                            const uint32_t negall = (((sbits >> l) & 1u) ^ (sx >> 31)) & 1u;
                            const mag_t r1 = P::presign(P::scale(m1, p), negall);
                            const mag_t r2 = P::presign(P::scale(m2, p), negall);
#pragma unroll
                            for (int j = 0; j < DC; ++j) {
                                if (UNIFORM || j < mdeg[l]) {
                                    r[l][j] = P::apply_sign(P::mag(q[j]) == m1 ? r2 : r1, q[j]);
                                    Q[v[j]] = P::add(q[j], r[l][j]);
                                }
                            }
                        }
                        __syncthreads();
                    }
                }
                all = __syncthreads_and(met());
                if (early && all) break;
            }
            if (k > p.max_iter) k = p.max_iter;
        }
        for (int v = tid; v < N; v += T) {
            err[v] = P::neg(Q[v]) ? 1 : 0;
            if (pr.post) pr.post[size_t(b) * N + v] = P::post(Q[v]);
        }
        if (tid == 0) {
            pr.iters[b] = k;
            pr.ok[b] = all ? 1 : 0;
        }
        __syncthreads();   // the next shot reuses shared memory
    }
}

}  // namespace kern

#define QLDPC_LAYERED_VARIANTS(X) X(6, true) X(7, true) X(8, true) X(9, true) X(8, false) X(16, false) X(32, false)

// Register-resident variants (at most 8 layers, rows of degree <= 8); KernelChoice::dvb = 1 selects them.
#define QLDPC_LAYERED_REG_VARIANTS(X) X(6, true) X(7, true) X(8, true) X(8, false)
constexpr int kLayeredRegMaxLayers = 8;

template <class P>
const void *layered_table(const KernelChoice &kc)
{
#define QLDPC_K(DCV, UNI)                                                                       \
    if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == 0) return reinterpret_cast<const void *>(&kern::msa_layered_kernel<P, DCV, UNI>);
    QLDPC_LAYERED_VARIANTS(QLDPC_K)
#undef QLDPC_K
#define QLDPC_K(DCV, UNI)                                                                       \
    if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == 1)                                       \
        return reinterpret_cast<const void *>(&kern::msa_layered_reg_kernel<P, DCV, UNI, kLayeredRegMaxLayers>);
    QLDPC_LAYERED_REG_VARIANTS(QLDPC_K)
#undef QLDPC_K
    return nullptr;
}

template <class P>
cudaError_t layered_launch(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads, size_t smem,
                           cudaStream_t stream)
{
#define QLDPC_L(DCV, UNI)                                                                       \
    if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == 0) {                                     \
        kern::msa_layered_kernel<P, DCV, UNI><<<grid, threads, smem, stream>>>(p);              \
        return cudaGetLastError();                                                              \
    }
    QLDPC_LAYERED_VARIANTS(QLDPC_L)
#undef QLDPC_L
#define QLDPC_L(DCV, UNI)                                                                       \
    if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == 1) {                                     \
        kern::msa_layered_reg_kernel<P, DCV, UNI, kLayeredRegMaxLayers><<<grid, threads, smem, stream>>>(p); \
        return cudaGetLastError();                                                              \
    }
    QLDPC_LAYERED_REG_VARIANTS(QLDPC_L)
#undef QLDPC_L
    return cudaErrorInvalidValue;
}

const void *msa_kernel_layered(int precision, const KernelChoice &kc)
{
    return precision == kINT16 ? layered_table<kern::I16>(kc)
           : precision == kINT8 ? layered_table<kern::I8>(kc)
                                : layered_table<kern::F32>(kc);
}

cudaError_t launch_msa_layered(int precision, const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                               size_t smem, cudaStream_t stream)
{
    return precision == kINT16 ? layered_launch<kern::I16>(p, kc, grid, threads, smem, stream)
           : precision == kINT8 ? layered_launch<kern::I8>(p, kc, grid, threads, smem, stream)
                                : layered_launch<kern::F32>(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc
