// Layered (row-serial) schedule of the normalized min-sum decoder, FP32, INT16 and INT8, for sm_103a.
//
// Algorithm 1 (Sec. 2 of arXiv 2508.07879) updates all checks from the previous iteration's
// messages (flooding).  The layered schedule applies the same check update to one check after
// another, each reading the a-posteriori LLRs already refreshed by the checks before it:
//   q_{m,n} = Q_n - r_{m,n};  r_{m,n} = (-1)^{s_m} prod_{j != n} sign(q_{m,j}) alpha min_{j != n} |q_{m,j}|;
//   Q_n = Q_n - r_old + r_new      (checks in ascending index; then decisions and the stop test)
// In fixed point Q is the exact 32-bit sum gamma + sum r of Algorithm 1's APP step and only the
// check's input q is clamped to the message range.
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
#include "server_kernel.cuh"

namespace qldpc {
namespace kern {

// One check of the layered schedule: Q - r_old, the min-sum update of q = clamp(Q - r_old),
// Q = (Q - r_old) + r_new.
template <class P, int DC, bool UNIFORM>
__device__ __forceinline__ void layered_check(int c, int M, int deg, uint32_t s_bit, typename P::acc_t *__restrict__ Q,
                                              typename P::msg_t *__restrict__ slots, const uint32_t *__restrict__ ecol,
                                              const LaunchParams &p)
{
    using acc_t = typename P::acc_t;
    using mag_t = typename P::mag_t;
    acc_t qu[DC], q[DC];
    uint32_t v[DC];
    uint32_t sx = 0;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            v[j] = __ldg(ecol + size_t(j) * M + c);
            qu[j] = P::sub(Q[v[j]], load_msg<P>(slots, uint32_t(j * M + c)));
            q[j] = P::clampq(qu[j]);
        }
    }
    mag_t m1, m2;
    row_minima<P, DC, UNIFORM>(q, deg, m1, m2, sx);
    const uint32_t negall = (s_bit ^ (sx >> 31)) & 1u;
    const mag_t r1 = P::presign(P::scale(m1, p), negall), r2 = P::presign(P::scale(m2, p), negall);
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        if (UNIFORM || j < deg) {
            const acc_t r = P::apply_sign(P::mag(q[j]) == m1 ? r2 : r1, q[j]);
            Q[v[j]] = P::add(qu[j], r);
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

// One shot on the shared-memory layout: Q [n] starts at the quantized priors, the messages at zero,
// sb [m] takes the syndrome bits syn(c).  Runs the layers of every iteration with one barrier each and
// the stop test after the last, and returns the iterations run (all = every check satisfied).  Ends
// with Q final and visible to the block.
template <class P, int DC, bool UNIFORM, class Syn>
__device__ __forceinline__ int layered_smem_shot(const DeviceGraph &g, int tid, int T, Syn syn,
                                                 const float *__restrict__ prior, typename P::acc_t *__restrict__ Q,
                                                 typename P::msg_t *__restrict__ slots, uint8_t *__restrict__ sb,
                                                 const LaunchParams &p, bool early, int &all)
{
    using msg_t = typename P::msg_t;
    const int M = g.m, N = g.n, L = g.nlayers;
    for (int v = tid; v < N; v += T) Q[v] = P::quantize(prior[v]);
    for (int c = tid; c < M; c += T) {
        sb[c] = syn(c) & 1u;
        const int deg = UNIFORM ? DC : int(__ldg(g.rdeg + c));
        for (int j = 0; j < deg; ++j) slots[j * M + c] = msg_t(0);
    }
    __syncthreads();
    int ok = 1;
    for (int c = tid; c < M; c += T)
        ok &= check_met<P, DC, UNIFORM>(c, M, UNIFORM ? DC : int(__ldg(g.rdeg + c)), sb[c], Q, g.ecol);
    all = __syncthreads_and(ok);
    int k = 0;
    if (!(early && all)) {
        for (k = 1; k <= p.max_iter; ++k) {
            for (int l = 0; l < L; ++l) {
                const int lo = __ldg(g.layer_ptr + l), hi = __ldg(g.layer_ptr + l + 1);
                for (int i = lo + tid; i < hi; i += T) {
                    const int c = int(__ldg(g.layer_chk + i));
                    layered_check<P, DC, UNIFORM>(c, M, UNIFORM ? DC : int(__ldg(g.rdeg + c)), sb[c], Q, slots,
                                                  g.ecol, p);
                }
                __syncthreads();
            }
            ok = 1;
            for (int c = tid; c < M; c += T)
                ok &= check_met<P, DC, UNIFORM>(c, M, UNIFORM ? DC : int(__ldg(g.rdeg + c)), sb[c], Q, g.ecol);
            all = __syncthreads_and(ok);
            if (early && all) break;
        }
        if (k > p.max_iter) k = p.max_iter;
    }
    return k;
}

template <class P, int DC, bool UNIFORM>
__global__ void __launch_bounds__(1024, 1) msa_layered_kernel(const LaunchParams p)
{
    using acc_t = typename P::acc_t;
    using msg_t = typename P::msg_t;
    const Problem pr = blockIdx.y == 0 ? p.prob[0] : p.prob[1];
    const int M = pr.g.m, N = pr.g.n;
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
        int all = 0;
        const int k = layered_smem_shot<P, DC, UNIFORM>(pr.g, tid, T, [&](int c) { return uint32_t(s[c]); }, pr.prior,
                                                        Q, slots, sb, p, early, all);
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
template <int DC, int MAXL>
struct LayeredOwned {
    int myc[MAXL], mdeg[MAXL];           // check of layer l owned by this thread (or -1), its degree
    uint32_t ev[MAXL][(DC + 1) / 2];     // its variables, two 16-bit indices per word
};

template <int DC, bool UNIFORM, int MAXL>
__device__ __forceinline__ void layered_own(const DeviceGraph &g, int tid, LayeredOwned<DC, MAXL> &o)
{
    const int M = g.m, L = g.nlayers;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        o.myc[l] = -1;
        o.mdeg[l] = 0;
        if (l < L) {
            const int i = __ldg(g.layer_ptr + l) + tid;
            if (i < __ldg(g.layer_ptr + l + 1)) {
                o.myc[l] = int(__ldg(g.layer_chk + i));
                o.mdeg[l] = UNIFORM ? DC : int(__ldg(g.rdeg + o.myc[l]));
            }
        }
#pragma unroll
        for (int j = 0; j < DC; j += 2) {
            uint32_t lo = 0, hi = 0;
            if (j < o.mdeg[l]) lo = __ldg(g.ecol + size_t(j) * M + o.myc[l]);
            if (j + 1 < DC && j + 1 < o.mdeg[l]) hi = __ldg(g.ecol + size_t(j + 1) * M + o.myc[l]);
            o.ev[l][j / 2] = lo | (hi << 16);
        }
    }
}

// One shot: Q [n] (shared) starts at the quantized priors, the messages at zero; syn(c) reads s_c.
// Runs the layers of every iteration with one barrier each and the stop test after the last, and
// returns the iterations run (all = every check satisfied).  Ends with Q final and visible to the
// block.  D <= DC: the row degree compiled into the loops (UNIFORM: every row has exactly D edges).
template <class P, int DC, int D, bool UNIFORM, int MAXL, class Syn>
__device__ __forceinline__ int layered_reg_shot(const LayeredOwned<DC, MAXL> &o, int L, int N, int tid, int T,
                                                Syn syn, const float *__restrict__ prior,
                                                typename P::acc_t *__restrict__ Q, const LaunchParams &p,
                                                bool early, int &all)
{
    static_assert(D <= DC, "compiled degree above the owned-check layout");
    using acc_t = typename P::acc_t;
    using mag_t = typename P::mag_t;
    acc_t r[MAXL][D];
    uint32_t sbits = 0;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        if (o.myc[l] >= 0) sbits |= (syn(o.myc[l]) & 1u) << l;
#pragma unroll
        for (int j = 0; j < D; ++j) r[l][j] = acc_t(0);
    }
    for (int v = tid; v < N; v += T) Q[v] = P::quantize(prior[v]);
    __syncthreads();
    // stop test over the thread's own checks
    auto met = [&]() {
        int ok = 1;
#pragma unroll
        for (int l = 0; l < MAXL; ++l) {
            if (o.myc[l] >= 0) {
                uint32_t par = (sbits >> l) & 1u;
#pragma unroll
                for (int j = 0; j < D; ++j)
                    if (UNIFORM || j < o.mdeg[l]) par ^= P::neg(Q[(o.ev[l][j / 2] >> (16 * (j & 1))) & 0xffffu]) ? 1u : 0u;
                ok &= par == 0;
            }
        }
        return ok;
    };
    all = __syncthreads_and(met());
    int k = 0;
    if (!(early && all)) {
        for (k = 1; k <= p.max_iter; ++k) {
#pragma unroll
            for (int l = 0; l < MAXL; ++l) {
                if (l < L) {
                    if (o.myc[l] >= 0) {
                        acc_t qu[D], q[D];
                        uint32_t v[D];
                        uint32_t sx = 0;
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            if (UNIFORM || j < o.mdeg[l]) {
                                v[j] = (o.ev[l][j / 2] >> (16 * (j & 1))) & 0xffffu;
                                qu[j] = P::sub(Q[v[j]], r[l][j]);
                                q[j] = P::clampq(qu[j]);
                            }
                        }
                        mag_t m1, m2;
                        row_minima<P, D, UNIFORM>(q, o.mdeg[l], m1, m2, sx);
                        const uint32_t negall = (((sbits >> l) & 1u) ^ (sx >> 31)) & 1u;
                        const mag_t r1 = P::presign(P::scale(m1, p), negall);
                        const mag_t r2 = P::presign(P::scale(m2, p), negall);
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            if (UNIFORM || j < o.mdeg[l]) {
                                r[l][j] = P::apply_sign(P::mag(q[j]) == m1 ? r2 : r1, q[j]);
                                Q[v[j]] = P::add(qu[j], r[l][j]);
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
    return k;
}

template <class P, int DC, bool UNIFORM, int MAXL>
__global__ void __launch_bounds__(256, 1) msa_layered_reg_kernel(const LaunchParams p)
{
    using acc_t = typename P::acc_t;
    const Problem pr = blockIdx.y == 0 ? p.prob[0] : p.prob[1];
    const int M = pr.g.m, N = pr.g.n, L = pr.g.nlayers;
    const int T = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem[];
    acc_t *Q = reinterpret_cast<acc_t *>(smem);

    LayeredOwned<DC, MAXL> own;
    layered_own<DC, UNIFORM, MAXL>(pr.g, tid, own);

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
        int all = 0;
        const int k = layered_reg_shot<P, DC, DC, UNIFORM, MAXL>(own, L, N, tid, T, [&](int c) { return uint32_t(s[c]); },
                                                                 pr.prior, Q, p, early, all);
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

// Persistent server worker on the layered schedule (QLDPC_LAYERED in the server's flags): the claim,
// publish and leave protocol of msa_server_kernel around one layered shot per request.  A code of at
// most MAXL layers runs layered_reg_shot (each thread owns one check per layer in registers, reloaded
// when the worker takes a request of another code); a code with more layers runs layered_smem_shot
// (messages in shared memory).  Results are those of msa_layered_kernel either way.
template <class P, int DC, bool UNIFORM, int MAXL>
__global__ void __launch_bounds__(256, 1) msa_server_layered_kernel(const ServerParams sp)
{
    using acc_t = typename P::acc_t;
    using msg_t = typename P::msg_t;
    const int T = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem[];
    acc_t *Q = reinterpret_cast<acc_t *>(smem);
    __shared__ uint64_t s_claim;

    LaunchParams p{};   // the arithmetic parameters the shared device functions read
    p.alpha = sp.alpha;
    p.alpha_q = sp.alpha_q;
    p.max_iter = sp.max_iter;
    p.flags = sp.flags;
    const bool early = (sp.flags & kFlagNoEarlyStop) == 0;

    int cur = -1;
    LayeredOwned<DC, MAXL> own;

    const uint64_t t_start = globaltimer();
    uint64_t t_idle_from = t_start;
    for (;;) {
        if (tid == 0) s_claim = claim_request(sp, t_start, t_idle_from);
        __syncthreads();
        const uint64_t e = s_claim;
        if (e == kQueueLeave) break;
        const int code = entry_code(e);
        const ServerCode &sc = sp.code[code];
        const bool reg = sc.layered_reg != 0;
        if (reg && code != cur) {
            layered_own<DC, UNIFORM, MAXL>(sc.g, tid, own);
            cur = code;
        }
        unsigned char *slot = sc.ring + size_t(entry_slot(e)) * size_t(sc.slot_bytes);
        const unsigned char *syn = slot + sc.syn_off;
        auto syn_bit = [&](int c) { return uint32_t(__ldcv(syn + c)); };
        const int N = sc.g.n;
        int all = 0, k;
        // a server whose codes differ in row degree still runs a code whose rows all have degree 6, 7
        // or 8 with that degree compiled in (block-uniform dispatch, no divergence)
        const int L = sc.g.nlayers;
        if (reg) {
            bool done = false;
            if constexpr (!UNIFORM && DC >= 8) {
                done = true;
                switch (sc.udc) {
                case 6: k = layered_reg_shot<P, DC, 6, true, MAXL>(own, L, N, tid, T, syn_bit, sc.prior, Q, p, early, all); break;
                case 7: k = layered_reg_shot<P, DC, 7, true, MAXL>(own, L, N, tid, T, syn_bit, sc.prior, Q, p, early, all); break;
                case 8: k = layered_reg_shot<P, DC, 8, true, MAXL>(own, L, N, tid, T, syn_bit, sc.prior, Q, p, early, all); break;
                default: done = false; break;
                }
            }
            if (!done)
                k = layered_reg_shot<P, DC, DC, UNIFORM, MAXL>(own, L, N, tid, T, syn_bit, sc.prior, Q, p, early, all);
        } else {
            const LayeredLayout lay = layered_layout(sc.g.m, N, sc.g.dc_max, int(sizeof(msg_t)));
            msg_t *slots = reinterpret_cast<msg_t *>(smem + lay.slot_off);
            uint8_t *sb = smem + lay.s_off;
            bool done = false;
            if constexpr (!UNIFORM && DC >= 8) {
                done = true;
                switch (sc.udc) {
                case 6: k = layered_smem_shot<P, 6, true>(sc.g, tid, T, syn_bit, sc.prior, Q, slots, sb, p, early, all); break;
                case 7: k = layered_smem_shot<P, 7, true>(sc.g, tid, T, syn_bit, sc.prior, Q, slots, sb, p, early, all); break;
                case 8: k = layered_smem_shot<P, 8, true>(sc.g, tid, T, syn_bit, sc.prior, Q, slots, sb, p, early, all); break;
                default: done = false; break;
                }
            }
            if (!done)
                k = layered_smem_shot<P, DC, UNIFORM>(sc.g, tid, T, syn_bit, sc.prior, Q, slots, sb, p, early, all);
        }
        unsigned char *err = slot + sc.err_off;
        for (int v = tid; v < N; v += T) err[v] = P::neg(Q[v]) ? 1 : 0;
        __syncthreads();
        if (tid == 0) publish_result(slot, k, all, entry_done(e));
    }
}

}  // namespace kern

#define QLDPC_LAYERED_VARIANTS(X) X(6, true) X(7, true) X(8, true) X(9, true) X(8, false) X(16, false) X(32, false)

// Register-resident variants (at most 8 layers, rows of degree <= 8); KernelChoice::dvb = 1 selects them.
#define QLDPC_LAYERED_REG_VARIANTS(X) X(6, true) X(7, true) X(8, true) X(8, false)
constexpr int kLayeredRegMaxLayers = 8;
static_assert(kLayeredRegMaxLayers == kLayeredServerMaxLayers, "the server workers use the register-resident layout");

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

template <class P>
const void *server_layered_table(const KernelChoice &kc)
{
#define QLDPC_K(DCV, UNI)                                                                       \
    if (kc.dc == DCV && kc.uniform == UNI)                                                      \
        return reinterpret_cast<const void *>(&kern::msa_server_layered_kernel<P, DCV, UNI, kLayeredRegMaxLayers>);
    QLDPC_LAYERED_REG_VARIANTS(QLDPC_K)
#undef QLDPC_K
    return nullptr;
}

template <class P>
cudaError_t server_layered_launch(const ServerParams &sp, const KernelChoice &kc, int blocks, int threads, size_t smem,
                                  cudaStream_t stream)
{
#define QLDPC_L(DCV, UNI)                                                                       \
    if (kc.dc == DCV && kc.uniform == UNI) {                                                    \
        kern::msa_server_layered_kernel<P, DCV, UNI, kLayeredRegMaxLayers><<<blocks, threads, smem, stream>>>(sp); \
        return cudaGetLastError();                                                              \
    }
    QLDPC_LAYERED_REG_VARIANTS(QLDPC_L)
#undef QLDPC_L
    return cudaErrorInvalidValue;
}

const void *server_kernel_layered(int precision, const KernelChoice &kc)
{
    return precision == kINT16 ? server_layered_table<kern::I16>(kc)
           : precision == kINT8 ? server_layered_table<kern::I8>(kc)
                                : server_layered_table<kern::F32>(kc);
}

cudaError_t launch_server_layered(int precision, const ServerParams &sp, const KernelChoice &kc, int blocks,
                                  int threads, size_t smem, cudaStream_t stream)
{
    return precision == kINT16 ? server_layered_launch<kern::I16>(sp, kc, blocks, threads, smem, stream)
           : precision == kINT8 ? server_layered_launch<kern::I8>(sp, kc, blocks, threads, smem, stream)
                                : server_layered_launch<kern::F32>(sp, kc, blocks, threads, smem, stream);
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
