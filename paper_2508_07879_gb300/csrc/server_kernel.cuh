// Persistent decoding server: a resident kernel whose worker blocks poll per-code request rings.
//
// The paper proposes launching decoders asynchronously so transfers overlap kernel execution
// (Table 1, Sec. 3 outlook).  On GB300 the lower-latency form is a kernel that never returns
// between requests: the host writes a syndrome into a ring slot in page-locked memory mapped into
// the GPU's address space (NVLink-C2C), publishes it by bumping the ring's tail, and a worker
// block of that code claims it (compare-and-swap on the ring's head), decodes it with the
// single-shot algorithm of msa_latency_kernel (graph, priors and per-thread state resident in
// registers since the kernel started), writes e_hat, iterations and ok into the slot, and
// releases a completion word.  No launch, copy or synchronize sits between a request and its
// result.  Requests of different codes are served concurrently by the workers of each code, and
// a request is admitted as soon as a worker of its code is free (continuous batching).
//
// Every wait is bounded: a worker leaves when the host sets the stop flag, after idle_ns without
// a request, after max_runtime_ns, or at a spin-count cap, and records why in the status word.
// The host relaunches the kernel when requests arrive after the workers left.
#pragma once

#include "msa_kernel.cuh"

namespace qldpc {
namespace kern {

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_sys(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr uint64_t kServerMaxSpins = uint64_t(1) << 34;   // safety cap far beyond the time limits

// Claim the next published request of one code (thread 0 of a worker).  Returns its sequence
// number, or -1 when the worker must leave (stop flag, idle, time limit, spin cap).
__device__ __forceinline__ int64_t claim_request(const ServerCode &sc, const ServerParams &sp,
                                                 uint64_t t_start, uint64_t &t_idle_from)
{
    for (uint64_t spin = 0; spin < kServerMaxSpins; ++spin) {
        const uint32_t tail = ld_acquire_sys(sc.tail);
        const uint32_t head = atomicAdd(sc.head, 0u);
        if (head != tail) {                       // head never passes tail: a request is waiting
            if (atomicCAS(sc.head, head, head + 1u) == head) {
                t_idle_from = globaltimer();
                return int64_t(head);
            }
            continue;                             // another worker took it
        }
        if (ld_relaxed_sys(sp.stop)) {
            atomicOr(sp.status, kServerStopped);
            return -1;
        }
        const uint64_t now = globaltimer();
        if (now - t_idle_from > sp.idle_ns) {
            atomicOr(sp.status, kServerIdleExit);
            return -1;
        }
        if (now - t_start > sp.max_runtime_ns) {
            atomicOr(sp.status, kServerTimeLimit);
            return -1;
        }
        __nanosleep(64);
    }
    atomicOr(sp.status, kServerSpinLimit);
    return -1;
}

// LEARNED (FP32): a code with weights decodes as the learned batch/latency kernels do (learned
// iterations, then the plain fallback from the prior); a code without weights decodes plainly.
template <class P, int DC, bool UNIFORM, int DV, bool LEARNED = false>
__global__ void __launch_bounds__(kLatencyMaxThreads, 1) msa_server_kernel(const ServerParams sp)
{
    using acc_t = typename P::acc_t;
    using msg_t = typename P::msg_t;

    int ci = 0;
    while (ci + 1 < sp.ncodes && int(blockIdx.x) >= sp.code[ci + 1].first_block) ++ci;
    const ServerCode sc = sp.code[ci];
    const int M = sc.g.m, N = sc.g.n, NV = sc.g.nv;
    const int T = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem[];
    const LatencyLayout L = latency_layout(M, sc.g.dc_max, int(sizeof(msg_t)));
    uint32_t *parity = reinterpret_cast<uint32_t *>(smem + L.par_off);
    msg_t *slots = reinterpret_cast<msg_t *>(smem + L.slot_off);
    __shared__ int64_t s_claim;

    LaunchParams p{};   // the arithmetic parameters the shared device functions read
    p.alpha = sp.alpha;
    p.alpha_q = sp.alpha_q;

    int cdeg[kLatCnPerThread];
#pragma unroll
    for (int i = 0; i < kLatCnPerThread; ++i) {
        const int c = tid + i * T;
        cdeg[i] = c < M ? (UNIFORM ? DC : int(__ldg(sc.g.rdeg + c))) : -1;
    }
    uint32_t ev[kLatVnPerThread][DV];
    int vdeg[kLatVnPerThread], vid[kLatVnPerThread];
    acc_t gam[kLatVnPerThread];
#pragma unroll
    for (int i = 0; i < kLatVnPerThread; ++i) {
        const int u = tid + i * T;
        const int v = u < NV ? int(__ldg(sc.g.vperm + u)) : N;   // N: idle lane
        vid[i] = v;
        vdeg[i] = u < NV ? int(__ldg(sc.g.vdeg + u)) : -1;
#pragma unroll
        for (int k = 0; k < DV; ++k) ev[i][k] = (k < vdeg[i]) ? __ldg(sc.g.vslot + size_t(k) * NV + u) : 0u;
        gam[i] = P::quantize(v < N ? sc.prior[v] : 0.0f);
    }

    const bool early = (sp.flags & kFlagNoEarlyStop) == 0;
    const size_t wstride = size_t(sc.g.dc_max) * M;
    const uint64_t t_start = globaltimer();
    uint64_t t_idle_from = t_start;
    for (;;) {
        if (tid == 0) s_claim = claim_request(sc, sp, t_start, t_idle_from);
        __syncthreads();
        const int64_t h = s_claim;
        if (h < 0) break;
        unsigned char *slot = sc.ring + size_t(uint32_t(h) & uint32_t(sp.ring_capacity - 1)) * size_t(sc.slot_bytes);
        const unsigned char *syn = slot + sc.syn_off;
        acc_t Q[kLatVnPerThread];
        // Initialization (Alg. 1), also the restart of the plain fallback; ends with a barrier.
        auto init_shot = [&]() {
#pragma unroll
            for (int i = 0; i < kLatCnPerThread; ++i)
                if (cdeg[i] >= 0) parity[tid + i * T] = (__ldcv(syn + tid + i * T) & 1u) * 3u;
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kLatVnPerThread; ++i) {
                Q[i] = gam[i];
                const bool d = P::neg(gam[i]);
#pragma unroll
                for (int k = 0; k < DV; ++k) {
                    if (k < vdeg[i]) {
                        slots[ev[i][k]] = P::to_msg(gam[i]);
                        if (d) flip_check(parity, CheckOf(sc.g)(ev[i][k]));
                    }
                }
            }
            __syncthreads();
        };
        init_shot();

        int k = 0, all = 0;
        bool learned = LEARNED && sc.weights != nullptr;
        int end = learned ? sc.learned_iters : sp.max_iter;
        for (;;) {
            const bool last = k >= end;
            const float *wk = nullptr;
            if constexpr (LEARNED) wk = (learned && !last) ? sc.weights + size_t(k) * wstride : nullptr;
            int ok = 1;
#pragma unroll
            for (int i = 0; i < kLatCnPerThread; ++i)
                if (cdeg[i] >= 0)
                    ok &= check_step<P, DC, UNIFORM, LEARNED>(tid + i * T, M, cdeg[i], parity[tid + i * T], !last,
                                                              slots, p, wk);
            all = __syncthreads_and(ok);
            if ((early || learned) && all) break;
            if (last) {
                if (!learned) break;
                learned = false;                  // fallback: plain min-sum from the prior
                end = k + sp.max_iter;
                init_shot();
                continue;
            }
#pragma unroll
            for (int i = 0; i < kLatVnPerThread; ++i)
                if (vdeg[i] >= 0)
                    Q[i] = var_step_regs<P, DV>(vdeg[i], ev[i], CheckOf(sc.g), gam[i], P::neg(Q[i]), slots, parity);
            __syncthreads();
            ++k;
        }

        unsigned char *err = slot + sc.err_off;
#pragma unroll
        for (int i = 0; i < kLatVnPerThread; ++i)
            if (vid[i] < N) err[vid[i]] = P::neg(Q[i]) ? 1 : 0;
        __syncthreads();
        if (tid == 0) {
            *reinterpret_cast<int32_t *>(slot + 4) = k;
            slot[8] = all ? 1 : 0;
            __threadfence_system();
            st_release_sys(reinterpret_cast<uint32_t *>(slot), uint32_t(h) + 1u);
        }
    }
}

}  // namespace kern

template <class P, bool LEARNED>
const void *server_table(const KernelChoice &kc)
{
#define QLDPC_K(DCV, UNI, DVV)                                                                  \
    if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == DVV)                                     \
        return reinterpret_cast<const void *>(&kern::msa_server_kernel<P, DCV, UNI, DVV, LEARNED>);
    QLDPC_VARIANTS(QLDPC_K)
#undef QLDPC_K
    return nullptr;
}

template <class P, bool LEARNED>
cudaError_t server_launch(const ServerParams &sp, const KernelChoice &kc, int blocks, int threads, size_t smem,
                          cudaStream_t stream)
{
#define QLDPC_L(DCV, UNI, DVV)                                                                  \
    if (kc.dc == DCV && kc.uniform == UNI && kc.dvb == DVV) {                                   \
        kern::msa_server_kernel<P, DCV, UNI, DVV, LEARNED><<<blocks, threads, smem, stream>>>(sp); \
        return cudaGetLastError();                                                              \
    }
    QLDPC_VARIANTS(QLDPC_L)
#undef QLDPC_L
    return cudaErrorInvalidValue;
}

}  // namespace qldpc
