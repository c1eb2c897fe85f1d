// Persistent decoding server: a resident kernel whose worker blocks take requests of any code from
// one arrival-ordered queue.
//
// The paper proposes launching decoders asynchronously so transfers overlap kernel execution
// (Table 1, Sec. 3 outlook).  On GB300 the lower-latency form is a kernel that never returns
// between requests: the host writes a syndrome into a slot of its code's ring in page-locked memory
// mapped into the GPU's address space (NVLink-C2C) and publishes the request by writing its entry
// (code, slot, arrival number) into the next position of a shared queue; a free worker block claims
// the oldest published entry (compare-and-swap on the queue's device-side head), decodes it with
// the single-shot algorithm of msa_latency_kernel, writes e_hat, iterations, ok and its own index
// into the slot and releases the slot's completion word.  No launch, copy or synchronize sits
// between a request and its result.
//
// Admission (continuous batching across codes): every worker has the same footprint, the largest
// any configured code needs (threads, shared memory, registers per thread for its edge lists), and
// as many workers run as fit on the GPU at that footprint, so a request starts as soon as any
// worker is free, whatever its code.  A worker keeps the per-thread state of the last code it
// decoded (edge lists, degrees, priors in registers) and reloads it from global memory (L1/L2
// resident) only when it takes a request of another code.
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
__device__ __forceinline__ uint64_t ld_acquire_sys64(const unsigned long long *p)
{
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
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

// Claim the oldest published request (thread 0 of a worker).  Returns its queue entry (code, slot
// and arrival number), or kQueueLeave when the worker must leave (stop flag, idle, time limit,
// spin cap).
__device__ __forceinline__ uint64_t claim_request(const ServerParams &sp, uint64_t t_start, uint64_t &t_idle_from)
{
    for (uint64_t spin = 0; spin < kServerMaxSpins; ++spin) {
        const uint32_t head = ld_relaxed_gpu(sp.head);
        const uint64_t e = ld_acquire_sys64(sp.queue + (head & sp.queue_mask));
        if (uint32_t(e >> 32) == head + 1u) {        // the entry at head is published
            if (atomicCAS(sp.head, head, head + 1u) == head) {
                t_idle_from = globaltimer();
                return e;
            }
            continue;                                 // another worker took it
        }
        if (ld_relaxed_sys(sp.stop)) {
            atomicOr(sp.status, kServerStopped);
            return kQueueLeave;
        }
        const uint64_t now = globaltimer();
        if (now - t_idle_from > sp.idle_ns) {
            atomicOr(sp.status, kServerIdleExit);
            return kQueueLeave;
        }
        if (now - t_start > sp.max_runtime_ns) {
            atomicOr(sp.status, kServerTimeLimit);
            return kQueueLeave;
        }
        __nanosleep(64);
    }
    atomicOr(sp.status, kServerSpinLimit);
    return kQueueLeave;
}

// Fields of a claimed entry; its high word (arrival number + 1) is the slot's completion word.
__device__ __forceinline__ int entry_code(uint64_t e) { return int(e >> kQueueCodeShift) & kQueueCodeMask; }
__device__ __forceinline__ uint32_t entry_slot(uint64_t e) { return uint32_t(e) & kQueueSlotMask; }
__device__ __forceinline__ uint32_t entry_done(uint64_t e) { return uint32_t(e >> 32); }

// Completion of a request (thread 0): iterations, ok and the worker's index into the slot header,
// then the completion word (the arrival number + 1) with a system-scope release.
__device__ __forceinline__ void publish_result(unsigned char *slot, int iters, int ok, uint32_t done)
{
    *reinterpret_cast<int32_t *>(slot + 4) = iters;
    slot[8] = ok ? 1 : 0;
    *reinterpret_cast<uint16_t *>(slot + 10) = uint16_t(blockIdx.x);
    __threadfence_system();
    st_release_sys(reinterpret_cast<uint32_t *>(slot), done);
}

// Per-thread state of one code in a flooding worker: the single-shot kernel's registers (degrees
// of the thread's checks; edge slots, degree, caller index and prior of its variable lanes).
template <class P, int DC, bool UNIFORM, int DV>
struct WorkerCode {
    int cdeg[kLatCnPerThread];
    uint32_t ev[kLatVnPerThread][DV];
    int vdeg[kLatVnPerThread], vid[kLatVnPerThread];
    typename P::acc_t gam[kLatVnPerThread];

    __device__ __forceinline__ void load(const ServerCode &sc, int tid, int T)
    {
        const int M = sc.g.m, N = sc.g.n, NV = sc.g.nv;
#pragma unroll
        for (int i = 0; i < kLatCnPerThread; ++i) {
            const int c = tid + i * T;
            cdeg[i] = c < M ? (UNIFORM ? DC : int(__ldg(sc.g.rdeg + c))) : -1;
        }
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
    }
};

// Check step and stop test of the thread's checks (tid + i*T) for rows of compiled degree D.
template <class P, int D, bool U, bool LEARNED>
__device__ __forceinline__ int server_checks(const int *cdeg, int tid, int T, int M, const uint32_t *parity, bool update,
                                             typename P::msg_t *slots, const LaunchParams &p, const float *wk)
{
    int ok = 1;
#pragma unroll
    for (int i = 0; i < kLatCnPerThread; ++i)
        if (cdeg[i] >= 0)
            ok &= check_step<P, D, U, LEARNED>(tid + i * T, M, cdeg[i], parity[tid + i * T], update, slots, p, wk);
    return ok;
}

// The check phase of one iteration.  A kernel compiled for rows of varying degree (a server whose
// codes differ in row degree) still runs each code whose rows all have one degree of 6..9 with that
// degree compiled in (pairwise minima, no per-edge predicates): the code is the same for the whole
// block, so the dispatch costs no divergence.
template <class P, int DC, bool UNIFORM, bool LEARNED>
__device__ __forceinline__ int server_check_phase(int udc, const int *cdeg, int tid, int T, int M,
                                                  const uint32_t *parity, bool update, typename P::msg_t *slots,
                                                  const LaunchParams &p, const float *wk)
{
    if constexpr (!UNIFORM) {
        switch (udc) {
        case 6: return server_checks<P, 6, true, LEARNED>(cdeg, tid, T, M, parity, update, slots, p, wk);
        case 7: return server_checks<P, 7, true, LEARNED>(cdeg, tid, T, M, parity, update, slots, p, wk);
        case 8: return server_checks<P, 8, true, LEARNED>(cdeg, tid, T, M, parity, update, slots, p, wk);
        case 9:
            if constexpr (DC >= 9) return server_checks<P, 9, true, LEARNED>(cdeg, tid, T, M, parity, update, slots, p, wk);
            break;
        default: break;
        }
    }
    return server_checks<P, DC, UNIFORM, LEARNED>(cdeg, tid, T, M, parity, update, slots, p, wk);
}

// LEARNED (FP32): a code with weights decodes as the learned batch/latency kernels do (learned
// iterations, then the plain fallback from the prior); a code without weights decodes plainly.
template <class P, int DC, bool UNIFORM, int DV, bool LEARNED = false>
__global__ void __launch_bounds__(kLatencyMaxThreads, 1) msa_server_kernel(const ServerParams sp)
{
    using acc_t = typename P::acc_t;
    using msg_t = typename P::msg_t;

    const int T = blockDim.x, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *parity = reinterpret_cast<uint32_t *>(smem);
    __shared__ uint64_t s_claim;

    LaunchParams p{};   // the arithmetic parameters the shared device functions read
    p.alpha = sp.alpha;
    p.alpha_q = sp.alpha_q;
    const bool early = (sp.flags & kFlagNoEarlyStop) == 0;

    // the code whose state the registers hold (-1: none yet) and its block-uniform parameters
    int cur = -1, M = 0, N = 0, learned_iters = 0, udc = 0;
    CheckOf ck;
    msg_t *slots = nullptr;
    const float *weights = nullptr;
    size_t wstride = 0;
    WorkerCode<P, DC, UNIFORM, DV> wc;

    const uint64_t t_start = globaltimer();
    uint64_t t_idle_from = t_start;
    for (;;) {
        if (tid == 0) s_claim = claim_request(sp, t_start, t_idle_from);
        __syncthreads();
        const uint64_t e = s_claim;
        if (e == kQueueLeave) break;
        const int code = entry_code(e);
        const ServerCode &sc = sp.code[code];
        unsigned char *slot = sc.ring + size_t(entry_slot(e)) * size_t(sc.slot_bytes);
        // The syndrome bits of the thread's checks, read from the host-memory slot once per request
        // and issued before the code's state is reloaded, so the two round trips overlap.
        uint32_t sbit[kLatCnPerThread];
#pragma unroll
        for (int i = 0; i < kLatCnPerThread; ++i) {
            const int c = tid + i * T;
            sbit[i] = c < sc.g.m ? uint32_t(__ldcv(slot + sc.syn_off + c)) & 1u : 0u;
        }
        if (code != cur) {
            cur = code;
            M = sc.g.m;
            N = sc.g.n;
            ck = CheckOf(sc.g);
            slots = reinterpret_cast<msg_t *>(smem + latency_layout(M, sc.g.dc_max, int(sizeof(msg_t))).slot_off);
            weights = LEARNED ? sc.weights : nullptr;
            learned_iters = sc.learned_iters;
            wstride = size_t(sc.g.dc_max) * M;
            udc = sc.udc;
            wc.load(sc, tid, T);
        }
        acc_t Q[kLatVnPerThread];
        // Initialization (Alg. 1), also the restart of the plain fallback; ends with a barrier.
        auto init_shot = [&]() {
#pragma unroll
            for (int i = 0; i < kLatCnPerThread; ++i)
                if (wc.cdeg[i] >= 0) parity[tid + i * T] = sbit[i] * 3u;
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kLatVnPerThread; ++i) {
                Q[i] = wc.gam[i];
                const bool d = P::neg(wc.gam[i]);
#pragma unroll
                for (int k = 0; k < DV; ++k) {
                    if (k < wc.vdeg[i]) {
                        slots[wc.ev[i][k]] = P::to_msg(wc.gam[i]);
                        if (d) flip_check(parity, ck(wc.ev[i][k]));
                    }
                }
            }
            __syncthreads();
        };
        init_shot();

        int k = 0, all = 0;
        bool learned = LEARNED && weights != nullptr;
        int end = learned ? learned_iters : sp.max_iter;
        for (;;) {
            const bool last = k >= end;
            const float *wk = nullptr;
            if constexpr (LEARNED) wk = (learned && !last) ? weights + size_t(k) * wstride : nullptr;
            const int ok = server_check_phase<P, DC, UNIFORM, LEARNED>(udc, wc.cdeg, tid, T, M, parity, !last, slots,
                                                                       p, wk);
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
                if (wc.vdeg[i] >= 0)
                    Q[i] = var_step_regs<P, DV>(wc.vdeg[i], wc.ev[i], ck, wc.gam[i], P::neg(Q[i]), slots, parity);
            __syncthreads();
            ++k;
        }

        unsigned char *err = slot + sc.err_off;
#pragma unroll
        for (int i = 0; i < kLatVnPerThread; ++i)
            if (wc.vid[i] < N) err[wc.vid[i]] = P::neg(Q[i]) ? 1 : 0;
        __syncthreads();
        if (tid == 0) publish_result(slot, k, all, entry_done(e));
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
