// Learned (neural) normalized min-sum decoding, FP32: the batch and latency kernels of
// msa_kernel.cuh with per-edge, per-iteration weights in place of alpha for the first
// learned_iters iterations and a plain min-sum fallback from the prior for unconverged shots.
#include "msa_kernel.cuh"

namespace qldpc {

const void *msa_kernel_learned(const KernelChoice &kc) { return kernel_table<kern::F32, true>(kc); }

cudaError_t launch_msa_learned(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                               size_t smem, cudaStream_t stream)
{
    return launch_table<kern::F32, true>(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc
