// FP32 instantiations of the flooding min-sum decoder kernels (see msa_kernel.cuh).
#include "msa_kernel.cuh"

namespace qldpc {

const void *msa_kernel_f32(const KernelChoice &kc) { return kernel_table<kern::F32>(kc); }

cudaError_t launch_msa_f32(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                           size_t smem, cudaStream_t stream)
{
    return launch_table<kern::F32>(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc
