// INT8 fixed-point instantiations of the flooding min-sum decoder kernels (see msa_kernel.cuh):
// LLRs with 2 fractional bits, messages clamped to +-127, sums in 32 bits.
#include "msa_kernel.cuh"

namespace qldpc {

const void *msa_kernel_i8(const KernelChoice &kc) { return kernel_table<kern::I8>(kc); }

cudaError_t launch_msa_i8(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                          size_t smem, cudaStream_t stream)
{
    return launch_table<kern::I8>(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc
