// INT16 fixed-point instantiations of the flooding min-sum decoder kernels (see msa_kernel.cuh).
#include "msa_kernel.cuh"

namespace qldpc {

const void *msa_kernel_i16(const KernelChoice &kc) { return kernel_table<kern::I16>(kc); }

cudaError_t launch_msa_i16(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads,
                           size_t smem, cudaStream_t stream)
{
    return launch_table<kern::I16>(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc
