// INT8 instantiations of the two-shots-per-word throughput kernel (see msa_packed.cuh): 8-bit
// messages held in 16-bit lanes, clamped to +-127.
#include "msa_packed.cuh"

namespace qldpc {

const void *msa_kernel_i8x2(const KernelChoice &kc) { return packed_table<kern::Pair16<kern::I8>>(kc); }

cudaError_t launch_msa_i8x2(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads, size_t smem,
                            cudaStream_t stream)
{
    return packed_launch<kern::Pair16<kern::I8>>(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc
