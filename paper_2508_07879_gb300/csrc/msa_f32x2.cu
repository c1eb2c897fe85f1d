// FP32 instantiations of the two-shots-per-block throughput kernel (see msa_packed.cuh): float2
// slots, each lane's arithmetic that of the one-shot FP32 kernel.
#include "msa_packed.cuh"

namespace qldpc {

const void *msa_kernel_f32x2(const KernelChoice &kc) { return packed_table<kern::PairF32>(kc); }

cudaError_t launch_msa_f32x2(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads, size_t smem,
                             cudaStream_t stream)
{
    return packed_launch<kern::PairF32>(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc
