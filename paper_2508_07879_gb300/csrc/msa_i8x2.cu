// INT8 instantiations of the two-shots-per-word throughput kernel (see msa_packed.cuh).  Codes with
// column degrees up to 8 carry the 8-bit messages in half-precision lanes (PairH8: every sum stays an
// integer of magnitude at most 1143, exact in FP16); higher column degrees hold them in 16-bit integer
// lanes clamped to +-127 (Pair16<I8>).  Both give the I8 integers exactly.
#include "msa_packed.cuh"

namespace qldpc {

const void *msa_kernel_i8x2(const KernelChoice &kc)
{
    return kc.dvb <= 8 ? packed_table<kern::PairH8, 0, 8>(kc) : packed_table<kern::Pair16<kern::I8>, 16, 16>(kc);
}

cudaError_t launch_msa_i8x2(const LaunchParams &p, const KernelChoice &kc, dim3 grid, int threads, size_t smem,
                            cudaStream_t stream)
{
    return kc.dvb <= 8 ? packed_launch<kern::PairH8, 0, 8>(p, kc, grid, threads, smem, stream)
                       : packed_launch<kern::Pair16<kern::I8>, 16, 16>(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc
