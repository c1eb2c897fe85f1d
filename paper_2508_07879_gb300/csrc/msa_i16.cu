// INT16 fixed-point instantiations of the flooding min-sum decoder (see msa_kernel.cuh).
#include "msa_kernel.cuh"

namespace qldpc {

const void *msa_kernel_i16(int dcb, int dvb) { return kernel_table<kern::I16>(dcb, dvb); }

cudaError_t launch_msa_i16(const LaunchParams &p, int dcb, int dvb, dim3 grid, int threads,
                           size_t smem, cudaStream_t stream)
{
    return launch_table<kern::I16>(p, dcb, dvb, grid, threads, smem, stream);
}

}  // namespace qldpc
