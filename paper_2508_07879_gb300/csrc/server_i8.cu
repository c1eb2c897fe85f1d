// INT8 fixed-point instantiations of the persistent decoding server kernel (see server_kernel.cuh).
#include "server_kernel.cuh"

namespace qldpc {

const void *server_kernel_i8(const KernelChoice &kc) { return server_table<kern::I8, false>(kc); }

cudaError_t launch_server_i8(const ServerParams &p, const KernelChoice &kc, int blocks, int threads,
                             size_t smem, cudaStream_t stream)
{
    return server_launch<kern::I8, false>(p, kc, blocks, threads, smem, stream);
}

}  // namespace qldpc
