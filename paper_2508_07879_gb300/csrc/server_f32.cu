// FP32 instantiations of the persistent decoding server kernel (see server_kernel.cuh); a code
// with learned weights decodes with them, then with the plain fallback.
#include "server_kernel.cuh"

namespace qldpc {

const void *server_kernel_f32(const KernelChoice &kc) { return server_table<kern::F32, true>(kc); }

cudaError_t launch_server_f32(const ServerParams &p, const KernelChoice &kc, int blocks, int threads,
                              size_t smem, cudaStream_t stream)
{
    return server_launch<kern::F32, true>(p, kc, blocks, threads, smem, stream);
}

}  // namespace qldpc
