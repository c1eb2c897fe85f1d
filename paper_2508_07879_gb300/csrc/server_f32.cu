// FP32 instantiations of the persistent decoding server kernel (see server_kernel.cuh): a plain one,
// and one in which a code with learned weights decodes with them, then with the plain fallback
// (chosen when the server decodes learned codes).
#include "server_kernel.cuh"

namespace qldpc {

const void *server_kernel_f32(const KernelChoice &kc)
{
    return kc.learned ? server_table<kern::F32, true>(kc) : server_table<kern::F32, false>(kc);
}

cudaError_t launch_server_f32(const ServerParams &p, const KernelChoice &kc, int blocks, int threads,
                              size_t smem, cudaStream_t stream)
{
    return kc.learned ? server_launch<kern::F32, true>(p, kc, blocks, threads, smem, stream)
                      : server_launch<kern::F32, false>(p, kc, blocks, threads, smem, stream);
}

}  // namespace qldpc
