// Test harness: runs the library's host-side graph layout (validate_and_layout in qldpc_host.cpp)
// on a CSR matrix read from stdin and prints the arrays it builds, one "name v0 v1 ..." line each.
// No CUDA call is made; the kernel tables the host file refers to are stubbed below.
#include "../paper_2508_07879_gb300/csrc/qldpc_host.cpp"

#include <cstdio>

namespace qldpc {
const void *msa_kernel_f32(const KernelChoice &) { return nullptr; }
const void *msa_kernel_i16(const KernelChoice &) { return nullptr; }
const void *msa_kernel_i8(const KernelChoice &) { return nullptr; }
const void *msa_kernel_learned(const KernelChoice &) { return nullptr; }
const void *msa_kernel_layered(int, const KernelChoice &) { return nullptr; }
const void *msa_kernel_i16x2(const KernelChoice &) { return nullptr; }
const void *msa_kernel_i8x2(const KernelChoice &) { return nullptr; }
const void *msa_kernel_f32x2(const KernelChoice &) { return nullptr; }
cudaError_t launch_msa_f32x2(const LaunchParams &, const KernelChoice &, dim3, int, size_t, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_msa_i16x2(const LaunchParams &, const KernelChoice &, dim3, int, size_t, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_msa_i8x2(const LaunchParams &, const KernelChoice &, dim3, int, size_t, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_msa_f32(const LaunchParams &, const KernelChoice &, dim3, int, size_t, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_msa_i16(const LaunchParams &, const KernelChoice &, dim3, int, size_t, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_msa_i8(const LaunchParams &, const KernelChoice &, dim3, int, size_t, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_msa_learned(const LaunchParams &, const KernelChoice &, dim3, int, size_t, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t launch_msa_layered(int, const LaunchParams &, const KernelChoice &, dim3, int, size_t, cudaStream_t) { return cudaErrorInvalidValue; }
}  // namespace qldpc

template <class V>
static void dump(const char *name, const V &v)
{
    std::printf("%s", name);
    for (const auto &x : v) std::printf(" %lld", static_cast<long long>(x));
    std::printf("\n");
}

int main()
{
    int m = 0, n = 0, nnz = 0;
    if (std::scanf("%d %d %d", &m, &n, &nnz) != 3 || m < 0 || n < 0 || nnz < 0) return 2;
    std::vector<int32_t> rp(static_cast<size_t>(m) + 1), ci(static_cast<size_t>(nnz));
    for (auto &x : rp)
        if (std::scanf("%d", &x) != 1) return 2;
    for (auto &x : ci)
        if (std::scanf("%d", &x) != 1) return 2;
    HostLayout hl;
    const int rc = validate_and_layout(rp.data(), nnz ? ci.data() : nullptr, m, n, hl);
    std::printf("rc %d\n", rc);
    if (rc) return 0;
    std::printf("dims %d %d %d %d\n", hl.dc_max, hl.dv_max, hl.nv, hl.uniform_rows ? 1 : 0);
    std::printf("magic %u %d\n", hl.m_magic, hl.m_shift);
    dump("vorder", hl.vorder);
    dump("vdeg", hl.vdeg);
    dump("vslot", hl.vslot);
    dump("eslot", hl.eslot);
    dump("layer_ptr", hl.layer_ptr);
    dump("layer_chk", hl.layer_chk);
    return 0;
}
