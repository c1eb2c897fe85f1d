// Host side of the learned-decoder entry points of include/qldpc.h: weight upload for learned
// decoding, workspace sizing, argument validation and launches of the training kernels
// (nms_train.cu), the Adam step, the device error sampler and the logical-failure test.  No
// arithmetic of the method runs here.
#include "qldpc.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "graph.h"
#include "msa_launch.h"

using namespace qldpc;
using namespace qldpc::detail;

namespace {

constexpr int32_t kMaxLearnedIters = 4096;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Compiled training variant for a graph (see nms_train.cu), or dc = -1 if none.
TrainChoice train_choice(const qldpc_graph *g)
{
    const int dvb = dv_bucket(g->dv_max);
    if (g->uniform_rows && g->dc_max >= 6 && g->dc_max <= 8 && dvb <= 8) return TrainChoice{g->dc_max, true, dvb};
    const int dcb = dc_bucket(g->dc_max);
    if (dcb < 0 || dvb < 0) return TrainChoice{-1, false, 0};
    return TrainChoice{dcb, false, std::max(8, dvb)};
}

struct TrainPlan {
    TrainChoice tc{};
    const void *fwd[2] = {nullptr, nullptr}, *bwd[2] = {nullptr, nullptr};   // [loss kind]
    size_t smem_f[2] = {0, 0}, smem_b[2] = {0, 0};   // [loss kind]
    int grid_f[2] = {0, 0}, grid_b[2] = {0, 0};
    size_t w_off = 0, state_off = 0, part_off = 0, total = 0;
};

int plan_training_uncached(const qldpc_graph *g, int32_t batch, int32_t T, TrainPlan &tp);

// The plan of the graph's last (batch, T), else a new one (occupancy queries cost host time on
// every training step otherwise).
int plan_training(const qldpc_graph *g, int32_t batch, int32_t T, TrainPlan &tp)
{
    static_assert(sizeof(TrainPlan) <= sizeof(g->train_plan), "plan cache too small");
    qldpc_graph *mg = const_cast<qldpc_graph *>(g);
    std::lock_guard<std::mutex> lk(mg->train_mu);
    if (mg->train_batch == batch && mg->train_T == T) {
        std::memcpy(&tp, mg->train_plan, sizeof(TrainPlan));
        return QLDPC_OK;
    }
    if (int rc = plan_training_uncached(g, batch, T, tp)) return rc;
    std::memcpy(mg->train_plan, &tp, sizeof(TrainPlan));
    mg->train_batch = batch;
    mg->train_T = T;
    return QLDPC_OK;
}

int plan_training_uncached(const qldpc_graph *g, int32_t batch, int32_t T, TrainPlan &tp)
{
    tp.tc = train_choice(g);
    if (tp.tc.dc < 0) return QLDPC_ERR_UNSUPPORTED;
    for (int kind = 0; kind < 2; ++kind) {
        const bool syn = kind == kLossSyndrome;
        tp.fwd[kind] = nms_forward_kernel_ptr(tp.tc, kind);
        tp.bwd[kind] = nms_backward_kernel_ptr(tp.tc, kind);
        if (!tp.fwd[kind] || !tp.bwd[kind]) return QLDPC_ERR_UNSUPPORTED;
        tp.smem_f[kind] = train_layout(g->m, g->nv, g->dc_max, false, syn).total;
        tp.smem_b[kind] = train_layout(g->m, g->nv, g->dc_max, true, syn).total;
        if (int rc = ensure_kernel_attrs(tp.fwd[kind], tp.smem_f[kind], g->smem_optin)) return rc;
        if (int rc = ensure_kernel_attrs(tp.bwd[kind], tp.smem_b[kind], g->smem_optin)) return rc;
    }
    for (int kind = 0; kind < 2; ++kind) {
        int per_f = 0, per_b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f, tp.fwd[kind], kTrainThreads, tp.smem_f[kind]) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_b, tp.bwd[kind], kTrainThreads, tp.smem_b[kind]) != cudaSuccess) {
            cudaGetLastError();
            return QLDPC_ERR_CUDA;
        }
        if (per_f < 1 || per_b < 1) return QLDPC_ERR_UNSUPPORTED;
        tp.grid_f[kind] = int(std::min<int64_t>(batch, int64_t(per_f) * g->sm_count));
        tp.grid_b[kind] = int(std::min<int64_t>(batch, int64_t(per_b) * g->sm_count));
    }
    const size_t S = size_t(g->dc_max) * size_t(g->m);
    tp.w_off = 0;
    tp.state_off = align_up(size_t(T) * S * sizeof(float));
    tp.part_off = tp.state_off + align_up(size_t(batch) * size_t(T) * kStateWords * size_t(g->m) * sizeof(uint32_t));
    tp.total = tp.part_off + align_up(size_t(T) * S * sizeof(float));
    return QLDPC_OK;
}

int check_workspace(const TrainPlan &tp, const void *ws, size_t bytes)
{
    if (!ws || bytes < tp.total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return QLDPC_ERR_INVALID_ARG;
    return QLDPC_OK;
}

TrainParams train_params(const qldpc_graph *g, const TrainPlan &tp, const uint8_t *syn, const uint8_t *target,
                         int32_t batch, const float *prior, int32_t T, void *ws)
{
    TrainParams p{};
    char *b = static_cast<char *>(ws);
    p.g = g->dg;
    p.syn = syn;
    p.target = target;
    p.prior = prior;
    p.w = reinterpret_cast<const float *>(b + tp.w_off);
    p.state = reinterpret_cast<uint32_t *>(b + tp.state_off);
    p.partial = reinterpret_cast<float *>(b + tp.part_off);
    p.T = T;
    p.batch = batch;
    return p;
}

}  // namespace

extern "C" {

int qldpc_graph_set_weights(qldpc_graph *g, const float *weights, int32_t T)
{
    if (!g || T < 0 || T > kMaxLearnedIters || (T > 0 && !weights)) return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    if (T == 0) {
        if (g->d_weights) cudaFree(g->d_weights);
        g->d_weights = nullptr;
        g->learned_T = 0;
        return QLDPC_OK;
    }
    const size_t count = size_t(T) * size_t(g->nnz);
    std::vector<float> host(count);
    cudaError_t e = cudaMemcpy(host.data(), weights, count * sizeof(float), cudaMemcpyDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QLDPC_ERR_INVALID_ARG;   // not a readable host or device range
    }
    for (float x : host)
        if (!std::isfinite(x)) return QLDPC_ERR_INVALID_ARG;
    // slot layout [T][dc_max * m]: the weight of CSR edge e at position j of row i sits at j*m + i
    const size_t S = size_t(g->dc_max) * size_t(g->m);
    std::vector<uint32_t> eslot(size_t(g->nnz));
    e = cudaMemcpy(eslot.data(), g->dg.eslot, eslot.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    std::vector<float> slot(size_t(T) * S, 0.0f);
    for (int32_t t = 0; t < T; ++t)
        for (int32_t i = 0; i < g->nnz; ++i) slot[size_t(t) * S + eslot[size_t(i)]] = host[size_t(t) * g->nnz + i];
    float *d = nullptr;
    e = cudaMalloc(&d, slot.size() * sizeof(float));
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemcpy(d, slot.data(), slot.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_status(e);
    }
    if (g->d_weights) cudaFree(g->d_weights);
    g->d_weights = d;
    g->learned_T = T;
    return QLDPC_OK;
}

int qldpc_nms_workspace_bytes(const qldpc_graph *g, int32_t batch, int32_t T, size_t *bytes)
{
    if (!g || !bytes || batch < 1 || T < 1 || T > kMaxLearnedIters) return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    TrainPlan tp;
    if (int rc = plan_training(g, batch, T, tp)) return rc;
    *bytes = tp.total;
    return QLDPC_OK;
}

int qldpc_nms_forward(const qldpc_graph *g, const uint8_t *syndromes, const uint8_t *targets, int32_t batch,
                      const float *prior, const float *weights, int32_t T, const float *loss_weights,
                      int32_t loss, float *out_loss, float *out_post, void *workspace, size_t workspace_bytes,
                      void *stream)
{
    if (loss != QLDPC_LOSS_ERROR && loss != QLDPC_LOSS_SYNDROME) return QLDPC_ERR_INVALID_ARG;
    if (!g || !syndromes || (!targets && loss == QLDPC_LOSS_ERROR) || !prior || !weights || !out_loss || batch < 1 ||
        T < 1 || T > kMaxLearnedIters)
        return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    TrainPlan tp;
    if (int rc = plan_training(g, batch, T, tp)) return rc;
    if (int rc = check_workspace(tp, workspace, workspace_bytes)) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TrainParams p = train_params(g, tp, syndromes, targets, batch, prior, T, workspace);
    p.loss = out_loss;
    p.post = out_post;
    p.loss_w = loss_weights;
    p.loss_kind = loss;
    const size_t S = size_t(g->dc_max) * size_t(g->m);
    cudaError_t e = launch_permute_weights(weights, g->dg.eslot, T, g->nnz, int32_t(S),
                                           const_cast<float *>(p.w), st);
    if (e == cudaSuccess) e = launch_nms_forward(p, tp.tc, tp.grid_f[loss], kTrainThreads, tp.smem_f[loss], st);
    return cuda_status(e);
}

int qldpc_nms_backward(const qldpc_graph *g, const uint8_t *syndromes, const uint8_t *targets, int32_t batch,
                       const float *prior, int32_t T, const float *loss_weights, int32_t loss,
                       const float *grad_loss, float *out_grad, void *workspace, size_t workspace_bytes,
                       void *stream)
{
    if (loss != QLDPC_LOSS_ERROR && loss != QLDPC_LOSS_SYNDROME) return QLDPC_ERR_INVALID_ARG;
    if (!g || !syndromes || (!targets && loss == QLDPC_LOSS_ERROR) || !prior || !grad_loss || !out_grad ||
        batch < 1 || T < 1 || T > kMaxLearnedIters)
        return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    TrainPlan tp;
    if (int rc = plan_training(g, batch, T, tp)) return rc;
    if (int rc = check_workspace(tp, workspace, workspace_bytes)) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TrainParams p = train_params(g, tp, syndromes, targets, batch, prior, T, workspace);
    p.grad_loss = grad_loss;
    p.loss_w = loss_weights;
    p.loss_kind = loss;
    const size_t S = size_t(g->dc_max) * size_t(g->m);
    cudaError_t e = cudaMemsetAsync(p.partial, 0, size_t(T) * S * sizeof(float), st);
    if (e == cudaSuccess) e = launch_nms_backward(p, tp.tc, tp.grid_b[loss], kTrainThreads, tp.smem_b[loss], st);
    if (e == cudaSuccess) e = launch_gather_grad(p.partial, g->dg.eslot, T, int32_t(S), g->nnz, out_grad, st);
    return cuda_status(e);
}

int qldpc_adam_step(float *params, const float *grads, float *exp_avg, float *exp_avg_sq, int64_t count,
                    int32_t step, float lr, float beta1, float beta2, float eps, void *stream)
{
    if (count < 0 || step < 1 || !std::isfinite(lr) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f) || !std::isfinite(eps))
        return QLDPC_ERR_INVALID_ARG;
    if (count == 0) return QLDPC_OK;
    if (!params || !grads || !exp_avg || !exp_avg_sq) return QLDPC_ERR_INVALID_ARG;
    return cuda_status(launch_adam(params, grads, exp_avg, exp_avg_sq, count, step, lr, beta1, beta2, eps,
                                   static_cast<cudaStream_t>(stream)));
}

int qldpc_sample_errors(const qldpc_graph *g, uint64_t seed, int64_t first_shot, int32_t batch, double p_lo,
                        double p_hi, uint8_t *out_err, uint8_t *out_syn, void *stream)
{
    if (!g || batch < 0 || first_shot < 0) return QLDPC_ERR_INVALID_ARG;
    if (!(p_lo >= 0.0 && p_hi <= 1.0 && p_lo <= p_hi)) return QLDPC_ERR_INVALID_ARG;
    if (batch == 0) return QLDPC_OK;
    if (!out_err || !out_syn) return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    const int grid = int(std::min<int64_t>(batch, int64_t(g->sm_count) * 8));
    return cuda_status(launch_sample(g->dg, seed, first_shot, batch, p_lo, p_hi, out_err, out_syn, grid,
                                     static_cast<cudaStream_t>(stream)));
}

int qldpc_logical_failures(const uint8_t *logicals, int32_t k, int32_t n, const uint8_t *errors,
                           const uint8_t *decisions, const uint8_t *ok, int32_t batch, uint8_t *out_fail,
                           void *stream)
{
    if (k < 1 || n < 1 || batch < 0) return QLDPC_ERR_INVALID_ARG;
    if (batch == 0) return QLDPC_OK;
    if (!logicals || !errors || !decisions || !ok || !out_fail) return QLDPC_ERR_INVALID_ARG;
    if ((size_t(k) + 1) * size_t((n + 31) / 32) * 4 > 48 * 1024) return QLDPC_ERR_UNSUPPORTED;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return QLDPC_ERR_CUDA;
    const int grid = int(std::min<int64_t>(batch, int64_t(sms) * 8));
    return cuda_status(launch_logical(logicals, k, n, errors, decisions, ok, batch, out_fail, grid,
                                      static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
