/*
 * qldpc.h -- C ABI of the GB300 (sm_103a) syndrome decoder for CSS quantum LDPC codes.
 *
 * The library runs normalized min-sum belief propagation driven by a syndrome (Algorithm 1,
 * "MSA for syndrome-based LDPC decoding", Sec. 2 of arXiv 2508.07879) on one GPU.  Given the
 * Tanner graph of a parity-check matrix H (M checks, N variables) and a batch of syndromes
 * s = H e^T over GF(2), it returns for every shot the estimate e_hat, the number of iterations run
 * and whether H e_hat^T = s holds.  For a CSS code, s_X = H_Z e_X^T is decoded with H_Z and
 * s_Z = H_X e_Z^T with H_X (Sec. 2); qldpc_decode_pair does both in one launch, as the paper's
 * decoder does (Fig. 2 caption).
 *
 * Arithmetic (identical, operation by operation, to the CPU oracle of the test suite):
 *   q_{m,n}^(0) = gamma_n                                        (Alg. 1 initialization)
 *   r_{m,n} = (-1)^{s_m} prod_{j in S_v(m)\n} sign(q_{m,j}) * (alpha * min_{j in S_v(m)\n} |q_{m,j}|)
 *   q_{m,n} = gamma_n + sum_{i in S_c(n)\m} r_{i,n}   (sum in ascending check order)
 *   Q_n     = gamma_n + sum_{i in S_c(n)} r_{i,n};    e_hat_n = [Q_n < 0]
 *   sign(x) = -1 iff x < 0.  The stop test H e_hat^T = s runs before the first iteration and
 *   after every iteration; decoding stops at the first success or after max_iter iterations.
 *   (FP32 treats a prior of -0 as +0; this can change only the sign of a zero a-posteriori LLR.)
 *
 * Precisions:
 *   QLDPC_FP32  IEEE binary32 messages, every add and multiply rounded to nearest (no fusion).
 *   QLDPC_INT16 16-bit fixed point with 8 fractional bits (the paper's integer proposal, Table 1):
 *               gamma_q = clamp(round_half_away(gamma*256), +-32767); alpha_q = round(alpha*2^15);
 *               |r| = floor(min*alpha_q/2^15); q = clamp(32-bit sum, +-32767); Q in 32 bits.
 *               Requires 0 < alpha <= 1.
 *   QLDPC_INT8  the same with 2 fractional bits and +-127 (8-bit messages; the paper names 8-bit
 *               integers without a scheme): gamma_q = clamp(round_half_away(gamma*4), +-127).
 *
 * Memory and ownership: graph arrays live on the device and are owned by the qldpc_graph.
 * Every buffer passed to qldpc_decode* is caller-owned DEVICE memory (e.g. torch tensors) unless
 * the function name says "host".  Row-major layouts: syndromes[b*m + i], out_err[b*n + j].
 * Decodes are asynchronous on the given stream and allocate nothing; qldpc_decode_host is
 * synchronous and uses device staging owned by the graph (grown on demand, or reserved ahead with
 * qldpc_graph_reserve).  A graph must be used on the device that was current when it was created.
 *
 * Entry points by group:
 *   graphs          qldpc_graph_create / _create_csc / _destroy / _dims / _footprint / _set_launch /
 *                   _reserve
 *   decoding        qldpc_decode, qldpc_decode_ex (flags: QLDPC_NO_EARLY_STOP, QLDPC_LAYERED for
 *                   the row-serial schedule, QLDPC_LEARNED), qldpc_decode_pair, qldpc_decode_host,
 *                   qldpc_decode_host_noalloc
 *   serving         qldpc_server_create / _submit / _poll / _replay / _status / _destroy
 *   learned decoder qldpc_graph_set_weights, qldpc_nms_workspace_bytes, qldpc_nms_forward,
 *                   qldpc_nms_backward, qldpc_adam_step
 *   workloads       qldpc_sample_errors (device error sampler), qldpc_logical_failures
 *
 * Soft syndromes: a syndrome bit read with error probability q is a degree-1 variable of its check
 * with prior LLR ln((1-q)/q).  Decoding the data-syndrome matrix [H | I_m] (create the graph from
 * it) with the data priors followed by the m read-error LLRs, and the measured bits as syndromes,
 * is soft-syndrome decoding; e_hat then holds the data error followed by the read errors.
 *
 * Errors: every function returns a qldpc_status.  Arguments are validated on the host before any
 * GPU work is enqueued; a rejected call enqueues nothing and writes no output.  A CUDA launch
 * failure returns QLDPC_ERR_CUDA; faults during execution surface at the caller's next
 * synchronization.  A non-finite prior LLR is detected on the device: every shot of that call
 * returns iters = -1, ok = 0 and e_hat = 0.
 */
#ifndef QLDPC_H
#define QLDPC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QLDPC_API __attribute__((visibility("default")))
#else
#define QLDPC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qldpc_graph qldpc_graph;   /* opaque; owned by the library */

typedef enum qldpc_status {
    QLDPC_OK = 0,
    QLDPC_PENDING = 1,            /* (server) the request is not finished yet: poll again */
    QLDPC_BUSY = 2,               /* (server) the code's ring is full: collect results first */
    QLDPC_ERR_INVALID_ARG = -1,   /* bad pointer, size, CSR structure, alpha, flag or precision */
    QLDPC_ERR_UNSUPPORTED = -2,   /* graph exceeds a kernel limit (degree, shared memory, size) */
    QLDPC_ERR_OOM = -3,           /* device or pinned host allocation failed */
    QLDPC_ERR_CUDA = -4,          /* CUDA runtime error (no device, launch failure, copy failure) */
    QLDPC_ERR_TIMEOUT = -5        /* a bounded device-side wait expired */
} qldpc_status;

/* Message precision.  FP32: Algorithm 1 in binary32.  INT16: LLRs in fixed point with 8 fractional
 * bits, messages clamped to +-32767, sums in 32 bits, alpha as round(alpha * 2^15) / 2^15.  INT8: the
 * same with 2 fractional bits and messages clamped to +-127 (LLRs within +-31.75). */
enum { QLDPC_FP32 = 0, QLDPC_INT16 = 1, QLDPC_INT8 = 2 };

/* Decode flags (bitwise OR). */
enum {
    QLDPC_NO_EARLY_STOP = 1u,     /* run exactly max_iter iterations (the paper's timed mode, Sec. 3);
                                     ok still reports H e_hat^T = s after the last one */
    QLDPC_LEARNED = 2u,           /* learned decoding with the graph's weights, then the plain
                                     fallback (see qldpc_graph_set_weights); FP32 and early stop only */
    QLDPC_LAYERED = 4u            /* layered (row-serial) schedule instead of flooding: the checks
                                     are updated one after another in ascending index, each from the
                                     a-posteriori LLRs the checks before it refreshed
                                     (q = Q - r_old, r = Algorithm 1's check update of q,
                                     Q = q + r); FP32, INT16 or INT8; not with QLDPC_LEARNED */
};

/* Limits of the compiled kernels. */
enum {
    QLDPC_MAX_ROW_DEGREE = 32,    /* check-node degree d_c */
    QLDPC_MAX_COL_DEGREE = 16,    /* variable-node degree d_v */
    QLDPC_MAX_CHECKS = 65535      /* rows m */
};

/*
 * Build a Tanner graph from H in CSR form (Sec. 2: S_v(m) = columns of row m).
 *   row_ptr  host int32[m+1], row_ptr[0] = 0, non-decreasing
 *   col_idx  host int32[row_ptr[m]], each in [0, n), no repeats within a row (any order)
 *   m, n     number of checks (rows) and variables (columns), both >= 1
 *   out      receives the new graph (set to NULL on failure)
 * The caller keeps its arrays; the library copies what it needs.
 * INVALID_ARG: null pointer, m or n <= 0, malformed row_ptr, column out of range, repeated column
 *              in a row, or a row of degree < 2 (the check update needs two neighbours).
 * UNSUPPORTED: a row degree > QLDPC_MAX_ROW_DEGREE, a column degree > QLDPC_MAX_COL_DEGREE,
 *              m > QLDPC_MAX_CHECKS, or one shot's working set (messages, priors, LLRs and parity
 *              words) larger than the device's shared memory per block.
 * CUDA / OOM:  no usable device or the upload failed.
 */
QLDPC_API int qldpc_graph_create(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                       qldpc_graph **out);

/* Same as qldpc_graph_create, from H in CSC form (S_c(n) = rows of column n):
 *   col_ptr host int32[n+1], row_idx host int32[col_ptr[n]] in [0, m). */
QLDPC_API int qldpc_graph_create_csc(const int32_t *col_ptr, const int32_t *row_idx, int32_t m, int32_t n,
                           qldpc_graph **out);

/* Release the graph and its device memory.  NULL is ignored.  The caller must ensure no decode
 * using the graph is still running. */
QLDPC_API void qldpc_graph_destroy(qldpc_graph *g);

/* Report the graph's shape: checks, variables, edges, maximum row and column degree (any output
 * pointer may be NULL). */
QLDPC_API int qldpc_graph_dims(const qldpc_graph *g, int32_t *m, int32_t *n, int32_t *nnz,
                     int32_t *max_row_degree, int32_t *max_col_degree);

/* The layered schedule the graph's row order gives (QLDPC_LAYERED): each check goes to the layer one
 * above the highest layer of an earlier row it shares a variable with, so the checks of a layer are
 * independent.  Reports the number of layers and the largest layer (any output pointer may be
 * NULL).  A caller who wants fewer layers reorders the rows of H, which is a different schedule. */
QLDPC_API int qldpc_graph_layers(const qldpc_graph *g, int32_t *layers, int32_t *widest);

/* On-chip footprint of the flooding kernels for one precision (QLDPC_FP32 / INT16 / INT8):
 *   lanes       variable lanes of the variable step, n plus idle lanes (variables are grouped by
 *               degree and packed into warps whose k-th edge slots fall in distinct shared-memory
 *               banks; an idle lane closes a warp early where that pays)
 *   shot_bytes  shared memory one shot takes in the throughput kernel: Q and gamma (4 B per lane),
 *               parity words (4 B per check), messages (max_row_degree * m slots and 32 scratch
 *               slots for the idle lanes), each section 16-byte aligned.  A decode whose
 *               shot_bytes plus the kernel's few bytes of static shared memory exceed the
 *               device's shared memory per block is refused with UNSUPPORTED.
 * Either output pointer may be NULL.  INVALID_ARG: null graph or unknown precision. */
QLDPC_API int qldpc_graph_footprint(const qldpc_graph *g, int32_t precision, int32_t *lanes, size_t *shot_bytes);

/* Kernels (qldpc_graph_set_launch). */
enum {
    QLDPC_KERNEL_AUTO = 0,      /* latency kernel when every shot gets its own SM, else the packed
                                   kernel where two shots fit a block's shared memory (learned
                                   decoding: the batch kernel) */
    QLDPC_KERNEL_BATCH = 1,     /* throughput kernel: one shot per block, thread per check / per
                                   variable, persistent blocks */
    QLDPC_KERNEL_LATENCY = 2,   /* single-shot kernel: per-thread state in registers, one block per
                                   shot; needs m <= 2*threads and n <= 2*threads, threads <= 640 */
    QLDPC_KERNEL_PACKED = 3     /* throughput kernel with two shots per block, their messages paired
                                   in one slot per edge (a float2 in FP32, two 16-bit integer lanes in
                                   INT16, two half-precision lanes holding the exact INT8 integers up
                                   to column degree 8 and 16-bit integer lanes above it); each shot
                                   stops at its own iteration */
};

/* Override the library's launch choice for this graph: the kernel, its threads per block (a
 * multiple of 32 in [32, 1024], at most 512 for QLDPC_KERNEL_PACKED; 0 = automatic) and the resident
 * blocks per SM used to size the grid (0 = from occupancy).  QLDPC_KERNEL_AUTO takes no shape (both
 * 0) and restores the default.  INVALID_ARG if out of range, UNSUPPORTED if the shape cannot run
 * this graph (in any precision) or the residency is not achievable.  Results never depend on the
 * launch choice. */
QLDPC_API int qldpc_graph_set_launch(qldpc_graph *g, int32_t kernel, int32_t threads_per_block,
                                     int32_t blocks_per_sm);

/* Pre-size the device staging that qldpc_decode_host uses, for up to max_batch shots. */
QLDPC_API int qldpc_graph_reserve(qldpc_graph *g, int32_t max_batch);

/*
 * Decode a batch of syndromes with H (Algorithm 1), FP32 messages, early stop on, legacy default
 * stream.  All pointers are DEVICE memory:
 *   syndromes  uint8[batch*m], values 0/1 (only bit 0 is read)
 *   prior_llr  float[n], gamma_n = ln(P(e_n=0)/P(e_n=1)); must be finite
 *   out_err    uint8[batch*n]  e_hat
 *   out_iters  int32[batch]    CN+VN iterations run (0 if the prior's decision already met s)
 *   out_ok     uint8[batch]    1 iff H e_hat^T = s
 * batch >= 0 (0 is a no-op); max_iter >= 0 (0 returns the prior's hard decision); alpha finite > 0.
 */
QLDPC_API int qldpc_decode(const qldpc_graph *g, const uint8_t *syndromes, int32_t batch,
                 const float *prior_llr, int32_t max_iter, float alpha,
                 uint8_t *out_err, int32_t *out_iters, uint8_t *out_ok);

/*
 * qldpc_decode with a precision (QLDPC_FP32 / QLDPC_INT16 / QLDPC_INT8), flags, a CUDA stream
 * (cudaStream_t cast to void*, NULL = legacy default stream) and an optional device output
 *   out_post  float[batch*n] or NULL: the a-posteriori LLR Q_n of the last iteration run
 *             (INT16: the fixed-point value / 256, exact).
 * A batch with more shots than the launch's resident blocks hands shots out dynamically: blocks
 * claim them from one of 1024 counter pairs held by the graph, zeroed on `stream` before the
 * launch (results do not depend on the order).  Only more than 1024 such decodes of one graph in
 * flight at once on different streams could share a pair.
 * With QLDPC_LAYERED the schedule is row-serial (see the flag): same outputs and stop rule; INT16
 * keeps Q in 32 bits and clamps q = Q - r to +-32767.  Its launch shape is chosen automatically
 * (qldpc_graph_set_launch does not apply).
 * With QLDPC_LEARNED the graph's learned weights (qldpc_graph_set_weights) drive the first T
 * iterations and max_iter bounds the plain fallback; INVALID_ARG if the graph has no weights, the
 * precision is not FP32 or QLDPC_NO_EARLY_STOP is also set.
 */
QLDPC_API int qldpc_decode_ex(const qldpc_graph *g, const uint8_t *syndromes, int32_t batch,
                    const float *prior_llr, int32_t max_iter, float alpha,
                    uint8_t *out_err, int32_t *out_iters, uint8_t *out_ok, float *out_post,
                    int32_t precision, uint32_t flags, void *stream);

/*
 * Decode both halves of a CSS syndrome round in one launch (Sec. 2 / Fig. 2: X and Z decoded in
 * the same kernel).  g_z decodes s_x (X errors, s_x = H_Z e_x^T, uint8[batch*m_z]) with prior_x;
 * g_x decodes s_z (Z errors, s_z = H_X e_z^T, uint8[batch*m_x]) with prior_z.  Each half stops at
 * its own convergence, so the results equal two qldpc_decode_ex calls bit for bit.  Outputs as in
 * qldpc_decode_ex (post pointers may be NULL).  Both graphs must have the same n.
 */
QLDPC_API int qldpc_decode_pair(const qldpc_graph *g_z, const qldpc_graph *g_x,
                      const uint8_t *s_x, const uint8_t *s_z, int32_t batch,
                      const float *prior_x, const float *prior_z, int32_t max_iter, float alpha,
                      uint8_t *err_x, uint8_t *err_z, int32_t *iters_x, int32_t *iters_z,
                      uint8_t *ok_x, uint8_t *ok_z, float *post_x, float *post_z,
                      int32_t precision, uint32_t flags, void *stream);

/*
 * End-to-end decode from HOST memory, as the paper times it (Sec. 3: latency includes the
 * host-to-device and device-to-host transfers).  Copies syndromes (host uint8[batch*m]) and the
 * prior (host float[n], uploaded only when it changed since the last call) into the graph's device
 * staging, decodes on `stream`, copies e_hat, iterations and ok back into the host buffers and
 * synchronizes the stream before returning.  When the syndrome and output buffers each lie inside
 * one page-locked allocation registered with CUDA (cudaHostAlloc, cudaMallocHost,
 * cudaHostRegister; torch pin_memory), no copy is issued: the kernel reads the syndromes from and
 * writes the results to host memory directly, and the call is one launch plus one synchronize.
 * Calls on the same graph are serialized by a lock inside the graph.
 */
QLDPC_API int qldpc_decode_host(qldpc_graph *g, const uint8_t *h_syndromes, int32_t batch,
                      const float *h_prior, int32_t max_iter, float alpha,
                      uint8_t *h_err, int32_t *h_iters, uint8_t *h_ok,
                      int32_t precision, uint32_t flags, void *stream);

/*
 * The X+Z pair decode of qldpc_decode_pair end to end with host buffers (the paper's latency
 * measurement, Sec. 3: transfers included, both halves in one kernel).  Arguments as for
 * qldpc_decode_pair, but every buffer is host memory: s_x [batch, m_z], s_z [batch, m_x], priors
 * float[n] each, outputs e_hat [batch, n], iters [batch], ok [batch] per half.  g_z and g_x must be
 * two different graphs (each stages its own half).  When every buffer lies in page-locked memory
 * the kernel reads and writes them in place (no copies); otherwise they are staged through each
 * graph's device staging (allocated on first use, as for qldpc_decode_host).  Synchronous: returns
 * after the results are in the host buffers.  Arguments and the launch plan are checked before
 * anything is enqueued (INVALID_ARG / UNSUPPORTED as for qldpc_decode_pair).
 */
QLDPC_API int qldpc_decode_pair_host(qldpc_graph *g_z, qldpc_graph *g_x, const uint8_t *h_sx,
                                     const uint8_t *h_sz, int32_t batch, const float *h_prior_x,
                                     const float *h_prior_z, int32_t max_iter, float alpha,
                                     uint8_t *h_err_x, uint8_t *h_err_z, int32_t *h_iters_x,
                                     int32_t *h_iters_z, uint8_t *h_ok_x, uint8_t *h_ok_z,
                                     int32_t precision, uint32_t flags, void *stream);

/* Static, human-readable name of a status code. */
QLDPC_API const char *qldpc_status_string(int status);

/* ===============================================================================================
 * Persistent decoding server (continuous batching of single syndrome rounds).
 *
 * The paper proposes launching decoders asynchronously so transfers overlap execution (Table 1,
 * Sec. 3 outlook).  The server takes that to its limit: one kernel stays resident and requests
 * flow through per-code rings of slots in page-locked host memory mapped into the GPU, announced
 * in arrival order through one shared queue.  Admission is by footprint: every worker block is
 * sized for the largest footprint among the server's codes (threads, shared memory, registers),
 * as many workers run as fit on the GPU at that footprint, and a request is admitted as soon as
 * any worker is free, oldest first, whatever its code; a worker keeps the last code's graph and
 * priors in registers and reloads them only when it switches codes.  Requests of different codes
 * and sizes decode concurrently; results come back in the slot.  Decoding is the single-shot
 * algorithm of qldpc_decode_ex, so a request decodes to the same result alone or in any mix.
 * Every device-side wait is bounded (idle timeout, maximum runtime); the library relaunches the
 * workers when requests arrive after they left.  submit/poll/replay on one server are serialized
 * by a lock inside it.
 * =============================================================================================== */
typedef struct qldpc_server qldpc_server;

enum { QLDPC_SERVER_MAX_CODES = 4 };

typedef struct qldpc_server_config {
    int32_t precision;            /* QLDPC_FP32, QLDPC_INT16 or QLDPC_INT8 */
    int32_t max_iter;             /* >= 0 */
    float alpha;                  /* as for qldpc_decode_ex */
    uint32_t flags;               /* QLDPC_NO_EARLY_STOP, or QLDPC_LEARNED (FP32: every code whose
                                     graph has weights decodes learned, the others plainly), and/or
                                     QLDPC_LAYERED (workers on the layered schedule: results equal
                                     qldpc_decode_ex with QLDPC_LAYERED; rows of degree <= 8 and at
                                     most 256 checks per layer; a code of at most 8 layers and
                                     n <= 65536 keeps its checks in registers, any other its messages
                                     in shared memory; not with QLDPC_LEARNED), or 0 */
    int32_t ring_capacity;        /* slots per code, a power of two in [2, 2^20]; 0 = 256 */
    int32_t threads_per_block;    /* 0 = automatic; QLDPC_LAYERED: a multiple of 32 in
                                     [widest layer, 256] */
    int32_t blocks[QLDPC_SERVER_MAX_CODES];   /* the worker pool's size is the sum (every worker
                                     serves every code); all 0 = as many as fit on the GPU */
    int64_t idle_timeout_ns;      /* workers leave after this long without a request; <= 0: 0.5 s */
    int64_t max_runtime_ns;       /* workers leave after this long; <= 0: 600 s */
} qldpc_server_config;

/* Create a server for ncodes (1..4) graphs of the current device with host priors[c] (float[n_c],
 * copied).  Allocates the rings (page-locked host memory) and device state; the kernel starts on
 * the first request.  INVALID_ARG on bad arguments or non-finite priors; UNSUPPORTED if a graph
 * exceeds the single-shot kernel's limits (with QLDPC_LAYERED: the layer and degree limits above)
 * or the workers cannot all be resident. */
QLDPC_API int qldpc_server_create(const qldpc_graph *const *graphs, const float *const *priors,
                                  int32_t ncodes, const qldpc_server_config *cfg,
                                  qldpc_server **out);

/* Publish one request: syndrome (host uint8[m_code]) for code `code`.  Returns QLDPC_OK and a
 * ticket (the code's request sequence number), or QLDPC_BUSY when all ring slots of the code hold
 * results not yet collected by qldpc_server_poll. */
QLDPC_API int qldpc_server_submit(qldpc_server *s, int32_t code, const uint8_t *syndrome,
                                  uint64_t *ticket);

/* Collect a request: QLDPC_OK with e_hat (host uint8[n_code]), iterations and ok copied out (any
 * output pointer may be NULL) and the slot released; QLDPC_PENDING while it runs; INVALID_ARG for
 * an unknown or already collected ticket. */
QLDPC_API int qldpc_server_poll(qldpc_server *s, int32_t code, uint64_t ticket, uint8_t *err,
                                int32_t *iters, uint8_t *ok);

/* Open-loop load generator and latency recorder: submits request i (code codes[i], syndrome at
 * syndromes + syn_offsets[i]) at arrival_ns[i] after the call starts (non-decreasing), collects
 * every result (e_hat at errs + err_offsets[i], iters[i], oks[i], and in workers[i] the index of
 * the worker block that decoded it, if workers is not NULL) and records latency_ns[i] = completion
 * seen by the host - scheduled arrival.  A request whose ring is full waits until a result of that
 * code is collected.  Returns QLDPC_ERR_TIMEOUT if results are still missing timeout_ns after the
 * last arrival (<= 0: 10 s). */
QLDPC_API int qldpc_server_replay(qldpc_server *s, int32_t nreq, const int32_t *codes,
                                  const uint8_t *syndromes, const int64_t *syn_offsets,
                                  const int64_t *arrival_ns, uint8_t *errs, const int64_t *err_offsets,
                                  int32_t *iters, uint8_t *oks, int64_t *latency_ns, int32_t *workers,
                                  int64_t timeout_ns);

/* The worker pool: number of worker blocks and the footprint each has (threads, dynamic shared
 * memory in bytes).  Any output pointer may be NULL. */
QLDPC_API int qldpc_server_info(const qldpc_server *s, int32_t *workers, int32_t *threads_per_block,
                                size_t *smem_per_block);

/* Status bits the workers left: 1 = idle timeout, 2 = maximum runtime, 4 = spin cap, 8 = stopped. */
QLDPC_API int qldpc_server_status(qldpc_server *s, uint32_t *status);

/* Stop the workers (they leave at their next poll), wait for the kernel and free everything.
 * Uncollected results are lost.  NULL is ignored. */
QLDPC_API void qldpc_server_destroy(qldpc_server *s);

/* ===============================================================================================
 * Learned (neural) normalized min-sum.
 *
 * The check-node update of Algorithm 1 (Sec. 2) with the normalization alpha replaced by a trained
 * weight per iteration t and edge e:
 *   r^(t)_{m,n} = (-1)^{s_m} prod_{j != n} sign(q_{m,j}) * (w[t][e(m,n)] * min_{j != n} |q_{m,j}|)
 * Weights are float[T][nnz] in CSR edge order (e = row_ptr[m] + position of n in row m of the
 * matrix given to qldpc_graph_create).  The variable step, APP and decision are Algorithm 1's.
 * Learned decoding runs iterations 1..T with the weights and the stop test; a shot whose syndrome
 * is still not met restarts from its prior with plain min-sum (alpha, up to max_iter iterations):
 * iters = T + plain iterations for such shots.  Training minimizes a BCE of the soft outputs,
 * with per-iteration loss weights lambda_t (default 1/T), one of
 *   QLDPC_LOSS_ERROR     loss_b = sum_t lambda_t / n sum_v BCE(sigma(-Q^(t)_v), y_v)
 *                        (y = the true error bits: the mean over iterations and variables)
 *   QLDPC_LOSS_SYNDROME  loss_b = sum_t lambda_t / m sum_c -log max(P^(t)_c, 1e-7),
 *                        P_c = (1 + (-1)^{s_c} prod_{v in row c} tanh(Q_v / 2)) / 2
 *                        (the BCE of the soft syndrome: P_c is the probability that row c's parity
 *                        under independent bits of P(e_v = 1) = sigma(-Q_v) equals s_c; every error
 *                        with the shot's syndrome scores alike, and targets are not read)
 * with a forward kernel that records a compressed check state per iteration and a backward
 * kernel that recomputes every message from it.  FP32 throughout.
 * =============================================================================================== */
enum { QLDPC_LOSS_ERROR = 0, QLDPC_LOSS_SYNDROME = 1 };

/* Set (T >= 1) or clear (T = 0, weights may be NULL) the graph's learned weights: float[T][nnz],
 * host or device memory, copied (synchronously) into the graph.  Decodes and servers created
 * afterwards with QLDPC_LEARNED use them; do not call while a decode using the graph is running.
 * INVALID_ARG: null graph, T < 0 or > 4096, null weights with T > 0, a non-finite weight. */
QLDPC_API int qldpc_graph_set_weights(qldpc_graph *g, const float *weights, int32_t T);

/* Device workspace (bytes) that qldpc_nms_forward / qldpc_nms_backward need for `batch` shots and
 * T iterations: the slot-layout weights, 16 bytes of recorded state per check, iteration and shot,
 * and the slot-layout gradient.  INVALID_ARG: null pointers, batch < 1, T < 1. */
QLDPC_API int qldpc_nms_workspace_bytes(const qldpc_graph *g, int32_t batch, int32_t T, size_t *bytes);

/*
 * Training forward: T learned iterations (no stop test) on every shot.
 *   syndromes  device uint8[batch][m];  targets device uint8[batch][n], the true error bits (may be
 *              NULL with QLDPC_LOSS_SYNDROME)
 *   prior      device float[n];         weights device float[T][nnz] (CSR edge order)
 *   loss_weights  device float[T] (lambda_t), or NULL for 1/T each
 *   loss       QLDPC_LOSS_ERROR or QLDPC_LOSS_SYNDROME
 *   out_loss   device float[batch], loss_b as above
 *   out_post   device float[batch][n], Q^(T) (the a-posteriori LLR of iteration T), or NULL
 *   workspace  device memory of at least qldpc_nms_workspace_bytes(g, batch, T), 256-byte aligned;
 *              it keeps the weights and the recorded state for qldpc_nms_backward
 * Enqueued on `stream`.  INVALID_ARG: null pointers, batch < 1, T < 1, workspace too small or
 * misaligned.  UNSUPPORTED: a degree combination without a compiled training kernel, or a shot
 * that does not fit in shared memory.  Non-finite priors give non-finite losses.
 */
QLDPC_API int qldpc_nms_forward(const qldpc_graph *g, const uint8_t *syndromes, const uint8_t *targets,
                                int32_t batch, const float *prior, const float *weights, int32_t T,
                                const float *loss_weights, int32_t loss, float *out_loss, float *out_post,
                                void *workspace, size_t workspace_bytes, void *stream);

/*
 * Training backward: out_grad (device float[T][nnz], overwritten) = sum_b grad_loss[b] d loss_b / d w,
 * with the subgradients d|q|/dq = sign(q) (+1 at 0), d sign/dq = 0, and the minimum's gradient going
 * to the lowest position attaining it.  The arguments must be those of the preceding
 * qldpc_nms_forward on the same workspace (same syndromes, targets, prior, batch, T, loss weights
 * and loss; the weights are read back from the workspace).  grad_loss is device float[batch].  The
 * sum over shots is taken with FP32 global reductions, so its rounding order (the last bits of the
 * result) follows the schedule and may differ between calls.
 */
QLDPC_API int qldpc_nms_backward(const qldpc_graph *g, const uint8_t *syndromes, const uint8_t *targets,
                                 int32_t batch, const float *prior, int32_t T, const float *loss_weights,
                                 int32_t loss, const float *grad_loss, float *out_grad, void *workspace,
                                 size_t workspace_bytes, void *stream);

/* One Adam step on device float arrays of `count` elements (Kingma and Ba, ICLR 2015), in the
 * arithmetic of PyTorch's single-tensor Adam: m += (1-beta1)(g-m); v = beta2 v + (1-beta2) g^2;
 * param -= lr/(1-beta1^step) * m / (sqrt(v)/sqrt(1-beta2^step) + eps).  step >= 1. */
QLDPC_API int qldpc_adam_step(float *params, const float *grads, float *exp_avg, float *exp_avg_sq,
                              int64_t count, int32_t step, float lr, float beta1, float beta2, float eps,
                              void *stream);

/*
 * Seeded synthetic i.i.d. bit-flip errors and their syndromes s = H e^T mod 2 for the graph's H,
 * on the device.  Counter-based SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) keyed by
 * (seed, shot, qubit): u(b, q) = (mix(mix(mix(seed) + shot) + q) >> 11) / 2^53 with
 * shot = first_shot + b.  Shot b's rate is p_b = p_lo + (p_hi - p_lo) * u(b, n), and
 * e[b][q] = [u(b, q) < p_b] for q < n (p_lo = p_hi: a fixed rate).  Outputs: device uint8
 * out_err[batch][n] and out_syn[batch][m].  INVALID_ARG: null pointers, batch < 0, first_shot < 0,
 * rates outside [0, 1] or p_hi < p_lo.
 */
QLDPC_API int qldpc_sample_errors(const qldpc_graph *g, uint64_t seed, int64_t first_shot, int32_t batch,
                                  double p_lo, double p_hi, uint8_t *out_err, uint8_t *out_syn,
                                  void *stream);

/*
 * Logical failure of each decoded shot: fail[b] = 1 if ok[b] = 0 or the residual e_b XOR e_hat_b
 * has odd overlap with one of the k logical operators (rows of `logicals`, device uint8[k][n],
 * 0/1), else 0.  For X errors decoded with H_Z the rows are Z logicals (a basis of
 * ker H_X modulo the row space of H_Z); a residual that meets the syndrome is then a stabilizer
 * iff it commutes with all of them.  All arrays device memory; INVALID_ARG on null pointers or
 * sizes < 1 (batch = 0 is a no-op); UNSUPPORTED if (k + 1) * ceil(n / 32) * 4 > 48 KB.
 */
QLDPC_API int qldpc_logical_failures(const uint8_t *logicals, int32_t k, int32_t n, const uint8_t *errors,
                                     const uint8_t *decisions, const uint8_t *ok, int32_t batch,
                                     uint8_t *out_fail, void *stream);

/* Size of the library's static device scratch used by qldpc_decode_host_noalloc (4 MiB). */
enum { QLDPC_NOALLOC_SCRATCH_BYTES = 4 * 1024 * 1024 };

/* The size of that scratch as compiled into the library, in bytes (a binding that carries its own
 * copy of the constant above can check it against this). */
QLDPC_API size_t qldpc_noalloc_scratch_bytes(void);

/*
 * qldpc_decode_host without any device allocation.  (No counterpart in the paper: this is a
 * deployment aid.)
 *
 * Some callers cannot call cudaMalloc once they are running: a real-time control process that
 * fixes its device memory at start-up because an allocation can synchronize the device and take
 * unbounded time inside the syndrome cycle, or a plug-in whose host application owns all device
 * memory.  qldpc_decode_host allocates device staging on first use (and grows it); this entry
 * point instead stages through one file-scope device array of QLDPC_NOALLOC_SCRATCH_BYTES.  It
 * calls no cudaMalloc, cudaFree or allocating library routine.  The driver places the array in a
 * device's memory when the library's module holding it is first loaded on that device, which
 * (with CUDA's default lazy module loading) is the first call of this function there, and keeps
 * it until the process exits.  So call it once with batch = 0 at start-up, on each device, with
 * that device current and before any stream capture: that call checks its arguments, resolves
 * the array's device address (cudaGetSymbolAddress) and returns.  The first decode of each kernel
 * variant (precision, schedule, learned weights) can likewise load that kernel's code: run one
 * decode of each kind you will use during start-up as well.
 *
 * Arguments, outputs and the synchronous behaviour are those of qldpc_decode_host (host buffers
 * in, host buffers out, stream synchronized before returning).  The prior is copied on every call.
 * The batch must fit the scratch: with a(x) = x rounded up to 256 bytes,
 *   a(4n) + a(batch*m) + a(batch*n) + a(4*batch) + a(batch) <= QLDPC_NOALLOC_SCRATCH_BYTES
 * (e.g. up to 2749 shots of a 465 x 1054 graph); a larger batch returns QLDPC_ERR_UNSUPPORTED
 * and enqueues nothing.  Invalid arguments (QLDPC_ERR_INVALID_ARG) and a launch plan the kernels
 * cannot run (QLDPC_ERR_UNSUPPORTED) are also reported before anything is enqueued.
 *
 * All calls in the process
 * share the one array and it keeps the last call's contents; nothing in it needs to start at zero
 * because every byte a call reads is first written by that call.  Calls whose work overlaps on the
 * GPU (other threads, other streams) race on the array: serialize them.
 */
QLDPC_API int qldpc_decode_host_noalloc(const qldpc_graph *g, const uint8_t *h_syndromes,
                                        int32_t batch, const float *h_prior, int32_t max_iter,
                                        float alpha, uint8_t *h_err, int32_t *h_iters,
                                        uint8_t *h_ok, int32_t precision, uint32_t flags,
                                        void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QLDPC_H */
