/*
 * CPU oracle for syndrome-based normalized min-sum (MSA) decoding -- Algorithm 1, Sec. 2 of
 * "GPU-Accelerated Syndrome Decoding for Quantum LDPC Codes below the 63 us Latency Threshold"
 * (arXiv 2508.07879).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load this file; the decoder library never does.  It shares no code,
 * header, table or helper with the CUDA decoder.
 *
 * What it computes (one shot; H given in CSR, S_v(m) = columns of row m, S_c(n) = rows of column n):
 *   init     q_{m,n} = gamma_n for every edge                                    (Alg. 1, init)
 *   CN       r_{m,n} = (-1)^{s_m} * prod_{j in S_v(m)\n} sign(q_{m,j})
 *                      * alpha * min_{j in S_v(m)\n} |q_{m,j}|                    (Alg. 1, CN step)
 *   VN       q_{m,n} = gamma_n + sum_{i in S_c(n)\m} r_{i,n}                     (Alg. 1, VN step)
 *   APP      Q_n     = gamma_n + sum_{i in S_c(n)} r_{i,n}                       (Alg. 1, APP)
 *   decision e_n     = 1 if Q_n < 0 else 0                                       (Alg. 1, decision)
 *   stop     after each iteration, when H e^T = s (early stop on) or after I_max iterations.
 *
 * Every sum and minimum is taken literally over the sets the algorithm names (no min1/min2
 * shortcut, no "total minus own" extrinsic trick): the CN step loops over S_v(m)\n for every n
 * and the VN step over S_c(n)\m for every m.  Sums run in ascending check order starting from
 * gamma_n.
 *
 * Readings of the printed algorithm (where it is garbled or silent):
 *   - The CN factor "alpha s_m prod sign" is read as alpha * (-1)^{s_m} * prod sign; a literal
 *     s_m in {0,1} would zero every message of a satisfied check.
 *   - sign(x) = -1 iff x < 0 (so +0 and -0 count as positive); the decision maps Q = 0 to 0.
 *   - gamma_n is the caller's prior LLR (the algorithm prints gamma_n = 1; any uniform positive
 *     gamma gives the same decisions in exact arithmetic because min-sum is positively homogeneous).
 *   - The UNTIL line is read as: repeat while k <= I_max and H e^(k-1) != s.  The test is also
 *     made before the first iteration on e^(0) = [gamma < 0]; an already satisfied syndrome returns
 *     0 iterations.  iters counts the CN+VN rounds run.  Without convergence the outputs are the
 *     decisions of iteration I_max with ok = 0.  With ORACLE_NO_EARLY_STOP no test stops the loop
 *     (the paper's timed runs use 10 fixed iterations, Sec. 3) and ok reports H e = s at the end.
 *   - CN messages are formed as sign * (alpha * min): the product alpha * min is rounded first.
 *
 * Precisions: f64 and f32 run the steps above in that type.  i16 is the fixed-point reading of
 * the paper's integer proposal (Table 1, Sec. 3 outlook): LLRs carry 8 fractional bits,
 *   gamma_q = clamp(round_half_away(gamma * 256), -32767, 32767),
 *   alpha_q = round_half_away(alpha * 32768) with 1 <= alpha_q <= 32768,
 *   |r| = floor(min * alpha_q / 2^15), sign applied afterwards,
 *   q = clamp(gamma_q + sum_{i != m} r, -32767, 32767) (sum in 32-bit integers),
 *   Q = gamma_q + sum r in 32-bit integers (not clamped), decision on Q.
 *
 * Diagnostic: margin[b] is the smallest |q| or |Q| (and |gamma|) the shot ever produced, in LLR
 * units.  A shot whose margin is tiny had a near-tie whose sign is decided by rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NO_EARLY_STOP 1u

enum { ORACLE_OK = 0, ORACLE_BAD_GRAPH = -1, ORACLE_BAD_ARG = -2, ORACLE_NO_MEMORY = -3 };

typedef struct {
    int32_t m, n, e;
    const int32_t *row_ptr, *col;   /* CSR: edge e = (check chk[e], variable col[e]) */
    int32_t *chk;                   /* [e] check of each edge */
    int32_t *vptr, *vedge;          /* S_c(n) as edge ids, ascending check: vedge[vptr[n]..vptr[n+1]) */
} tanner;

static int tanner_build(tanner *t, const int32_t *row_ptr, const int32_t *col, int32_t m, int32_t n)
{
    if (!row_ptr || !col || m <= 0 || n <= 0 || row_ptr[0] != 0) return ORACLE_BAD_GRAPH;
    for (int32_t c = 0; c < m; ++c)
        if (row_ptr[c + 1] < row_ptr[c]) return ORACLE_BAD_GRAPH;
    int32_t e = row_ptr[m];
    for (int32_t i = 0; i < e; ++i)
        if (col[i] < 0 || col[i] >= n) return ORACLE_BAD_GRAPH;
    t->m = m; t->n = n; t->e = e; t->row_ptr = row_ptr; t->col = col;
    t->chk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(e > 0 ? e : 1));
    t->vptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    t->vedge = (int32_t *)malloc(sizeof(int32_t) * (size_t)(e > 0 ? e : 1));
    int32_t *fill = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!t->chk || !t->vptr || !t->vedge || !fill) {
        free(t->chk); free(t->vptr); free(t->vedge); free(fill);
        return ORACLE_NO_MEMORY;
    }
    for (int32_t c = 0; c < m; ++c)
        for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {
            t->chk[i] = c;
            t->vptr[col[i] + 1]++;
        }
    for (int32_t v = 0; v < n; ++v) t->vptr[v + 1] += t->vptr[v];
    /* rows are visited in ascending order, so each S_c(n) list comes out in ascending check order */
    for (int32_t c = 0; c < m; ++c)
        for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {
            int32_t v = col[i];
            t->vedge[t->vptr[v] + fill[v]++] = i;
        }
    free(fill);
    return ORACLE_OK;
}

static void tanner_free(tanner *t)
{
    free(t->chk); free(t->vptr); free(t->vedge);
}

/* 1 iff H e^T = s over GF(2) */
static int syndrome_met(const tanner *t, const uint8_t *e_hat, const uint8_t *s)
{
    for (int32_t c = 0; c < t->m; ++c) {
        int par = s[c] & 1;
        for (int32_t i = t->row_ptr[c]; i < t->row_ptr[c + 1]; ++i) par ^= e_hat[t->col[i]];
        if (par) return 0;
    }
    return 1;
}

/* ---------------------------------------------------------------------------------------------
 * Floating-point decoder, instantiated for double and float.
 * ------------------------------------------------------------------------------------------- */
#define DEFINE_MSA_REAL(NAME, REAL, FABS)                                                          \
int NAME(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,                   \
         const uint8_t *syn, int32_t batch, const REAL *prior, int32_t max_iter, REAL alpha,      \
         uint32_t flags, uint8_t *out_err, int32_t *out_iters, uint8_t *out_ok,                   \
         REAL *out_post, double *out_margin)                                                      \
{                                                                                                 \
    if (batch < 0 || max_iter < 0 || !syn || !prior || !out_err || !out_iters || !out_ok)        \
        return ORACLE_BAD_ARG;                                                                    \
    tanner t;                                                                                     \
    int rc = tanner_build(&t, row_ptr, col_idx, m, n);                                            \
    if (rc) return rc;                                                                            \
    const int early = !(flags & ORACLE_NO_EARLY_STOP);                                           \
    REAL *q = (REAL *)malloc(sizeof(REAL) * (size_t)(t.e > 0 ? t.e : 1));                        \
    REAL *r = (REAL *)malloc(sizeof(REAL) * (size_t)(t.e > 0 ? t.e : 1));                        \
    REAL *post = (REAL *)malloc(sizeof(REAL) * (size_t)n);                                        \
    if (!q || !r || !post) { free(q); free(r); free(post); tanner_free(&t); return ORACLE_NO_MEMORY; } \
    for (int32_t b = 0; b < batch; ++b) {                                                         \
        const uint8_t *s = syn + (size_t)b * m;                                                   \
        uint8_t *e_hat = out_err + (size_t)b * n;                                                 \
        double margin = INFINITY;                                                                 \
        /* iteration 0: decisions from the prior alone */                                        \
        for (int32_t v = 0; v < n; ++v) {                                                         \
            post[v] = prior[v];                                                                   \
            e_hat[v] = prior[v] < 0;                                                              \
            if ((double)FABS(prior[v]) < margin) margin = (double)FABS(prior[v]);                 \
        }                                                                                         \
        int met = syndrome_met(&t, e_hat, s);                                                     \
        int32_t iters = 0;                                                                        \
        if (!(early && met) && max_iter > 0) {                                                    \
            for (int32_t i = 0; i < t.e; ++i) q[i] = prior[t.col[i]];                             \
            for (int32_t k = 1; k <= max_iter; ++k) {                                             \
                /* check-node processing */                                                       \
                for (int32_t c = 0; c < m; ++c)                                                   \
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {                       \
                        int neg = s[c] & 1;                                                       \
                        REAL mn = (REAL)INFINITY;                                                 \
                        for (int32_t j = row_ptr[c]; j < row_ptr[c + 1]; ++j) {                   \
                            if (j == i) continue;                                                 \
                            if (q[j] < 0) neg ^= 1;                                               \
                            if (FABS(q[j]) < mn) mn = FABS(q[j]);                                 \
                        }                                                                         \
                        REAL mag = alpha * mn;                                                    \
                        r[i] = neg ? -mag : mag;                                                  \
                    }                                                                             \
                /* variable-node processing (extrinsic sums) */                                   \
                for (int32_t v = 0; v < n; ++v)                                                   \
                    for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) {                         \
                        REAL acc = prior[v];                                                      \
                        for (int32_t bb = t.vptr[v]; bb < t.vptr[v + 1]; ++bb)                    \
                            if (bb != a) acc = acc + r[t.vedge[bb]];                              \
                        q[t.vedge[a]] = acc;                                                      \
                        if ((double)FABS(acc) < margin) margin = (double)FABS(acc);               \
                    }                                                                             \
                /* a-posteriori LLR and tentative decision */                                     \
                for (int32_t v = 0; v < n; ++v) {                                                 \
                    REAL acc = prior[v];                                                          \
                    for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) acc = acc + r[t.vedge[a]]; \
                    post[v] = acc;                                                                \
                    e_hat[v] = acc < 0;                                                           \
                    if ((double)FABS(acc) < margin) margin = (double)FABS(acc);                   \
                }                                                                                 \
                iters = k;                                                                        \
                met = syndrome_met(&t, e_hat, s);                                                 \
                if (early && met) break;                                                          \
            }                                                                                     \
        }                                                                                         \
        out_iters[b] = iters;                                                                     \
        out_ok[b] = (uint8_t)met;                                                                 \
        if (out_post) memcpy(out_post + (size_t)b * n, post, sizeof(REAL) * (size_t)n);           \
        if (out_margin) out_margin[b] = margin;                                                   \
    }                                                                                             \
    free(q); free(r); free(post); tanner_free(&t);                                                \
    return ORACLE_OK;                                                                             \
}

DEFINE_MSA_REAL(oracle_msa_f64, double, fabs)
DEFINE_MSA_REAL(oracle_msa_f32, float, fabsf)

/* ---------------------------------------------------------------------------------------------
 * 16-bit fixed-point decoder (8 fractional bits, 32-bit accumulation).
 * ------------------------------------------------------------------------------------------- */
static int32_t clamp16(int64_t x)
{
    if (x > 32767) return 32767;
    if (x < -32767) return -32767;
    return (int32_t)x;
}

/* gamma_q = clamp(round_half_away(gamma * 256)); returns 0 on a non-finite gamma */
static int quantize_prior(float g, int32_t *out)
{
    if (!isfinite(g)) return 0;
    float t = roundf(g * 256.0f);          /* roundf rounds halves away from zero */
    if (t > 32767.0f) t = 32767.0f;
    if (t < -32767.0f) t = -32767.0f;
    *out = (int32_t)t;
    return 1;
}

int oracle_alpha_q(float alpha)
{
    if (!isfinite(alpha) || alpha <= 0.0f || alpha > 1.0f) return -1;
    int32_t a = (int32_t)roundf(alpha * 32768.0f);
    return (a >= 1 && a <= 32768) ? a : -1;
}

int oracle_msa_i16(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                   const uint8_t *syn, int32_t batch, const float *prior, int32_t max_iter,
                   float alpha, uint32_t flags, uint8_t *out_err, int32_t *out_iters,
                   uint8_t *out_ok, int32_t *out_post_q, double *out_margin)
{
    if (batch < 0 || max_iter < 0 || !syn || !prior || !out_err || !out_iters || !out_ok)
        return ORACLE_BAD_ARG;
    const int32_t alpha_q = oracle_alpha_q(alpha);
    if (alpha_q < 0) return ORACLE_BAD_ARG;
    tanner t;
    int rc = tanner_build(&t, row_ptr, col_idx, m, n);
    if (rc) return rc;
    const int early = !(flags & ORACLE_NO_EARLY_STOP);
    int32_t *gq = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(t.e > 0 ? t.e : 1));
    int32_t *r = (int32_t *)malloc(sizeof(int32_t) * (size_t)(t.e > 0 ? t.e : 1));
    int32_t *post = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!gq || !q || !r || !post) {
        free(gq); free(q); free(r); free(post); tanner_free(&t);
        return ORACLE_NO_MEMORY;
    }
    for (int32_t v = 0; v < n; ++v)
        if (!quantize_prior(prior[v], &gq[v])) {
            free(gq); free(q); free(r); free(post); tanner_free(&t);
            return ORACLE_BAD_ARG;
        }
    for (int32_t b = 0; b < batch; ++b) {
        const uint8_t *s = syn + (size_t)b * m;
        uint8_t *e_hat = out_err + (size_t)b * n;
        int64_t margin = INT64_MAX;
        for (int32_t v = 0; v < n; ++v) {
            post[v] = gq[v];
            e_hat[v] = gq[v] < 0;
            if (llabs((long long)gq[v]) < margin) margin = llabs((long long)gq[v]);
        }
        int met = syndrome_met(&t, e_hat, s);
        int32_t iters = 0;
        if (!(early && met) && max_iter > 0) {
            for (int32_t i = 0; i < t.e; ++i) q[i] = gq[t.col[i]];
            for (int32_t k = 1; k <= max_iter; ++k) {
                for (int32_t c = 0; c < m; ++c)
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {
                        int neg = s[c] & 1;
                        int64_t mn = INT64_MAX;
                        for (int32_t j = row_ptr[c]; j < row_ptr[c + 1]; ++j) {
                            if (j == i) continue;
                            if (q[j] < 0) neg ^= 1;
                            int64_t a = llabs((long long)q[j]);
                            if (a < mn) mn = a;
                        }
                        int32_t mag = (int32_t)((mn * (int64_t)alpha_q) >> 15);
                        r[i] = neg ? -mag : mag;
                    }
                for (int32_t v = 0; v < n; ++v)
                    for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) {
                        int64_t acc = gq[v];
                        for (int32_t bb = t.vptr[v]; bb < t.vptr[v + 1]; ++bb)
                            if (bb != a) acc += r[t.vedge[bb]];
                        q[t.vedge[a]] = clamp16(acc);
                        if (llabs((long long)q[t.vedge[a]]) < margin) margin = llabs((long long)q[t.vedge[a]]);
                    }
                for (int32_t v = 0; v < n; ++v) {
                    int64_t acc = gq[v];
                    for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) acc += r[t.vedge[a]];
                    post[v] = (int32_t)acc;
                    e_hat[v] = acc < 0;
                    if (llabs((long long)acc) < margin) margin = llabs((long long)acc);
                }
                iters = k;
                met = syndrome_met(&t, e_hat, s);
                if (early && met) break;
            }
        }
        out_iters[b] = iters;
        out_ok[b] = (uint8_t)met;
        if (out_post_q) memcpy(out_post_q + (size_t)b * n, post, sizeof(int32_t) * (size_t)n);
        if (out_margin) out_margin[b] = (double)margin / 256.0;
    }
    free(gq); free(q); free(r); free(post); tanner_free(&t);
    return ORACLE_OK;
}
