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
 * Precisions: f64 and f32 run the steps above in that type.  i8 is i16 below with 2 fractional
 * bits and messages saturated to +-127 (the paper names 8-bit integers without a scheme).  i16 is the fixed-point reading of
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
 * Fixed-point decoders with 32-bit accumulation: i16 (8 fractional bits, messages within
 * +-32767) and i8 (2 fractional bits, messages within +-127).
 * ------------------------------------------------------------------------------------------- */
static int32_t clampq(int64_t x, int32_t lim)
{
    if (x > lim) return lim;
    if (x < -lim) return -lim;
    return (int32_t)x;
}

/* gamma_q = clamp(round_half_away(gamma * 2^frac), -lim, lim); returns 0 on a non-finite gamma */
static int quantize_fixed(float g, int frac, int32_t lim, int32_t *out)
{
    if (!isfinite(g)) return 0;
    float t = roundf(g * (float)(1 << frac));   /* exact scaling; roundf rounds halves away from zero */
    if (t > (float)lim) t = (float)lim;
    if (t < -(float)lim) t = -(float)lim;
    *out = (int32_t)t;
    return 1;
}


int oracle_alpha_q(float alpha)
{
    if (!isfinite(alpha) || alpha <= 0.0f || alpha > 1.0f) return -1;
    int32_t a = (int32_t)roundf(alpha * 32768.0f);
    return (a >= 1 && a <= 32768) ? a : -1;
}

static int msa_fixed(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                     const uint8_t *syn, int32_t batch, const float *prior, int32_t max_iter,
                     float alpha, uint32_t flags, uint8_t *out_err, int32_t *out_iters,
                     uint8_t *out_ok, int32_t *out_post_q, double *out_margin, int frac, int32_t lim)
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
        if (!quantize_fixed(prior[v], frac, lim, &gq[v])) {
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
                        q[t.vedge[a]] = clampq(acc, lim);
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
        if (out_margin) out_margin[b] = (double)margin / (double)(1 << frac);
    }
    free(gq); free(q); free(r); free(post); tanner_free(&t);
    return ORACLE_OK;
}

int oracle_msa_i16(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                   const uint8_t *syn, int32_t batch, const float *prior, int32_t max_iter,
                   float alpha, uint32_t flags, uint8_t *out_err, int32_t *out_iters,
                   uint8_t *out_ok, int32_t *out_post_q, double *out_margin)
{
    return msa_fixed(row_ptr, col_idx, m, n, syn, batch, prior, max_iter, alpha, flags, out_err, out_iters,
                     out_ok, out_post_q, out_margin, 8, 32767);
}

/* i8: LLRs with 2 fractional bits (a quarter), messages saturated to +-127 (+-31.75), Q in 32 bits,
 * alpha_q and |r| = floor(min * alpha_q / 2^15) as for i16. */
int oracle_msa_i8(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                  const uint8_t *syn, int32_t batch, const float *prior, int32_t max_iter,
                  float alpha, uint32_t flags, uint8_t *out_err, int32_t *out_iters,
                  uint8_t *out_ok, int32_t *out_post_q, double *out_margin)
{
    return msa_fixed(row_ptr, col_idx, m, n, syn, batch, prior, max_iter, alpha, flags, out_err, out_iters,
                     out_ok, out_post_q, out_margin, 2, 127);
}

/* ---------------------------------------------------------------------------------------------
 * Layered (row-serial) schedule.  Algorithm 1 updates every check from the previous iteration's
 * messages (flooding); the layered schedule, a standard alternative for the same min-sum update,
 * visits the checks one after another within an iteration and lets each use the a-posteriori LLRs
 * already refreshed by the checks before it:
 *   start    Q_n = gamma_n, r_{m,n} = 0
 *   check m (ascending index), for n in S_v(m):
 *            q_{m,n} = Q_n - r_{m,n}
 *            r_{m,n} = (-1)^{s_m} prod_{j != n} sign(q_{m,j}) * (alpha * min_{j != n} |q_{m,j}|)
 *            Q_n     = q_{m,n} + r_{m,n}                     (with the new r)
 *   after the last check: e_n = [Q_n < 0] and the stop test, exactly as for flooding (iteration-0
 *   test, early stop, ok, iters).
 * Fixed point (i16, i8): the a-posteriori LLR stays the exact 32-bit sum of Algorithm 1's APP step,
 * Q_n = gamma_n + sum_m r_{m,n}, updated per check as Q_n <- Q_n - r_old + r_new; only the check's
 * input is clamped, q = clamp(Q - r_old, +-lim), and |r| = floor(min * alpha_q / 2^15).
 * --------------------------------------------------------------------------------------------- */
#define DEFINE_LAYERED_REAL(NAME, REAL, FABS)                                                     \
int NAME(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,                   \
         const uint8_t *syn, int32_t batch, const REAL *prior, int32_t max_iter, REAL alpha,      \
         uint32_t flags, uint8_t *out_err, int32_t *out_iters, uint8_t *out_ok, REAL *out_post)   \
{                                                                                                 \
    if (batch < 0 || max_iter < 0 || !syn || !prior || !out_err || !out_iters || !out_ok)        \
        return ORACLE_BAD_ARG;                                                                    \
    tanner t;                                                                                     \
    int rc = tanner_build(&t, row_ptr, col_idx, m, n);                                            \
    if (rc) return rc;                                                                            \
    const int early = !(flags & ORACLE_NO_EARLY_STOP);                                           \
    const size_t E = (size_t)(t.e > 0 ? t.e : 1);                                                 \
    REAL *q = (REAL *)malloc(sizeof(REAL) * E), *r = (REAL *)malloc(sizeof(REAL) * E);           \
    REAL *rn = (REAL *)malloc(sizeof(REAL) * E), *Q = (REAL *)malloc(sizeof(REAL) * (size_t)n);  \
    if (!q || !r || !rn || !Q) { free(q); free(r); free(rn); free(Q); tanner_free(&t); return ORACLE_NO_MEMORY; } \
    for (int32_t b = 0; b < batch; ++b) {                                                         \
        const uint8_t *s = syn + (size_t)b * m;                                                   \
        uint8_t *e_hat = out_err + (size_t)b * n;                                                 \
        for (int32_t v = 0; v < n; ++v) { Q[v] = prior[v]; e_hat[v] = prior[v] < 0; }           \
        int met = syndrome_met(&t, e_hat, s);                                                     \
        int32_t iters = 0;                                                                        \
        if (!(early && met) && max_iter > 0) {                                                    \
            for (int32_t i = 0; i < t.e; ++i) r[i] = 0;                                           \
            for (int32_t k = 1; k <= max_iter; ++k) {                                             \
                for (int32_t c = 0; c < m; ++c) {                                                 \
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) q[i] = Q[col_idx[i]] - r[i]; \
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {                       \
                        int neg = s[c] & 1;                                                       \
                        REAL mn = (REAL)INFINITY;                                                 \
                        for (int32_t j = row_ptr[c]; j < row_ptr[c + 1]; ++j) {                   \
                            if (j == i) continue;                                                 \
                            if (q[j] < 0) neg ^= 1;                                               \
                            if (FABS(q[j]) < mn) mn = FABS(q[j]);                                 \
                        }                                                                         \
                        REAL mag = alpha * mn;                                                    \
                        rn[i] = neg ? -mag : mag;                                                 \
                    }                                                                             \
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {                       \
                        Q[col_idx[i]] = q[i] + rn[i];                                             \
                        r[i] = rn[i];                                                             \
                    }                                                                             \
                }                                                                                 \
                for (int32_t v = 0; v < n; ++v) e_hat[v] = Q[v] < 0;                              \
                iters = k;                                                                        \
                met = syndrome_met(&t, e_hat, s);                                                 \
                if (early && met) break;                                                          \
            }                                                                                     \
        }                                                                                         \
        out_iters[b] = iters;                                                                     \
        out_ok[b] = (uint8_t)met;                                                                 \
        if (out_post) memcpy(out_post + (size_t)b * n, Q, sizeof(REAL) * (size_t)n);              \
    }                                                                                             \
    free(q); free(r); free(rn); free(Q); tanner_free(&t);                                         \
    return ORACLE_OK;                                                                             \
}

DEFINE_LAYERED_REAL(oracle_layered_f64, double, fabs)
DEFINE_LAYERED_REAL(oracle_layered_f32, float, fabsf)

static int layered_fixed(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                         const uint8_t *syn, int32_t batch, const float *prior, int32_t max_iter,
                         float alpha, uint32_t flags, uint8_t *out_err, int32_t *out_iters,
                         uint8_t *out_ok, int32_t *out_post_q, int frac, int32_t lim)
{
    if (batch < 0 || max_iter < 0 || !syn || !prior || !out_err || !out_iters || !out_ok)
        return ORACLE_BAD_ARG;
    const int32_t alpha_q = oracle_alpha_q(alpha);
    if (alpha_q < 0) return ORACLE_BAD_ARG;
    tanner t;
    int rc = tanner_build(&t, row_ptr, col_idx, m, n);
    if (rc) return rc;
    const int early = !(flags & ORACLE_NO_EARLY_STOP);
    const size_t E = (size_t)(t.e > 0 ? t.e : 1);
    int32_t *gq = (int32_t *)malloc(sizeof(int32_t) * (size_t)n), *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * E), *r = (int32_t *)malloc(sizeof(int32_t) * E);
    int32_t *rn = (int32_t *)malloc(sizeof(int32_t) * E);
    if (!gq || !Q || !q || !r || !rn) {
        free(gq); free(Q); free(q); free(r); free(rn); tanner_free(&t);
        return ORACLE_NO_MEMORY;
    }
    for (int32_t v = 0; v < n; ++v)
        if (!quantize_fixed(prior[v], frac, lim, &gq[v])) {
            free(gq); free(Q); free(q); free(r); free(rn); tanner_free(&t);
            return ORACLE_BAD_ARG;
        }
    for (int32_t b = 0; b < batch; ++b) {
        const uint8_t *s = syn + (size_t)b * m;
        uint8_t *e_hat = out_err + (size_t)b * n;
        for (int32_t v = 0; v < n; ++v) { Q[v] = gq[v]; e_hat[v] = gq[v] < 0; }
        int met = syndrome_met(&t, e_hat, s);
        int32_t iters = 0;
        if (!(early && met) && max_iter > 0) {
            for (int32_t i = 0; i < t.e; ++i) r[i] = 0;
            for (int32_t k = 1; k <= max_iter; ++k) {
                for (int32_t c = 0; c < m; ++c) {
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i)
                        q[i] = clampq((int64_t)Q[col_idx[i]] - r[i], lim);
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {
                        int neg = s[c] & 1;
                        int32_t mn = INT32_MAX;
                        for (int32_t j = row_ptr[c]; j < row_ptr[c + 1]; ++j) {
                            if (j == i) continue;
                            if (q[j] < 0) neg ^= 1;
                            const int32_t a = q[j] < 0 ? -q[j] : q[j];
                            if (a < mn) mn = a;
                        }
                        const int32_t mag = (int32_t)(((int64_t)mn * alpha_q) >> 15);
                        rn[i] = neg ? -mag : mag;
                    }
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {
                        Q[col_idx[i]] = Q[col_idx[i]] - r[i] + rn[i];   /* exact: Q = gamma + sum r */
                        r[i] = rn[i];
                    }
                }
                for (int32_t v = 0; v < n; ++v) e_hat[v] = Q[v] < 0;
                iters = k;
                met = syndrome_met(&t, e_hat, s);
                if (early && met) break;
            }
        }
        out_iters[b] = iters;
        out_ok[b] = (uint8_t)met;
        if (out_post_q) memcpy(out_post_q + (size_t)b * n, Q, sizeof(int32_t) * (size_t)n);
    }
    free(gq); free(Q); free(q); free(r); free(rn); tanner_free(&t);
    return ORACLE_OK;
}

int oracle_layered_i16(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                       const uint8_t *syn, int32_t batch, const float *prior, int32_t max_iter,
                       float alpha, uint32_t flags, uint8_t *out_err, int32_t *out_iters,
                       uint8_t *out_ok, int32_t *out_post_q)
{
    return layered_fixed(row_ptr, col_idx, m, n, syn, batch, prior, max_iter, alpha, flags, out_err, out_iters,
                         out_ok, out_post_q, 8, 32767);
}

int oracle_layered_i8(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                      const uint8_t *syn, int32_t batch, const float *prior, int32_t max_iter,
                      float alpha, uint32_t flags, uint8_t *out_err, int32_t *out_iters,
                      uint8_t *out_ok, int32_t *out_post_q)
{
    return layered_fixed(row_ptr, col_idx, m, n, syn, batch, prior, max_iter, alpha, flags, out_err, out_iters,
                         out_ok, out_post_q, 2, 127);
}

/* ---------------------------------------------------------------------------------------------
 * Neural normalized min-sum: Algorithm 1 with the scale alpha replaced by a learned weight
 * w[t][e] per iteration t (0-based here, iteration t+1 of the algorithm) and per edge e (CSR edge
 * order: e = row_ptr[m] + position of n in row m):
 *   r^(t)_{m,n} = (-1)^{s_m} prod_{j != n} sign(q^(t-1)_{m,j}) * (w[t][e] * min_{j != n} |q^(t-1)_{m,j}|)
 * with the variable step and a-posteriori LLR of Algorithm 1 unchanged (literal sums over
 * S_c(n)\m in ascending check order, as in the plain decoder above).
 *
 * Training loss of one shot with true error y (the sampled e), over T iterations, no stop test:
 *   loss = sum_{t=1..T} lambda_t / N sum_n BCE(sigma(-Q^(t)_n), y_n),  BCE(p, y) = -y log p - (1-y) log(1-p)
 * with per-iteration loss weights lambda_t (default 1/T: the mean over iterations and variables)
 * evaluated as softplus(Q) for y = 1 and softplus(-Q) for y = 0 (softplus(x) = log(1 + e^x)):
 * Q = log P(e_n = 0)/P(e_n = 1), so P(e_n = 1) = sigma(-Q).
 *
 * Syndrome loss (loss_kind 1): the same unrolled decoder scored on the syndrome instead of the
 * sampled error.  With independent bits of P(e_n = 1) = sigma(-Q_n), the parity of row m is odd
 * with probability (1 - prod_{n in S_v(m)} tanh(Q_n / 2)) / 2 (the product of the bits' 1 - 2p),
 * so the probability that the soft output reproduces s_m is
 *   P_m = (1 + (-1)^{s_m} prod_{n in S_v(m)} tanh(Q_n / 2)) / 2,
 *   loss = sum_{t=1..T} lambda_t / M sum_m -log(max(P^(t)_m, 1e-7)),
 * the BCE of the soft syndrome against s.  It is blind to which error of a coset the outputs
 * point at (any e with H e = s scores the same), as a quantum code's decoder may be.
 *   dloss_m/dQ_n = -(1 / P_m) (-1)^{s_m} / 2 prod_{j in S_v(m)\n} tanh(Q_j / 2) (1 - tanh^2(Q_n / 2)) / 2,
 * and 0 where the floor 1e-7 is active.
 *
 * Reverse mode (the gradient of sum_b g_b loss_b with respect to w), with the subgradient rules
 *   d|q|/dq = +1 for q >= 0, -1 for q < 0;  d sign(q)/dq = 0;
 *   the minimum over S_v(m)\n flows to the lowest-index edge attaining it.
 * The forward runs in REAL (double or float, the float one operation for operation the learned
 * decoder below); losses and the whole reverse sweep are evaluated in double from the recorded
 * forward values.
 * --------------------------------------------------------------------------------------------- */
static double softplus_d(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
static double sigmoid_d(double x) { return x >= 0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x)); }
#define SYN_LOSS_FLOOR 1e-7

/* P_m of the syndrome loss for row c from a-posteriori LLRs Q (any precision, evaluated in double). */
static double syndrome_match_prob(const tanner *t, int32_t c, const uint8_t *s, const double *Qd)
{
    double prod = 1.0;
    for (int32_t i = t->row_ptr[c]; i < t->row_ptr[c + 1]; ++i) prod *= tanh(0.5 * Qd[t->col[i]]);
    return 0.5 * (1.0 + ((s[c] & 1) ? -prod : prod));
}

/* Adds scale * dloss_c/dQ_n to gQ[n] for every n of row c (the product over S_v(c)\n taken literally). */
static void syndrome_loss_grad(const tanner *t, int32_t c, const uint8_t *s, const double *Qd, double scale,
                               double *gQ)
{
    const double P = syndrome_match_prob(t, c, s, Qd);
    if (!(P > SYN_LOSS_FLOOR)) return;
    const double sg = (s[c] & 1) ? -1.0 : 1.0;
    for (int32_t i = t->row_ptr[c]; i < t->row_ptr[c + 1]; ++i) {
        double others = 1.0;
        for (int32_t j = t->row_ptr[c]; j < t->row_ptr[c + 1]; ++j)
            if (j != i) others *= tanh(0.5 * Qd[t->col[j]]);
        const double th = tanh(0.5 * Qd[t->col[i]]);
        gQ[t->col[i]] += scale * (-(1.0 / P) * 0.5 * sg * others * 0.5 * (1.0 - th * th));
    }
}

#define DEFINE_NMS_TRAIN(SUFFIX, REAL, FABS)                                                          \
/* CN update of check c with weights w_t; records per edge the sign factor, the minimum over the    \
 * other edges and the edge attaining it (lowest index on ties; -1 for a row of degree 1). */       \
static void nms_check_##SUFFIX(const tanner *t, int32_t c, const uint8_t *s, const REAL *q,           \
                               const REAL *w_t, REAL *r, double *sgn, REAL *mu, int32_t *arg)        \
{                                                                                                     \
    for (int32_t i = t->row_ptr[c]; i < t->row_ptr[c + 1]; ++i) {                                     \
        int neg = s[c] & 1;                                                                           \
        REAL mn = (REAL)INFINITY;                                                                     \
        int32_t am = -1;                                                                              \
        for (int32_t j = t->row_ptr[c]; j < t->row_ptr[c + 1]; ++j) {                                 \
            if (j == i) continue;                                                                     \
            if (q[j] < 0) neg ^= 1;                                                                   \
            if (FABS(q[j]) < mn) { mn = FABS(q[j]); am = j; }                                         \
        }                                                                                             \
        sgn[i] = neg ? -1.0 : 1.0;                                                                    \
        mu[i] = mn;                                                                                   \
        arg[i] = am;                                                                                  \
        const REAL mag = w_t[i] * mn;                                                                 \
        r[i] = neg ? -mag : mag;                                                                      \
    }                                                                                                 \
}                                                                                                     \
                                                                                                      \
int oracle_nms_train_##SUFFIX(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,   \
                              const uint8_t *syn, const uint8_t *target, int32_t batch,               \
                              const REAL *prior, const REAL *weights, int32_t T,                      \
                              const double *loss_w, int32_t loss_kind, const double *grad_loss,       \
                              double *out_loss, REAL *out_post, double *out_grad)                     \
{                                                                                                     \
    if (batch < 0 || T < 1 || !syn || !target || !prior || !weights || !out_loss) return ORACLE_BAD_ARG; \
    if (loss_kind != 0 && loss_kind != 1) return ORACLE_BAD_ARG;                                      \
    if (out_grad && !grad_loss) return ORACLE_BAD_ARG;                                                \
    tanner t;                                                                                         \
    int rc = tanner_build(&t, row_ptr, col_idx, m, n);                                                \
    if (rc) return rc;                                                                                \
    const size_t E = (size_t)(t.e > 0 ? t.e : 1), TE = E * (size_t)T;                                 \
    REAL *qs = (REAL *)malloc(sizeof(REAL) * TE);      /* q^(k): input of iteration k+1 */            \
    REAL *rs = (REAL *)malloc(sizeof(REAL) * TE);                                                     \
    REAL *mus = (REAL *)malloc(sizeof(REAL) * TE);                                                    \
    double *sgs = (double *)malloc(sizeof(double) * TE);                                              \
    int32_t *ams = (int32_t *)malloc(sizeof(int32_t) * TE);                                           \
    REAL *Qs = (REAL *)malloc(sizeof(REAL) * (size_t)n * (size_t)T);                                  \
    double *gq = (double *)malloc(sizeof(double) * E), *gq_prev = (double *)malloc(sizeof(double) * E); \
    double *gr = (double *)malloc(sizeof(double) * E), *gQ = (double *)malloc(sizeof(double) * (size_t)n); \
    double *Qd = (double *)malloc(sizeof(double) * (size_t)n);                                         \
    if (!qs || !rs || !mus || !sgs || !ams || !Qs || !gq || !gq_prev || !gr || !gQ || !Qd) {          \
        rc = ORACLE_NO_MEMORY;                                                                        \
        goto done;                                                                                    \
    }                                                                                                 \
    for (int32_t b = 0; b < batch; ++b) {                                                             \
        const uint8_t *s = syn + (size_t)b * m, *y = target + (size_t)b * n;                          \
        /* forward: T iterations of CN, VN and APP */                                                 \
        for (int32_t i = 0; i < t.e; ++i) qs[i] = prior[t.col[i]];                                    \
        double loss = 0.0;                                                                            \
        for (int32_t k = 0; k < T; ++k) {                                                             \
            const double lw = loss_w ? loss_w[k] : 1.0 / T;                                           \
            double it_loss = 0.0;                                                                     \
            const REAL *q = qs + (size_t)k * E;                                                       \
            REAL *r = rs + (size_t)k * E;                                                             \
            for (int32_t c = 0; c < m; ++c)                                                           \
                nms_check_##SUFFIX(&t, c, s, q, weights + (size_t)k * t.e, r, sgs + (size_t)k * E,     \
                                   mus + (size_t)k * E, ams + (size_t)k * E);                         \
            for (int32_t v = 0; v < n; ++v) {                                                         \
                REAL Q = prior[v];                                                                    \
                for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) Q = Q + r[t.vedge[a]];            \
                Qs[(size_t)k * n + v] = Q;                                                            \
                Qd[v] = (double)Q;                                                                    \
                if (loss_kind == 0) it_loss += y[v] ? softplus_d((double)Q) : softplus_d(-(double)Q); \
                if (out_post) out_post[((size_t)b * T + k) * n + v] = Q;                              \
                if (k + 1 < T) {                                                                      \
                    REAL *qn = qs + (size_t)(k + 1) * E;                                              \
                    for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) {                             \
                        REAL acc = prior[v];                                                          \
                        for (int32_t bb = t.vptr[v]; bb < t.vptr[v + 1]; ++bb)                        \
                            if (bb != a) acc = acc + r[t.vedge[bb]];                                  \
                        qn[t.vedge[a]] = acc;                                                         \
                    }                                                                                 \
                }                                                                                     \
            }                                                                                         \
            if (loss_kind == 1) {                                                                     \
                for (int32_t c = 0; c < m; ++c) {                                                     \
                    const double P = syndrome_match_prob(&t, c, s, Qd);                               \
                    it_loss += -log(P > SYN_LOSS_FLOOR ? P : SYN_LOSS_FLOOR);                         \
                }                                                                                     \
                loss += lw * (it_loss / m);                                                           \
            } else {                                                                                  \
                loss += lw * (it_loss / n);                                                           \
            }                                                                                         \
        }                                                                                             \
        out_loss[b] = loss;                                                                           \
        if (!out_grad) continue;                                                                      \
        /* reverse sweep, iteration T down to 1 */                                                    \
        const double scale = grad_loss[b] / (loss_kind == 1 ? m : n);                                 \
        for (int32_t i = 0; i < t.e; ++i) gq[i] = 0.0;    /* d/d q^(k+1): feeds iteration k+2 */      \
        for (int32_t k = T - 1; k >= 0; --k) {                                                        \
            const double lw = loss_w ? loss_w[k] : 1.0 / T;                                           \
            if (loss_kind == 1) {                                                                     \
                for (int32_t v = 0; v < n; ++v) {                                                     \
                    gQ[v] = 0.0;                                                                      \
                    Qd[v] = (double)Qs[(size_t)k * n + v];                                            \
                }                                                                                     \
                for (int32_t c = 0; c < m; ++c) syndrome_loss_grad(&t, c, s, Qd, scale * lw, gQ);     \
            } else {                                                                                  \
                for (int32_t v = 0; v < n; ++v)                                                       \
                    gQ[v] = scale * lw * ((double)y[v] - sigmoid_d(-(double)Qs[(size_t)k * n + v]));  \
            }                                                                                         \
            /* r^(k+1)_{m,n} enters Q^(k+1)_n and every q^(k+1)_{i,n} with i != m */                  \
            for (int32_t v = 0; v < n; ++v)                                                           \
                for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) {                                 \
                    double acc = gQ[v];                                                               \
                    for (int32_t bb = t.vptr[v]; bb < t.vptr[v + 1]; ++bb)                            \
                        if (bb != a) acc += gq[t.vedge[bb]];                                          \
                    gr[t.vedge[a]] = acc;                                                             \
                }                                                                                     \
            const REAL *q = qs + (size_t)k * E;                                                       \
            for (int32_t i = 0; i < t.e; ++i) gq_prev[i] = 0.0;                                       \
            for (int32_t i = 0; i < t.e; ++i) {                                                       \
                const double sg = sgs[(size_t)k * E + i], mn = (double)mus[(size_t)k * E + i];        \
                out_grad[(size_t)k * t.e + i] += gr[i] * sg * mn;            /* d r / d w = sg mn */  \
                const int32_t j = ams[(size_t)k * E + i];                                             \
                if (j >= 0) {                                /* d r / d q_j = w sg d|q_j|/dq_j */     \
                    const double dabs = q[j] >= 0 ? 1.0 : -1.0;                                       \
                    gq_prev[j] += gr[i] * (double)weights[(size_t)k * t.e + i] * sg * dabs;           \
                }                                                                                     \
            }                                                                                         \
            for (int32_t i = 0; i < t.e; ++i) gq[i] = gq_prev[i];                                     \
        }                                                                                             \
    }                                                                                                 \
done:                                                                                                 \
    free(qs); free(rs); free(mus); free(sgs); free(ams); free(Qs);                                    \
    free(gq); free(gq_prev); free(gr); free(gQ); free(Qd);                                            \
    tanner_free(&t);                                                                                  \
    return rc;                                                                                        \
}

DEFINE_NMS_TRAIN(f64, double, fabs)
DEFINE_NMS_TRAIN(f32, float, fabsf)

/* Learned decoding for inference, FP32: iterations 1..T use the weights with the stop test of
 * Algorithm 1; a shot whose syndrome is not met after T iterations is decoded again from its prior
 * by plain min-sum (alpha, early stop, up to max_iter_plain iterations).  iters = learned
 * iterations run, plus T + the plain iterations for a fallback shot; ok and the outputs are those
 * of the decoder that produced them.  out_fallback[b] = 1 for fallback shots. */
int oracle_nms_decode_f32(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                          const uint8_t *syn, int32_t batch, const float *prior, const float *weights,
                          int32_t T, int32_t max_iter_plain, float alpha, uint8_t *out_err,
                          int32_t *out_iters, uint8_t *out_ok, float *out_post, uint8_t *out_fallback)
{
    if (batch < 0 || T < 0 || max_iter_plain < 0 || !syn || !prior || !weights || !out_err || !out_iters || !out_ok)
        return ORACLE_BAD_ARG;
    tanner t;
    int rc = tanner_build(&t, row_ptr, col_idx, m, n);
    if (rc) return rc;
    const size_t E = (size_t)(t.e > 0 ? t.e : 1);
    float *q = (float *)malloc(sizeof(float) * E), *r = (float *)malloc(sizeof(float) * E);
    float *post = (float *)malloc(sizeof(float) * (size_t)n);
    if (!q || !r || !post) { free(q); free(r); free(post); tanner_free(&t); return ORACLE_NO_MEMORY; }
    for (int32_t b = 0; b < batch; ++b) {
        const uint8_t *s = syn + (size_t)b * m;
        uint8_t *e_hat = out_err + (size_t)b * n;
        for (int32_t v = 0; v < n; ++v) { post[v] = prior[v]; e_hat[v] = prior[v] < 0; }
        int met = syndrome_met(&t, e_hat, s);
        int32_t iters = 0;
        int fell_back = 0;
        if (!met) {
            for (int32_t i = 0; i < t.e; ++i) q[i] = prior[t.col[i]];
            for (int32_t k = 1; k <= T && !met; ++k) {
                const float *w = weights + (size_t)(k - 1) * t.e;
                for (int32_t c = 0; c < m; ++c)
                    for (int32_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) {
                        int neg = s[c] & 1;
                        float mn = INFINITY;
                        for (int32_t j = row_ptr[c]; j < row_ptr[c + 1]; ++j) {
                            if (j == i) continue;
                            if (q[j] < 0) neg ^= 1;
                            if (fabsf(q[j]) < mn) mn = fabsf(q[j]);
                        }
                        const float mag = w[i] * mn;
                        r[i] = neg ? -mag : mag;
                    }
                for (int32_t v = 0; v < n; ++v)
                    for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) {
                        float acc = prior[v];
                        for (int32_t bb = t.vptr[v]; bb < t.vptr[v + 1]; ++bb)
                            if (bb != a) acc = acc + r[t.vedge[bb]];
                        q[t.vedge[a]] = acc;
                    }
                for (int32_t v = 0; v < n; ++v) {
                    float acc = prior[v];
                    for (int32_t a = t.vptr[v]; a < t.vptr[v + 1]; ++a) acc = acc + r[t.vedge[a]];
                    post[v] = acc;
                    e_hat[v] = acc < 0;
                }
                iters = k;
                met = syndrome_met(&t, e_hat, s);
            }
            if (!met) {
                int32_t it2 = 0;
                uint8_t ok2 = 0;
                float *post2 = (float *)malloc(sizeof(float) * (size_t)n);
                if (!post2) { free(q); free(r); free(post); tanner_free(&t); return ORACLE_NO_MEMORY; }
                rc = oracle_msa_f32(row_ptr, col_idx, m, n, s, 1, prior, max_iter_plain, alpha, 0u, e_hat, &it2, &ok2,
                                    post2, NULL);
                memcpy(post, post2, sizeof(float) * (size_t)n);
                free(post2);
                if (rc) { free(q); free(r); free(post); tanner_free(&t); return rc; }
                iters = T + it2;
                met = ok2;
                fell_back = 1;
            }
        }
        out_iters[b] = iters;
        out_ok[b] = (uint8_t)met;
        if (out_post) memcpy(out_post + (size_t)b * n, post, sizeof(float) * (size_t)n);
        if (out_fallback) out_fallback[b] = (uint8_t)fell_back;
    }
    free(q); free(r); free(post); tanner_free(&t);
    return ORACLE_OK;
}
