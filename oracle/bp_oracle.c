/*
 * FP64 reference sum-product (belief-propagation) decoder with the paper's
 * early-termination rules.  TEST INFRASTRUCTURE ONLY: the parity tests, the
 * smoke check and the benchmark's CPU-baseline leg call it; the product path
 * never does.  It shares no code, header or table with the CUDA decoder.
 *
 * What it computes (paper, section "Early Termination"):
 *   - flooding BP over the Tanner graph of H, at most D_max iterations;
 *   - check-node rule with tanh / atanh, the sign flipped by the syndrome bit
 *     of the check (syndrome-based reconciliation: H x = s);
 *   - l_out,i^(k): the log a-posteriori value of bit i after iteration k;
 *   - PCE-ET: stop with success when the hard decision meets H x^ = s;
 *   - VNR-ET: q^(k) = sum over variable nodes of degree > 1 of |l_out,i^(k)|;
 *     stop (abort) when q^(k) < q^(k-1).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   LLR L = ln P(x=0)/P(x=1); hard decision x^ = 1 iff L < 0 (a tie gives 0);
 *   q uses magnitudes |L|; the first VNR comparison is at k = vnr_first_iter
 *   (2: q^(2) vs q^(1); 1: q^(1) vs q^(0) = sum over V of |Lch|); the
 *   comparison is strict; PCE is tested before VNR in the same iteration;
 *   no test is made before the first iteration; v2c and c2v messages are
 *   clamped to [-lmax, lmax]; the APP value is not clamped.
 *
 * oracle_decode_weighted adds learned weights (one per iteration and edge
 * class) on the check-to-variable messages, the reading the weighted-BP
 * oracle (wbp_oracle.c) also takes; the early-termination rules are unchanged.
 *
 * Everything is plain loops in the order the algorithm states them; the
 * exclusive sums and products are taken by explicit loops, never by removing
 * one's own term from a total.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { RULE_NONE = 0, RULE_PCE = 1, RULE_PCE_VNR = 2 };
enum { FLAG_SUCCESS = 1, FLAG_ABORTED = 2 };

static double clampd(double x, double lim)
{
    if (x > lim) return lim;
    if (x < -lim) return -lim;
    return x;
}

/* Variable-node adjacency: for variable v, the edge ids (positions in the
 * check-major CSR arrays) that touch it, in increasing edge id. */
typedef struct {
    int64_t *ptr;   /* [n+1] */
    int64_t *edge;  /* [E]   */
} var_adj;

static int build_var_adj(int64_t n, int64_t m, const int64_t *rowptr,
                         const int32_t *colidx, var_adj *a)
{
    int64_t E = rowptr[m];
    a->ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    a->edge = (int64_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!a->ptr || !a->edge || !fill) { free(fill); return -1; }
    for (int64_t e = 0; e < E; e++) a->ptr[colidx[e] + 1]++;
    for (int64_t v = 0; v < n; v++) a->ptr[v + 1] += a->ptr[v];
    for (int64_t e = 0; e < E; e++) {
        int64_t v = colidx[e];
        a->edge[a->ptr[v] + fill[v]++] = e;
    }
    free(fill);
    return 0;
}

/* 1 if the hard decision satisfies every check: XOR over N(c) of x^_v = s_c. */
static int syndrome_ok(int64_t m, const int64_t *rowptr, const int32_t *colidx,
                       const uint8_t *xhat, const uint8_t *s)
{
    for (int64_t c = 0; c < m; c++) {
        int par = s[c];
        for (int64_t e = rowptr[c]; e < rowptr[c + 1]; e++) par ^= xhat[colidx[e]];
        if (par) return 0;
    }
    return 1;
}

/* Decode one frame.  Returns 0, or -1 on allocation failure. */
static int decode_frame(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                        const var_adj *va, const float *llr_f, const uint8_t *s,
                        int max_iter, int rule, int vnr_first_iter, double lmax,
                        uint8_t *bits_out, uint8_t *flag_out, int32_t *iters_out,
                        double *app_out, int trace_iters, int64_t frame, int64_t frames,
                        double *trace_c2v, double *trace_app, double *trace_q,
                        const double *w, int w_iters, int n_classes, const int32_t *edge_class)
{
    int64_t E = rowptr[m];
    double *c2v = (double *)calloc((size_t)(E > 0 ? E : 1), sizeof(double));
    double *v2c = (double *)calloc((size_t)(E > 0 ? E : 1), sizeof(double));
    double *Lch = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *app = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    uint8_t *xhat = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!c2v || !v2c || !Lch || !app || !xhat) {
        free(c2v); free(v2c); free(Lch); free(app); free(xhat);
        return -1;
    }
    for (int64_t v = 0; v < n; v++) Lch[v] = (double)llr_f[v];

    /* V: variable nodes of degree higher than 1. */
    double q_prev = 0.0;
    if (vnr_first_iter <= 1) { /* q^(0) from the channel values */
        for (int64_t v = 0; v < n; v++)
            if (va->ptr[v + 1] - va->ptr[v] > 1) q_prev += fabs(Lch[v]);
    }

    int success = 0, aborted = 0, D = max_iter;
    for (int k = 1; k <= max_iter; k++) {
        /* 1. variable-to-check: channel value plus all other incoming c2v. */
        for (int64_t v = 0; v < n; v++) {
            for (int64_t a = va->ptr[v]; a < va->ptr[v + 1]; a++) {
                int64_t e = va->edge[a];
                double sum = Lch[v];
                for (int64_t b = va->ptr[v]; b < va->ptr[v + 1]; b++)
                    if (b != a) sum += c2v[va->edge[b]];
                v2c[e] = clampd(sum, lmax);
            }
        }
        /* 2. check-to-variable: tanh rule over the other edges of the check,
         *    sign flipped when the syndrome bit is 1. */
        for (int64_t c = 0; c < m; c++) {
            double sgn = s[c] ? -1.0 : 1.0;
            for (int64_t e = rowptr[c]; e < rowptr[c + 1]; e++) {
                double prod = 1.0;
                for (int64_t f = rowptr[c]; f < rowptr[c + 1]; f++)
                    if (f != e) prod *= tanh(0.5 * v2c[f]);
                c2v[e] = clampd(sgn * 2.0 * atanh(prod), lmax);
                if (w) /* weighted decoding: iteration k scales by row min(k, w_iters) */
                    c2v[e] *= w[(int64_t)((k < w_iters ? k : w_iters) - 1) * n_classes + edge_class[e]];
            }
        }
        /* 3. a-posteriori LLR and hard decision. */
        for (int64_t v = 0; v < n; v++) {
            double L = Lch[v];
            for (int64_t a = va->ptr[v]; a < va->ptr[v + 1]; a++) L += c2v[va->edge[a]];
            app[v] = L;
            xhat[v] = (uint8_t)(L < 0.0);
        }
        double q = 0.0;
        for (int64_t v = 0; v < n; v++)
            if (va->ptr[v + 1] - va->ptr[v] > 1) q += fabs(app[v]);
        if (k <= trace_iters) {
            int64_t base = (int64_t)(k - 1) * frames + frame;
            if (trace_c2v) memcpy(trace_c2v + base * E, c2v, (size_t)E * sizeof(double));
            if (trace_app) memcpy(trace_app + base * n, app, (size_t)n * sizeof(double));
            if (trace_q) trace_q[base] = q;
        }
        /* 4. PCE-ET, then VNR-ET. */
        if (rule != RULE_NONE && syndrome_ok(m, rowptr, colidx, xhat, s)) {
            success = 1; D = k; break;
        }
        if (rule == RULE_PCE_VNR && k >= vnr_first_iter && q < q_prev) {
            aborted = 1; D = k; break;
        }
        q_prev = q;
        if (k == max_iter) success = syndrome_ok(m, rowptr, colidx, xhat, s);
    }
    memcpy(bits_out, xhat, (size_t)n);
    if (app_out) memcpy(app_out, app, (size_t)n * sizeof(double));
    *flag_out = (uint8_t)((success ? FLAG_SUCCESS : 0) | (aborted ? FLAG_ABORTED : 0));
    *iters_out = D;
    free(c2v); free(v2c); free(Lch); free(app); free(xhat);
    return 0;
}

/*
 * Decode `frames` frames of the code H (m x n, check-major CSR with 64-bit
 * row pointers).  llr: [frames][n] float; syndrome: [frames][m] bytes 0/1.
 * Outputs: bits [frames][n], flags [frames] (bit0 success, bit1 aborted),
 * iters [frames], and (optional, may be NULL) app [frames][n], the APP values
 * of the last iteration run.  Traces (optional, may be NULL): c2v [trace_iters][frames][E]
 * in CSR edge order, app [trace_iters][frames][n], q [trace_iters][frames];
 * entries of iterations a frame did not run are left untouched.
 * threads <= 0 uses the OpenMP default.  Returns 0, or -1 on bad input or
 * allocation failure.
 */
static int decode_all(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                      int64_t frames, const float *llr, const uint8_t *syndrome,
                      int max_iter, int rule, int vnr_first_iter, double lmax,
                      uint8_t *bits_out, uint8_t *flags_out, int32_t *iters_out, double *app_out,
                      int trace_iters, double *trace_c2v, double *trace_app, double *trace_q,
                      int threads, const double *w, int w_iters, int n_classes, const int32_t *edge_class)
{
    if (m < 0 || n < 0 || frames < 0 || rule < 0 || rule > 2 || max_iter < 1) return -1;
    var_adj va;
    if (build_var_adj(n, m, rowptr, colidx, &va) != 0) return -1;
    int err = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (int64_t f = 0; f < frames; f++) {
        if (decode_frame(m, n, rowptr, colidx, &va, llr + f * n, syndrome + f * m,
                         max_iter, rule, vnr_first_iter, lmax, bits_out + f * n,
                         flags_out + f, iters_out + f, app_out ? app_out + f * n : NULL,
                         trace_iters, f, frames,
                         trace_c2v, trace_app, trace_q, w, w_iters, n_classes, edge_class) != 0)
            err |= 1;
    }
    free(va.ptr);
    free(va.edge);
    return err ? -1 : 0;
}

int oracle_decode(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                  int64_t frames, const float *llr, const uint8_t *syndrome,
                  int max_iter, int rule, int vnr_first_iter, double lmax,
                  uint8_t *bits_out, uint8_t *flags_out, int32_t *iters_out, double *app_out,
                  int trace_iters, double *trace_c2v, double *trace_app, double *trace_q,
                  int threads)
{
    return decode_all(m, n, rowptr, colidx, frames, llr, syndrome, max_iter, rule, vnr_first_iter, lmax,
                      bits_out, flags_out, iters_out, app_out, trace_iters, trace_c2v, trace_app, trace_q,
                      threads, NULL, 0, 0, NULL);
}

/*
 * The same decoder with the check-to-variable messages of iteration k scaled
 * by w[min(k, w_iters) - 1][edge_class[e]] (learned weights; iterations past
 * the last trained one keep its weights).  w: [w_iters][n_classes] doubles,
 * edge_class: [E] in CSR edge order with values in [0, n_classes).
 */
int oracle_decode_weighted(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                           int64_t frames, const float *llr, const uint8_t *syndrome,
                           int max_iter, int rule, int vnr_first_iter, double lmax,
                           uint8_t *bits_out, uint8_t *flags_out, int32_t *iters_out, double *app_out,
                           int trace_iters, double *trace_c2v, double *trace_app, double *trace_q,
                           int threads, const double *w, int w_iters, int n_classes,
                           const int32_t *edge_class)
{
    if (!w || w_iters < 1 || n_classes < 1 || !edge_class || m < 0) return -1;
    for (int64_t e = 0; e < rowptr[m]; e++)
        if (edge_class[e] < 0 || edge_class[e] >= n_classes) return -1;
    return decode_all(m, n, rowptr, colidx, frames, llr, syndrome, max_iter, rule, vnr_first_iter, lmax,
                      bits_out, flags_out, iters_out, app_out, trace_iters, trace_c2v, trace_app, trace_q,
                      threads, w, w_iters, n_classes, edge_class);
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
