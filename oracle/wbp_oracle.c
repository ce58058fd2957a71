/*
 * FP64 reference for weighted belief propagation unrolled over T iterations,
 * with its loss and its exact reverse-mode gradient.  TEST INFRASTRUCTURE
 * ONLY: the parity tests, the smoke check and the benchmark's CPU-baseline
 * leg call it; the product path never does.  It shares no code, header or
 * table with the CUDA kernels (nor with bp_oracle.c).
 *
 * What it computes.  The decoder is the flooding sum-product decoder of the
 * paper (section "Early Termination": tanh/atanh check rule, syndrome sign,
 * l_out as the a-posteriori value), run for exactly T iterations with no early
 * termination, and with one scaling weight per (iteration, edge class) on the
 * check-to-variable messages:
 *
 *   u_e^(k)   = Lch_v + sum_{e' in M(v), e' != e} c2v_e'^(k-1)       (v2c before the clamp)
 *   a_e^(k)   = clamp(u_e^(k), -lmax, lmax)
 *   t_e^(k)   = (1 - 2 s_c) * 2 atanh( prod_{e' in N(c), e' != e} tanh(a_e'^(k) / 2) )
 *               (a check of degree 1: (1 - 2 s_c) * lmax)
 *   c2v_e^(k) = w[k][class(e)] * t_e^(k)
 *   APP_v^(k) = Lch_v + sum_{e in M(v)} c2v_e^(k)
 *
 * with c2v^(0) = 0, e an edge (c, v), N(c) the edges of check c and M(v) those
 * of variable v.  The loss is the mean binary cross-entropy of the soft
 * output of the last iteration against the transmitted bits x, with
 * P(x_v = 1) = 1 / (1 + exp(APP_v)) (L = ln P(0)/P(1)):
 *
 *   loss = 1/(F n) * sum_f sum_v softplus(-(1 - 2 x_v) APP_v^(T)).
 *
 * Readings (the paper trains no weights; these fix what the weights mean):
 *   the weight multiplies the check's outgoing message after the clamp; the
 *   check-side clamp only binds for degree-1 checks (|a (+) b| <= min(|a|,|b|)
 *   <= lmax otherwise), so its derivative is 0 there and 1 elsewhere; the
 *   variable-side clamp passes the gradient where |u| <= lmax (closed
 *   interval, as torch.clamp does); only the last iteration's output enters
 *   the loss.
 *
 * The gradient is the chain rule taken backwards through the stored forward
 * values, written as plain loops:
 *
 *   G_e   = dloss/dc2v_e^(T) = g_v with g_v = dloss/dAPP_v^(T)
 *   for k = T .. 1:
 *     dloss/dw[k][cl] += sum_{e in cl} G_e t_e^(k)
 *     dt_e  = G_e w[k][class(e)] (0 at degree-1 checks)
 *     da_j  = (1 - 2 s_c) sum_{e in N(c), e != j} dt_e dPhi_e/da_j,
 *             dPhi_e/da_j = (1 - tanh^2(a_j/2)) prod_{i != e, j} tanh(a_i/2) / (1 - P_e^2),
 *             P_e = prod_{i in N(c), i != e} tanh(a_i/2)
 *     du_j  = da_j [|u_j| <= lmax]
 *     dloss/dLch_v += sum_{e in M(v)} du_e
 *     G_e  <- sum_{e' in M(v), e' != e} du_e'       (now dloss/dc2v^(k-1))
 *
 * Per-frame results are combined in frame order, so the output does not
 * depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double clamp_lim(double x, double lim)
{
    if (x > lim) return lim;
    if (x < -lim) return -lim;
    return x;
}

/* log(1 + exp(z)) without overflow */
static double softplus(double z)
{
    return z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
}

static double sigmoid(double z)
{
    return z >= 0.0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
}

typedef struct {
    int64_t m, n, E;
    const int64_t *rowptr;   /* [m+1] check-major edges */
    const int32_t *colidx;   /* [E] variable of each edge */
    int64_t *vptr;           /* [n+1] variable-major adjacency */
    int64_t *vedge;          /* [E] edge ids of variable v, ascending */
    int64_t *echeck;         /* [E] check of each edge */
} graph;

static int graph_init(graph *g, int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx)
{
    g->m = m;
    g->n = n;
    g->E = rowptr[m];
    g->rowptr = rowptr;
    g->colidx = colidx;
    g->vptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->vedge = (int64_t *)malloc((size_t)(g->E > 0 ? g->E : 1) * sizeof(int64_t));
    g->echeck = (int64_t *)malloc((size_t)(g->E > 0 ? g->E : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->vptr || !g->vedge || !g->echeck || !fill) {
        free(fill);
        return -1;
    }
    for (int64_t e = 0; e < g->E; ++e) g->vptr[colidx[e] + 1] += 1;
    for (int64_t v = 0; v < n; ++v) g->vptr[v + 1] += g->vptr[v];
    for (int64_t c = 0; c < m; ++c)
        for (int64_t e = rowptr[c]; e < rowptr[c + 1]; ++e) {
            const int64_t v = colidx[e];
            g->vedge[g->vptr[v] + fill[v]] = e;
            fill[v] += 1;
            g->echeck[e] = c;
        }
    free(fill);
    return 0;
}

static void graph_free(graph *g)
{
    free(g->vptr);
    free(g->vedge);
    free(g->echeck);
}

/* One frame: forward over T iterations (every iteration's values kept), loss,
 * and, if want_grad, the backward pass.  gw: [T][n_classes] (this frame's
 * contribution), gl: [n] (dloss/dLch of this frame). */
static int wbp_frame(const graph *g, const float *llr, const uint8_t *s, const uint8_t *x, int T,
                     int n_classes, const int32_t *cls, const double *w, double lmax, double scale,
                     double *app, double *loss, int want_grad, double *gw, double *gl)
{
    const int64_t E = g->E, n = g->n, m = g->m;
    double *c2v = (double *)calloc((size_t)(T + 1) * (size_t)(E > 0 ? E : 1), sizeof(double));
    double *tt = (double *)calloc((size_t)(T + 1) * (size_t)(E > 0 ? E : 1), sizeof(double));
    double *uu = (double *)calloc((size_t)(T + 1) * (size_t)(E > 0 ? E : 1), sizeof(double));
    double *G = (double *)calloc((size_t)(E > 0 ? E : 1), sizeof(double));
    double *dt = (double *)calloc((size_t)(E > 0 ? E : 1), sizeof(double));
    double *du = (double *)calloc((size_t)(E > 0 ? E : 1), sizeof(double));
    if (!c2v || !tt || !uu || !G || !dt || !du) {
        free(c2v); free(tt); free(uu); free(G); free(dt); free(du);
        return -1;
    }
    (void)n_classes;

    /* ---- forward ---- */
    for (int k = 1; k <= T; ++k) {
        const double *cold = c2v + (size_t)(k - 1) * E;
        double *cnew = c2v + (size_t)k * E;
        double *u = uu + (size_t)k * E;
        double *t = tt + (size_t)k * E;
        /* variable to check: explicit exclusive sums */
        for (int64_t v = 0; v < n; ++v) {
            for (int64_t a = g->vptr[v]; a < g->vptr[v + 1]; ++a) {
                double sum = (double)llr[v];
                for (int64_t b = g->vptr[v]; b < g->vptr[v + 1]; ++b)
                    if (b != a) sum += cold[g->vedge[b]];
                u[g->vedge[a]] = sum;
            }
        }
        /* check to variable: explicit exclusive products */
        for (int64_t c = 0; c < m; ++c) {
            const double sgn = s[c] ? -1.0 : 1.0;
            const int64_t e0 = g->rowptr[c], e1 = g->rowptr[c + 1];
            for (int64_t e = e0; e < e1; ++e) {
                double val;
                if (e1 - e0 == 1) {
                    val = sgn * lmax;
                } else {
                    double prod = 1.0;
                    for (int64_t f = e0; f < e1; ++f)
                        if (f != e) prod *= tanh(0.5 * clamp_lim(u[f], lmax));
                    val = clamp_lim(sgn * 2.0 * atanh(prod), lmax);
                }
                t[e] = val;
                cnew[e] = w[(size_t)(k - 1) * n_classes + cls[e]] * val;
            }
        }
    }
    const double *cT = c2v + (size_t)T * E;
    double lsum = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        double L = (double)llr[v];
        for (int64_t a = g->vptr[v]; a < g->vptr[v + 1]; ++a) L += cT[g->vedge[a]];
        app[v] = L;
        const double sx = x[v] ? -1.0 : 1.0;
        lsum += softplus(-sx * L);
    }
    *loss = lsum * scale;
    if (!want_grad) {
        free(c2v); free(tt); free(uu); free(G); free(dt); free(du);
        return 0;
    }

    /* ---- backward ---- */
    for (int64_t v = 0; v < n; ++v) {
        const double sx = x[v] ? -1.0 : 1.0;
        const double gv = -sx * sigmoid(-sx * app[v]) * scale;
        gl[v] = gv;
        for (int64_t a = g->vptr[v]; a < g->vptr[v + 1]; ++a) G[g->vedge[a]] = gv;
    }
    for (int k = T; k >= 1; --k) {
        const double *t = tt + (size_t)k * E;
        const double *u = uu + (size_t)k * E;
        const double *wk = w + (size_t)(k - 1) * n_classes;
        double *gwk = gw + (size_t)(k - 1) * n_classes;
        for (int64_t e = 0; e < E; ++e) gwk[cls[e]] += G[e] * t[e];
        for (int64_t c = 0; c < m; ++c) {
            const int64_t e0 = g->rowptr[c], e1 = g->rowptr[c + 1];
            for (int64_t e = e0; e < e1; ++e) dt[e] = (e1 - e0 == 1) ? 0.0 : G[e] * wk[cls[e]];
        }
        for (int64_t c = 0; c < m; ++c) {
            const double sgn = s[c] ? -1.0 : 1.0;
            const int64_t e0 = g->rowptr[c], e1 = g->rowptr[c + 1];
            for (int64_t j = e0; j < e1; ++j) {
                double da = 0.0;
                if (e1 - e0 > 1) {
                    const double tj = tanh(0.5 * clamp_lim(u[j], lmax));
                    for (int64_t e = e0; e < e1; ++e) {
                        if (e == j) continue;
                        double P = 1.0, rest = 1.0;
                        for (int64_t i = e0; i < e1; ++i) {
                            if (i == e) continue;
                            const double ti = tanh(0.5 * clamp_lim(u[i], lmax));
                            P *= ti;
                            if (i != j) rest *= ti;
                        }
                        const double dphi = (1.0 - tj * tj) * rest / (1.0 - P * P);
                        da += dt[e] * sgn * dphi;
                    }
                }
                du[j] = fabs(u[j]) <= lmax ? da : 0.0;
            }
        }
        for (int64_t v = 0; v < n; ++v) {
            double S = 0.0;
            for (int64_t a = g->vptr[v]; a < g->vptr[v + 1]; ++a) S += du[g->vedge[a]];
            gl[v] += S;
            for (int64_t a = g->vptr[v]; a < g->vptr[v + 1]; ++a) {
                double ex = 0.0;
                for (int64_t b = g->vptr[v]; b < g->vptr[v + 1]; ++b)
                    if (b != a) ex += du[g->vedge[b]];
                G[g->vedge[a]] = ex;
            }
        }
    }
    free(c2v); free(tt); free(uu); free(G); free(dt); free(du);
    return 0;
}

/* Weighted BP over F frames.  app_out [F][n] (APP of the last iteration);
 * loss_out [1]; grad_w [T][n_classes] and grad_llr [F][n] may be NULL (then
 * no backward pass).  Returns 0, or -1 on allocation failure / bad input. */
int oracle_wbp(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx, int64_t frames,
               const float *llr, const uint8_t *syn, const uint8_t *x, int32_t T, int32_t n_classes,
               const int32_t *edge_class, const double *w, double lmax, double *app_out, double *loss_out,
               double *grad_w, double *grad_llr, int32_t threads)
{
    if (T < 1 || n_classes < 1 || frames < 0) return -1;
    graph g;
    if (graph_init(&g, m, n, rowptr, colidx) != 0) return -1;
    for (int64_t e = 0; e < g.E; ++e)
        if (edge_class[e] < 0 || edge_class[e] >= n_classes) {
            graph_free(&g);
            return -1;
        }
    const int want_grad = grad_w != NULL || grad_llr != NULL;
    const size_t nw = (size_t)T * (size_t)n_classes;
    double *fl = (double *)calloc((size_t)(frames > 0 ? frames : 1), sizeof(double));
    double *fgw = want_grad ? (double *)calloc((size_t)(frames > 0 ? frames : 1) * nw, sizeof(double)) : NULL;
    double *fgl = want_grad ? (double *)calloc((size_t)(frames > 0 ? frames : 1) * (size_t)(n > 0 ? n : 1),
                                               sizeof(double)) : NULL;
    if (!fl || (want_grad && (!fgw || !fgl))) {
        free(fl); free(fgw); free(fgl);
        graph_free(&g);
        return -1;
    }
    const double scale = (frames > 0 && n > 0) ? 1.0 / ((double)frames * (double)n) : 0.0;
    int failed = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t f = 0; f < frames; ++f) {
        int r = wbp_frame(&g, llr + (size_t)f * n, syn + (size_t)f * m, x + (size_t)f * n, T, n_classes,
                          edge_class, w, lmax, scale, app_out + (size_t)f * n, fl + f, want_grad,
                          want_grad ? fgw + (size_t)f * nw : NULL, want_grad ? fgl + (size_t)f * n : NULL);
        if (r != 0) {
#pragma omp atomic write
            failed = 1;
        }
    }
    double L = 0.0;
    for (int64_t f = 0; f < frames; ++f) L += fl[f];
    *loss_out = L;
    if (want_grad) {
        if (grad_w) {
            for (size_t i = 0; i < nw; ++i) grad_w[i] = 0.0;
            for (int64_t f = 0; f < frames; ++f)
                for (size_t i = 0; i < nw; ++i) grad_w[i] += fgw[(size_t)f * nw + i];
        }
        if (grad_llr) memcpy(grad_llr, fgl, (size_t)frames * (size_t)n * sizeof(double));
    }
    free(fl); free(fgw); free(fgl);
    graph_free(&g);
    return failed ? -1 : 0;
}
