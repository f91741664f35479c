/*
 * CPU oracle of the joint (all-pulsar) likelihood with a Hellings-Downs
 * correlated gravitational-wave background.  TEST INFRASTRUCTURE ONLY.
 *
 * theta = [log10 h_a, log10 gamma_a, (log10 sigma_p, log10 gamma_p, EFAC_p)_p],
 * D = 2 + 3P.  The model is stated in gwb_body.h.  Hellings-Downs:
 *   G_nm = 3/2 x ln x - x/4 + 1/2,  x = (1 - c_n.c_m) / 2  (n != m),  G_nn = 1
 * (the autocorrelation includes the pulsar-term noise, which doubles the
 * n -> m limit 1/2).  Gradients by the complex-step method (Squire & Trapp
 * 1998) through the same filter in complex arithmetic.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LOG2PI 1.8378770664093454836
#define CS_H 1e-20

typedef double complex cplx;

#define KF_T double
#define GWB_NAME gwb_real
#define KF_NAME gwb_unused_real
#define KF_PHI gwb_phi_real
#define KF_EXP exp
#define KF_LOG log
#define KF_RE(x) (x)
#define KF_LOG2PI LOG2PI
#include "ou_phi.h"
#include "gwb_body.h"
#undef KF_T
#undef GWB_NAME
#undef KF_NAME
#undef KF_PHI
#undef KF_EXP
#undef KF_LOG
#undef KF_RE

#define KF_T cplx
#define GWB_NAME gwb_cplx
#define KF_NAME gwb_unused_cplx
#define KF_PHI gwb_phi_cplx
#define KF_EXP cexp
#define KF_LOG clog
#define KF_RE(x) creal(x)
#include "ou_phi.h"
#include "gwb_body.h"

/* Hellings-Downs matrix of the pulsar positions pos[P][3] -> G[P][P] */
void oracle_hellings_downs(int P, const double* pos, double* G)
{
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            if (a == b) { G[a * P + b] = 1.0; continue; }
            double c = pos[3 * a] * pos[3 * b] + pos[3 * a + 1] * pos[3 * b + 1] +
                       pos[3 * a + 2] * pos[3 * b + 2];
            double x = 0.5 * (1.0 - c);
            G[a * P + b] = (x > 0.0 ? 1.5 * x * log(x) : 0.0) - 0.25 * x + 0.5;
        }
}

typedef struct {
    int P;
    const int64_t* off;
    const double *t, *r, *sigma, *pos, *equad, *p0;
    double* G;
    int64_t* order;
    int* psr_of;
    int64_t N;
} gwb_view;

static int cmp_time_idx(const void* x, const void* y, void* ctx)
{
    const gwb_view* v = ctx;
    int64_t a = *(const int64_t*)x, b = *(const int64_t*)y;
    if (v->t[a] < v->t[b]) return -1;
    if (v->t[a] > v->t[b]) return 1;
    return (a > b) - (a < b);     /* global index: pulsar, then TOA */
}

static void view_init(gwb_view* v)
{
    v->N = v->off[v->P];
    v->G = malloc(sizeof(double) * v->P * v->P);
    oracle_hellings_downs(v->P, v->pos, v->G);
    v->order = malloc(sizeof(int64_t) * (v->N > 0 ? v->N : 1));
    v->psr_of = malloc(sizeof(int) * (v->N > 0 ? v->N : 1));
    for (int64_t g = 0; g < v->N; ++g) v->order[g] = g;
    qsort_r(v->order, (size_t)v->N, sizeof(int64_t), cmp_time_idx, v);
    for (int64_t j = 0; j < v->N; ++j) {
        int q = 0;
        while (v->order[j] >= v->off[q + 1]) ++q;
        v->psr_of[j] = q;
    }
}

static void view_free(gwb_view* v) { free(v->G); free(v->order); free(v->psr_of); }

static int gwb_in_domain(const gwb_view* v, const double* th)
{
    const int D = 2 + 3 * v->P;
    for (int j = 0; j < D; ++j)
        if (!isfinite(th[j])) return 0;
    for (int p = 0; p < v->P; ++p)
        if (!(th[2 + 3 * p + 2] > 0.0)) return 0;
    return 1;
}

static cplx gwb_ll_c(const gwb_view* v, const cplx* th, int* bad)
{
    const int P = v->P;
    cplx* s2 = malloc(sizeof(cplx) * P);
    cplx* gp = malloc(sizeof(cplx) * P);
    cplx* ef = malloc(sizeof(cplx) * P);
    for (int p = 0; p < P; ++p) {
        s2[p] = cpow(10.0, 2.0 * th[2 + 3 * p]);
        gp[p] = cpow(10.0, th[2 + 3 * p + 1]);
        ef[p] = th[2 + 3 * p + 2];
    }
    cplx ll = v->N == 0 ? 0.0
                        : gwb_cplx(P, v->off, v->t, v->r, v->sigma, v->equad, v->p0, v->G, v->order,
                                   v->psr_of, v->N, cpow(10.0, 2.0 * th[0]), cpow(10.0, th[1]), s2,
                                   gp, ef, bad);
    free(s2); free(gp); free(ef);
    return ll;
}

static double gwb_ll_r(const gwb_view* v, const double* th, int* bad)
{
    const int P = v->P;
    double* s2 = malloc(sizeof(double) * P);
    double* gp = malloc(sizeof(double) * P);
    double* ef = malloc(sizeof(double) * P);
    for (int p = 0; p < P; ++p) {
        s2[p] = pow(10.0, 2.0 * th[2 + 3 * p]);
        gp[p] = pow(10.0, th[2 + 3 * p + 1]);
        ef[p] = th[2 + 3 * p + 2];
    }
    double ll = v->N == 0 ? 0.0
                          : gwb_real(P, v->off, v->t, v->r, v->sigma, v->equad, v->p0, v->G, v->order,
                                     v->psr_of, v->N, pow(10.0, 2.0 * th[0]), pow(10.0, th[1]), s2, gp,
                                     ef, bad);
    free(s2); free(gp); free(ef);
    return ll;
}

/* Joint log-likelihood of B parameter vectors theta[B][2 + 3P] -> out[B]. */
int oracle_gwb_loglik(int P, const int64_t* off, const double* t, const double* r,
                      const double* sigma, const double* pos, const double* equad,
                      const double* p0, const double* theta, int64_t B, double* out)
{
    gwb_view v = {P, off, t, r, sigma, pos, equad, p0, NULL, NULL, NULL, 0};
    view_init(&v);
    const int D = 2 + 3 * P;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b) {
        const double* th = theta + b * D;
        int bad = 0;
        double ll = gwb_in_domain(&v, th) ? gwb_ll_r(&v, th, &bad) : -INFINITY;
        out[b] = (bad || isnan(ll)) ? -INFINITY : ll;
    }
    view_free(&v);
    return 0;
}

/* ... and its gradient out_grad[B][2 + 3P] (complex step). */
int oracle_gwb_loglik_grad(int P, const int64_t* off, const double* t, const double* r,
                           const double* sigma, const double* pos, const double* equad,
                           const double* p0, const double* theta, int64_t B, double* out_ll,
                           double* out_grad)
{
    gwb_view v = {P, off, t, r, sigma, pos, equad, p0, NULL, NULL, NULL, 0};
    view_init(&v);
    const int D = 2 + 3 * P;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b) {
        const double* th = theta + b * D;
        double* g = out_grad + b * D;
        int bad = 0;
        double ll = gwb_in_domain(&v, th) ? gwb_ll_r(&v, th, &bad) : -INFINITY;
        out_ll[b] = (bad || isnan(ll)) ? -INFINITY : ll;
        memset(g, 0, sizeof(double) * D);
        if (isinf(out_ll[b])) continue;
        cplx* thc = malloc(sizeof(cplx) * D);
        for (int j = 0; j < D; ++j) {
            for (int k = 0; k < D; ++k) thc[k] = th[k];
            thc[j] += I * CS_H;
            g[j] = cimag(gwb_ll_c(&v, thc, &bad)) / CS_H;
        }
        free(thc);
    }
    view_free(&v);
    return 0;
}
