/*
 * CPU oracle: plain, slow FP64 Kalman-filter log-likelihood of a pulsar timing
 * array and its gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the CUDA product path shares
 * no code with it.
 *
 * What it computes (paper, Functionality: the likelihood of the TOA data
 * evaluated by a Kalman filter in O(N); pulsars are independent given the
 * parameters of a deterministic continuous-wave source, so the array
 * log-likelihood is the sum of the pulsar log-likelihoods):
 *
 *   ll(theta) = sum_p ll_p(theta),  theta = [log10 f, Phi0, psi, cos iota,
 *               sin delta, alpha, log10 h0, (log10 sigma_p, EFAC_p)_p]
 *
 * Model flags (bit 0: Ornstein-Uhlenbeck red noise, adding log10 gamma_p after
 * log10 sigma_p; bit 1: the pulsar term of the wave, adding the pulsar's
 * distance d_p in kpc after EFAC_p).
 *
 * The continuous-wave residual is the Earth term of a monochromatic source
 * (paper, Future Directions, and the prior work it cites):
 *   n = (cos d cos a, cos d sin a, sin d), u = (sin a, -cos a, 0),
 *   v = (sin d cos a, sin d sin a, -cos d), p = cos psi u + sin psi v,
 *   q = -sin psi u + cos psi v,
 *   F+ = ((c.p)^2 - (c.q)^2) / (2 (1 - n.c)),  Fx = (c.p)(c.q) / (1 - n.c),
 *   s(t) = A sin(W t + Phi0) + B cos(W t + Phi0),
 *   A = F+ h0 (1 + cos^2 i) / W,  B = -2 Fx h0 cos i / W,  W = 2 pi f.
 * The pulsar term (the source of the paper's cited prior work on pulsar
 * terms) is the same wave met by the pulsar at the retarded time
 * t - tau_p, tau_p = d_p (1 - n.c) / c, and enters with the opposite sign:
 *   s(t) = A sin(W t + Phi0) + B cos(W t + Phi0)
 *          - [A sin(W t + Phi0 - W tau_p) + B cos(W t + Phi0 - W tau_p)].
 * 1 - n.c is clamped at 1e-12 in both terms.
 *
 * The gradient is taken by the complex-step method (Squire & Trapp 1998):
 * d ll / d theta_j = Im ll(theta + i h e_j) / h with h = 1e-20, evaluated
 * through the same filter code in complex arithmetic.  It shares nothing with
 * the reverse-mode adjoint of the CUDA path.
 *
 * Out-of-domain parameter vectors (non-finite, EFAC <= 0, |cos i| > 1,
 * |sin d| > 1) and filters that meet S_k <= 0 get ll = -inf and a zero
 * gradient.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#define LOG2PI 1.8378770664093454836
#define CS_H 1e-20
#define N_GW 7
/* light-travel time over one kiloparsec, s: 1 pc = (648000 / pi) au,
   1 au = 149597870700 m, c = 299792458 m/s (IAU 2012 / 2015 definitions) */
#define KPC_LIGHT_S (1e3 * (648000.0 / M_PI) * 149597870700.0 / 299792458.0)

typedef double complex cplx;

/* ---- the filter, instantiated for double and for double complex ---- */
#define KF_T double
#define KF_NAME kf_real
#define KF_PHI ou_phi_real
#define KF_EXP exp
#define KF_SIN sin
#define KF_COS cos
#define KF_LOG log
#define KF_RE(x) (x)
#define KF_LOG2PI LOG2PI
#include "kf_body.h"
#undef KF_T
#undef KF_NAME
#undef KF_PHI
#undef KF_EXP
#undef KF_SIN
#undef KF_COS
#undef KF_LOG
#undef KF_RE

#define KF_T cplx
#define KF_NAME kf_cplx
#define KF_PHI ou_phi_cplx
#define KF_EXP cexp
#define KF_SIN csin
#define KF_COS ccos
#define KF_LOG clog
#define KF_RE(x) creal(x)
#include "kf_body.h"

/* ---- continuous-wave projection, in complex arithmetic ---- */
static void cw_project(const cplx th[N_GW], const double c[3],
                       cplx* A, cplx* B, cplx* Om, cplx* Phi0, cplx* Dn)
{
    cplx f = cpow(10.0, th[0]);
    cplx W = 2.0 * M_PI * f;
    cplx psi = th[2], cosi = th[3], sind = th[4], al = th[5];
    cplx h0 = cpow(10.0, th[6]);
    cplx cosd = csqrt(1.0 - sind * sind);
    cplx n[3] = {cosd * ccos(al), cosd * csin(al), sind};
    cplx u[3] = {csin(al), -ccos(al), 0.0};
    cplx v[3] = {sind * ccos(al), sind * csin(al), -cosd};
    cplx p[3], q[3];
    for (int i = 0; i < 3; ++i) {
        p[i] = ccos(psi) * u[i] + csin(psi) * v[i];
        q[i] = -csin(psi) * u[i] + ccos(psi) * v[i];
    }
    cplx cp = c[0] * p[0] + c[1] * p[1] + c[2] * p[2];
    cplx cq = c[0] * q[0] + c[1] * q[1] + c[2] * q[2];
    cplx D = 1.0 - (c[0] * n[0] + c[1] * n[1] + c[2] * n[2]);
    if (creal(D) < 1e-12) D = 1e-12 + I * cimag(D);   /* source behind the pulsar */
    cplx Fp = 0.5 * (cp * cp - cq * cq) / D;
    cplx Fx = cp * cq / D;
    *A = Fp * h0 * (1.0 + cosi * cosi) / W;
    *B = -2.0 * Fx * h0 * cosi / W;
    *Om = W;
    *Phi0 = th[1];
    *Dn = D;
}

typedef struct {
    int P;
    const int64_t* off;
    const double *t, *r, *sigma, *pos, *equad, *p0;
    int ou;    /* Ornstein-Uhlenbeck red noise: log10 gamma after log10 sigma */
    int pt;    /* pulsar term: distance d (kpc) after EFAC */
} array_view;

/* parameters per pulsar: (log10 sigma, [log10 gamma], EFAC, [d]) */
static int n_noise(const array_view* a) { return 2 + a->ou + a->pt; }
static int efac_slot(const array_view* a) { return 1 + a->ou; }

static int theta_in_domain(const array_view* a, const double* th)
{
    int np = n_noise(a), D = N_GW + np * a->P;
    for (int j = 0; j < D; ++j)
        if (!isfinite(th[j])) return 0;
    if (fabs(th[3]) > 1.0 || fabs(th[4]) > 1.0) return 0;
    for (int p = 0; p < a->P; ++p) {
        if (!(th[N_GW + np * p + efac_slot(a)] > 0.0)) return 0;
        if (a->pt && !(th[N_GW + np * p + np - 1] > 0.0)) return 0;
    }
    return 1;
}

/* one pulsar, complex parameters; nz = its own parameters (n_noise of them) */
static cplx pulsar_ll_c(const array_view* a, int p, const cplx thgw[N_GW], const cplx* nz,
                        int* bad)
{
    cplx A, B, Om, Phi0, Dn;
    cw_project(thgw, a->pos + 3 * p, &A, &B, &Om, &Phi0, &Dn);
    cplx sig2 = cpow(10.0, 2.0 * nz[0]);
    cplx gam = a->ou ? cpow(10.0, nz[1]) : 0.0;
    cplx efac = nz[efac_slot(a)];
    cplx Dp = a->pt ? Om * (nz[n_noise(a) - 1] * KPC_LIGHT_S * Dn) : 0.0;
    int64_t o = a->off[p], n = a->off[p + 1] - a->off[p];
    return kf_cplx(n, a->t + o, a->r + o, a->sigma + o, a->equad[p], a->p0 + 3 * p,
                   A, B, Om, Phi0, sig2, efac, a->ou, gam, a->pt, Dp, bad, NULL, NULL);
}

/* one pulsar, real parameters */
static double pulsar_ll_r(const array_view* a, int p, const double* th, int* bad)
{
    cplx thc[N_GW];
    for (int j = 0; j < N_GW; ++j) thc[j] = th[j];
    cplx A, B, Om, Phi0, Dn;
    cw_project(thc, a->pos + 3 * p, &A, &B, &Om, &Phi0, &Dn);
    int np = n_noise(a);
    const double* nz = th + N_GW + np * p;
    double sig2 = pow(10.0, 2.0 * nz[0]);
    double gam = a->ou ? pow(10.0, nz[1]) : 0.0;
    double efac = nz[efac_slot(a)];
    double Dp = a->pt ? creal(Om) * (nz[np - 1] * KPC_LIGHT_S * creal(Dn)) : 0.0;
    int64_t o = a->off[p], n = a->off[p + 1] - a->off[p];
    return kf_real(n, a->t + o, a->r + o, a->sigma + o, a->equad[p], a->p0 + 3 * p,
                   creal(A), creal(B), creal(Om), creal(Phi0), sig2, efac, a->ou, gam, a->pt, Dp,
                   bad, NULL, NULL);
}

static double walker_ll(const array_view* a, const double* th, double* lane_ll)
{
    if (!theta_in_domain(a, th)) {
        if (lane_ll) for (int p = 0; p < a->P; ++p) lane_ll[p] = -INFINITY;
        return -INFINITY;
    }
    double ll = 0.0;
    int bad = 0;
    for (int p = 0; p < a->P; ++p) {
        int b = 0;
        double lp = pulsar_ll_r(a, p, th, &b);
        if (b || isnan(lp)) lp = -INFINITY;
        if (lane_ll) lane_ll[p] = lp;
        bad |= b;
        ll += lp;
    }
    if (bad || isnan(ll)) ll = -INFINITY;
    return ll;
}

static void walker_grad(const array_view* a, const double* th, double* g)
{
    int P = a->P, np = n_noise(a), D = N_GW + np * P;
    memset(g, 0, sizeof(double) * D);
    cplx thgw[N_GW];
    for (int j = 0; j < N_GW; ++j) thgw[j] = th[j];
    int bad = 0;
    /* continuous-wave parameters: every pulsar depends on them */
    for (int j = 0; j < N_GW; ++j) {
        cplx tj[N_GW];
        memcpy(tj, thgw, sizeof(tj));
        tj[j] += I * CS_H;
        double acc = 0.0;
        for (int p = 0; p < P; ++p) {
            cplx nz[4];   /* at most (log10 sigma, log10 gamma, EFAC, d) */
            for (int i = 0; i < np; ++i) nz[i] = th[N_GW + np * p + i];
            cplx lp = pulsar_ll_c(a, p, tj, nz, &bad);
            acc += cimag(lp) / CS_H;
        }
        g[j] = acc;
    }
    /* per-pulsar noise parameters: only their own pulsar depends on them */
    for (int p = 0; p < P; ++p) {
        for (int i = 0; i < np; ++i) {
            cplx nz[4];   /* at most (log10 sigma, log10 gamma, EFAC, d) */
            for (int k = 0; k < np; ++k) nz[k] = th[N_GW + np * p + k];
            nz[i] += I * CS_H;
            cplx lp = pulsar_ll_c(a, p, thgw, nz, &bad);
            g[N_GW + np * p + i] = cimag(lp) / CS_H;
        }
    }
    if (bad) memset(g, 0, sizeof(double) * D);
}

/* ---------------------------- exported API ---------------------------- */

/* Array log-likelihood for B parameter vectors theta[B][D] -> out[B],
   D = 7 + (2 + (model & 1) + ((model >> 1) & 1)) P: model bit 0 selects the
   Ornstein-Uhlenbeck red noise, bit 1 the pulsar term.
   lane_out (optional, may be NULL): per-pulsar terms [B][P]. */
int oracle_loglik(int P, const int64_t* off, const double* t, const double* r,
                  const double* sigma, const double* pos, const double* equad,
                  const double* p0, int model, const double* theta, int64_t B,
                  double* out, double* lane_out)
{
    array_view a = {P, off, t, r, sigma, pos, equad, p0, model & 1, (model >> 1) & 1};
    int D = N_GW + n_noise(&a) * P;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        out[b] = walker_ll(&a, theta + b * D, lane_out ? lane_out + b * P : NULL);
    return 0;
}

/* Log-likelihood and gradient: out_ll[B], out_grad[B][D] (D as above). */
int oracle_loglik_grad(int P, const int64_t* off, const double* t, const double* r,
                       const double* sigma, const double* pos, const double* equad,
                       const double* p0, int model, const double* theta, int64_t B,
                       double* out_ll, double* out_grad)
{
    array_view a = {P, off, t, r, sigma, pos, equad, p0, model & 1, (model >> 1) & 1};
    int D = N_GW + n_noise(&a) * P;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b) {
        const double* th = theta + b * D;
        out_ll[b] = walker_ll(&a, th, NULL);
        if (isinf(out_ll[b]) && out_ll[b] < 0)
            memset(out_grad + b * D, 0, sizeof(double) * D);
        else
            walker_grad(&a, th, out_grad + b * D);
    }
    return 0;
}

/* Threads of the OpenMP loops over parameter vectors (n >= 1). */
#ifdef _OPENMP
#include <omp.h>
#endif
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Continuous-wave projection of one parameter vector onto one pulsar:
   out = {A, B, Omega, Phi0, 1 - n.c (clamped)}. */
int oracle_cw_project(const double* theta_gw, const double* pos, double* out)
{
    cplx th[N_GW];
    for (int j = 0; j < N_GW; ++j) th[j] = theta_gw[j];
    cplx A, B, Om, Phi0, Dn;
    cw_project(th, pos, &A, &B, &Om, &Phi0, &Dn);
    out[0] = creal(A); out[1] = creal(B); out[2] = creal(Om); out[3] = creal(Phi0);
    out[4] = creal(Dn);
    return 0;
}

/* One pulsar's filter with explicit lane parameters lane = {A, B, Omega,
   Phi0, sigma^2, EFAC, gamma, Dp}; gamma > 0 selects the Ornstein-Uhlenbeck
   model, 0 the random walk; Dp != 0 adds the pulsar term with that phase lag
   (rad); optionally returns the innovations e_k and their variances S_k (used
   by the calibration tests). */
double oracle_pulsar_filter(int64_t n, const double* t, const double* r, const double* sigma,
                            double equad, const double* p0, const double* lane,
                            double* e_out, double* S_out)
{
    int bad = 0;
    double ll = kf_real(n, t, r, sigma, equad, p0, lane[0], lane[1], lane[2], lane[3],
                        lane[4], lane[5], lane[6] > 0.0, lane[6], lane[7] != 0.0, lane[7],
                        &bad, e_out, S_out);
    return bad ? -INFINITY : ll;
}
