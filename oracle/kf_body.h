/*
 * One pulsar's Kalman-filter log-likelihood, written once for a scalar type
 * KF_T and included twice by kalman.c: once with KF_T = double (the value) and
 * once with KF_T = double complex (complex-step derivatives).
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle; the product path never
 * links it.
 *
 * Model (paper, Functionality: "State-space model construction" and "Kalman
 * filter likelihood evaluation"): state x = (rho, y), rho the timing residual
 * (s) and y the fractional frequency deviation; d rho/dt = y, dy/dt = xi(t),
 * <xi(t) xi(t')> = sigma_p^2 delta(t - t').  Measurement r_k = rho(t_k) +
 * s(t_k) + eps_k, eps_k ~ N(0, R_k), R_k = EFAC^2 sigma_k^2 + EQUAD^2 (the
 * paper's separation of process noise from the EFAC/EQUAD measurement noise).
 * Prior x(t_1) ~ N(0, P0).  The log-likelihood is the prediction-error
 * decomposition: sum_k -1/2 (ln 2 pi + ln S_k + e_k^2 / S_k).
 *
 * With ou != 0 the frequency deviation is an Ornstein-Uhlenbeck process
 * instead (paper, Functionality: pulsar-intrinsic red noise as an OU
 * process): dy/dt = -gam y + xi(t).  Over dt, with x = gam dt,
 *   F = [[1, dt phi1(x)], [0, exp(-x)]],
 *   Q = sigma^2 [[dt^3/3 phi4(x), dt^2/2 phi1(x)^2], [., dt phi1(2x)]],
 *   phi1(x) = (1 - e^-x)/x,  phi4(x) = 3 (x - 2 (1 - e^-x) + (1 - e^-2x)/2) / x^3,
 * (both -> 1 as gam -> 0, the random walk), by their Taylor series below
 * x = 0.5 and the closed forms above.
 *
 * With pt != 0 the continuous-wave residual also carries its pulsar term:
 * the wave that passed the pulsar a time tau_p earlier, with the opposite
 * sign; for a monochromatic source that is the Earth-term sinusoid with its
 * phase lagging by Dp = Om tau_p (the caller forms Dp).
 *
 * Steps per TOA in textbook order: predict the mean (m = F m) and covariance
 * (P = F P F^T + Q), form the signal and the innovation e = r - s - H m with
 * H = (1, 0) and its variance S = H P H^T + R, gain K = P H^T / S, update
 * m = m + K e and P = P - K S K^T, accumulate the likelihood term.
 */
#include "ou_phi.h"

static KF_T KF_NAME(int64_t n, const double* t, const double* r, const double* sigma,
                    double equad, const double p0[3],
                    KF_T A, KF_T B, KF_T Om, KF_T Phi0, KF_T sig2, KF_T efac,
                    int ou, KF_T gam, int pt, KF_T Dp, int* bad, double* e_out, double* S_out)
{
    KF_T m0 = 0.0, m1 = 0.0;
    KF_T p00 = p0[0], p01 = p0[1], p11 = p0[2];
    KF_T ll = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double dt = (k == 0) ? 0.0 : t[k] - t[k - 1];
        /* transition F = [[1, b], [0, a]] and process noise Q; for the
           random walk b = dt, a = 1, Q = sigma^2 [[dt^3/3, dt^2/2], [dt^2/2, dt]] */
        KF_T b = dt, a = 1.0;
        KF_T q00 = sig2 * (dt * dt * dt / 3.0);
        KF_T q01 = sig2 * (dt * dt / 2.0);
        KF_T q11 = sig2 * dt;
        if (ou) {
            KF_T p1, p2, p4;
            KF_PHI(gam * dt, &p1, &p2, &p4);
            b = dt * p1;
            a = 1.0 - gam * dt * p1;
            q00 = q00 * p4;
            q01 = q01 * p1 * p1;
            q11 = q11 * p2;
        }
        /* predict */
        KF_T mp0 = m0 + b * m1;
        KF_T mp1 = a * m1;
        KF_T a00 = p00 + b * p01 + b * p01 + b * b * p11 + q00;
        KF_T a01 = a * (p01 + b * p11) + q01;
        KF_T a11 = a * a * p11 + q11;
        /* continuous-wave timing residual at this TOA */
        KF_T phase = Om * t[k] + Phi0;
        KF_T s = A * KF_SIN(phase) + B * KF_COS(phase);
        if (pt) s -= A * KF_SIN(phase - Dp) + B * KF_COS(phase - Dp);
        /* innovation and its variance */
        KF_T R = efac * efac * (sigma[k] * sigma[k]) + equad * equad;
        KF_T e = r[k] - s - mp0;
        KF_T S = a00 + R;
        if (!(KF_RE(S) > 0.0)) *bad = 1;
        /* gain and update */
        KF_T K0 = a00 / S, K1 = a01 / S;
        m0 = mp0 + K0 * e;
        m1 = mp1 + K1 * e;
        p00 = a00 - K0 * S * K0;
        p01 = a01 - K0 * S * K1;
        p11 = a11 - K1 * S * K1;
        ll += -0.5 * (KF_LOG2PI + KF_LOG(S) + e * e / S);
        if (e_out) e_out[k] = KF_RE(e);
        if (S_out) S_out[k] = KF_RE(S);
    }
    return ll;
}
