// The per-lane model shared by the filter kernels (sequential K2/K3 and the
// associative scan): lane constants, the filter state, the transition of the
// Ornstein-Uhlenbeck red noise over one step, and one Kalman step.
#pragma once

#include <cstdint>

#include "kf_internal.cuh"
#include "kf_math.cuh"

namespace argus {

struct Lane {
    double A, B, f, phc, sig2, efac2, equad2, gam;
};

struct State {
    double m0, m1, p00, p01, p11;
};

// ---------------------------------------------------------------------------
// Ornstein-Uhlenbeck red noise, dy = -gamma y dt + sigma dW.  Over one step,
// with x = gamma dt:
//   F = [[1, b], [0, a]],  a = e^-x,  b = dt psi1(x),
//   Q / sigma^2 = [[dt^3/3 phi4(x), dt^2/2 psi1(x)^2], [., dt psi1(2x)]],
// where psi_k(x) = sum_m (-x)^m / (m + k)! are the exponential-integrator
// phi-functions at -x (psi_{k-1} = 1/(k-1)! - x psi_k), so that
//   psi1(2x) = psi1 (1 - x psi1 / 2),   phi4 = 3 (psi2 - psi3 - x psi2^2 / 2),
// and their x-derivatives, for the adjoint, follow from psi_k' = k psi_{k+1} - psi_k:
//   a' = -a,  psi1' = psi2 - psi1,  psi1(2x)' = a (psi2 - psi1) - psi1^2 / 2,
//   phi4' = 3 ((2 psi3 - psi2)(1 - x psi2) - (3 psi4 - psi3) - psi2^2 / 2).
// Below x = 0.5 psi4 is its Taylor series, cut where the next term falls
// below 2^-54 of the sum (5, 7, 10 or 14 terms for x below 2^-8, 2^-6, 2^-3,
// 2^-1; psi4 enters everything else multiplied by x or, in phi4', beside
// terms 8x larger), and psi3, psi2, psi1, a follow by the recurrence without
// cancellation.  Above, a = exp(-x) and closed forms with u = 1 - a:
//   psi1 = u / x,  psi2 = (1 - psi1) / x,  phi4 = 3 (x - u (1 + u/2)) / x^3,
//   phi4' = 3 u^2 / x^3 - 3 phi4 / x.
// The range tests compare the high word of x (x >= 0, thresholds powers of
// two) on the integer pipe.  As gamma -> 0 every factor tends to the random
// walk's (a = 1, b = dt, Q = sigma^2 [[dt^3/3, dt^2/2], [., dt]]).
// With kDeriv the gamma-derivatives (d/dgamma = dt d/dx) of b and of the
// three Q / sigma^2 entries are formed here too, in the forward step, so that
// the reverse sweep reads them from the tape instead of re-deriving them.
// ---------------------------------------------------------------------------
struct OuCoef {
    double a, b, c00, c01, c11;        // F entries and Q / sigma^2
    double db, dc00, dc01, dc11;       // their derivatives in gamma (with kDeriv)
};

// Taylor coefficients (-1)^m / (m + 4)!, each fixed at compile time (a static
// constexpr member must be a constant expression; (m + 4)! <= 17! is exact
// in a double, so each coefficient is one correctly rounded division).
constexpr double factorial(int n) { return n <= 1 ? 1.0 : double(n) * factorial(n - 1); }
template <int M>
struct Psi4Coef {
    static constexpr double value = ((M & 1) ? -1.0 : 1.0) / factorial(M + 4);
};

template <int M>
__device__ __forceinline__ double psi4_horner(double x, double s) {
    if constexpr (M < 0) {
        return s;
    } else {
        return psi4_horner<M - 1>(x, fma(s, x, Psi4Coef<M>::value));
    }
}

template <int N>
__device__ __forceinline__ double psi4_series(double x) {
    return psi4_horner<N - 2>(x, Psi4Coef<N - 1>::value);
}

// hsel: the high word that picks the series length (x's own, or a larger
// one shared by a warp; a longer series is never less accurate)
template <bool kDeriv>
__device__ __forceinline__ void ou_coef_sel(double x, int hsel, double dt, double h2, double h3,
                                            double dt2, OuCoef& c) {
    double p1, p2, phi4, dphi4 = 0.0;
    const int hx = __double2hiint(x);
    if (hx < 0x3FE00000) {                       // x < 2^-1
        double p4;
        if (hsel < 0x3F700000) p4 = psi4_series<5>(x);          // x < 2^-8
        else if (hsel < 0x3F900000) p4 = psi4_series<7>(x);     // x < 2^-6
        else if (hsel < 0x3FC00000) p4 = psi4_series<10>(x);    // x < 2^-3
        else p4 = psi4_series<14>(x);
        const double p3 = fma(-x, p4, 1.0 / 6.0);
        p2 = fma(-x, p3, 0.5);
        p1 = fma(-x, p2, 1.0);
        c.a = fma(-x, p1, 1.0);
        phi4 = 3.0 * fma(-0.5 * x * p2, p2, p2 - p3);
        if (kDeriv)
            dphi4 = 3.0 * fma(-0.5 * p2, p2, fma(2.0 * p3 - p2, fma(-x, p2, 1.0), fma(-3.0, p4, p3)));
    } else {
        c.a = exp(-x);
        const double r = 1.0 / x;
        const double u = 1.0 - c.a;
        p1 = u * r;
        p2 = (1.0 - p1) * r;
        phi4 = 3.0 * (x - u * fma(0.5, u, 1.0)) * (r * r * r);
        if (kDeriv) dphi4 = 3.0 * r * fma(u * u, r * r, -phi4);
    }
    const double p1sq = p1 * p1;
    c.b = dt * p1;
    c.c00 = h3 * phi4;
    c.c01 = h2 * p1sq;
    c.c11 = dt * fma(-0.5 * x, p1sq, p1);
    if (kDeriv) {
        const double dp1 = p2 - p1;
        c.db = dt2 * dp1;                          // dt^2 psi1'
        c.dc00 = (h3 * dt) * dphi4;                // dt^4/3 phi4'
        c.dc01 = (3.0 * h3) * (p1 * dp1);          // dt^3 psi1 psi1'
        c.dc11 = dt2 * fma(c.a, dp1, -0.5 * p1sq); // dt^2 (a psi1' - psi1^2 / 2)
    }
}

template <bool kDeriv>
__device__ __forceinline__ void ou_coef(double x, double dt, double h2, double h3, double dt2,
                                        OuCoef& c) {
    ou_coef_sel<kDeriv>(x, __double2hiint(x), dt, h2, h3, dt2, c);
}

// The same for lanes of one warp with different x (e.g. the pulsars of an
// array): every lane on the series branch uses the series length of the
// warp's largest such x, so the warp runs one series instead of several in
// turn.  All active lanes must call it together.
template <bool kDeriv>
__device__ __forceinline__ void ou_coef_warp(double x, double dt, double h2, double h3, double dt2,
                                             OuCoef& c) {
    const int hx = __double2hiint(x);
    const unsigned key = (hx < 0x3FE00000) ? unsigned(hx) : 0u;
    const int hmax = int(__reduce_max_sync(__activemask(), key));
    ou_coef_sel<kDeriv>(x, hmax, dt, h2, h3, dt2, c);
}

template <bool kOU>
__device__ __forceinline__ void load_lane(const FilterArgs& a, int p, int64_t b, double equad2,
                                          Lane& L) {
    const int64_t lanes = a.B * a.P;
    const double* o = a.lc + int64_t(p) * a.B + b;
    L.A = o[0 * lanes];
    L.B = o[1 * lanes];
    L.f = o[2 * lanes];
    L.phc = o[3 * lanes];
    L.sig2 = o[4 * lanes];
    L.efac2 = o[5 * lanes];
    L.equad2 = equad2;
    L.gam = kOU ? o[7 * lanes] : 0.0;
}


struct StepOut {   // what the adjoint needs from the forward step
    // w = R/S = 1 - K0, K1 = M01/S, g = e/S, h2 = g^2 - 1/S (= -(1 - e^2/S)/S)
    double w, K1, g, h2, sn, cs;
    uint64_t F;    // the phase's fraction in 2^-64 cycles (sin, cos follow from it: sincos_frac)
    // Ornstein-Uhlenbeck only: m1, p01 + b p11 and a p11 before the step, the
    // transition a, b, Q / sigma^2 and the gamma-derivatives of b and Q / sigma^2
    double m1, t1, ap11;
    double a, b, c00, c01, c11, db, dc00, dc01, dc11;
};

// ---------------------------------------------------------------------------
// One Kalman step (predict, innovate, update), FP64.
//   predict:  m = F m,  M = F P F^T + sigma^2 Q~(dt)
//   innovate: e = r - s - m0,  S = M00 + R,  R = EFAC^2 sigma_k^2 + EQUAD^2
//   update:   m += M[:,0] e / S,  P = M - M[:,0] M[0,:] / S
// The covariance update is written as P00 = M00 R/S, P01 = M01 R/S,
// P11 = M11 - M01^2/S, algebraically equal to M - K S K^T.
// The signal's sin/cos run on the FP32/integer pipes (phase_sincos); the
// log-determinant is a running mantissa product (LogProd).
// ---------------------------------------------------------------------------
// kTape: produce what the adjoint needs; kLL: accumulate the log-likelihood;
// kOU: Ornstein-Uhlenbeck red noise (else the random walk); kShort: the
// short-latency reciprocal (rcp_nr3) for the latency-bound scan paths.
template <bool kTape, bool kLL, bool kOU, bool kShort = false>
__device__ __forceinline__ void kf_step(State& x, const double* __restrict__ rec, const Lane& L,
                                        PhaseTable tab, double& quad, LogProd& lp,
                                        StepOut& so) {
    const double t = rec[0], dt = rec[1], h2 = rec[2], h3 = rec[3], r = rec[4], s2k = rec[5];
    // predict
    double m0, mp1, t1, M00, M01, M11;
    if (kOU) {
        OuCoef c;
        ou_coef<kTape>(L.gam * dt, dt, h2, h3, rec[6], c);
        m0 = fma(c.b, x.m1, x.m0);
        mp1 = c.a * x.m1;
        t1 = fma(c.b, x.p11, x.p01);
        const double ap11 = c.a * x.p11;
        M00 = fma(L.sig2, c.c00, fma(c.b, x.p01 + t1, x.p00));
        M01 = fma(L.sig2, c.c01, c.a * t1);
        M11 = fma(L.sig2, c.c11, c.a * ap11);
        if (kTape) {
            so.m1 = x.m1; so.t1 = t1; so.ap11 = ap11;
            so.a = c.a; so.b = c.b; so.c00 = c.c00; so.c01 = c.c01; so.c11 = c.c11;
            so.db = c.db; so.dc00 = c.dc00; so.dc01 = c.dc01; so.dc11 = c.dc11;
        }
    } else {
        m0 = fma(dt, x.m1, x.m0);
        mp1 = x.m1;
        t1 = fma(dt, x.p11, x.p01);
        M00 = fma(L.sig2, h3, fma(dt, x.p01 + t1, x.p00));
        M01 = fma(L.sig2, h2, t1);
        M11 = fma(L.sig2, dt, x.p11);
    }
    // signal at phase f t + Phi0/(2 pi) cycles
    double sn, cs;
    const uint64_t F = frac_cycles_u64(fma(L.f, t, L.phc));
    sincos_frac(F, tab, sn, cs);
    // innovation e = r - (A sin + B cos) - m0
    const double e = fma(-L.A, sn, fma(-L.B, cs, r - m0));
    const double R = fma(L.efac2, s2k, L.equad2);
    const double S = M00 + R;
    const double rS = kShort ? rcp_nr3(S) : rcp_nr(S);
    const double g = e * rS;
    const double w = R * rS;
    const double K1 = M01 * rS;
    // update
    x.m0 = fma(M00, g, m0);
    x.m1 = fma(M01, g, mp1);
    x.p00 = M00 * w;
    x.p01 = M01 * w;
    x.p11 = fma(-K1, M01, M11);
    if (kTape) {
        so.w = w; so.K1 = K1; so.g = g; so.h2 = fma(g, g, -rS); so.sn = sn; so.cs = cs; so.F = F;
    }
    if (kLL) {
        quad = fma(e, g, quad);
        lp.add(S);
    }
}

}  // namespace argus
