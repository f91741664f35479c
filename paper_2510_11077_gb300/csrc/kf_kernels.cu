// Filter kernels for sm_103a: K2 forward filter and K3 adjoint (the K1
// projection and K4 reduction are in kf_project.cu).
//
// Lane = (walker b, pulsar p), one CUDA thread each.  A thread block holds
// W lanes of ONE pulsar, so every thread walks the same TOAs in lock-step and
// reads each staged TOA record from shared memory as a broadcast.  All filter
// arithmetic is FP64 (TOA residuals need it).
#include <cmath>
#include <cstdint>

#include "kf_internal.cuh"
#include "kf_math.cuh"

namespace argus {

namespace {

constexpr double kLog2Pi = 1.8378770664093454836;
constexpr int kChunk = 128;  // TOA records per shared-memory chunk (forward kernel)

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
struct Lane {
    double A, B, f, phc, sig2, efac2, equad2, gam;
};

struct State {
    double m0, m1, p00, p01, p11;
};

struct StepOut {   // what the adjoint needs from the forward step (w = R/S = 1 - K0)
    double w, K1, rS, e, sn, cs;
    // Ornstein-Uhlenbeck only: m1, p01 + b p11 and a p11 before the step, the
    // transition a, b, Q / sigma^2 and the gamma-derivatives of b and Q / sigma^2
    double m1, t1, ap11;
    double a, b, c00, c01, c11, db, dc00, dc01, dc11;
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

template <bool kDeriv>
__device__ __forceinline__ void ou_coef(double x, double dt, double h2, double h3, double dt2,
                                        OuCoef& c) {
    double p1, p2, phi4, dphi4 = 0.0;
    const int hx = __double2hiint(x);
    if (hx < 0x3FE00000) {                       // x < 2^-1
        double p4;
        if (hx < 0x3F700000) p4 = psi4_series<5>(x);          // x < 2^-8
        else if (hx < 0x3F900000) p4 = psi4_series<7>(x);     // x < 2^-6
        else if (hx < 0x3FC00000) p4 = psi4_series<10>(x);    // x < 2^-3
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

// kTape: produce what the adjoint needs; kLL: accumulate the log-likelihood;
// kOU: Ornstein-Uhlenbeck red noise (else the random walk).
template <bool kTape, bool kLL, bool kOU>
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
    phase_sincos(fma(L.f, t, L.phc), tab, sn, cs);
    const double s = fma(L.A, sn, L.B * cs);
    // innovation
    const double e = (r - s) - m0;
    const double R = fma(L.efac2, s2k, L.equad2);
    const double S = M00 + R;
    const double rS = rcp_nr(S);
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
        so.w = w; so.K1 = K1; so.rS = rS; so.e = e; so.sn = sn; so.cs = cs;
    }
    if (kLL) {
        quad = fma(e, g, quad);
        lp.add(S);
    }
}

struct Adjoint {
    double mu0, mu1, pi00, pi01, pi11;   // adjoints of the post-update state
};

// Per-lane gradient accumulators: dll/dA, dll/dB, sum sbar t sin, sum sbar t
// cos, dll/dsigma^2, sum Sbar sigma_k^2 (= dll/dEFAC / (2 EFAC)) and, for
// Ornstein-Uhlenbeck red noise, dll/dgamma.  The Phi0 and Omega derivatives
// follow as A gB - B gA and A gBt - B gAt.
struct LaneGrad {
    double A, B, At, Bt, s2, E, G;
};

// Reverse of kf_step: consumes the adjoint of the step's output state and the
// step's own loglik term, produces the adjoint of its input state and adds the
// step's contribution to the lane gradient.
template <bool kOU>
__device__ __forceinline__ void kf_step_adjoint(Adjoint& a, const StepOut& so,
                                                const double* __restrict__ rec, const Lane& L,
                                                LaneGrad& g) {
    const double t = rec[0], dt = rec[1], h2 = rec[2], h3 = rec[3], s2k = rec[5], dt2 = rec[6];
    const double twodt = rec[7];
    // K0 = M00/S = 1 - w
    const double w = so.w, K1 = so.K1, gg = so.e * so.rS;
    const double t1 = fma(-a.mu0, w, fma(a.mu1, K1, a.mu0));    // mu0 K0 + mu1 K1
    const double ebar = t1 - gg;                                // dL/de
    const double u = fma(-a.pi00, w, fma(a.pi01, K1, a.pi00));  // pi00 K0 + pi01 K1
    const double v = a.pi11 * K1;
    const double ku = fma(-w, u, fma(v, K1, u));                // K0 u + K1 v
    const double Sbar = fma(-0.5 * so.rS, fma(-so.e, gg, 1.0), fma(-gg, t1, ku));
    const double a0 = a.mu0 - ebar;                             // dL/d(predicted m0)
    const double M00b = fma(a.mu0, gg, fma(a.pi00, fma(2.0, w, -1.0), fma(-a.pi01, K1, Sbar)));
    const double M01b = fma(a.mu1, gg, fma(a.pi01, w, -2.0 * v));
    const double M11b = a.pi11;
    g.E = fma(Sbar, s2k, g.E);
    // dL/ds_k = -ebar
    g.A = fma(-ebar, so.sn, g.A);
    g.B = fma(-ebar, so.cs, g.B);
    const double st = -ebar * t;
    g.At = fma(st, so.sn, g.At);
    g.Bt = fma(st, so.cs, g.Bt);
    // back through the prediction m = F m, M = F P F^T + Q
    if (kOU) {
        g.s2 = fma(M00b, so.c00, fma(M01b, so.c01, fma(M11b, so.c11, g.s2)));
        // adjoints of a and b; da/dgamma = -dt a
        const double abar = fma(a.mu1, so.m1, fma(M01b, so.t1, 2.0 * M11b * so.ap11));
        const double bbar = fma(a0, so.m1, fma(2.0 * M00b, so.t1, M01b * so.ap11));
        const double qg = fma(M00b, so.dc00, fma(M01b, so.dc01, M11b * so.dc11));
        g.G = fma(-dt * so.a, abar, fma(bbar, so.db, fma(L.sig2, qg, g.G)));
        a.mu0 = a0;
        a.mu1 = fma(so.b, a0, so.a * a.mu1);
        a.pi00 = M00b;
        a.pi01 = fma(2.0 * so.b, M00b, so.a * M01b);
        a.pi11 = fma(so.b * so.b, M00b, so.a * fma(so.b, M01b, so.a * M11b));
    } else {
        g.s2 = fma(M00b, h3, fma(M01b, h2, fma(M11b, dt, g.s2)));
        a.mu0 = a0;
        a.mu1 = fma(dt, a0, a.mu1);
        a.pi00 = M00b;
        a.pi01 = fma(twodt, M00b, M01b);
        a.pi11 = fma(dt2, M00b, fma(dt, M01b, M11b));
    }
}

// One step's tape record, field-major within the step: [field][W].
template <bool kOU>
__device__ __forceinline__ void tape_put(double* tk, int W, const StepOut& so) {
    tk[0 * W] = so.w; tk[1 * W] = so.K1; tk[2 * W] = so.rS;
    tk[3 * W] = so.e; tk[4 * W] = so.sn; tk[5 * W] = so.cs;
    if (kOU) {
        tk[6 * W] = so.m1; tk[7 * W] = so.t1; tk[8 * W] = so.ap11;
        tk[9 * W] = so.a; tk[10 * W] = so.b; tk[11 * W] = so.c00; tk[12 * W] = so.c01;
        tk[13 * W] = so.c11; tk[14 * W] = so.db; tk[15 * W] = so.dc00; tk[16 * W] = so.dc01;
        tk[17 * W] = so.dc11;
    }
}

template <bool kOU>
__device__ __forceinline__ StepOut tape_get(const double* tk, int W) {
    StepOut so{};
    so.w = tk[0 * W]; so.K1 = tk[1 * W]; so.rS = tk[2 * W];
    so.e = tk[3 * W]; so.sn = tk[4 * W]; so.cs = tk[5 * W];
    if (kOU) {
        so.m1 = tk[6 * W]; so.t1 = tk[7 * W]; so.ap11 = tk[8 * W];
        so.a = tk[9 * W]; so.b = tk[10 * W]; so.c00 = tk[11 * W]; so.c01 = tk[12 * W];
        so.c11 = tk[13 * W]; so.db = tk[14 * W]; so.dc00 = tk[15 * W]; so.dc01 = tk[16 * W];
        so.dc11 = tk[17 * W];
    }
    return so;
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

// Cooperative copy of `cnt` records into shared memory (16-byte vector loads).
__device__ __forceinline__ void stage_records(double* __restrict__ s, const double* __restrict__ g,
                                              int cnt) {
    const double2* g2 = reinterpret_cast<const double2*>(g);
    double2* s2 = reinterpret_cast<double2*>(s);
    const int n2 = cnt * (kRecDoubles / 2);
    for (int i = threadIdx.x; i < n2; i += blockDim.x) s2[i] = __ldg(g2 + i);
}

__device__ __forceinline__ int next_item(const FilterArgs& a, int iter, int* s_item) {
    if (a.counter == nullptr) return iter == 0 ? int(blockIdx.x) : a.n_items;
    if (threadIdx.x == 0) *s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    return *s_item;
}

__device__ __forceinline__ double finish_ll(int n, double quad, const LogProd& lp) {
    if (n == 0) return 0.0;
    const double ll = -0.5 * (double(n) * kLog2Pi + lp.value() + quad);
    return (lp.bad || !isfinite(ll)) ? -INFINITY : ll;
}

// shared memory of a filter block: phase table, then the staged TOA records
struct FilterSmem {
    PhaseTable tab;
    double* rec;
};

__device__ __forceinline__ FilterSmem filter_smem() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FilterSmem s;
    s.tab.d = reinterpret_cast<double2*>(smem_raw);
    s.tab.f = reinterpret_cast<float4*>(smem_raw + kPhaseTable * sizeof(double2));
    s.rec = reinterpret_cast<double*>(smem_raw + kPhaseTableBytes);
    return s;
}

// ---------------------------------------------------------------------------
// K2: forward filter, one lane per thread.
// ---------------------------------------------------------------------------
template <bool kOU>
__global__ void __launch_bounds__(256) k_filter_fwd(FilterArgs a) {
    const FilterSmem sm = filter_smem();
    __shared__ int s_item;
    fill_phase_table(sm.tab);
    for (int iter = 0;; ++iter) {
        const int it = next_item(a, iter, &s_item);
        if (it >= a.n_items) break;
        const WorkItem wi = a.items[it];
        const PulsarDev& ps = a.psr[wi.p];
        const int n = ps.n;
        const int64_t b = int64_t(wi.b0) + threadIdx.x;
        const bool active = b < a.B;
        Lane L;
        State x{0.0, 0.0, ps.p0[0], ps.p0[1], ps.p0[2]};
        if (active) load_lane<kOU>(a, wi.p, b, ps.equad2, L);
        double quad = 0.0;
        LogProd lp;
        StepOut so;
        for (int k0 = 0; k0 < n; k0 += kChunk) {
            const int cnt = min(kChunk, n - k0);
            __syncthreads();
            stage_records(sm.rec, a.rec + (ps.off + k0) * kRecDoubles, cnt);
            __syncthreads();
            if (active) {
                for (int k = 0; k < cnt; ++k)
                    kf_step<false, true, kOU>(x, sm.rec + k * kRecDoubles, L, sm.tab, quad, lp, so);
            }
        }
        if (active) a.lane_out[int64_t(wi.p) * a.B + b] = finish_ll(n, quad, lp);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K3: log-likelihood and its gradient by a reverse-mode adjoint sweep.
// Pass 1 runs the filter forward segment by segment (stride TOAs each) and
// checkpoints the state at the start of every segment.  Pass 2 walks the
// segments backwards: restore the checkpoint, re-run the segment forward
// recording (R/S, K1, 1/S, e, sin, cos) per step in the block's tape, then
// run the adjoint steps in reverse.  Checkpoints and tape live in the block's
// own slot of global scratch ([..][field][W], so a warp's accesses coalesce).
// With kCache the tape of every segment is written during pass 1 and kept in
// HBM (the slot holds the whole pulsar), so pass 2 skips the re-run: HBM
// traffic is traded for FP64 work, which is the scarce resource here.
// ---------------------------------------------------------------------------
template <bool kCache, bool kOU>
__global__ void __launch_bounds__(256) k_filter_grad(FilterArgs a) {
    constexpr int kTd = kOU ? kTapeDoublesOU : kTapeDoubles;
    const FilterSmem sm = filter_smem();
    __shared__ int s_item;
    const int W = blockDim.x;
    const int tid = threadIdx.x;
    double* ck = a.ckpt + int64_t(blockIdx.x) * a.ckpt_slot + tid;
    double* tp = a.tape + int64_t(blockIdx.x) * a.tape_slot + tid;
    fill_phase_table(sm.tab);
    for (int iter = 0;; ++iter) {
        const int it = next_item(a, iter, &s_item);
        if (it >= a.n_items) break;
        const WorkItem wi = a.items[it];
        const PulsarDev& ps = a.psr[wi.p];
        const int n = ps.n, c = ps.stride, nseg = ps.nseg;
        const int64_t b = int64_t(wi.b0) + tid;
        const bool active = b < a.B;
        Lane L;
        if (active) load_lane<kOU>(a, wi.p, b, ps.equad2, L);
        State x{0.0, 0.0, ps.p0[0], ps.p0[1], ps.p0[2]};
        double quad = 0.0;
        LogProd lp;
        StepOut so;
        // pass 1: forward with checkpoints (and, with kCache, the whole tape)
        for (int seg = 0; seg < nseg; ++seg) {
            const int k0 = seg * c, cnt = min(c, n - k0);
            __syncthreads();
            stage_records(sm.rec, a.rec + (ps.off + k0) * kRecDoubles, cnt);
            __syncthreads();
            if (active) {
                double* cp = ck + int64_t(seg) * kCkptDoubles * W;
                cp[0 * W] = x.m0; cp[1 * W] = x.m1; cp[2 * W] = x.p00; cp[3 * W] = x.p01; cp[4 * W] = x.p11;
                for (int k = 0; k < cnt; ++k) {
                    kf_step<kCache, true, kOU>(x, sm.rec + k * kRecDoubles, L, sm.tab, quad, lp, so);
                    if (kCache) tape_put<kOU>(tp + int64_t(k0 + k) * kTd * W, W, so);
                }
            }
        }
        const double ll = finish_ll(n, quad, lp);
        // pass 2: reverse sweep
        Adjoint adj{0.0, 0.0, 0.0, 0.0, 0.0};
        LaneGrad g{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int seg = nseg - 1; seg >= 0; --seg) {
            const int k0 = seg * c, cnt = min(c, n - k0);
            __syncthreads();
            stage_records(sm.rec, a.rec + (ps.off + k0) * kRecDoubles, cnt);
            __syncthreads();
            if (active) {
                const double* ts = tp + int64_t(kCache ? k0 : 0) * kTd * W;
                if (!kCache) {
                    const double* cp = ck + int64_t(seg) * kCkptDoubles * W;
                    State y{cp[0 * W], cp[1 * W], cp[2 * W], cp[3 * W], cp[4 * W]};
                    double q2 = 0.0;
                    LogProd l2;
                    for (int k = 0; k < cnt; ++k) {
                        kf_step<true, false, kOU>(y, sm.rec + k * kRecDoubles, L, sm.tab, q2, l2, so);
                        tape_put<kOU>(tp + int64_t(k) * kTd * W, W, so);
                    }
                }
                for (int k = cnt - 1; k >= 0; --k) {
                    const StepOut sk = tape_get<kOU>(ts + int64_t(k) * kTd * W, W);
                    kf_step_adjoint<kOU>(adj, sk, sm.rec + k * kRecDoubles, L, g);
                }
            }
        }
        if (active) {
            const int64_t lanes = a.B * a.P;
            double* o = a.lane_out + int64_t(wi.p) * a.B + b;
            o[0] = ll;
            o[1 * lanes] = g.A;
            o[2 * lanes] = g.B;
            o[3 * lanes] = g.At;
            o[4 * lanes] = g.Bt;
            o[5 * lanes] = g.s2;
            o[6 * lanes] = g.E;
            if (kOU) o[7 * lanes] = g.G;
        }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t filter_smem_bytes(bool grad, int stride_max) {
    const int recs = grad ? stride_max : kChunk;
    return kPhaseTableBytes + size_t(recs) * kRecDoubles * sizeof(double);
}

void launch_filter_fwd(const FilterArgs& a, int W, int grid, cudaStream_t s) {
    const size_t smem = filter_smem_bytes(false, 0);
    if (a.model == kOrnsteinUhlenbeck) k_filter_fwd<true><<<grid, W, smem, s>>>(a);
    else k_filter_fwd<false><<<grid, W, smem, s>>>(a);
}

void launch_filter_grad(const FilterArgs& a, int W, int grid, cudaStream_t s) {
    const size_t smem = filter_smem_bytes(true, a.stride_max);
    const bool ou = a.model == kOrnsteinUhlenbeck;
    if (a.tape_cache) {
        if (ou) k_filter_grad<true, true><<<grid, W, smem, s>>>(a);
        else k_filter_grad<true, false><<<grid, W, smem, s>>>(a);
    } else {
        if (ou) k_filter_grad<false, true><<<grid, W, smem, s>>>(a);
        else k_filter_grad<false, false><<<grid, W, smem, s>>>(a);
    }
}

}  // namespace argus
