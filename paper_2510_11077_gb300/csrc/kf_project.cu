// Projection (K1) and reduction (K4) kernels for sm_103a: the parameter
// vector's continuous-wave source mapped onto each pulsar's lane constants,
// and the per-walker sum over pulsars with the chain rule of the gradient back
// through that mapping.  Both are O(B x P) and run once per call; the O(B x N)
// filter kernels are in kf_kernels.cu.
#include <cmath>
#include <cstdint>

#include "kf_internal.cuh"
#include "kf_few.cuh"
#include "lib_internal.cuh"

namespace argus {

namespace {

constexpr double kLn10 = 2.302585092994045684;
constexpr double kTwoPi = 6.283185307179586477;
constexpr double kPi = 3.141592653589793238;
constexpr int kFewThreads = 128;   // one block of four warps per walker (k_project_few)
constexpr int kFewReduceThreads = 160;   // k_reduce_few: the four, and a fifth for the walker's ll
constexpr int kFewTerms = 10;      // a pulsar's terms of the source-parameter gradient sums

// light-travel time over one kiloparsec [s]: 1 pc = (648000 / pi) au,
// 1 au = 149597870700 m, c = 299792458 m/s
constexpr double kKpcLightS = 1e3 * (648000.0 / kPi) * 149597870700.0 / 299792458.0;

// ---------------------------------------------------------------------------
// Continuous-wave projection (Earth term of a monochromatic source).
// Source direction n = (cos d cos a, cos d sin a, sin d); polarisation basis
// u = (sin a, -cos a, 0), v = (sin d cos a, sin d sin a, -cos d) rotated by psi:
// p = cos psi u + sin psi v, q = -sin psi u + cos psi v.  For a pulsar at c:
// F+ = ((c.p)^2 - (c.q)^2) / (2 (1 - n.c)), Fx = (c.p)(c.q) / (1 - n.c).
// The residual is the time integral of the redshift F+ h+ + Fx hx with
// h+ = h0 (1 + cos^2 i) cos Phi(t), hx = 2 h0 cos i sin Phi(t):
// s(t) = A sin Phi + B cos Phi, A = F+ h0 (1 + cos^2 i) / W,
// B = -2 Fx h0 cos i / W, Phi(t) = W t + Phi0, W = 2 pi f.
//
// Pulsar term: the wave met the pulsar tau = d (1 - n.c) / c earlier, and its
// redshift enters with the opposite sign, so for a monochromatic source
// s(t) = A sin Phi + B cos Phi - A sin(Phi - L) - B cos(Phi - L), L = W tau,
// which is again one sinusoid: s = A' sin Phi + B' cos Phi with
// A' = A (1 - cos L) - B sin L,  B' = B (1 - cos L) + A sin L
// (1 - cos L = 2 sin^2(L/2)).  K1 hands the filter A', B'; K4 carries the
// gradient back through them to A, B and L.
// ---------------------------------------------------------------------------
struct SourceFrame {
    double W, f, h0, ampP, ampX;        // ampP = h0 (1 + ci^2)/W, ampX = -2 h0 ci / W
    double ci;
    double n[3], P[3], Q[3];
    // derivatives with respect to alpha (_a) and sin(delta) (_x)
    double n_a[3], P_a[3], Q_a[3];
    double n_x[3], P_x[3], Q_x[3];
};

__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}

// The frame's transcendentals: f = 10^log10 f, h0 = 10^log10 h0 and the
// sines and cosines of alpha and psi.
struct FrameTrig {
    double f, h0, sa, ca, sp, cp;
};

__device__ __forceinline__ void frame_trig(const double* th, FrameTrig& T) {
    T.f = exp10(th[0]);
    T.h0 = exp10(th[6]);
    sincos(th[5], &T.sa, &T.ca);
    sincos(th[2], &T.sp, &T.cp);
}

__device__ void source_frame(const double* th, const FrameTrig& T, bool with_derivs, SourceFrame& F) {
    F.f = T.f;
    F.W = kTwoPi * F.f;
    F.h0 = T.h0;
    F.ci = th[3];
    F.ampP = F.h0 * fma(F.ci, F.ci, 1.0) / F.W;
    F.ampX = -2.0 * F.h0 * F.ci / F.W;
    const double x = th[4];
    const double cd = sqrt(fmax(0.0, 1.0 - x * x));
    const double sa = T.sa, ca = T.ca, sp = T.sp, cp = T.cp;
    const double u[3] = {sa, -ca, 0.0};
    const double v[3] = {x * ca, x * sa, -cd};
    F.n[0] = cd * ca; F.n[1] = cd * sa; F.n[2] = x;
    for (int i = 0; i < 3; ++i) {
        F.P[i] = cp * u[i] + sp * v[i];
        F.Q[i] = -sp * u[i] + cp * v[i];
    }
    if (!with_derivs) return;
    const double u_a[3] = {ca, sa, 0.0};
    const double v_a[3] = {-x * sa, x * ca, 0.0};
    F.n_a[0] = -cd * sa; F.n_a[1] = cd * ca; F.n_a[2] = 0.0;
    const double cd_x = -x / cd;
    const double v_x[3] = {ca, sa, -cd_x};
    F.n_x[0] = cd_x * ca; F.n_x[1] = cd_x * sa; F.n_x[2] = 1.0;
    for (int i = 0; i < 3; ++i) {
        F.P_a[i] = cp * u_a[i] + sp * v_a[i];
        F.Q_a[i] = -sp * u_a[i] + cp * v_a[i];
        F.P_x[i] = sp * v_x[i];
        F.Q_x[i] = cp * v_x[i];
    }
}

__device__ __forceinline__ void source_frame(const double* th, bool with_derivs, SourceFrame& F) {
    FrameTrig T;
    frame_trig(th, T);
    source_frame(th, T, with_derivs, F);
}

struct Antenna {
    double Fp, Fx;
    double D;                       // 1 - n.c, clamped at 1e-12
    double Fp_a, Fx_a, Fp_x, Fx_x;  // derivatives (alpha, sin delta)
    double D_a, D_x;
};

__device__ void antenna(const SourceFrame& F, const double* c, bool with_derivs, Antenna& R) {
    const double a = dot3(c, F.P), b = dot3(c, F.Q);
    double D = 1.0 - dot3(c, F.n);
    const bool clamped = D < 1e-12;
    if (clamped) D = 1e-12;
    const double iD = 1.0 / D;
    R.D = D;
    R.Fp = 0.5 * (a * a - b * b) * iD;
    R.Fx = a * b * iD;
    if (!with_derivs) return;
    {
        const double a_z = dot3(c, F.P_a), b_z = dot3(c, F.Q_a);
        const double D_z = clamped ? 0.0 : -dot3(c, F.n_a);
        R.D_a = D_z;
        R.Fp_a = (a * a_z - b * b_z - R.Fp * D_z) * iD;
        R.Fx_a = (a_z * b + a * b_z - R.Fx * D_z) * iD;
    }
    {
        const double a_z = dot3(c, F.P_x), b_z = dot3(c, F.Q_x);
        const double D_z = clamped ? 0.0 : -dot3(c, F.n_x);
        R.D_x = D_z;
        R.Fp_x = (a * a_z - b * b_z - R.Fp * D_z) * iD;
        R.Fx_x = (a_z * b + a * b_z - R.Fx * D_z) * iD;
    }
}

// Where each pulsar's own parameters sit: (log10 sigma, [log10 gamma], EFAC, [d_kpc]).
struct Layout {
    int nq, efac;
    bool ou, pt;
    __device__ explicit Layout(int32_t flags)
        : nq(params_per_pulsar(flags)), efac((flags & kFlagOU) ? 2 : 1),
          ou((flags & kFlagOU) != 0), pt((flags & kFlagPulsarTerm) != 0) {}
};

__device__ __forceinline__ bool theta_in_domain(const double* th, int P, const Layout& ly) {
    const int D = kNgw + ly.nq * P;
    bool ok = true;
    for (int j = 0; j < D; ++j) ok = ok && isfinite(th[j]);
    ok = ok && fabs(th[3]) <= 1.0 && fabs(th[4]) <= 1.0;
    for (int p = 0; p < P; ++p) {
        ok = ok && th[kNgw + ly.nq * p + ly.efac] > 0.0;
        if (ly.pt) ok = ok && th[kNgw + ly.nq * p + ly.nq - 1] > 0.0;
    }
    return ok;
}

// ---------------------------------------------------------------------------
// K1: lane constants.  lc[k][p][b], k = A, B, f, Phi0/(2 pi), sigma^2, EFAC^2,
// EFAC, gamma (the last only for Ornstein-Uhlenbeck red noise).  With the
// pulsar term A and B are the folded A', B'.
// ---------------------------------------------------------------------------
// One lane's constants (o: its first entry, rows `lanes` apart) from its
// walker's frame; sig2 = 10^(2 log10 sigma), gam = 10^log10 gamma.
__device__ __forceinline__ void project_lane(const double* th, const SourceFrame& F, const PulsarDev& ps,
                                             int p, const Layout& ly, double sig2, double gam, double* o,
                                             int64_t lanes) {
    Antenna R;
    antenna(F, ps.pos, false, R);
    const double* nz = th + kNgw + ly.nq * p;
    const double efac = nz[ly.efac];
    double A = R.Fp * F.ampP, Bc = R.Fx * F.ampX;
    if (ly.pt) {
        // lag L = W d (1 - n.c) / c;  1 - cos L = 2 sin^2(L/2), sin L = 2 sin(L/2) cos(L/2)
        const double L = F.W * (nz[ly.nq - 1] * kKpcLightS * R.D);
        double sh, ch;
        sincos(0.5 * L, &sh, &ch);
        const double omc = 2.0 * sh * sh, sl = 2.0 * sh * ch;
        const double Ap = fma(A, omc, -Bc * sl), Bp = fma(Bc, omc, A * sl);
        A = Ap;
        Bc = Bp;
    }
    o[0 * lanes] = A;
    o[1 * lanes] = Bc;
    o[2 * lanes] = F.f;
    o[3 * lanes] = th[1] / kTwoPi;
    o[4 * lanes] = sig2;
    o[5 * lanes] = efac * efac;
    o[6 * lanes] = efac;
    if (ly.ou) o[7 * lanes] = gam;
}

__global__ void k_project(const double* __restrict__ theta, int64_t B, int32_t P, int32_t flags,
                          const PulsarDev* __restrict__ psr, double* __restrict__ lc) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t lanes = B * P;
    if (idx >= lanes) return;
    const Layout ly(flags);
    const int p = int(idx / B);
    const int64_t b = idx - int64_t(p) * B;
    const int D = kNgw + ly.nq * P;
    const double* th = theta + b * D;
    SourceFrame F;
    source_frame(th, false, F);
    const double* nz = th + kNgw + ly.nq * p;
    project_lane(th, F, psr[p], p, ly, exp10(2.0 * nz[0]), ly.ou ? exp10(nz[1]) : 0.0, lc + idx, lanes);
}

// ---------------------------------------------------------------------------
// K1 and K4 for a few walkers (the time-parallel plan's batches): one block
// of four warps per walker.  A warp's 32-lane FP64 instruction runs on one
// SM sub-partition, a quarter of the SM's FP64 units, so at one thread per
// lane the serial transcendentals of a walker's frame dominate K1 and K4.
// Here they run on the four warps at once (few_trig); then one thread per
// pulsar finishes its lane with the batched kernels' arithmetic.
// ---------------------------------------------------------------------------
// s[0, P): 10^(2 log10 sigma_p); s[P, 2P): 10^log10 gamma_p (Ornstein-Uhlenbeck).
// Called by the block's first four warps (a fifth, if any, does nothing here).
__device__ __forceinline__ void few_trig(const double* th, int P, const Layout& ly, FrameTrig& T,
                                         double* s) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w == 0) {
        if (l < 2) {
            const double v = exp10(th[l == 0 ? 0 : 6]);
            if (l == 0) T.f = v;
            else T.h0 = v;
        }
    } else if (w == 1) {
        if (l == 0) sincos(th[5], &T.sa, &T.ca);
    } else if (w == 2) {
        if (l == 0) sincos(th[2], &T.sp, &T.cp);
    } else if (w == 3) {
        const int n = ly.ou ? 2 * P : P;
        for (int i = l; i < n; i += 32) {
            const int p = i < P ? i : i - P;
            const double* nz = th + kNgw + ly.nq * p;
            s[i] = exp10(i < P ? 2.0 * nz[0] : nz[1]);
        }
    }
}

__global__ void __launch_bounds__(kFewThreads) k_project_few(const double* __restrict__ theta, int64_t B,
                                                            int32_t P, int32_t flags,
                                                            const PulsarDev* __restrict__ psr,
                                                            double* __restrict__ lc) {
    extern __shared__ double s_few[];   // [2P]
    __shared__ FrameTrig T;
    const Layout ly(flags);
    const int64_t b = blockIdx.x;
    const double* th = theta + b * (kNgw + ly.nq * P);
    few_trig(th, P, ly, T, s_few);
    __syncthreads();
    const int64_t lanes = B * P;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        SourceFrame F;
        source_frame(th, T, false, F);
        project_lane(th, F, psr[p], p, ly, s_few[p], ly.ou ? s_few[P + p] : 0.0, lc + int64_t(p) * B + b,
                     lanes);
    }
}


// ---------------------------------------------------------------------------
// K4: per walker, fixed-order sum over pulsars; for the gradient, the chain
// rule through K1 for the 7 source parameters and each pulsar's own ones.
// ---------------------------------------------------------------------------
// One pulsar's part of a walker's gradient: its own parameters' entries (gz)
// and its terms of the 7 source-parameter sums, c[0..6], with the pulsar term
// also c[7..9], further terms of entries 0, 4 and 5 (each sum adds c[j], then
// c[7..9], pulsar by pulsar).  o: the lane's row 0 entry of lane_out.
__device__ __forceinline__ void pulsar_grad(const SourceFrame& F, const PulsarDev& ps, const double* o,
                                            int64_t lanes, const double* nz, double* gz, const Layout& ly,
                                            double sig2, double gam, double* c) {
    const int nq = ly.nq;
    const double gA = o[1 * lanes], gB = o[2 * lanes], gAt = o[3 * lanes];
    const double gBt = o[4 * lanes], gs2 = o[5 * lanes], gE = o[6 * lanes];
    Antenna R;
    antenna(F, ps.pos, true, R);
    const double A = R.Fp * F.ampP, Bc = R.Fx * F.ampX;
    // (Af, Bf): the filter's amplitudes; (hA, hB): dll/dA, dll/dB of the
    // Earth-term amplitudes; hL: dll/dL of the pulsar-term lag
    double Af = A, Bf = Bc, hA = gA, hB = gB, hL = 0.0, L = 0.0;
    if (ly.pt) {
        L = F.W * (nz[nq - 1] * kKpcLightS * R.D);
        double sh, ch;
        sincos(0.5 * L, &sh, &ch);
        const double omc = 2.0 * sh * sh, sl = 2.0 * sh * ch, cl = 1.0 - omc;
        Af = fma(A, omc, -Bc * sl);
        Bf = fma(Bc, omc, A * sl);
        hA = fma(gA, omc, gB * sl);
        hB = fma(gB, omc, -gA * sl);
        hL = fma(gA, fma(A, sl, -Bc * cl), gB * fma(Bc, sl, A * cl));
    }
    // through the phase: ds/dPhi0 = Af cos - Bf sin, ds/dOmega = t (Af cos - Bf sin)
    const double gP = fma(Af, gB, -Bf * gA);
    const double gW = fma(Af, gBt, -Bf * gAt);
    const double gAB = fma(hA, A, hB * Bc);
    c[0] = fma(gW, F.W * kLn10, -gAB * kLn10);
    c[1] = gP;
    c[2] = fma(hA, 2.0 * R.Fx * F.ampP, hB * (-2.0 * R.Fp) * F.ampX);
    c[3] = fma(hA, R.Fp * 2.0 * F.h0 * F.ci / F.W, hB * R.Fx * (-2.0 * F.h0 / F.W));
    c[4] = fma(hA, R.Fp_x * F.ampP, hB * R.Fx_x * F.ampX);
    c[5] = fma(hA, R.Fp_a * F.ampP, hB * R.Fx_a * F.ampX);
    // rounded products (__dmul_rn): the sums add exactly these terms whichever
    // kernel forms them, none fused into an FMA with the running sum
    c[6] = __dmul_rn(gAB, kLn10);
    if (ly.pt) {
        // L = W d K D: dL/dlog10 f = L ln 10, dL/dx = W d K dD/dx, dL/dd = W K D
        const double WdK = F.W * nz[nq - 1] * kKpcLightS;
        c[7] = __dmul_rn(hL * L, kLn10);
        c[8] = __dmul_rn(hL * WdK, R.D_x);
        c[9] = __dmul_rn(hL * WdK, R.D_a);
        gz[nq - 1] = hL * F.W * kKpcLightS * R.D;
    }
    gz[0] = gs2 * 2.0 * kLn10 * sig2;
    gz[ly.efac] = gE * 2.0 * nz[ly.efac];
    if (ly.ou) gz[1] = o[7 * lanes] * kLn10 * gam;
}

// gw[0..6] += one pulsar's terms, in the order pulsar_grad states
__device__ __forceinline__ void add_pulsar_terms(double* gw, const double* c, const Layout& ly) {
    for (int j = 0; j < kNgw; ++j) gw[j] += c[j];
    if (ly.pt) {
        gw[0] += c[7];
        gw[4] += c[8];
        gw[5] += c[9];
    }
}

// The walker's log-likelihood (and each lane's), from lane_out row 0 in
// pulsar order; returns whether it is finite and theta in the domain.
__device__ __forceinline__ bool walker_ll(const double* th, int64_t b, int64_t B, int32_t P,
                                          const Layout& ly, const double* lane_out, double* loglik,
                                          double* lane_ll) {
    const bool ok = theta_in_domain(th, P, ly);
    double ll = 0.0;
    for (int p = 0; p < P; ++p) {
        const double lp = lane_out[int64_t(p) * B + b];
        if (lane_ll) lane_ll[b * P + p] = ok ? lp : -INFINITY;
        ll += lp;
    }
    const bool good = ok && isfinite(ll);
    if (loglik) loglik[b] = good ? ll : -INFINITY;
    return good;
}

__global__ void k_reduce(const double* __restrict__ theta, int64_t B, int32_t P, int32_t flags,
                         const PulsarDev* __restrict__ psr, const double* __restrict__ lane_out,
                         double* __restrict__ loglik, double* __restrict__ grad,
                         double* __restrict__ lane_ll) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const Layout ly(flags);
    const int nq = ly.nq;
    const int D = kNgw + nq * P;
    const int64_t lanes = B * P;
    const double* th = theta + b * D;
    const bool good = walker_ll(th, b, B, P, ly, lane_out, loglik, lane_ll);
    if (!grad) return;
    double* gout = grad + b * D;
    if (!good) {
        for (int j = 0; j < D; ++j) gout[j] = 0.0;
        return;
    }
    SourceFrame F;
    source_frame(th, true, F);
    double gw[kNgw] = {0, 0, 0, 0, 0, 0, 0};
    for (int p = 0; p < P; ++p) {
        const double* nz = th + kNgw + nq * p;
        double c[kFewTerms];
        pulsar_grad(F, psr[p], lane_out + int64_t(p) * B + b, lanes, nz, gout + kNgw + nq * p, ly,
                    exp10(2.0 * nz[0]), ly.ou ? exp10(nz[1]) : 0.0, c);
        add_pulsar_terms(gw, c, ly);
    }
    for (int j = 0; j < kNgw; ++j) gout[j] = gw[j];
}

// K4 with the gradient for a few walkers (see k_project_few): the walker's
// frame and the pulsars' exponentials on four warps at once while a fifth
// sums the walker's log-likelihood, each pulsar's terms on its own thread,
// and the sums over pulsars in pulsar order on one.
__global__ void __launch_bounds__(kFewReduceThreads) k_reduce_few(const double* __restrict__ theta, int64_t B,
                                                           int32_t P, int32_t flags,
                                                           const PulsarDev* __restrict__ psr,
                                                           const double* __restrict__ lane_out,
                                                           double* __restrict__ loglik,
                                                           double* __restrict__ grad,
                                                           double* __restrict__ lane_ll) {
    extern __shared__ double s_few[];   // [2P] exponentials, then [P][kFewTerms] terms
    __shared__ FrameTrig T;
    __shared__ int s_good;
    const Layout ly(flags);
    const int nq = ly.nq;
    const int64_t b = blockIdx.x;
    const int D = kNgw + nq * P;
    const int64_t lanes = B * P;
    const double* th = theta + b * D;
    if (threadIdx.x == 4 * 32) s_good = walker_ll(th, b, B, P, ly, lane_out, loglik, lane_ll) ? 1 : 0;
    few_trig(th, P, ly, T, s_few);
    __syncthreads();
    double* gout = grad + b * D;
    if (!s_good) {   // the whole block
        for (int j = threadIdx.x; j < D; j += blockDim.x) gout[j] = 0.0;
        return;
    }
    double* terms = s_few + 2 * P;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        SourceFrame F;
        source_frame(th, T, true, F);
        const double* nz = th + kNgw + nq * p;
        pulsar_grad(F, psr[p], lane_out + int64_t(p) * B + b, lanes, nz, gout + kNgw + nq * p, ly,
                    s_few[p], ly.ou ? s_few[P + p] : 0.0, terms + int64_t(p) * kFewTerms);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double gw[kNgw] = {0, 0, 0, 0, 0, 0, 0};
        for (int p = 0; p < P; ++p) add_pulsar_terms(gw, terms + int64_t(p) * kFewTerms, ly);
        for (int j = 0; j < kNgw; ++j) gout[j] = gw[j];
    }
}

// Per-walker status of a finished call: 0 = finite log-likelihood, 1 = theta
// outside the domain, 2 = theta in the domain but the filter met an innovation
// variance that is not a positive normal finite number (or the sum is not
// finite).  Bit 0 of *any2 is set if some walker has status 2.
__global__ void k_walker_flags(const double* __restrict__ theta, int64_t B, int32_t P, int32_t flags,
                               const double* __restrict__ loglik, int32_t* __restrict__ out,
                               int* __restrict__ any2) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const Layout ly(flags);
    const int D = kNgw + ly.nq * P;
    int32_t f = 0;
    if (!isfinite(loglik[b])) f = theta_in_domain(theta + b * D, P, ly) ? 2 : 1;
    if (out) out[b] = f;
    if (f == 2 && any2) atomicOr(any2, 1);
}

// s[off_p + k] = A_p sin(W t_k + Phi0) + B_p cos(W t_k + Phi0); grid (TOA blocks, P)
__global__ void k_cw_signal(const double* __restrict__ thg, const PulsarDev* __restrict__ psr,
                            const double* __restrict__ rec, double* __restrict__ s) {
    const int p = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const PulsarDev& ps = psr[p];
    if (k >= ps.n) return;
    double th[kNgw];
    for (int j = 0; j < kNgw; ++j) th[j] = thg[j];
    SourceFrame F;
    source_frame(th, false, F);
    Antenna R;
    antenna(F, ps.pos, false, R);
    const double t = rec[(ps.off + k) * kRecDoubles];
    double sn, cs;
    sincospi(2.0 * fma(F.f, t, th[1] / kTwoPi), &sn, &cs);
    s[ps.off + k] = fma(R.Fp * F.ampP, sn, R.Fx * F.ampX * cs);
}

}  // namespace

void launch_project(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                    double* lc, cudaStream_t s) {
    const int64_t lanes = B * P;
    const int threads = 128;
    const int64_t blocks = (lanes + threads - 1) / threads;
    k_project<<<unsigned(blocks), threads, 0, s>>>(theta, B, P, flags, psr, lc);
}

void launch_cw_signal(const double* theta_gw, int32_t P, const PulsarDev* psr, const double* rec,
                      int max_n, double* s, cudaStream_t st) {
    if (max_n <= 0) return;
    dim3 grid((max_n + 127) / 128, P);
    k_cw_signal<<<grid, 128, 0, st>>>(theta_gw, psr, rec, s);
}

bool few_walkers(int64_t B, int32_t P) { return B >= 1 && B <= kFewMaxWalkers && P >= 1 && P <= kFewMaxPulsars; }

void launch_project_few(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                        double* lc, cudaStream_t s) {
    k_project_few<<<unsigned(B), kFewThreads, size_t(2) * P * sizeof(double), s>>>(theta, B, P, flags, psr, lc);
}

void launch_reduce_few(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                       const double* lane_out, double* loglik, double* grad, double* lane_ll,
                       cudaStream_t s) {
    const size_t smem = size_t(2 + kFewTerms) * P * sizeof(double);
    k_reduce_few<<<unsigned(B), kFewReduceThreads, smem, s>>>(theta, B, P, flags, psr, lane_out, loglik,
                                                              grad, lane_ll);
}

void launch_walker_flags(const double* theta, int64_t B, int32_t P, int32_t flags, const double* loglik,
                         int32_t* out, int* any2, cudaStream_t s) {
    const int threads = 128;
    const int64_t blocks = (B + threads - 1) / threads;
    k_walker_flags<<<unsigned(blocks), threads, 0, s>>>(theta, B, P, flags, loglik, out, any2);
}

void launch_reduce(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                   const double* lane_out, double* loglik, double* grad, double* lane_ll,
                   cudaStream_t s) {
    const int threads = 128;
    const int64_t blocks = (B + threads - 1) / threads;
    k_reduce<<<unsigned(blocks), threads, 0, s>>>(theta, B, P, flags, psr, lane_out, loglik, grad,
                                                  lane_ll);
}

}  // namespace argus
