// Projection (K1) and reduction (K4) kernels for sm_103a: the parameter
// vector's continuous-wave source mapped onto each pulsar's lane constants,
// and the per-walker sum over pulsars with the chain rule of the gradient back
// through that mapping.  Both are O(B x P) and run once per call; the O(B x N)
// filter kernels are in kf_kernels.cu.
#include <cmath>
#include <cstdint>

#include "kf_internal.cuh"

namespace argus {

namespace {

constexpr double kLn10 = 2.302585092994045684;
constexpr double kTwoPi = 6.283185307179586477;
constexpr double kPi = 3.141592653589793238;
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

__device__ void source_frame(const double* th, bool with_derivs, SourceFrame& F) {
    F.f = exp10(th[0]);
    F.W = kTwoPi * F.f;
    F.h0 = exp10(th[6]);
    F.ci = th[3];
    F.ampP = F.h0 * fma(F.ci, F.ci, 1.0) / F.W;
    F.ampX = -2.0 * F.h0 * F.ci / F.W;
    const double x = th[4];
    const double cd = sqrt(fmax(0.0, 1.0 - x * x));
    double sa, ca, sp, cp;
    sincos(th[5], &sa, &ca);
    sincos(th[2], &sp, &cp);
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
    double thg[kNgw];
    for (int j = 0; j < kNgw; ++j) thg[j] = th[j];
    SourceFrame F;
    source_frame(thg, false, F);
    Antenna R;
    antenna(F, psr[p].pos, false, R);
    const double* nz = th + kNgw + ly.nq * p;
    const double efac = nz[ly.efac];
    const double sig2 = exp10(2.0 * nz[0]);
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
    double* o = lc + idx;
    o[0 * lanes] = A;
    o[1 * lanes] = Bc;
    o[2 * lanes] = F.f;
    o[3 * lanes] = thg[1] / kTwoPi;
    o[4 * lanes] = sig2;
    o[5 * lanes] = efac * efac;
    o[6 * lanes] = efac;
    if (ly.ou) o[7 * lanes] = exp10(nz[1]);
}


// ---------------------------------------------------------------------------
// K4: per walker, fixed-order sum over pulsars; for the gradient, the chain
// rule through K1 for the 7 source parameters and each pulsar's own ones.
// ---------------------------------------------------------------------------
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
    const bool ok = theta_in_domain(th, P, ly);
    double ll = 0.0;
    for (int p = 0; p < P; ++p) {
        const double lp = lane_out[int64_t(p) * B + b];
        if (lane_ll) lane_ll[b * P + p] = ok ? lp : -INFINITY;
        ll += lp;
    }
    const bool good = ok && isfinite(ll);
    if (loglik) loglik[b] = good ? ll : -INFINITY;
    if (!grad) return;
    double* gout = grad + b * D;
    if (!good) {
        for (int j = 0; j < D; ++j) gout[j] = 0.0;
        return;
    }
    double thg[kNgw];
    for (int j = 0; j < kNgw; ++j) thg[j] = th[j];
    SourceFrame F;
    source_frame(thg, true, F);
    double gw[kNgw] = {0, 0, 0, 0, 0, 0, 0};
    for (int p = 0; p < P; ++p) {
        const double* o = lane_out + int64_t(p) * B + b;
        const double gA = o[1 * lanes], gB = o[2 * lanes], gAt = o[3 * lanes];
        const double gBt = o[4 * lanes], gs2 = o[5 * lanes], gE = o[6 * lanes];
        Antenna R;
        antenna(F, psr[p].pos, true, R);
        const double A = R.Fp * F.ampP, Bc = R.Fx * F.ampX;
        const double* nz = th + kNgw + nq * p;
        double* gz = gout + kNgw + nq * p;
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
        gw[0] += fma(gW, F.W * kLn10, -gAB * kLn10);
        gw[1] += gP;
        gw[2] += fma(hA, 2.0 * R.Fx * F.ampP, hB * (-2.0 * R.Fp) * F.ampX);
        gw[3] += fma(hA, R.Fp * 2.0 * F.h0 * F.ci / F.W, hB * R.Fx * (-2.0 * F.h0 / F.W));
        gw[4] += fma(hA, R.Fp_x * F.ampP, hB * R.Fx_x * F.ampX);
        gw[5] += fma(hA, R.Fp_a * F.ampP, hB * R.Fx_a * F.ampX);
        gw[6] += gAB * kLn10;
        if (ly.pt) {
            // L = W d K D: dL/dlog10 f = L ln 10, dL/dx = W d K dD/dx, dL/dd = W K D
            const double WdK = F.W * nz[nq - 1] * kKpcLightS;
            gw[0] += hL * L * kLn10;
            gw[4] += hL * WdK * R.D_x;
            gw[5] += hL * WdK * R.D_a;
            gz[nq - 1] = hL * F.W * kKpcLightS * R.D;
        }
        gz[0] = gs2 * 2.0 * kLn10 * exp10(2.0 * nz[0]);
        gz[ly.efac] = gE * 2.0 * nz[ly.efac];
        if (ly.ou) gz[1] = o[7 * lanes] * kLn10 * exp10(nz[1]);
    }
    for (int j = 0; j < kNgw; ++j) gout[j] = gw[j];
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

void launch_reduce(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                   const double* lane_out, double* loglik, double* grad, double* lane_ll,
                   cudaStream_t s) {
    const int threads = 128;
    const int64_t blocks = (B + threads - 1) / threads;
    k_reduce<<<unsigned(blocks), threads, 0, s>>>(theta, B, P, flags, psr, lane_out, loglik, grad,
                                                  lane_ll);
}

}  // namespace argus
