// Joint Kalman-filter likelihood of a pulsar timing array with a stochastic
// GW background coupled by the Hellings-Downs correlation (include/argus_gwb.h).
//
// The state of all P pulsars, (rho_n, y_n, a_n), evolves together, and every
// TOA of every pulsar updates it, so the work per TOA is O(P^2) and the lanes
// are parameter vectors, not pulsars: one thread block per parameter vector
// with the 3P x 3P covariance in shared memory.  Per TOA:
//   1. transition coefficients over dt: each pulsar's OU red noise
//      (a_p, b_p, Q_p / sigma_p^2 by ou_coef) and the GW process's;
//   2. predict: F is block diagonal (3 x 3 per pulsar,
//      F_n = [[1, b_p, b_a], [0, a_p, 0], [0, 0, a_a]]), so each 3 x 3 block
//      of P becomes F_I P_IJ F_J^T + Q_IJ on its own.  P is symmetric and
//      only its upper triangle is stored, packed row by row (up to 64
//      pulsars fit): blocks I <= J are computed, the diagonal blocks read
//      symmetrically.  Q_IJ holds the intrinsic noise
//      (I = J) and h_a^2 G_IJ times the integrated-OU increment covariance of
//      the GW process in the (rho, a) slots;
//   3. innovate on rho_q of the TOA's pulsar q: c = P e_{3q}, S = c_{3q} + R,
//      e = r - m_{3q}; the threads that form c also form c / S;
//   4. update: m += c e / S and, over the upper triangle only,
//      P_ij -= c_i (c_j / S); accumulate -1/2 (ln 2 pi + ln S + e^2 / S).
// Steps 2-4 are spread over the block's threads with a barrier between them;
// a TOA at the same time as the previous one skips the predict (F = I, Q = 0).
//
// Scaled frame (the likelihood pass).  The decays a_p of y_p and a_a of the
// GW state are diagonal, so they are carried in scale factors instead of
// the covariance: P = S Ph S, m = S mh with S = diag(1, s_p, s_a) per pulsar.
// Since F_I S_I = S'_I Fh_I with S' = diag(1, s_p a_p, s_a a_a) and
// Fh_I = [[1, b_p s_p, b_a s_a], [0, 1, 0], [0, 0, 1]], the predict becomes
// Ph <- Fh Ph Fh^T + S'^-1 Q S'^-1 and only the rho rows and columns of each
// block change (16 FP64 operations per block instead of 28).  The
// observation picks rho_q, whose scale is 1, so c, S, e and the update keep
// their form with Ph, mh.  A scale below 2^-200 (a fast decay over a long
// gap) folds S back into Ph and takes that one predict unscaled.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/argus.h"
#include "../../include/argus_gwb.h"
#include "kf_internal.cuh"
#include "lib_internal.cuh"
#include "kf_math.cuh"
#include "kf_model.cuh"

namespace argus {
namespace {

constexpr double kLog2PiGwb = 1.8378770664093454836;
constexpr double kLn10Gwb = 2.302585092994045684;
constexpr int kGwbThreads = 256;      // gradient kernel
constexpr int kGwbFwdThreads = 32;    // likelihood kernel: one warp per block
constexpr int kGwbGradMaxPulsars = 48;   // gradient: two packed 3P x 3P triangles in shared memory
constexpr int kCo = 9;                   // per-pulsar coefficients (see GwbSmem::co)

struct GwbRec {     // one TOA of the merged, time-ordered stream (32 bytes)
    double dt;      // time since the previous TOA of any pulsar (0 for the first)
    double r;       // residual, s
    double s2;      // sigma_k^2
    int32_t q;      // pulsar
    int32_t pad;
};

struct GwbArgs {
    const GwbRec* rec;
    int64_t N;
    int32_t P;
    const double* p0;       // [P][3]
    const double* equad2;   // [P]
    const double* G;        // [P][P] Hellings-Downs
    const double* theta;    // [B][2 + 3P]
    int64_t B;
    double* loglik;         // [B]
    double* grad;           // [B][2 + 3P] (gradient kernel)
    double* ckpt;           // per block: [nseg][ne + n] state at each segment start
    double* tape;           // per block: [L][ne + n] state before each step of a segment
    int64_t slot;           // doubles per block in ckpt and in tape
    int32_t L;              // segment length (TOAs)
    int32_t nseg;
};

// Shared memory of a block.  The covariance P and, for the gradient, its
// adjoint Pb are symmetric and stored as packed upper triangles (see pk).
struct GwbSmem {
    int P, n, nb, ne;
    double* Pm;     // packed upper triangle, n (n + 1) / 2
    double* m;      // [n]
    double* c;      // [n]
    double* co;     // [P][9]: a, b, Q/sigma^2 (c00, c01, c11), d/dgamma of b and of c00, c01, c11
    double* cs;     // [P + 1][5], scaled frame, per pulsar and for the GW process (row P):
                    // b s, v c00, v c01 / s', v c11 / s'^2, 1 / s' (v = sigma_p^2 or h_a^2, s' = s a)
    double* ct;     // [n]: c / S
    double* sg;     // [P + 1]: scale factors s_p and s_a (scaled frame)
    double* sg0;    // [P + 1]: the scale factors before the current predict
    const double* G;   // [P][P] Hellings-Downs, in global memory (read through the read-only cache)
    double* par;    // [P][4]: sigma^2, gamma_p, EFAC^2, EFAC
    double* gw;     // GW process: a, b, c00, c01, c11, db, dc00, dc01, dc11 (per unit h_a^2); scalars
    double* Pb;     // packed upper triangle (gradient)
    double* mb;     // [n]      (gradient)
    double* u;      // [n]      (gradient)
    double* v;      // [n]      (gradient)
    double* acc;    // [P][5]: d/d sigma^2, d/d gamma_p, d/d EFAC, d/d h_a^2 part, d/d gamma_a part
    double* part;   // [P][chunks][6]: partial sums of the parameter terms
    double* sgb;    // [2P]: adjoints of s_p, and pulsar I's share of the adjoint of s_a (gradient)
    uint16_t* pairs;
    uint8_t* ent;
};
// scalar slots of gw[]
enum { kGwA = 0, kGwHa2 = 9, kGwGa, kGwE, kGwS, kGwRS, kGwG, kGwOk, kGwSb, kGwEb, kGwR0, kGwRn, kGwRnAny,
       kGwSlots = 24 };
constexpr double kGwbTiny = 0x1p-200;   // smallest scale factor kept (scaled frame)

// chunks per pulsar of the adjoint's parameter sums (J ranges of about 5)
__host__ __device__ inline int gwb_jchunks(int P) { return (P + 4) / 5 < 8 ? (P + 4) / 5 : 8; }
// doubles of one saved state: the upper triangle of P, m and the P + 1 scales
__host__ __device__ inline int64_t gwb_rec_len(int P) {
    const int64_t n = 3 * int64_t(P);
    return n * (n + 1) / 2 + n + P + 1;
}

__host__ __device__ inline size_t gwb_smem_doubles(int P, bool grad) {
    const size_t n = 3 * size_t(P), ne = n * (n + 1) / 2;
    size_t d = ne + 3 * n + kCo * size_t(P) + 5 * (size_t(P) + 1) + 4 * size_t(P) + 2 * (size_t(P) + 1) +
               kGwSlots;
    if (grad) d += ne + 3 * n + 5 * size_t(P) + 6 * size_t(P) * gwb_jchunks(P) + 2 * size_t(P);
    return d;
}

// dynamic shared memory of a block: the doubles, the (I, J) pairs of the
// upper 3x3 blocks (uint16) and the (i, j) pairs of the upper entries (uint8)
__host__ __device__ inline size_t gwb_smem_bytes(int P, bool grad) {
    const size_t n = 3 * size_t(P);
    return gwb_smem_doubles(P, grad) * sizeof(double) + size_t(P) * (P + 1) * sizeof(uint16_t) +
           n * (n + 1) * sizeof(uint8_t);
}

__device__ GwbSmem gwb_carve(double* base, int P, bool grad, const double* G) {
    GwbSmem s;
    s.P = P; s.n = 3 * P; s.nb = P * (P + 1) / 2; s.ne = s.n * (s.n + 1) / 2;
    const int n = s.n;
    double* q = base;
    s.Pm = q; q += s.ne;
    s.m = q; q += n;
    s.c = q; q += n;
    s.co = q; q += kCo * P;
    s.cs = q; q += 5 * (P + 1);
    s.ct = q; q += n;
    s.sg = q; q += P + 1;
    s.sg0 = q; q += P + 1;
    s.G = G;
    s.par = q; q += 4 * P;
    s.gw = q; q += kGwSlots;
    if (grad) {
        s.Pb = q; q += s.ne;
        s.mb = q; q += n;
        s.u = q; q += n;
        s.v = q; q += n;
        s.acc = q; q += 5 * P;
        s.part = q; q += 6 * P * gwb_jchunks(P);
        s.sgb = q; q += 2 * P;
    } else {
        s.Pb = s.mb = s.u = s.v = s.acc = s.part = s.sgb = nullptr;
    }
    s.pairs = reinterpret_cast<uint16_t*>(q);
    s.ent = reinterpret_cast<uint8_t*>(s.pairs + 2 * s.nb);
    return s;
}

__device__ __forceinline__ double gwb_G(const GwbSmem& s, int I, int J) { return __ldg(s.G + I * s.P + J); }

// Symmetric matrices (P and its adjoint) are stored as packed upper
// triangles, row by row: entry (i, j), i <= j, at i n - i (i - 1) / 2 + j - i
// (the order of the (i, j) pair table and of a saved state).
__device__ __forceinline__ int pk(int n, int i, int j) { return i * n - ((i * (i - 1)) >> 1) + (j - i); }
// row i of a packed triangle: prow(M, n, i)[j] is entry (i, j) for j >= i
__device__ __forceinline__ double* prow(double* M, int n, int i) { return M + (i * n - ((i * (i - 1)) >> 1) - i); }
__device__ __forceinline__ double psym(const double* M, int n, int i, int j) {
    return i <= j ? M[pk(n, i, j)] : M[pk(n, j, i)];
}

// sum over a warp in a fixed order (the same tree on every call)
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    return x;
}

// tables and HD matrix, once per block
__device__ void gwb_tables(const GwbSmem& s, const GwbArgs& a) {
    if (threadIdx.x == 0) {
        // the diagonal blocks first, so that only the first warp(s) take their extra terms
        int k = 0;
        for (int I = 0; I < s.P; ++I) { s.pairs[2 * k] = uint16_t(I); s.pairs[2 * k + 1] = uint16_t(I); ++k; }
        for (int I = 0; I < s.P; ++I)
            for (int J = I + 1; J < s.P; ++J) { s.pairs[2 * k] = uint16_t(I); s.pairs[2 * k + 1] = uint16_t(J); ++k; }
        k = 0;
        for (int i = 0; i < s.n; ++i)
            for (int j = i; j < s.n; ++j) { s.ent[2 * k] = uint8_t(i); s.ent[2 * k + 1] = uint8_t(j); ++k; }
    }
}

// parameters of walker th and the prior at the array's earliest TOA; returns
// false (uniformly) when theta is out of the domain
__device__ bool gwb_setup(const GwbSmem& s, const GwbArgs& a, const double* th) {
    const int P = s.P, n = s.n, D = 2 + 3 * P;
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int j = 0; j < D; ++j) ok = ok && isfinite(th[j]);
        for (int p = 0; p < P; ++p) ok = ok && th[2 + 3 * p + 2] > 0.0;
        s.gw[kGwHa2] = exp10(2.0 * th[0]);
        s.gw[kGwGa] = exp10(th[1]);
        s.gw[kGwOk] = ok ? 1.0 : 0.0;
        s.gw[kGwRn] = 0.0;
        s.gw[kGwRnAny] = 0.0;
    }
    for (int p = threadIdx.x; p <= P; p += blockDim.x) s.sg[p] = 1.0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        s.par[4 * p] = exp10(2.0 * th[2 + 3 * p]);
        s.par[4 * p + 1] = exp10(th[2 + 3 * p + 1]);
        const double ef = th[2 + 3 * p + 2];
        s.par[4 * p + 2] = ef * ef;
        s.par[4 * p + 3] = ef;
    }
    __syncthreads();
    if (s.gw[kGwOk] == 0.0) return false;
    const double ha2 = s.gw[kGwHa2], ga = s.gw[kGwGa];
    for (int q = threadIdx.x; q < s.ne; q += blockDim.x) {
        const int r = s.ent[2 * q], col = s.ent[2 * q + 1];
        const int I = r / 3, J = col / 3, uu = r - 3 * I, vv = col - 3 * J;
        double x = 0.0;
        if (uu == 2 && vv == 2) x = ha2 * gwb_G(s, I, J) / (2.0 * ga);
        else if (I == J && uu < 2 && vv < 2) x = a.p0[3 * I + uu + vv];
        s.Pm[q] = x;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) s.m[i] = 0.0;
    __syncthreads();
    return true;
}

// 1. transition coefficients over dt (threads 0..P-1 the pulsars, thread P the GW process)
template <bool kDeriv>
__device__ void gwb_coef(const GwbSmem& s, double dt) {
    const double h2 = 0.5 * dt * dt, h3 = dt * dt * dt / 3.0, dt2 = dt * dt;
    for (int p = threadIdx.x; p <= s.P; p += blockDim.x) {
        OuCoef oc;
        const double gam = (p < s.P) ? s.par[4 * p + 1] : s.gw[kGwGa];
        ou_coef_warp<kDeriv>(gam * dt, dt, h2, h3, dt2, oc);
        double* o = (p < s.P) ? s.co + kCo * p : s.gw + kGwA;
        o[0] = oc.a; o[1] = oc.b; o[2] = oc.c00; o[3] = oc.c01; o[4] = oc.c11;
        if (kDeriv) { o[5] = oc.db; o[6] = oc.dc00; o[7] = oc.dc01; o[8] = oc.dc11; }
    }
}

// 2. predict: the mean and every upper 3x3 block, F_I P_IJ F_J^T + Q_IJ
__device__ void gwb_predict(const GwbSmem& s) {
    const int P = s.P, n = s.n;
    const double* gw = s.gw;
    const double aa = gw[0], ba = gw[1], ha2 = gw[kGwHa2];
    const double qa00 = ha2 * gw[2], qa01 = ha2 * gw[3], qa11 = ha2 * gw[4];
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        double* mp = s.m + 3 * p;
        mp[0] = fma(s.co[kCo * p + 1], mp[1], fma(ba, mp[2], mp[0]));
        mp[1] *= s.co[kCo * p];
        mp[2] *= aa;
    }
    for (int q = threadIdx.x; q < s.nb; q += blockDim.x) {
        const int I = s.pairs[2 * q], J = s.pairs[2 * q + 1];
        const double apI = s.co[kCo * I], bpI = s.co[kCo * I + 1];
        const double apJ = s.co[kCo * J], bpJ = s.co[kCo * J + 1];
        double X[3][3];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v)
                X[u][v] = (I < J || u <= v) ? s.Pm[pk(n, 3 * I + u, 3 * J + v)] : s.Pm[pk(n, 3 * I + v, 3 * J + u)];
        double Y[3][3];   // F_I X
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            Y[0][v] = fma(bpI, X[1][v], fma(ba, X[2][v], X[0][v]));
            Y[1][v] = apI * X[1][v];
            Y[2][v] = aa * X[2][v];
        }
        double Z[3][3];   // (F_I X) F_J^T
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            Z[u][0] = fma(bpJ, Y[u][1], fma(ba, Y[u][2], Y[u][0]));
            Z[u][1] = apJ * Y[u][1];
            Z[u][2] = aa * Y[u][2];
        }
        const double g = gwb_G(s, I, J);
        Z[0][0] = fma(g, qa00, Z[0][0]);
        Z[0][2] = fma(g, qa01, Z[0][2]);
        Z[2][0] = fma(g, qa01, Z[2][0]);
        Z[2][2] = fma(g, qa11, Z[2][2]);
        if (I == J) {
            const double s2 = s.par[4 * I];
            Z[0][0] = fma(s2, s.co[kCo * I + 2], Z[0][0]);
            Z[0][1] = fma(s2, s.co[kCo * I + 3], Z[0][1]);
            Z[1][0] = fma(s2, s.co[kCo * I + 3], Z[1][0]);
            Z[1][1] = fma(s2, s.co[kCo * I + 4], Z[1][1]);
        }
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v)
                if (I < J || u <= v) s.Pm[pk(n, 3 * I + u, 3 * J + v)] = Z[u][v];
    }
}

// 1'. scaled frame: the coefficients of 1. (with their gamma-derivatives when
// kDeriv) and those of Fh and S'^-1 Q S'^-1 (cs).  With kAdvance the scales
// advance to s' = s a, and a scale below kGwbTiny raises the flag.
template <bool kDeriv, bool kAdvance>
__device__ void gwb_coef_scaled(const GwbSmem& s, double dt) {
    const double h2 = 0.5 * dt * dt, h3 = dt * dt * dt / 3.0, dt2 = dt * dt;
    for (int p = threadIdx.x; p <= s.P; p += blockDim.x) {
        OuCoef oc;
        const bool psr = p < s.P;
        ou_coef_warp<kDeriv>((psr ? s.par[4 * p + 1] : s.gw[kGwGa]) * dt, dt, h2, h3, dt2, oc);
        const double sg = s.sg[p], sn = sg * oc.a;
        if (kAdvance) {
            s.sg0[p] = sg;
            s.sg[p] = sn;
            if (!(sn >= kGwbTiny)) s.gw[kGwRn] = 1.0;
        }
        const double w = rcp_nr(sn), sc = psr ? s.par[4 * p] : s.gw[kGwHa2];
        double* o = psr ? s.co + kCo * p : s.gw + kGwA;
        o[0] = oc.a; o[1] = oc.b; o[2] = oc.c00; o[3] = oc.c01; o[4] = oc.c11;
        if (kDeriv) { o[5] = oc.db; o[6] = oc.dc00; o[7] = oc.dc01; o[8] = oc.dc11; }
        double* h = s.cs + 5 * p;
        h[0] = oc.b * sg;
        h[1] = sc * oc.c00;
        h[2] = sc * oc.c01 * w;
        h[3] = sc * oc.c11 * w * w;
        h[4] = w;
    }
}

// 2'. scaled predict: mh <- Fh mh, Ph <- Fh Ph Fh^T + S'^-1 Q S'^-1 (upper
// blocks); Fh is the identity but for the rho row (b_p s_p, b_a s_a)
__device__ void gwb_predict_scaled(const GwbSmem& s) {
    const int P = s.P, n = s.n;
    const double* ca = s.cs + 5 * P;
    const double al = ca[0], qa00 = ca[1], qa01 = ca[2], qa11 = ca[3];
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        double* mp = s.m + 3 * p;
        mp[0] = fma(s.cs[5 * p], mp[1], fma(al, mp[2], mp[0]));
    }
    for (int q = threadIdx.x; q < s.nb; q += blockDim.x) {
        const int I = s.pairs[2 * q], J = s.pairs[2 * q + 1];
        const double bI = s.cs[5 * I], bJ = s.cs[5 * J];
        // rows 3I, 3I+1, 3I+2 of the block (entry (3I+u, 3J+v) is R_u[v])
        double* R0 = prow(s.Pm, n, 3 * I) + 3 * J;
        double* R1 = prow(s.Pm, n, 3 * I + 1) + 3 * J;
        double* R2 = prow(s.Pm, n, 3 * I + 2) + 3 * J;
        const double x00 = R0[0], x01 = R0[1], x02 = R0[2], x11 = R1[1], x12 = R1[2], x22 = R2[2];
        const double x10 = I < J ? R1[0] : x01, x20 = I < J ? R2[0] : x02, x21 = I < J ? R2[1] : x12;
        // row 0 of Fh_I X, then column 0 of (Fh_I X) Fh_J^T
        const double y0 = fma(bI, x10, fma(al, x20, x00));
        const double y1 = fma(bI, x11, fma(al, x21, x01));
        const double y2 = fma(bI, x12, fma(al, x22, x02));
        const double g = gwb_G(s, I, J);
        double z00 = fma(g, qa00, fma(bJ, y1, fma(al, y2, y0)));
        double z01 = y1;
        const double z02 = fma(g, qa01, y2);
        double z11 = x11;
        const double z22 = fma(g, qa11, x22);
        if (I == J) {
            const double* cI = s.cs + 5 * I;
            z00 += cI[1];
            z01 += cI[2];
            z11 += cI[3];
        } else {
            R1[0] = fma(bJ, x11, fma(al, x12, x10));
            R2[0] = fma(g, qa01, fma(bJ, x21, fma(al, x22, x20)));
        }
        R0[0] = z00; R0[1] = z01; R0[2] = z02; R1[1] = z11; R2[2] = z22;
    }
}

// scale of state i: 1 for rho, s_p for y_p, s_a for a_p
__device__ __forceinline__ double gwb_scale_of(const double* sc, int P, int i) {
    const int J = i / 3, cmp = i - 3 * J;
    return cmp == 0 ? 1.0 : sc[cmp == 1 ? J : P];
}

// P = S Ph S, m = S mh for the scales sc (the upper triangle and the mean)
__device__ void gwb_fold(const GwbSmem& s, const double* sc) {
    const int n = s.n, P = s.P;
    for (int q = threadIdx.x; q < s.ne; q += blockDim.x) {
        const int r = s.ent[2 * q], col = s.ent[2 * q + 1];
        s.Pm[q] *= gwb_scale_of(sc, P, r) * gwb_scale_of(sc, P, col);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) s.m[i] *= gwb_scale_of(sc, P, i);
}

// 3. innovate on rho of pulsar q: c = P e_i and c / S (the threads that form
// c each form 1/S); thread 0 records e, S, 1/S, e/S
__device__ void gwb_innovate(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk) {
    const int n = s.n, i0 = 3 * rk.q;
    if (threadIdx.x < n) {
        const double R = fma(s.par[4 * rk.q + 2], rk.s2, a.equad2[rk.q]);
        const double S = s.Pm[pk(n, i0, i0)] + R;
        const double rS = rcp_nr(S);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double ci = psym(s.Pm, n, i, i0);
            s.c[i] = ci;
            s.ct[i] = ci * rS;
        }
        if (threadIdx.x == 0) {
            const double e = rk.r - s.m[i0];
            s.gw[kGwE] = e;
            s.gw[kGwS] = S;
            s.gw[kGwRS] = rS;
            s.gw[kGwG] = e * rS;
        }
    }
}

// 4. update (upper triangle, P_ij -= c_i (c_j / S)) and mean
__device__ void gwb_update(const GwbSmem& s) {
    const int n = s.n;
    const double g = s.gw[kGwG];
    for (int q = threadIdx.x; q < s.ne; q += blockDim.x) {
        const int r = s.ent[2 * q], col = s.ent[2 * q + 1];
        s.Pm[q] = fma(-s.c[r], s.ct[col], s.Pm[q]);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) s.m[i] = fma(s.c[i], g, s.m[i]);
}

// one forward step; thread 0 accumulates the likelihood when kLL; kScaled
// keeps Ph, mh in the scaled frame
template <bool kLL, bool kScaled = false>
__device__ void gwb_step(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk, double& quad, LogProd& lp) {
    if (rk.dt > 0.0) {
        if (kScaled) {
            gwb_coef_scaled<false, true>(s, rk.dt);
            __syncthreads();
            if (s.gw[kGwRn] != 0.0) {          // block-uniform and rare: unscale, predict unscaled
                gwb_fold(s, s.sg0);
                __syncthreads();
                gwb_predict(s);
                for (int p = threadIdx.x; p <= s.P; p += blockDim.x) s.sg[p] = 1.0;
                if (threadIdx.x == 0) {
                    s.gw[kGwRn] = 0.0;
                    s.gw[kGwRnAny] = 1.0;
                }
            } else {
                gwb_predict_scaled(s);
            }
        } else {
            gwb_coef<false>(s, rk.dt);
            __syncthreads();
            gwb_predict(s);
        }
        __syncthreads();
    }
    gwb_innovate(s, a, rk);
    __syncthreads();
    if (kLL && threadIdx.x == 0) {
        quad = fma(s.gw[kGwE], s.gw[kGwG], quad);
        lp.add(s.gw[kGwS]);
    }
    gwb_update(s);
    __syncthreads();
}

__device__ __forceinline__ double gwb_finish(int64_t N, double quad, const LogProd& lp) {
    double ll = (N == 0) ? 0.0 : -0.5 * (double(N) * kLog2PiGwb + lp.value() + quad);
    return (lp.bad || !isfinite(ll)) ? -INFINITY : ll;
}

__global__ void __launch_bounds__(kGwbFwdThreads) k_gwb_filter(GwbArgs a) {
    extern __shared__ __align__(16) double gsm[];
    const GwbSmem s = gwb_carve(gsm, a.P, false, a.G);
    gwb_tables(s, a);
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        __syncthreads();
        if (!gwb_setup(s, a, a.theta + b * (2 + 3 * a.P))) {
            if (threadIdx.x == 0) a.loglik[b] = -INFINITY;
            continue;
        }
        double quad = 0.0;
        LogProd lp;
        for (int64_t k = 0; k < a.N; ++k) gwb_step<true, true>(s, a, a.rec[k], quad, lp);
        if (threadIdx.x == 0) a.loglik[b] = gwb_finish(a.N, quad, lp);
    }
}

// state (upper triangle of P, then m) to / from a global slot
__device__ void gwb_save(const GwbSmem& s, double* dst) {
    for (int q = threadIdx.x; q < s.ne; q += blockDim.x) dst[q] = s.Pm[q];
    for (int i = threadIdx.x; i < s.n; i += blockDim.x) dst[s.ne + i] = s.m[i];
    for (int p = threadIdx.x; p <= s.P; p += blockDim.x) dst[s.ne + s.n + p] = s.sg[p];
}

__device__ void gwb_load(const GwbSmem& s, const double* src) {
    for (int q = threadIdx.x; q < s.ne; q += blockDim.x) s.Pm[q] = src[q];
    for (int i = threadIdx.x; i < s.n; i += blockDim.x) s.m[i] = src[s.ne + i];
    for (int p = threadIdx.x; p <= s.P; p += blockDim.x) s.sg[p] = src[s.ne + s.n + p];
}

// Reverse of the observation of TOA rk (either frame).  On entry c holds the
// predicted covariance's column i = 3q, gw[kGwE] the innovation and
// gw[kGwR0] the measurement variance; Pb, mb the adjoints after the update.
// On exit Pb holds M-bar, the symmetric adjoint of the predicted covariance,
// and mb mu-bar, that of the predicted mean; EFAC_q's term is accumulated.
__device__ void gwb_adjoint_observation(const GwbSmem& s, const GwbRec& rk) {
    const int n = s.n, q = rk.q, i0 = 3 * q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* gw = s.gw;
    if (tid == 0) {
        const double S = s.c[i0] + gw[kGwR0];
        const double rS = rcp_nr(S);
        gw[kGwS] = S; gw[kGwRS] = rS; gw[kGwG] = gw[kGwE] * rS;
    }
    // v = Pb c, one thread per entry: row j of the symmetric Pb is its packed
    // column above the diagonal, then its packed row (k in order either way)
    for (int j = tid; j < n; j += blockDim.x) {
        double acc = 0.0;
        int idx = j;                      // packed (0, j)
        for (int k = 0; k < j; ++k) {
            acc = fma(s.Pb[idx], s.c[k], acc);
            idx += n - k - 1;             // packed (k + 1, j)
        }
        const double* Rj = prow(s.Pb, n, j);
        for (int k = j; k < n; ++k) acc = fma(Rj[k], s.c[k], acc);
        s.v[j] = acc;
    }
    __syncthreads();
    if (warp == 0) {
        double gb = 0.0, cv = 0.0;
        for (int k = lane; k < n; k += 32) { gb = fma(s.mb[k], s.c[k], gb); cv = fma(s.c[k], s.v[k], cv); }
        gb = warp_sum(gb);
        cv = warp_sum(cv);
        if (lane == 0) {
            const double rS = gw[kGwRS], g = gw[kGwG];
            const double Sb = rS * rS * cv - gb * g * rS - 0.5 * rS + 0.5 * g * g;
            gw[kGwSb] = Sb;
            gw[kGwEb] = gb * rS - g;
            s.acc[5 * q + 2] += Sb * 2.0 * s.par[4 * q + 3] * rk.s2;     // d/d EFAC_q
        }
    }
    __syncthreads();
    // c-bar, the symmetric M-bar (row and column i of Pb) and mu-bar (in mb)
    {
        const double rS = gw[kGwRS], g = gw[kGwG], Sb = gw[kGwSb], eb = gw[kGwEb];
        for (int j = tid; j < n; j += blockDim.x) {
            const double cb = fma(s.mb[j], g, -2.0 * rS * s.v[j]);
            if (j == i0) {
                s.Pb[pk(n, j, j)] += cb + Sb;
                s.mb[j] -= eb;
            } else {   // the one stored entry of the symmetric pair (j, i), (i, j)
                double& e = s.Pb[j < i0 ? pk(n, j, i0) : pk(n, i0, j)];
                e = fma(0.5, cb, e);
            }
        }
    }
    __syncthreads();
}

// Reverse of one forward step k, the state before it in Pm, m.  On entry Pb,
// mb hold the adjoints of the state after the step; on exit, before it.
__device__ void gwb_step_adjoint(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk) {
    const int P = s.P, n = s.n, q = rk.q, i0 = 3 * q;
    const int tid = threadIdx.x;
    const double dt = rk.dt;
    const bool pred = dt > 0.0;
    double* gw = s.gw;
    if (pred) {
        gwb_coef<true>(s, dt);
        __syncthreads();
    }
    // u = P (F^T e_i), and mu_i = (F m)_i
    const double bq = pred ? s.co[kCo * q + 1] : 0.0, ba = pred ? gw[1] : 0.0;
    for (int j = tid; j < n; j += blockDim.x)
        s.u[j] = fma(bq, psym(s.Pm, n, j, i0 + 1), fma(ba, psym(s.Pm, n, j, i0 + 2), psym(s.Pm, n, j, i0)));
    __syncthreads();
    // c = F u + Q e_i (the predicted covariance's column i)
    const double ha2 = gw[kGwHa2];
    for (int J = tid; J < P; J += blockDim.x) {
        const double* uJ = s.u + 3 * J;
        if (pred) {
            const double aJ = s.co[kCo * J], bJ = s.co[kCo * J + 1], aa = gw[0];
            const double g = gwb_G(s, J, q) * ha2;
            double c0 = fma(bJ, uJ[1], fma(ba, uJ[2], uJ[0])) + g * gw[2];
            double c1 = aJ * uJ[1];
            const double c2 = fma(aa, uJ[2], g * gw[3]);
            if (J == q) {
                const double s2 = s.par[4 * q];
                c0 = fma(s2, s.co[kCo * q + 2], c0);
                c1 = fma(s2, s.co[kCo * q + 3], c1);
            }
            s.c[3 * J] = c0; s.c[3 * J + 1] = c1; s.c[3 * J + 2] = c2;
        } else {
            s.c[3 * J] = uJ[0]; s.c[3 * J + 1] = uJ[1]; s.c[3 * J + 2] = uJ[2];
        }
    }
    if (tid == 0) {
        const double mu = fma(bq, s.m[i0 + 1], fma(ba, s.m[i0 + 2], s.m[i0]));
        const double R = fma(s.par[4 * q + 2], rk.s2, a.equad2[q]);
        gw[kGwE] = rk.r - mu;
        gw[kGwR0] = R;   // this TOA's measurement variance
    }
    __syncthreads();
    gwb_adjoint_observation(s, rk);
    if (!pred) return;   // F = I, Q = 0: the adjoints pass through
    // parameters through F and Q, in two levels: work item (I, chunk of J)
    // forms partial sums of (M-bar F P) at (rho_I, y_I), (y_I, y_I),
    // (rho_I, a_I), (a_I, a_I) and of the GW noise's contractions with G;
    // then one thread per pulsar adds its chunks in fixed order
    const double aa = gw[0], dba = gw[5], dca00 = gw[6], dca01 = gw[7], dca11 = gw[8];
    const int nch = gwb_jchunks(P), jc = (P + nch - 1) / nch;
    for (int it = tid; it < P * nch; it += blockDim.x) {
        const int I = it / nch, ch = it - I * nch;
        const int rI = 3 * I, yI = rI + 1, aI = rI + 2;
        auto Mr = [&](int j) { return psym(s.Pb, n, rI, j); };   // row rho_I of M-bar
        auto My = [&](int j) { return psym(s.Pb, n, yI, j); };
        auto Ma = [&](int j) { return psym(s.Pb, n, aI, j); };
        double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, h = 0.0, gd = 0.0;
        const int j_hi = min(P, (ch + 1) * jc);
        for (int J = ch * jc; J < j_hi; ++J) {
            const int rJ = 3 * J;
            const double aJ = s.co[kCo * J], bJ = s.co[kCo * J + 1];
            const double py0 = psym(s.Pm, n, rJ, yI), py1 = psym(s.Pm, n, rJ + 1, yI), py2 = psym(s.Pm, n, rJ + 2, yI);
            const double pa0 = psym(s.Pm, n, rJ, aI), pa1 = psym(s.Pm, n, rJ + 1, aI), pa2 = psym(s.Pm, n, rJ + 2, aI);
            // (F P)[k, y_I] and (F P)[k, a_I] for k = rho_J, y_J, a_J
            const double fy0 = fma(bJ, py1, fma(ba, py2, py0)), fy1 = aJ * py1, fy2 = aa * py2;
            const double fa0 = fma(bJ, pa1, fma(ba, pa2, pa0)), fa1 = aJ * pa1, fa2 = aa * pa2;
            s1 = fma(Mr(rJ), fy0, fma(Mr(rJ + 1), fy1, fma(Mr(rJ + 2), fy2, s1)));
            s2 = fma(My(rJ), fy0, fma(My(rJ + 1), fy1, fma(My(rJ + 2), fy2, s2)));
            s3 = fma(Mr(rJ), fa0, fma(Mr(rJ + 1), fa1, fma(Mr(rJ + 2), fa2, s3)));
            s4 = fma(Ma(rJ), fa0, fma(Ma(rJ + 1), fa1, fma(Ma(rJ + 2), fa2, s4)));
            const double g = gwb_G(s, I, J);
            const double X00 = Mr(rJ), X02 = Mr(rJ + 2), X20 = Ma(rJ), X22 = Ma(rJ + 2);
            h = fma(g, fma(X00, gw[2], fma(X02 + X20, gw[3], X22 * gw[4])), h);
            gd = fma(g, fma(X00, dca00, fma(X02 + X20, dca01, X22 * dca11)), gd);
        }
        double* pt = s.part + 6 * it;
        pt[0] = s1; pt[1] = s2; pt[2] = s3; pt[3] = s4; pt[4] = h; pt[5] = gd;
    }
    __syncthreads();
    for (int I = tid; I < P; I += blockDim.x) {
        const int rI = 3 * I, yI = rI + 1, aI = rI + 2;
        double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, h = 0.0, gd = 0.0;
        for (int ch = 0; ch < nch; ++ch) {
            const double* pt = s.part + 6 * (I * nch + ch);
            s1 += pt[0]; s2 += pt[1]; s3 += pt[2]; s4 += pt[3]; h += pt[4]; gd += pt[5];
        }
        const double* co = s.co + kCo * I;
        const double bbar_p = fma(2.0, s1, s.mb[rI] * s.m[yI]);
        const double abar_p = fma(2.0, s2, s.mb[yI] * s.m[yI]);
        const double bbar_a = fma(2.0, s3, s.mb[rI] * s.m[aI]);
        const double abar_a = fma(2.0, s4, s.mb[aI] * s.m[aI]);
        const double M00 = s.Pb[pk(n, rI, rI)], M01 = s.Pb[pk(n, rI, yI)], M11 = s.Pb[pk(n, yI, yI)];
        const double s2p = s.par[4 * I];
        double* acc = s.acc + 5 * I;
        acc[0] += fma(M00, co[2], fma(2.0 * M01, co[3], M11 * co[4]));
        acc[1] += fma(-dt * co[0], abar_p, fma(bbar_p, co[5],
                      s2p * fma(M00, co[6], fma(2.0 * M01, co[7], M11 * co[8]))));
        acc[3] += h;
        acc[4] += fma(-dt * aa, abar_a, fma(bbar_a, dba, ha2 * gd));
    }
    __syncthreads();
    // Pb <- F^T Pb F (upper blocks) and mb <- F^T mb
    for (int qq = tid; qq < s.nb; qq += blockDim.x) {
        const int I = s.pairs[2 * qq], J = s.pairs[2 * qq + 1];
        const double aI = s.co[kCo * I], bI = s.co[kCo * I + 1], aJ = s.co[kCo * J], bJ = s.co[kCo * J + 1];
        double X[3][3];
        for (int u = 0; u < 3; ++u)
            for (int v = 0; v < 3; ++v)
                X[u][v] = (I < J || u <= v) ? s.Pb[pk(n, 3 * I + u, 3 * J + v)] : s.Pb[pk(n, 3 * I + v, 3 * J + u)];
        double Y[3][3];   // F_I^T X
        for (int v = 0; v < 3; ++v) {
            Y[0][v] = X[0][v];
            Y[1][v] = fma(bI, X[0][v], aI * X[1][v]);
            Y[2][v] = fma(ba, X[0][v], aa * X[2][v]);
        }
        for (int u = 0; u < 3; ++u) {   // (F_I^T X) F_J
            const double z0 = Y[u][0];
            const double z1 = fma(bJ, Y[u][0], aJ * Y[u][1]);
            const double z2 = fma(ba, Y[u][0], aa * Y[u][2]);
            double* R = prow(s.Pb, n, 3 * I + u) + 3 * J;   // a diagonal block keeps v >= u
            if (I < J || u == 0) R[0] = z0;
            if (I < J || u <= 1) R[1] = z1;
            R[2] = z2;
        }
    }
    for (int J = tid; J < P; J += blockDim.x) {
        double* mJ = s.mb + 3 * J;
        const double m0 = mJ[0];
        mJ[1] = fma(s.co[kCo * J + 1], m0, s.co[kCo * J] * mJ[1]);
        mJ[2] = fma(ba, m0, aa * mJ[2]);
    }
    __syncthreads();
}

// Reverse of one forward step k in the scaled frame: the state before it
// (Ph, mh and the scales s) in Pm, m, sg.  On entry Pb, mb and sgb hold the
// adjoints of Ph, mh and s after the step; on exit, before it.  With M-bar the
// adjoint of the predicted Ph and mu-bar that of the predicted mh:
//   Fh-bar = 2 M-bar Fh Ph + mu-bar mh^T, of which b s (rho_I, y_I) and
//   b_a s_a (rho_I, a_I, every I) are parameters;
//   the process noise v c / s'^k (k = 0, 1, 2) passes its adjoint to v, c and
//   s' = s a; s' passes its adjoint to s and a;
//   Ph-bar = Fh^T M-bar Fh, mh-bar = Fh^T mu-bar.
// The GW scale s_a is common to all pulsars; its adjoint is carried as P
// shares (pulsar I's terms), so every sum over pulsars stays in fixed order.
__device__ void gwb_step_adjoint_scaled(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk) {
    const int P = s.P, n = s.n, q = rk.q, i0 = 3 * q;
    const int tid = threadIdx.x;
    const double dt = rk.dt;
    const bool pred = dt > 0.0;
    double* gw = s.gw;
    if (pred) {
        gwb_coef_scaled<true, false>(s, dt);
        __syncthreads();
    }
    const double* ca = s.cs + 5 * P;
    const double bq = pred ? s.cs[5 * q] : 0.0, al = pred ? ca[0] : 0.0;
    // u = Ph (Fh^T e_i); c = Fh u + Qh e_i, the predicted column i
    for (int j = tid; j < n; j += blockDim.x)
        s.u[j] = fma(bq, psym(s.Pm, n, j, i0 + 1), fma(al, psym(s.Pm, n, j, i0 + 2), psym(s.Pm, n, j, i0)));
    __syncthreads();
    for (int J = tid; J < P; J += blockDim.x) {
        const double* uJ = s.u + 3 * J;
        if (pred) {
            const double g = gwb_G(s, J, q);
            double c0 = fma(g, ca[1], fma(s.cs[5 * J], uJ[1], fma(al, uJ[2], uJ[0])));
            double c1 = uJ[1];
            const double c2 = fma(g, ca[2], uJ[2]);
            if (J == q) {
                c0 += s.cs[5 * q + 1];
                c1 += s.cs[5 * q + 2];
            }
            s.c[3 * J] = c0; s.c[3 * J + 1] = c1; s.c[3 * J + 2] = c2;
        } else {
            s.c[3 * J] = uJ[0]; s.c[3 * J + 1] = uJ[1]; s.c[3 * J + 2] = uJ[2];
        }
    }
    if (tid == 0) {
        const double mu = fma(bq, s.m[i0 + 1], fma(al, s.m[i0 + 2], s.m[i0]));
        gw[kGwE] = rk.r - mu;
        gw[kGwR0] = fma(s.par[4 * q + 2], rk.s2, a.equad2[q]);
    }
    __syncthreads();
    gwb_adjoint_observation(s, rk);
    if (!pred) return;   // Fh = I, Q = 0, s unchanged: the adjoints pass through
    // sums over J for each pulsar I, in chunks of J: (M-bar Fh Ph) at (rho_I,
    // y_I) and (rho_I, a_I), and the GW noise's contractions with G
    const int nch = gwb_jchunks(P), jc = (P + nch - 1) / nch;
    for (int it = tid; it < P * nch; it += blockDim.x) {
        const int I = it / nch, ch = it - I * nch;
        const int rI = 3 * I, yI = rI + 1, aI = rI + 2;
        auto Mr = [&](int j) { return psym(s.Pb, n, rI, j); };   // row rho_I of M-bar
        auto Ma = [&](int j) { return psym(s.Pb, n, aI, j); };
        double sB = 0.0, sA = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
        const int j_hi = min(P, (ch + 1) * jc);
        for (int J = ch * jc; J < j_hi; ++J) {
            const int rJ = 3 * J;
            const double bJ = s.cs[5 * J];
            const double py0 = psym(s.Pm, n, rJ, yI), py1 = psym(s.Pm, n, rJ + 1, yI), py2 = psym(s.Pm, n, rJ + 2, yI);
            const double pa0 = psym(s.Pm, n, rJ, aI), pa1 = psym(s.Pm, n, rJ + 1, aI), pa2 = psym(s.Pm, n, rJ + 2, aI);
            const double m0 = Mr(rJ), m1 = Mr(rJ + 1), m2 = Mr(rJ + 2);
            sB = fma(m0, fma(bJ, py1, fma(al, py2, py0)), fma(m1, py1, fma(m2, py2, sB)));
            sA = fma(m0, fma(bJ, pa1, fma(al, pa2, pa0)), fma(m1, pa1, fma(m2, pa2, sA)));
            const double g = gwb_G(s, I, J);
            t1 = fma(g, m0, t1);
            t2 = fma(g, m2 + Ma(rJ), t2);
            t3 = fma(g, Ma(rJ + 2), t3);
        }
        double* pt = s.part + 6 * it;
        pt[0] = sB; pt[1] = sA; pt[2] = t1; pt[3] = t2; pt[4] = t3;
    }
    __syncthreads();
    const double ha2 = gw[kGwHa2], sga = s.sg[P], wa = ca[4];
    for (int I = tid; I < P; I += blockDim.x) {
        const int rI = 3 * I, yI = rI + 1, aI = rI + 2;
        double sB = 0.0, sA = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (int ch = 0; ch < nch; ++ch) {
            const double* pt = s.part + 6 * (I * nch + ch);
            sB += pt[0]; sA += pt[1]; t1 += pt[2]; t2 += pt[3]; t3 += pt[4];
        }
        const double* co = s.co + kCo * I;
        const double* cI = s.cs + 5 * I;
        const double w = cI[4], sgI = s.sg[I], s2p = s.par[4 * I];
        const double bhb = fma(2.0, sB, s.mb[rI] * s.m[yI]);     // adjoint of b_I s_I
        const double alb = fma(2.0, sA, s.mb[rI] * s.m[aI]);     // pulsar I's share of that of b_a s_a
        const double M00 = s.Pb[pk(n, rI, rI)], q1b = 2.0 * s.Pb[pk(n, rI, yI)], M11 = s.Pb[pk(n, yI, yI)];
        // intrinsic noise v c00, v c01 / s', v c11 / s'^2 and the scale s'_I
        const double sbt = s.sgb[I] - w * fma(q1b, cI[2], 2.0 * M11 * cI[3]);
        double* acc = s.acc + 5 * I;
        acc[0] += fma(M00, co[2], w * fma(q1b, co[3], w * M11 * co[4]));
        acc[1] += fma(s2p, fma(M00, co[6], w * fma(q1b, co[7], w * M11 * co[8])),
                      sgI * fma(bhb, co[5], -dt * co[0] * sbt));
        s.sgb[I] = fma(sbt, co[0], bhb * co[1]);
        // pulsar I's share of the GW terms
        const double sbat = s.sgb[P + I] - wa * fma(t2, ca[2], 2.0 * t3 * ca[3]);
        acc[3] += fma(t1, gw[2], wa * fma(t2, gw[3], wa * t3 * gw[4]));
        acc[4] += fma(ha2, fma(t1, gw[6], wa * fma(t2, gw[7], wa * t3 * gw[8])),
                      sga * fma(alb, gw[5], -dt * gw[0] * sbat));
        s.sgb[P + I] = fma(sbat, gw[0], alb * gw[1]);
    }
    __syncthreads();
    // Pb <- Fh^T Pb Fh (upper blocks) and mb <- Fh^T mb
    for (int qq = tid; qq < s.nb; qq += blockDim.x) {
        const int I = s.pairs[2 * qq], J = s.pairs[2 * qq + 1];
        const double bI = s.cs[5 * I], bJ = s.cs[5 * J];
        double X[3][3];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v)
                X[u][v] = (I < J || u <= v) ? s.Pb[pk(n, 3 * I + u, 3 * J + v)] : s.Pb[pk(n, 3 * I + v, 3 * J + u)];
#pragma unroll
        for (int v = 0; v < 3; ++v) {   // Fh_I^T X: rows y, a gain b_I s_I, b_a s_a times row rho
            X[1][v] = fma(bI, X[0][v], X[1][v]);
            X[2][v] = fma(al, X[0][v], X[2][v]);
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {   // (Fh_I^T X) Fh_J
            const double z0 = X[u][0];
            const double z1 = fma(bJ, z0, X[u][1]);
            const double z2 = fma(al, z0, X[u][2]);
            double* R = prow(s.Pb, n, 3 * I + u) + 3 * J;   // a diagonal block keeps v >= u
            if (I < J || u == 0) R[0] = z0;
            if (I < J || u <= 1) R[1] = z1;
            R[2] = z2;
        }
    }
    for (int J = tid; J < P; J += blockDim.x) {
        double* mJ = s.mb + 3 * J;
        const double m0 = mJ[0];
        mJ[1] = fma(s.cs[5 * J], m0, mJ[1]);
        mJ[2] = fma(al, m0, mJ[2]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kGwbThreads, 4) k_gwb_grad(GwbArgs a) {
    extern __shared__ __align__(16) double gsm[];
    const GwbSmem s = gwb_carve(gsm, a.P, true, a.G);
    const int P = s.P, n = s.n, D = 2 + 3 * P;
    const int64_t rec_len = gwb_rec_len(P);
    double* ck = a.ckpt + int64_t(blockIdx.x) * a.slot;
    double* tp = a.tape + int64_t(blockIdx.x) * a.slot;
    gwb_tables(s, a);
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        double* gout = a.grad + b * D;
        __syncthreads();
        if (!gwb_setup(s, a, a.theta + b * D)) {
            for (int j = threadIdx.x; j < D; j += blockDim.x) gout[j] = 0.0;
            if (threadIdx.x == 0) a.loglik[b] = -INFINITY;
            continue;
        }
        // forward in the scaled frame, with the state saved at each segment
        // start; a vector whose scales had to be folded back (a fast decay
        // over a long gap) runs the whole gradient unscaled instead
        double quad = 0.0;
        LogProd lp;
        for (int seg = 0; seg < a.nseg; ++seg) {
            gwb_save(s, ck + seg * rec_len);
            const int64_t k1 = min(int64_t(seg + 1) * a.L, a.N);
            for (int64_t k = int64_t(seg) * a.L; k < k1; ++k) gwb_step<true, true>(s, a, a.rec[k], quad, lp);
        }
        const bool scaled = s.gw[kGwRnAny] == 0.0;
        if (!scaled) {
            __syncthreads();
            gwb_setup(s, a, a.theta + b * D);
            quad = 0.0;
            lp = LogProd();
            for (int seg = 0; seg < a.nseg; ++seg) {
                gwb_save(s, ck + seg * rec_len);
                const int64_t k1 = min(int64_t(seg + 1) * a.L, a.N);
                for (int64_t k = int64_t(seg) * a.L; k < k1; ++k) gwb_step<true>(s, a, a.rec[k], quad, lp);
            }
        }
        if (threadIdx.x == 0) {
            const double ll = gwb_finish(a.N, quad, lp);
            a.loglik[b] = ll;
            s.gw[kGwOk] = isfinite(ll) ? 1.0 : 0.0;
        }
        for (int i = threadIdx.x; i < s.ne; i += blockDim.x) s.Pb[i] = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s.mb[i] = 0.0;
        for (int i = threadIdx.x; i < 5 * P; i += blockDim.x) s.acc[i] = 0.0;
        for (int i = threadIdx.x; i < 2 * P; i += blockDim.x) s.sgb[i] = 0.0;
        __syncthreads();
        if (s.gw[kGwOk] == 0.0 || a.N == 0) {
            for (int j = threadIdx.x; j < D; j += blockDim.x) gout[j] = 0.0;
            continue;
        }
        // reverse, segment by segment: re-run the segment saving the state
        // before each step, then the adjoint steps in reverse order
        for (int seg = a.nseg - 1; seg >= 0; --seg) {
            const int64_t k0 = int64_t(seg) * a.L, k1 = min(k0 + a.L, a.N);
            gwb_load(s, ck + seg * rec_len);
            __syncthreads();
            for (int64_t k = k0; k < k1; ++k) {
                gwb_save(s, tp + (k - k0) * rec_len);
                if (scaled) gwb_step<false, true>(s, a, a.rec[k], quad, lp);
                else gwb_step<false>(s, a, a.rec[k], quad, lp);
            }
            for (int64_t k = k1 - 1; k >= k0; --k) {
                __syncthreads();
                gwb_load(s, tp + (k - k0) * rec_len);
                __syncthreads();
                if (scaled) gwb_step_adjoint_scaled(s, a, a.rec[k]);
                else gwb_step_adjoint(s, a, a.rec[k]);
            }
        }
        // the stationary prior of the a block: h_a^2 G / (2 gamma_a)
        const double ha2 = s.gw[kGwHa2], ga = s.gw[kGwGa];
        for (int I = threadIdx.x; I < P; I += blockDim.x) {
            double h = 0.0;
            for (int J = 0; J < P; ++J) h = fma(psym(s.Pb, n, 3 * I + 2, 3 * J + 2), gwb_G(s, I, J), h);
            s.acc[5 * I + 3] += h / (2.0 * ga);
            s.acc[5 * I + 4] -= h * ha2 / (2.0 * ga * ga);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double hb = 0.0, gb = 0.0;
            for (int I = 0; I < P; ++I) { hb += s.acc[5 * I + 3]; gb += s.acc[5 * I + 4]; }
            gout[0] = hb * 2.0 * kLn10Gwb * ha2;
            gout[1] = gb * kLn10Gwb * ga;
        }
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            gout[2 + 3 * p] = s.acc[5 * p] * 2.0 * kLn10Gwb * s.par[4 * p];
            gout[3 + 3 * p] = s.acc[5 * p + 1] * kLn10Gwb * s.par[4 * p + 1];
            gout[4 + 3 * p] = s.acc[5 * p + 2];
        }
    }
}

}  // namespace
}  // namespace argus

using namespace argus;

struct argus_gwb {
    int device = 0;
    int n_sm = 0;
    int P = 0;
    int64_t N = 0;
    GwbRec* d_rec = nullptr;
    double* d_p0 = nullptr;
    double* d_equad2 = nullptr;
    double* d_G = nullptr;
    double* d_stage = nullptr;
    size_t cap_stage = 0;
    // gradient: per resident block, the segment-start states and one segment's tape
    double* d_ckpt = nullptr;
    double* d_tape = nullptr;
    size_t cap_ckpt = 0;
};

namespace {

int gwb_fail(int st, const std::string& msg) { return record_error(st, msg.c_str()); }

int gwb_cuda(cudaError_t e, const char* what) {
    return record_error(e == cudaErrorMemoryAllocation ? ARGUS_ERR_OOM : ARGUS_ERR_CUDA,
                        (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

// Hellings-Downs matrix: G_nm = 3/2 x ln x - x/4 + 1/2, x = (1 - c_n.c_m)/2; G_nn = 1.
std::vector<double> hellings_downs(const argus_pulsar* psrs, int P) {
    std::vector<double> G(size_t(P) * P);
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            if (a == b) { G[size_t(a) * P + b] = 1.0; continue; }
            double cth = 0.0;
            for (int i = 0; i < 3; ++i) cth += psrs[a].pos[i] * psrs[b].pos[i];
            cth = std::min(1.0, std::max(-1.0, cth));
            const double x = 0.5 * (1.0 - cth);
            G[size_t(a) * P + b] = (x > 0.0 ? 1.5 * x * std::log(x) : 0.0) - 0.25 * x + 0.5;
        }
    return G;
}

bool gwb_is_device_ptr(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

argus_status argus_gwb_create(const argus_pulsar* psrs, int32_t n_pulsars, int32_t device,
                              argus_gwb** out) {
    if (!out) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "out is NULL"));
    if (!psrs || n_pulsars < 1) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "need at least one pulsar"));
    if (n_pulsars > kGwbMaxPulsars)
        return argus_status(gwb_fail(ARGUS_ERR_UNSUPPORTED, "the joint filter holds at most 64 pulsars"));
    if (device < 0) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "device must be >= 0"));
    int64_t total = 0;
    if (int st = validate_pulsars(psrs, n_pulsars, &total)) return argus_status(st);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return argus_status(gwb_cuda(e, "cudaGetDeviceCount"));
    if (device >= ndev) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "no such device"));
    cudaDeviceProp prop{};
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess)
        return argus_status(gwb_cuda(e, "cudaGetDeviceProperties"));
    if (prop.major != 10 || prop.minor != 3)
        return argus_status(gwb_fail(ARGUS_ERR_UNSUPPORTED, std::string("built for sm_103a, device is ") + prop.name));
    // merged TOA stream, time order; ties keep (pulsar, TOA) order
    std::vector<int32_t> psr_of;
    std::vector<int64_t> loc;
    psr_of.reserve(size_t(total));
    loc.reserve(size_t(total));
    for (int p = 0; p < n_pulsars; ++p)
        for (int64_t k = 0; k < psrs[p].n_toa; ++k) { psr_of.push_back(p); loc.push_back(k); }
    std::vector<int64_t> order(static_cast<size_t>(total));
    std::iota(order.begin(), order.end(), int64_t(0));
    auto tof = [&](int64_t g) { return psrs[psr_of[g]].t[loc[g]]; };
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return tof(x) < tof(y); });
    std::vector<GwbRec> rec(size_t(std::max<int64_t>(total, 1)));
    double t_prev = total ? tof(order[0]) : 0.0;
    for (int64_t j = 0; j < total; ++j) {
        const int64_t g = order[j];
        const argus_pulsar& ps = psrs[psr_of[g]];
        const double t = ps.t[loc[g]];
        rec[j] = GwbRec{t - t_prev, ps.r[loc[g]], ps.sigma[loc[g]] * ps.sigma[loc[g]], psr_of[g], 0};
        t_prev = t;
    }
    std::vector<double> p0(size_t(3) * n_pulsars), eq2(n_pulsars);
    for (int p = 0; p < n_pulsars; ++p) {
        for (int i = 0; i < 3; ++i) p0[3 * p + i] = psrs[p].p0[i];
        eq2[p] = psrs[p].equad * psrs[p].equad;
    }
    const std::vector<double> G = hellings_downs(psrs, n_pulsars);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    argus_gwb* h = new argus_gwb();
    h->device = device;
    h->n_sm = prop.multiProcessorCount;
    h->P = n_pulsars;
    h->N = total;
    auto bail = [&](cudaError_t err, const char* what) {
        argus_gwb_destroy(h);
        if (prev >= 0) cudaSetDevice(prev);
        return argus_status(gwb_cuda(err, what));
    };
    if ((e = cudaMalloc(&h->d_rec, sizeof(GwbRec) * rec.size())) != cudaSuccess) return bail(e, "cudaMalloc(records)");
    if ((e = cudaMalloc(&h->d_p0, sizeof(double) * p0.size())) != cudaSuccess) return bail(e, "cudaMalloc(p0)");
    if ((e = cudaMalloc(&h->d_equad2, sizeof(double) * eq2.size())) != cudaSuccess) return bail(e, "cudaMalloc(equad)");
    if ((e = cudaMalloc(&h->d_G, sizeof(double) * G.size())) != cudaSuccess) return bail(e, "cudaMalloc(G)");
    if ((e = cudaMemcpy(h->d_rec, rec.data(), sizeof(GwbRec) * rec.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_p0, p0.data(), sizeof(double) * p0.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_equad2, eq2.data(), sizeof(double) * eq2.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_G, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "cudaMemcpy");
    // the kernel's dynamic shared memory limit, set for the largest array any
    // handle may hold (a per-function setting shared by all handles)
    if ((e = cudaFuncSetAttribute(k_gwb_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(gwb_smem_bytes(kGwbMaxPulsars, false)))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_gwb_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(gwb_smem_bytes(kGwbGradMaxPulsars, true)))) != cudaSuccess ||
        // all of the unified L1 as shared memory: blocks per SM are set by shared memory
        (e = cudaFuncSetAttribute(k_gwb_filter, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  int(cudaSharedmemCarveoutMaxShared))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_gwb_grad, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  int(cudaSharedmemCarveoutMaxShared))) != cudaSuccess)
        return bail(e, "cudaFuncSetAttribute");
    if (prev >= 0) cudaSetDevice(prev);
    *out = h;
    return ARGUS_OK;
}

void argus_gwb_destroy(argus_gwb* h) {
    if (!h) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->d_rec);
    cudaFree(h->d_p0);
    cudaFree(h->d_equad2);
    cudaFree(h->d_G);
    cudaFree(h->d_stage);
    cudaFree(h->d_ckpt);
    cudaFree(h->d_tape);
    if (prev >= 0) cudaSetDevice(prev);
    delete h;
}

int32_t argus_gwb_dim(const argus_gwb* h) { return h ? 2 + 3 * h->P : -1; }

argus_status argus_gwb_loglik(argus_gwb* h, const double* theta, int64_t B, double* loglik,
                              void* stream) {
    if (!h) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "handle is NULL"));
    if (B < 0) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "B must be >= 0"));
    if (B == 0) return ARGUS_OK;
    if (!theta || !loglik) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "theta or loglik is NULL"));
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int D = 2 + 3 * h->P;
    const bool dev_in = gwb_is_device_ptr(theta), dev_out = gwb_is_device_ptr(loglik);
    const double* th_d = theta;
    double* ll_d = loglik;
    cudaError_t e = cudaSuccess;
    argus_status st = ARGUS_OK;
    if (!dev_in || !dev_out) {
        const size_t need = size_t(B) * (D + 1);
        if (need > h->cap_stage) {
            cudaFree(h->d_stage);
            h->d_stage = nullptr;
            h->cap_stage = 0;
            if ((e = cudaMalloc(&h->d_stage, need * sizeof(double))) != cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMalloc(stage)"));
                goto done;
            }
            h->cap_stage = need;
        }
        if (!dev_in) {
            if ((e = cudaMemcpyAsync(h->d_stage, theta, sizeof(double) * B * D, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMemcpyAsync(theta)"));
                goto done;
            }
            th_d = h->d_stage;
        }
        if (!dev_out) ll_d = h->d_stage + size_t(B) * D;
    }
    {
        GwbArgs a{};
        a.rec = h->d_rec; a.N = h->N; a.P = h->P; a.p0 = h->d_p0; a.equad2 = h->d_equad2; a.G = h->d_G;
        a.theta = th_d; a.B = B; a.loglik = ll_d;
        const size_t smem = gwb_smem_bytes(h->P, false);
        const int grid = int(std::min<int64_t>(B, int64_t(h->n_sm) * 8));
        k_gwb_filter<<<grid, kGwbFwdThreads, smem, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "k_gwb_filter"));
            goto done;
        }
        if (!dev_out) {
            if ((e = cudaMemcpyAsync(loglik, ll_d, sizeof(double) * B, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMemcpyAsync(loglik)"));
                goto done;
            }
        }
        if (!dev_in || !dev_out) {
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) st = argus_status(gwb_cuda(e, "cudaStreamSynchronize"));
        }
    }
done:
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

argus_status argus_gwb_loglik_grad(argus_gwb* h, const double* theta, int64_t B, double* loglik,
                                   double* grad, void* stream) {
    if (!h) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "handle is NULL"));
    if (B < 0) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "B must be >= 0"));
    if (B == 0) return ARGUS_OK;
    if (!theta || !loglik || !grad)
        return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "theta, loglik or grad is NULL"));
    if (h->P > kGwbGradMaxPulsars)
        return argus_status(gwb_fail(ARGUS_ERR_UNSUPPORTED, "the joint filter's gradient holds at most 48 pulsars"));
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int D = 2 + 3 * h->P;
    const bool dev_in = gwb_is_device_ptr(theta), dev_ll = gwb_is_device_ptr(loglik),
               dev_g = gwb_is_device_ptr(grad);
    const double* th_d = theta;
    double *ll_d = loglik, *g_d = grad;
    cudaError_t e = cudaSuccess;
    argus_status st = ARGUS_OK;
    const size_t smem = gwb_smem_bytes(h->P, true);
    int per_sm = 1;
    const int L = std::max(1, int(std::ceil(std::sqrt(double(std::max<int64_t>(h->N, 1))))));
    const int nseg = int((h->N + L - 1) / L);
    const size_t slot = size_t(std::max(nseg, L)) * size_t(gwb_rec_len(h->P));
    int grid = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gwb_grad, kGwbThreads, smem)) != cudaSuccess) {
        st = argus_status(gwb_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor"));
        goto done;
    }
    grid = int(std::min<int64_t>(B, int64_t(h->n_sm) * std::max(per_sm, 1)));
    if (slot * grid > h->cap_ckpt) {
        cudaFree(h->d_ckpt);
        cudaFree(h->d_tape);
        h->d_ckpt = h->d_tape = nullptr;
        h->cap_ckpt = 0;
        if ((e = cudaMalloc(&h->d_ckpt, slot * grid * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&h->d_tape, slot * grid * sizeof(double))) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "cudaMalloc(gradient scratch)"));
            goto done;
        }
        h->cap_ckpt = slot * grid;
    }
    if (!dev_in || !dev_ll || !dev_g) {
        const size_t need = size_t(B) * (2 * D + 1);
        if (need > h->cap_stage) {
            cudaFree(h->d_stage);
            h->d_stage = nullptr;
            h->cap_stage = 0;
            if ((e = cudaMalloc(&h->d_stage, need * sizeof(double))) != cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMalloc(stage)"));
                goto done;
            }
            h->cap_stage = need;
        }
        if (!dev_in) {
            if ((e = cudaMemcpyAsync(h->d_stage, theta, sizeof(double) * B * D, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMemcpyAsync(theta)"));
                goto done;
            }
            th_d = h->d_stage;
        }
        if (!dev_ll) ll_d = h->d_stage + size_t(B) * D;
        if (!dev_g) g_d = h->d_stage + size_t(B) * (D + 1);
    }
    {
        GwbArgs a{};
        a.rec = h->d_rec; a.N = h->N; a.P = h->P; a.p0 = h->d_p0; a.equad2 = h->d_equad2; a.G = h->d_G;
        a.theta = th_d; a.B = B; a.loglik = ll_d; a.grad = g_d;
        a.ckpt = h->d_ckpt; a.tape = h->d_tape; a.slot = int64_t(slot); a.L = L; a.nseg = nseg;
        k_gwb_grad<<<grid, kGwbThreads, smem, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "k_gwb_grad"));
            goto done;
        }
        if (!dev_ll &&
            (e = cudaMemcpyAsync(loglik, ll_d, sizeof(double) * B, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "cudaMemcpyAsync(loglik)"));
            goto done;
        }
        if (!dev_g &&
            (e = cudaMemcpyAsync(grad, g_d, sizeof(double) * B * D, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "cudaMemcpyAsync(grad)"));
            goto done;
        }
        if (!dev_in || !dev_ll || !dev_g) {
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) st = argus_status(gwb_cuda(e, "cudaStreamSynchronize"));
        }
    }
done:
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
