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
//
// Gradient (two kernels).  The likelihood kernel, with one warp per vector,
// also saves the state every L = ceil(sqrt N) TOAs ("checkpoints") and flags
// a vector whose scales had to be folded.  The reverse kernel then takes one
// vector per block of 64 threads (more for large arrays): segment by segment,
// last first, it re-runs the segment from its checkpoint and writes each
// step's "tape entry" to global memory -- the state before the step and the
// step's transition coefficients with their gamma-derivatives -- and then
// runs the adjoint steps backwards, each reading its entry into one of two
// shared-memory buffers by cp.async while the step before it computes.  A
// flagged vector runs the whole gradient unscaled instead.
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
constexpr int kGwbFwdThreads = 32;    // likelihood kernel: one warp per block
constexpr int kGwbRevMaxThreads = 256;   // reverse kernel: 64, 128 or 256 threads per block
constexpr int kGwbGradMaxPulsars = 48;   // gradient: the adjoint and a tape entry in shared memory
constexpr int kCo = 9;                   // per-pulsar coefficients (see GwbSmem::co)
constexpr int kDotChunks = 2;            // lanes per dot product in the adjoint's parameter sums

struct GwbRec {     // one TOA of the merged, time-ordered stream (56 bytes)
    double dt;      // time since the previous TOA of any pulsar (0 for the first)
    double r;       // residual, s
    double s2;      // sigma_k^2
    double h2;      // dt^2 / 2
    double h3;      // dt^3 / 3
    double dt2;     // dt^2
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
    double* grad;           // [B][2 + 3P] (reverse kernel)
    double* ckpt;           // per vector: [nseg][rec_len] state at each segment start, or NULL
    int32_t* flags;         // per vector: 1 if the likelihood pass folded its scales (with ckpt)
    double* tape;           // per reverse block: [L][tape_len] tape entries of one segment
    int64_t ck_slot;        // doubles per vector in ckpt
    int64_t tape_slot;      // doubles per block in tape
    int32_t L;              // segment length (TOAs)
    int32_t nseg;
    int32_t nbuf;           // tape-entry buffers in the reverse kernel's shared memory (1 or 2)
};

// Shared memory of a block.  The covariance P and, for the gradient, its
// adjoint Pb are symmetric and stored as packed upper triangles (see pk).
// The state and the step's coefficients sit in one contiguous "entry" in the
// order of a tape entry: Pm, m, sg, co, gc, cs.
struct GwbSmem {
    int P, n, nb, ne;
    double* Pm;     // packed upper triangle, n (n + 1) / 2
    double* m;      // [n]
    double* sg;     // [P + 1]: scale factors s_p and s_a (scaled frame)
    double* co;     // [P][9]: a, b, Q/sigma^2 (c00, c01, c11), d/dgamma of b and of c00, c01, c11
    double* gc;     // [9]: the same for the GW process (per unit h_a^2)
    double* cs;     // [P + 1][5], scaled frame, per pulsar and for the GW process (row P):
                    // b s, v c00, v c01 / s', v c11 / s'^2, 1 / s' (v = sigma_p^2 or h_a^2, s' = s a)
    double* c;      // [n]
    double* ct;     // [n]: c / S
    double* sg0;    // [P + 1]: the scale factors before the current predict
    const double* G;   // [P][P] Hellings-Downs, in global memory (read through the read-only cache)
    double* par;    // [P][4]: sigma^2, gamma_p, EFAC^2, EFAC
    double* gw;     // scalar slots (enum below)
    // reverse kernel only
    double* E1;     // second tape-entry buffer (== Pm's entry when there is one buffer)
    double* Pb;     // packed upper triangle: adjoint of Ph
    double* mb;     // [n]: adjoint of mh
    double* v;      // [n]
    double* acc;    // [P][5]: d/d sigma^2, d/d gamma_p, d/d EFAC, d/d h_a^2 part, d/d gamma_a part
    double* sgb;    // [P]: adjoints of the scales s_p
    double* sbt;    // [P]: this step's adjoint of s'_p from the intrinsic noise
    double* n1;     // [P]: this step's intrinsic-noise term of d/d gamma_p (before the factor sigma_p^2)
    double* dd;     // [2P]: this step's Fh-bar dot products, (rho_I, y_I) then (rho_I, a_I)
    double* td;     // [3P]: the diagonal blocks' Hellings-Downs contraction terms
    double* red;    // [2 x warps]: block reductions
    double* u;      // [n]      (unscaled fallback)
    double* part;   // [P][chunks][6]: partial sums of the parameter terms (unscaled fallback)
    uint16_t* pairs;
};
// scalar slots of gw[]
// (kGwK..kGwK+10: the GW share update's per-step products, reverse kernel)
enum { kGwHa2 = 0, kGwGa, kGwE, kGwS, kGwRS, kGwG, kGwOk, kGwSb, kGwEb, kGwR0, kGwRn, kGwRnAny,
       kGwK = 16, kGwSlots = 32 };
constexpr double kGwbTiny = 0x1p-200;   // smallest scale factor kept (scaled frame)

// chunks per pulsar of the unscaled adjoint's parameter sums (J ranges of about 5)
__host__ __device__ inline int gwb_jchunks(int P) { return (P + 4) / 5 < 8 ? (P + 4) / 5 : 8; }
// doubles of one saved state (a checkpoint): the upper triangle of P, m and the P + 1 scales
__host__ __device__ inline int64_t gwb_rec_len(int P) {
    const int64_t n = 3 * int64_t(P);
    return n * (n + 1) / 2 + n + P + 1;
}
// doubles of one tape entry: a saved state, then co, gc and cs, then the
// step's predicted column c = M e_i (3P), 1/S and e/S; even, so that entries
// start on 16-byte boundaries
__host__ __device__ inline int64_t gwb_tape_c_off(int P) {
    return gwb_rec_len(P) + kCo * int64_t(P) + 9 + 5 * (int64_t(P) + 1);
}
__host__ __device__ inline int64_t gwb_tape_len(int P) {
    const int64_t d = gwb_tape_c_off(P) + 3 * int64_t(P) + 2;
    return (d + 1) & ~int64_t(1);
}

// dynamic shared memory of the likelihood kernel: one entry, c, ct, sg0,
// par, the scalar slots and the (I, J) pairs of the upper 3x3 blocks (uint16)
__host__ __device__ inline size_t gwb_fwd_smem_bytes(int P) {
    const size_t n = 3 * size_t(P);
    const size_t d = size_t(gwb_tape_len(P)) + 2 * n + (size_t(P) + 1) + 4 * size_t(P) + kGwSlots;
    return d * sizeof(double) + size_t(P) * (P + 1) * sizeof(uint16_t);
}

// doubles of the reverse kernel's arrays after the entry buffers
__host__ __device__ inline size_t gwb_rev_tail_doubles(int P, int threads) {
    const size_t n = 3 * size_t(P), ne = n * (n + 1) / 2;
    return ne + 4 * n + (size_t(P) + 1) + 4 * size_t(P) + kGwSlots + 5 * size_t(P) + 8 * size_t(P) +
           2 * size_t(threads / 32);
}
// the unscaled fallback's u and part: in the second entry buffer when there is one
__host__ __device__ inline size_t gwb_rev_fallback_doubles(int P) {
    return 3 * size_t(P) + 6 * size_t(P) * gwb_jchunks(P);
}
__host__ __device__ inline size_t gwb_rev_smem_bytes(int P, int nbuf, int threads) {
    size_t d = size_t(nbuf) * size_t(gwb_tape_len(P)) + gwb_rev_tail_doubles(P, threads);
    if (nbuf == 1) d += gwb_rev_fallback_doubles(P);
    return d * sizeof(double) + size_t(P) * (P + 1) * sizeof(uint16_t);
}

// pointers of an entry at e
__device__ __forceinline__ void gwb_entry_ptrs(GwbSmem& s, double* e) {
    const int P = s.P;
    s.Pm = e;
    s.m = e + s.ne;
    s.sg = s.m + s.n;
    s.co = s.sg + P + 1;
    s.gc = s.co + kCo * P;
    s.cs = s.gc + 9;
}

__device__ GwbSmem gwb_carve_fwd(double* base, int P, const double* G) {
    GwbSmem s{};
    s.P = P; s.n = 3 * P; s.nb = P * (P + 1) / 2; s.ne = s.n * (s.n + 1) / 2;
    gwb_entry_ptrs(s, base);
    double* q = base + gwb_tape_len(P);
    s.c = q; q += s.n;
    s.ct = q; q += s.n;
    s.sg0 = q; q += P + 1;
    s.par = q; q += 4 * P;
    s.gw = q; q += kGwSlots;
    s.G = G;
    s.E1 = base;
    s.pairs = reinterpret_cast<uint16_t*>(q);
    return s;
}

__device__ GwbSmem gwb_carve_rev(double* base, int P, int nbuf, const double* G) {
    GwbSmem s{};
    s.P = P; s.n = 3 * P; s.nb = P * (P + 1) / 2; s.ne = s.n * (s.n + 1) / 2;
    const int64_t tl = gwb_tape_len(P);
    const int n = s.n;
    gwb_entry_ptrs(s, base);
    s.E1 = base + (nbuf == 2 ? tl : 0);
    double* q = base + nbuf * tl;
    s.Pb = q; q += s.ne;
    s.mb = q; q += n;
    s.c = q; q += n;
    s.ct = q; q += n;
    s.v = q; q += n;
    s.sg0 = q; q += P + 1;
    s.par = q; q += 4 * P;
    s.gw = q; q += kGwSlots;
    s.acc = q; q += 5 * P;
    s.sgb = q; q += P;
    s.sbt = q; q += P;
    s.n1 = q; q += P;
    s.dd = q; q += 2 * P;
    s.td = q; q += 3 * P;
    s.red = q; q += 2 * (blockDim.x / 32);
    if (nbuf == 2) {
        s.u = s.E1;
        s.part = s.E1 + n;
    } else {
        s.u = q; q += n;
        s.part = q; q += 6 * P * gwb_jchunks(P);
    }
    s.G = G;
    s.pairs = reinterpret_cast<uint16_t*>(q);
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

// the (I, J) pairs of the upper 3x3 blocks, once per block: the diagonal
// blocks first, then I < J row by row
__device__ void gwb_tables(const GwbSmem& s) {
    if (threadIdx.x == 0) {
        int k = 0;
        for (int I = 0; I < s.P; ++I) { s.pairs[2 * k] = uint16_t(I); s.pairs[2 * k + 1] = uint16_t(I); ++k; }
        for (int I = 0; I < s.P; ++I)
            for (int J = I + 1; J < s.P; ++J) { s.pairs[2 * k] = uint16_t(I); s.pairs[2 * k + 1] = uint16_t(J); ++k; }
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
    for (int r = threadIdx.x; r < n; r += blockDim.x) {   // one packed row per thread
        const int I = r / 3, uu = r - 3 * I;
        double* row = prow(s.Pm, n, r);
        for (int col = r; col < n; ++col) {
            const int J = col / 3, vv = col - 3 * J;
            double x = 0.0;
            if (uu == 2 && vv == 2) x = ha2 * gwb_G(s, I, J) / (2.0 * ga);
            else if (I == J && uu < 2 && vv < 2) x = a.p0[3 * I + uu + vv];
            row[col] = x;
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) s.m[i] = 0.0;
    __syncthreads();
    return true;
}

// 1. transition coefficients over dt (threads 0..P-1 the pulsars, thread P the GW process)
template <bool kDeriv>
__device__ void gwb_coef(const GwbSmem& s, const GwbRec& rk) {
    const double dt = rk.dt, h2 = rk.h2, h3 = rk.h3, dt2 = rk.dt2;
    for (int p = threadIdx.x; p <= s.P; p += blockDim.x) {
        OuCoef oc;
        const double gam = (p < s.P) ? s.par[4 * p + 1] : s.gw[kGwGa];
        ou_coef_warp<kDeriv>(gam * dt, dt, h2, h3, dt2, oc);
        double* o = (p < s.P) ? s.co + kCo * p : s.gc;
        o[0] = oc.a; o[1] = oc.b; o[2] = oc.c00; o[3] = oc.c01; o[4] = oc.c11;
        if (kDeriv) { o[5] = oc.db; o[6] = oc.dc00; o[7] = oc.dc01; o[8] = oc.dc11; }
    }
}

// 2. predict: the mean and every upper 3x3 block, F_I P_IJ F_J^T + Q_IJ
__device__ void gwb_predict(const GwbSmem& s) {
    const int P = s.P, n = s.n;
    const double* gc = s.gc;
    const double aa = gc[0], ba = gc[1], ha2 = s.gw[kGwHa2];
    const double qa00 = ha2 * gc[2], qa01 = ha2 * gc[3], qa11 = ha2 * gc[4];
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
// advance to s' = s a, and a scale below kGwbTiny raises the flag.  tape_sg,
// if given, receives the scales before the step (each by the thread that
// advances it).
template <bool kDeriv, bool kAdvance>
__device__ void gwb_coef_scaled(const GwbSmem& s, const GwbRec& rk, double* tape_sg = nullptr) {
    const double dt = rk.dt, h2 = rk.h2, h3 = rk.h3, dt2 = rk.dt2;
    for (int p = threadIdx.x; p <= s.P; p += blockDim.x) {
        OuCoef oc;
        const bool psr = p < s.P;
        ou_coef_warp<kDeriv>((psr ? s.par[4 * p + 1] : s.gw[kGwGa]) * dt, dt, h2, h3, dt2, oc);
        const double sg = s.sg[p], sn = sg * oc.a;
        if (tape_sg) tape_sg[p] = sg;
        if (kAdvance) {
            s.sg0[p] = sg;
            s.sg[p] = sn;
            if (!(sn >= kGwbTiny)) s.gw[kGwRn] = 1.0;
        }
        const double w = rcp_nr3(sn), sc = psr ? s.par[4 * p] : s.gw[kGwHa2];
        double* o = psr ? s.co + kCo * p : s.gc;
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
    for (int r = threadIdx.x; r < n; r += blockDim.x) {   // one packed row per thread
        const double sr = gwb_scale_of(sc, P, r);
        double* row = prow(s.Pm, n, r);
        for (int col = r; col < n; ++col) row[col] *= sr * gwb_scale_of(sc, P, col);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) s.m[i] *= gwb_scale_of(sc, P, i);
}

// 2'' the scaled predict, or (a scale fell below kGwbTiny: block-uniform and
// rare) unscale and predict unscaled
__device__ void gwb_predict_scaled_or_fold(const GwbSmem& s) {
    if (s.gw[kGwRn] != 0.0) {
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
}

// first item of a role whose item x runs on thread (o + x) mod T: single-warp
// roles start on different warps, so that the four sub-partitions' FP64
// pipes share the serial work of a step
__device__ __forceinline__ int gwb_role_first(int o) {
    const int T = blockDim.x;
    return (int(threadIdx.x) + T - o % T) % T;
}

// 3. innovate on rho of pulsar q: c = P e_i and c / S (the threads that form
// c each form 1/S; in blocks of 128 threads or more the second half, while
// the first computes the coefficients); item 0 records e, S, 1/S, e/S
__device__ void gwb_innovate(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk) {
    const int n = s.n, i0 = 3 * rk.q, T = blockDim.x;
    int i = gwb_role_first(T >= 128 ? T / 2 : 0);
    if (i < n) {
        const double R = fma(s.par[4 * rk.q + 2], rk.s2, a.equad2[rk.q]);
        const double S = s.Pm[pk(n, i0, i0)] + R;
        const double rS = rcp_nr3(S);
        for (; i < n; i += T) {
            const double ci = psym(s.Pm, n, i, i0);
            s.c[i] = ci;
            s.ct[i] = ci * rS;
            if (i == 0) {
                const double e = rk.r - s.m[i0];
                s.gw[kGwE] = e;
                s.gw[kGwS] = S;
                s.gw[kGwRS] = rS;
                s.gw[kGwG] = e * rS;
            }
        }
    }
}

// 4. update (upper triangle, P_ij -= c_i (c_j / S)) and mean.  Thread t takes
// packed entries t, t + T, ...; the row r and the offset in the row follow
// the index along.  Four entries at a time, their loads ahead of their
// stores, so that the FMAs do not wait on each other.
__device__ __forceinline__ void gwb_advance(int n, int T, int& r, int& off) {
    off += T;
    while (r < n && off >= n - r) { off -= n - r; ++r; }
}
__device__ void gwb_update(const GwbSmem& s) {
    const int n = s.n, T = blockDim.x, ne = s.ne;
    const double g = s.gw[kGwG];
    int r = 0, off = threadIdx.x;
    while (r < n && off >= n - r) { off -= n - r; ++r; }
    int q = threadIdx.x;
    for (; q + 3 * T < ne; q += 4 * T) {
        double x[4], ci[4], cj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[u] = s.Pm[q + u * T];
            ci[u] = s.c[r];
            cj[u] = s.ct[r + off];
            gwb_advance(n, T, r, off);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s.Pm[q + u * T] = fma(-ci[u], cj[u], x[u]);
    }
    for (; q < ne; q += T) {
        s.Pm[q] = fma(-s.c[r], s.ct[r + off], s.Pm[q]);
        gwb_advance(n, T, r, off);
    }
    for (int i = threadIdx.x; i < n; i += T) s.m[i] = fma(s.c[i], g, s.m[i]);
}

// one forward step; thread 0 accumulates the likelihood when kLL; kScaled
// keeps Ph, mh in the scaled frame
template <bool kLL, bool kScaled = false>
__device__ void gwb_step(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk, double& quad, LogProd& lp) {
    if (rk.dt > 0.0) {
        if (kScaled) {
            gwb_coef_scaled<false, true>(s, rk);
            __syncthreads();
            gwb_predict_scaled_or_fold(s);
        } else {
            gwb_coef<false>(s, rk);
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

// state (upper triangle of P, m, scales) to a global slot; each scale is
// written by the thread that advances it in the next step
__device__ void gwb_save(const GwbSmem& s, double* dst) {
    for (int q = threadIdx.x; q < s.ne + s.n; q += blockDim.x) dst[q] = s.Pm[q];
    for (int p = threadIdx.x; p <= s.P; p += blockDim.x) dst[s.ne + s.n + p] = s.sg[p];
}

// Likelihood; with a.ckpt also the state at every segment start (the
// checkpoints of the gradient) and the fold flag of each vector.
__global__ void __launch_bounds__(kGwbFwdThreads) k_gwb_filter(GwbArgs a) {
    extern __shared__ __align__(16) double gsm[];
    const GwbSmem s = gwb_carve_fwd(gsm, a.P, a.G);
    const int64_t rec_len = gwb_rec_len(a.P);
    gwb_tables(s);
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        __syncthreads();
        if (!gwb_setup(s, a, a.theta + b * (2 + 3 * a.P))) {
            if (threadIdx.x == 0) {
                a.loglik[b] = -INFINITY;
                if (a.flags) a.flags[b] = 0;
            }
            continue;
        }
        double quad = 0.0;
        LogProd lp;
        if (a.ckpt) {
            double* ck = a.ckpt + b * a.ck_slot;
            for (int seg = 0; seg < a.nseg; ++seg) {
                gwb_save(s, ck + seg * rec_len);
                const int64_t k1 = min(int64_t(seg + 1) * a.L, a.N);
                for (int64_t k = int64_t(seg) * a.L; k < k1; ++k) gwb_step<true, true>(s, a, a.rec[k], quad, lp);
            }
        } else {
            for (int64_t k = 0; k < a.N; ++k) gwb_step<true, true>(s, a, a.rec[k], quad, lp);
        }
        if (threadIdx.x == 0) {
            a.loglik[b] = gwb_finish(a.N, quad, lp);
            if (a.flags) a.flags[b] = s.gw[kGwRnAny] != 0.0 ? 1 : 0;
        }
    }
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
        const double rS = rcp_nr3(S);
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

// Reverse of one forward step k in the unscaled frame (the fallback for a
// vector whose scales fold), the state before it in Pm, m.  On entry Pb, mb
// hold the adjoints of the state after the step; on exit, before it.
__device__ void gwb_step_adjoint(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk) {
    const int P = s.P, n = s.n, q = rk.q, i0 = 3 * q;
    const int tid = threadIdx.x;
    const double dt = rk.dt;
    const bool pred = dt > 0.0;
    double* gw = s.gw;
    const double* gc = s.gc;
    if (pred) {
        gwb_coef<true>(s, rk);
        __syncthreads();
    }
    // u = P (F^T e_i), and mu_i = (F m)_i
    const double bq = pred ? s.co[kCo * q + 1] : 0.0, ba = pred ? gc[1] : 0.0;
    for (int j = tid; j < n; j += blockDim.x)
        s.u[j] = fma(bq, psym(s.Pm, n, j, i0 + 1), fma(ba, psym(s.Pm, n, j, i0 + 2), psym(s.Pm, n, j, i0)));
    __syncthreads();
    // c = F u + Q e_i (the predicted covariance's column i)
    const double ha2 = gw[kGwHa2];
    for (int J = tid; J < P; J += blockDim.x) {
        const double* uJ = s.u + 3 * J;
        if (pred) {
            const double aJ = s.co[kCo * J], bJ = s.co[kCo * J + 1], aa = gc[0];
            const double g = gwb_G(s, J, q) * ha2;
            double c0 = fma(bJ, uJ[1], fma(ba, uJ[2], uJ[0])) + g * gc[2];
            double c1 = aJ * uJ[1];
            const double c2 = fma(aa, uJ[2], g * gc[3]);
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
    const double aa = gc[0], dba = gc[5], dca00 = gc[6], dca01 = gc[7], dca11 = gc[8];
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
            h = fma(g, fma(X00, gc[2], fma(X02 + X20, gc[3], X22 * gc[4])), h);
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

// ---------------------------------------------------------------------------
// Reverse kernel: tape entries, the scaled adjoint step, the kernel
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(double* dst_smem, const double* src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// all threads: start copying one tape entry (tl doubles, 16-byte aligned) to
// shared memory; cp_async_wait_all and a barrier make it visible
__device__ __forceinline__ void gwb_fetch_entry(double* dst, const double* src, int64_t tl) {
    for (int64_t i = threadIdx.x; i < tl / 2; i += blockDim.x) cp_async16(dst + 2 * i, src + 2 * i);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The transition coefficients, with their gamma-derivatives, of steps
// k0..k1-1 (scaled frame) straight into their tape entries' co and gc fields
// (tape entry k - k0).  They depend on gamma and dt only, not on the state,
// so the whole segment's are formed at once: one (step, pulsar) pair per
// thread (pulsar P: the GW process), all lanes busy.  The lanes of a warp
// share the longest series any of them needs (ou_coef_warp); a longer
// series is never less accurate, so these may differ from the likelihood
// pass's by rounding only.
__device__ void gwb_segment_coefs(const GwbSmem& s, const GwbArgs& a, int64_t k0, int64_t k1, double* tp,
                                  int64_t tl) {
    const int P = s.P, np = P + 1;
    const int64_t off = gwb_rec_len(P);        // co's offset in an entry; gc follows co
    const int64_t items = (k1 - k0) * np;
    for (int64_t it = threadIdx.x; it < items; it += blockDim.x) {
        const int64_t j = it / np;
        const int p = int(it - j * np);
        const GwbRec& rk = a.rec[k0 + j];
        if (!(rk.dt > 0.0)) continue;
        OuCoef oc;
        ou_coef_warp<true>((p < P ? s.par[4 * p + 1] : s.gw[kGwGa]) * rk.dt, rk.dt, rk.h2, rk.h3, rk.dt2, oc);
        double* o = tp + j * tl + off + kCo * p;
        o[0] = oc.a; o[1] = oc.b; o[2] = oc.c00; o[3] = oc.c01; o[4] = oc.c11;
        o[5] = oc.db; o[6] = oc.dc00; o[7] = oc.dc01; o[8] = oc.dc11;
    }
}

// One forward step in the scaled frame that also writes its tape entry to
// slot: the state before the step (Ph, mh, scales), the scale-dependent
// coefficients cs (co and gc are already there, gwb_segment_coefs), the
// predicted column c, 1/S and e/S.  Thread p forms cs_p and advances s_p
// from co_p as gwb_coef_scaled does, and keeps a, b and Q / sigma^2 in
// shared memory for a fold's unscaled predict.
__device__ void gwb_tape_step_scaled(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk, double* slot) {
    const int ne = s.ne, n = s.n, P = s.P, T = blockDim.x;
    double* tsg = slot + ne + n;
    const double* tco = tsg + P + 1;
    double* tcs = tsg + P + 1 + kCo * P + 9;
    const bool pred = rk.dt > 0.0;
    double oa = 0.0, ob = 0.0, q00 = 0.0, q01 = 0.0, q11 = 0.0;
    if (pred && int(threadIdx.x) <= P) {        // loads first, under the state's stores
        const double* o = tco + kCo * threadIdx.x;
        oa = o[0]; ob = o[1]; q00 = o[2]; q01 = o[3]; q11 = o[4];
    }
    for (int i = threadIdx.x; i < ne + n; i += T) slot[i] = s.Pm[i];
    if (pred) {
        for (int p = threadIdx.x; p <= P; p += T) {
            if (p != int(threadIdx.x)) {
                const double* o = tco + kCo * p;
                oa = o[0]; ob = o[1]; q00 = o[2]; q01 = o[3]; q11 = o[4];
            }
            const double sg = s.sg[p], sn = sg * oa;
            tsg[p] = sg;
            s.sg0[p] = sg;
            s.sg[p] = sn;
            if (!(sn >= kGwbTiny)) s.gw[kGwRn] = 1.0;
            const double w = rcp_nr3(sn), sc = p < P ? s.par[4 * p] : s.gw[kGwHa2];
            double* h = s.cs + 5 * p;
            h[0] = ob * sg;
            h[1] = sc * q00;
            h[2] = sc * q01 * w;
            h[3] = sc * q11 * w * w;
            h[4] = w;
            double* th = tcs + 5 * p;
            th[0] = h[0]; th[1] = h[1]; th[2] = h[2]; th[3] = h[3]; th[4] = h[4];
            double* o = p < P ? s.co + kCo * p : s.gc;
            o[0] = oa; o[1] = ob; o[2] = q00; o[3] = q01; o[4] = q11;
        }
        __syncthreads();
        gwb_predict_scaled_or_fold(s);
        __syncthreads();
    } else {
        for (int p = threadIdx.x; p <= P; p += T) tsg[p] = s.sg[p];
    }
    gwb_innovate(s, a, rk);
    __syncthreads();
    double* tc = slot + gwb_tape_c_off(P);
    for (int i = threadIdx.x; i < n; i += T) tc[i] = s.c[i];
    if (threadIdx.x == 0) {
        tc[n] = s.gw[kGwRS];
        tc[n + 1] = s.gw[kGwG];
    }
    gwb_update(s);
    __syncthreads();
}

// The same in the unscaled frame (the fallback): the entry holds the state
// only; its adjoint forms the coefficients itself.
__device__ void gwb_tape_step_unscaled(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk, double* slot) {
    for (int i = threadIdx.x; i < s.ne + s.n; i += blockDim.x) slot[i] = s.Pm[i];
    if (rk.dt > 0.0) {
        gwb_coef<false>(s, rk);
        __syncthreads();
        gwb_predict(s);
        __syncthreads();
    }
    gwb_innovate(s, a, rk);
    __syncthreads();
    gwb_update(s);
    __syncthreads();
}

// This thread's shares of the GW scale's adjoint and of the two GW
// parameters' sums.  Every term is linear in the per-block contractions, so
// each thread carries its own part through the steps and the parts are added
// once per vector, in a fixed order.
struct GwShare {
    double sg, a3, a4;
};

// The per-pulsar end of scaled adjoint step rk whose Fh-bar dot products are
// in dd, on thread I's share: d/d gamma_p through b_p s_p and the adjoint of
// the scale s_p, and pulsar I's part of the adjoint of b_a s_a (into the GW
// shares).  E: that step's tape entry.
__device__ __forceinline__ void gwb_finish_pulsar(const GwbSmem& s, const double* E, double dt, int I,
                                                  GwShare& sh) {
    const int P = s.P, rI = 3 * I;
    const double* mh = E + s.ne;
    const double* sg = mh + s.n;
    const double* co = sg + P + 1;
    const double* gc = co + kCo * P;
    const double* coI = co + kCo * I;
    const double mbr = s.mb[rI];
    const double bhb = fma(2.0, s.dd[I], mbr * mh[rI + 1]);         // adjoint of b_I s_I
    const double sbt = s.sbt[I];
    s.acc[5 * I + 1] += fma(s.par[4 * I], s.n1[I], sg[I] * fma(bhb, coI[5], -dt * coI[0] * sbt));
    s.sgb[I] = fma(sbt, coI[0], bhb * coI[1]);
    const double alb = fma(2.0, s.dd[P + I], mbr * mh[rI + 2]);     // pulsar I's part of that of b_a s_a
    sh.a4 = fma(sg[P] * gc[5], alb, sh.a4);
    sh.sg = fma(gc[1], alb, sh.sg);
}

// Reverse of forward step rk in the scaled frame.  E holds its tape entry:
// the state before the step (Ph, mh, the scales s) and the step's
// coefficients.  On entry Pb, mb and sgb hold the adjoints of Ph, mh and s_p
// after the step (sh those of s_a); on exit, before it.  With M-bar the
// adjoint of the predicted Ph and mu-bar that of the predicted mh:
//   Fh-bar = 2 M-bar Fh Ph + mu-bar mh^T, of which b s (rho_I, y_I) and
//   b_a s_a (rho_I, a_I, every I) are parameters;
//   the process noise v c / s'^k (k = 0, 1, 2) passes its adjoint to v, c and
//   s' = s a; s' passes its adjoint to s and a;
//   Ph-bar = Fh^T M-bar Fh, mh-bar = Fh^T mu-bar.
// Row rho_I of Fh^T M-bar Fh equals that of M-bar Fh, so the two Fh-bar
// entries of pulsar I are dot products of that row of the new Pb with columns
// y_I and a_I of Ph.  nxt_src: a tape entry to fetch into nxt_dst meanwhile
// (NULL: none).  Eprev: the entry of the step reversed before this one, whose
// per-pulsar ends (gwb_finish_pulsar) run here, during the second phase, on
// the threads of the role that starts at thread 32 (NULL: none pending).
// The forward step left c, 1/S and e/S in the entry.  Four phases and
// barriers; on return the fetch has landed, Pb is complete and this step's
// per-pulsar ends are pending.
__device__ void gwb_adjoint_scaled(const GwbSmem& s, const GwbArgs& a, const GwbRec& rk, const double* E,
                                   double* nxt_dst, const double* nxt_src, const double* Eprev, double dt_prev,
                                   int64_t tl, GwShare& sh) {
    const int P = s.P, n = s.n, q = rk.q, i0 = 3 * q;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const double* Ph = E;
    const double* mh = E + s.ne;
    const double* sg = mh + n;
    const double* co = sg + P + 1;
    const double* gc = co + kCo * P;
    const double* cs = gc + 9;
    const double* ca = cs + 5 * P;
    const double dt = rk.dt;
    const bool pred = dt > 0.0;
    double* gw = s.gw;
    const double al = pred ? ca[0] : 0.0;
    // the predicted column c = M e_i (i = rho_q), 1/S and e/S, from the forward step
    const double* c = E + gwb_tape_c_off(P);
    const double rS = c[n], g = c[n + 1];
    __syncthreads();
    // the previous step's per-pulsar ends (its Fh-bar dot products were
    // written after its last barrier)
    if (Eprev)
        for (int I = gwb_role_first(32); I < P; I += T) gwb_finish_pulsar(s, Eprev, dt_prev, I, sh);
    // 2. v = Pb c, a row per thread (two threads per row when the block has
    //    twice as many threads as rows)
    const int parts = T >= 2 * n ? 2 : 1, half = (n + 1) / 2;
    for (int base = 0; base < parts * n; base += T) {
        const int it = base + tid, j = it / parts, h = it - j * parts;
        const bool valid = it < parts * n;
        double a0 = 0.0, a1 = 0.0;
        if (valid) {
            const int klo = parts == 2 && h ? half : 0, khi = parts == 2 && !h ? half : n;
            // row j of Pb along k (see the dot products below)
            int k = klo;
            int ib = k < j ? pk(n, k, j) : pk(n, j, k);
            auto step = [&](int kk, int& idx) { idx = kk + 1 < j ? idx + n - kk - 1 : kk + 1 == j ? pk(n, j, j) : idx + 1; };
            for (; k + 1 < khi; k += 2) {
                const double b0 = s.Pb[ib];
                step(k, ib);
                const double b1 = s.Pb[ib];
                step(k + 1, ib);
                a0 = fma(b0, c[k], a0);
                a1 = fma(b1, c[k + 1], a1);
            }
            if (k < khi) a0 = fma(s.Pb[ib], c[k], a0);
        }
        double acc = a0 + a1;
        if (parts == 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (valid && h == 0) s.v[j] = acc;
    }
    __syncthreads();
    // the previous step's entry is no longer read: fetch the next one into its buffer
    if (nxt_src) gwb_fetch_entry(nxt_dst, nxt_src, tl);
    // 3. M-bar: c-bar and S-bar into row and column i of Pb; mu-bar = mb - e-bar e_i.
    //    The warp of the thread that takes row i forms mb.c (lanes 0-15) and
    //    c.v (lanes 16-31), each half summing its 16 lanes in a fixed tree.
    double gb = 0.0, cv = 0.0;
    if (warp == (i0 % T) / 32) {
        const bool hv = lane >= 16;
        const double* x = hv ? c : s.mb;
        const double* y = hv ? s.v : c;
        double d = 0.0;
        for (int k = lane & 15; k < n; k += 16) d = fma(x[k], y[k], d);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        gb = __shfl_sync(0xffffffffu, d, 0);
        cv = __shfl_sync(0xffffffffu, d, 16);
    }
    for (int j = tid; j < n; j += T) {
        const double cb = fma(s.mb[j], g, -2.0 * rS * s.v[j]);
        if (j == i0) {     // S-bar and e-bar
            const double Sb = rS * rS * cv - gb * g * rS - 0.5 * rS + 0.5 * g * g;
            const double eb = gb * rS - g;
            s.acc[5 * q + 2] += Sb * 2.0 * s.par[4 * q + 3] * rk.s2;     // d/d EFAC_q
            s.Pb[pk(n, j, j)] += cb + Sb;
            s.mb[j] -= eb;
        } else {   // the one stored entry of the symmetric pair (j, i), (i, j)
            double& e = s.Pb[j < i0 ? pk(n, j, i0) : pk(n, i0, j)];
            e = fma(0.5, cb, e);
        }
    }
    if (!pred) {   // Fh = I, Q = 0, scales unchanged: the adjoints pass through
        cp_async_wait_all();
        __syncthreads();
        return;
    }
    __syncthreads();
    if (tid >= T - 10) {   // the GW share update's products for this step, one per lane:
        // K_i = ((f0 f1) f2) f3, the factors picked per lane, the products on all ten at once
        //   K0 = wa ca2, K1 = 2 wa ca3, K2 = gc2, K3 = wa gc3, K4 = wa wa gc4, K5 = ha2 gc6,
        //   K6 = ha2 wa gc7, K7 = ha2 wa wa gc8, K8 = sga (-dt) gc0, K9 = gc0
        const int i = tid - (T - 10);
        const double wa = ca[4];
        double f0 = wa, f1 = 1.0, f2 = 1.0, f3 = 1.0;
        switch (i) {
            case 0: f1 = ca[2]; break;
            case 1: f0 = 2.0; f1 = wa; f2 = ca[3]; break;
            case 2: f0 = gc[2]; break;
            case 3: f1 = gc[3]; break;
            case 4: f1 = wa; f2 = gc[4]; break;
            case 5: f0 = gw[kGwHa2]; f1 = gc[6]; break;
            case 6: f0 = gw[kGwHa2]; f1 = wa; f2 = gc[7]; break;
            case 7: f0 = gw[kGwHa2]; f1 = wa; f2 = wa; f3 = gc[8]; break;
            case 8: f0 = sg[P]; f1 = -dt; f2 = gc[0]; break;
            default: f0 = gc[0]; break;
        }
        gw[kGwK + i] = ((f0 * f1) * f2) * f3;
    }
    // 4. Pb <- Fh^T M-bar Fh, block by block, with this thread's parts of the
    //    Hellings-Downs contractions of M-bar: sum_IJ G_IJ times its (rho_I,
    //    rho_J), (rho_I, a_J) + (a_I, rho_J) and (a_I, a_J) entries
    // The off-diagonal blocks on the first 64 threads (all, in smaller
    // blocks): they, the first P threads and the per-pulsar ends' threads
    // carry the GW shares
    const int Tc = T >= 128 ? 64 : T;
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
    for (int it = tid < Tc ? tid : s.nb; it < s.nb - P; it += Tc) {   // blocks I < J
        const int I = s.pairs[2 * (P + it)], J = s.pairs[2 * (P + it) + 1];
        const double bI = cs[5 * I], bJ = cs[5 * J];
        double* R[3];
        double X[3][3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            R[u] = prow(s.Pb, n, 3 * I + u) + 3 * J;
#pragma unroll
            for (int v = 0; v < 3; ++v) X[u][v] = R[u][v];
        }
        const double g2 = 2.0 * gwb_G(s, I, J);           // the (J, I) block's terms too
        t1 = fma(g2, X[0][0], t1);
        t2 = fma(g2, X[0][2] + X[2][0], t2);
        t3 = fma(g2, X[2][2], t3);
#pragma unroll
        for (int v = 0; v < 3; ++v) {   // Fh_I^T X: rows y, a gain b_I s_I, b_a s_a times row rho
            X[1][v] = fma(bI, X[0][v], X[1][v]);
            X[2][v] = fma(al, X[0][v], X[2][v]);
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {   // (Fh_I^T X) Fh_J
            R[u][0] = X[u][0];
            R[u][1] = fma(bJ, X[u][0], X[u][1]);
            R[u][2] = fma(al, X[u][0], X[u][2]);
        }
    }
    // diagonal blocks: on the third warp of larger blocks (the first two take
    // the off-diagonal ones); their contraction terms go to thread I's share
    for (int I = gwb_role_first(T >= 128 ? 64 : 32); I < P; I += T) {
        const int rI = 3 * I;
        const double bI = cs[5 * I];
        double* R0 = prow(s.Pb, n, rI) + rI;
        double* R1 = prow(s.Pb, n, rI + 1) + rI;
        double* R2 = prow(s.Pb, n, rI + 2) + rI;
        const double x00 = R0[0], x01 = R0[1], x02 = R0[2], x11 = R1[1], x12 = R1[2], x22 = R2[2];
        const double g = gwb_G(s, I, I);
        s.td[3 * I] = g * x00;
        s.td[3 * I + 1] = g * (x02 + x02);
        s.td[3 * I + 2] = g * x22;
        // intrinsic noise sigma^2 c00, sigma^2 c01 / s', sigma^2 c11 / s'^2 and the scale s'_I
        const double* cI = cs + 5 * I;
        const double* coI = co + kCo * I;
        const double w = cI[4], q1b = 2.0 * x01;
        s.sbt[I] = s.sgb[I] - w * fma(q1b, cI[2], 2.0 * x11 * cI[3]);
        s.acc[5 * I] += fma(x00, coI[2], w * fma(q1b, coI[3], w * x11 * coI[4]));
        s.n1[I] = fma(x00, coI[6], w * fma(q1b, coI[7], w * x11 * coI[8]));
        double X[3][3] = {{x00, x01, x02}, {x01, x11, x12}, {x02, x12, x22}};
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            X[1][v] = fma(bI, X[0][v], X[1][v]);
            X[2][v] = fma(al, X[0][v], X[2][v]);
        }
        R0[0] = X[0][0];
        R0[1] = fma(bI, X[0][0], X[0][1]);
        R0[2] = fma(al, X[0][0], X[0][2]);
        R1[1] = fma(bI, X[1][0], X[1][1]);
        R1[2] = fma(al, X[1][0], X[1][2]);
        R2[2] = fma(al, X[2][0], X[2][2]);
        double* mI = s.mb + rI;                             // mu-bar <- Fh^T mu-bar
        mI[1] = fma(bI, mI[0], mI[1]);
        mI[2] = fma(al, mI[0], mI[2]);
    }
    cp_async_wait_all();
    __syncthreads();
    // 5. the adjoints of b_I s_I and of b_a s_a: 2 (M-bar Fh Ph) at (rho_I, y_I)
    //    and (rho_I, a_I) plus the mean's terms; kDotChunks lanes per dot product
    const int items = 2 * kDotChunks * P, clen = (n + kDotChunks - 1) / kDotChunks;
    for (int base = 0; base < items; base += T) {
        if (base + (tid & ~31) >= items) break;             // warp-uniform
        const int it = base + tid;
        const bool valid = it < items;
        const int dp = it / kDotChunks, ch = it % kDotChunks;
        const int I = dp >> 1, kind = dp & 1, rI = 3 * I;
        double d = 0.0, d1 = 0.0;
        if (valid) {
            // row rho_I of Pb and column col of Ph along k: packed (k, x) for
            // k < x steps by n - k - 1, then (x, k) by one
            const int col = rI + 1 + kind, k1 = min(n, (ch + 1) * clen);
            int k = ch * clen;
            int ib = k < rI ? pk(n, k, rI) : pk(n, rI, k);
            int ih = k < col ? pk(n, k, col) : pk(n, col, k);
            auto step = [&](int kk, int x, int& idx) { idx = kk + 1 < x ? idx + n - kk - 1 : kk + 1 == x ? pk(n, x, x) : idx + 1; };
            for (; k + 1 < k1; k += 2) {
                const double b0 = s.Pb[ib], h0 = Ph[ih];
                step(k, rI, ib); step(k, col, ih);
                const double b1 = s.Pb[ib], h1 = Ph[ih];
                step(k + 1, rI, ib); step(k + 1, col, ih);
                d = fma(b0, h0, d);
                d1 = fma(b1, h1, d1);
            }
            if (k < k1) d = fma(s.Pb[ib], Ph[ih], d);
        }
        d += d1;
        static_assert(kDotChunks == 1 || kDotChunks == 2 || kDotChunks == 4, "lane groups within a warp");
#pragma unroll
        for (int o = 1; o < kDotChunks; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (valid && ch == 0) s.dd[kind * P + I] = d;
    }
    for (int I = tid; I < P; I += T) {   // the diagonal blocks' contraction terms
        t1 += s.td[3 * I];
        t2 += s.td[3 * I + 1];
        t3 += s.td[3 * I + 2];
    }
    // GW: h_a^2 c / s'^k and the scale s'_a = s_a a_a, on this thread's parts
    // (the pulsars' parts of b_a s_a's adjoint follow in gwb_finish_pulsar)
    if (tid < min(T, max(Tc, 32 + P))) {   // the threads that hold shares
        const double* K = gw + kGwK;
        const double sbat = sh.sg - fma(t2, K[0], t3 * K[1]);
        sh.a3 = fma(t1, K[2], fma(t2, K[3], fma(t3, K[4], sh.a3)));
        sh.a4 = fma(t1, K[5], fma(t2, K[6], fma(t3, K[7], fma(sbat, K[8], sh.a4))));
        sh.sg = sbat * K[9];
    }
}

// Gradient: one vector per block.  The likelihood kernel has written
// loglik, the checkpoints and the fold flags of this launch's vectors.
// kMaxT threads at most per block, kMinB blocks per SM: <128, 4> keeps the
// registers to 128 per thread, so that shared memory alone limits the
// blocks per SM (4 blocks of 128 threads up to 20 pulsars); <256, 1> gives
// large arrays, one block per SM, 8 warps.
template <int kMaxT, int kMinB>
__global__ void __launch_bounds__(kMaxT, kMinB) k_gwb_reverse(GwbArgs a) {
    extern __shared__ __align__(16) double gsm[];
    GwbSmem s = gwb_carve_rev(gsm, a.P, a.nbuf, a.G);
    const int P = s.P, n = s.n, ne = s.ne, D = 2 + 3 * P;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int64_t rec_len = gwb_rec_len(P), tl = gwb_tape_len(P);
    double* tp = a.tape + int64_t(blockIdx.x) * a.tape_slot;
    double* const Ebuf[2] = {s.Pm, s.E1};
    gwb_tables(s);
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        double* gout = a.grad + b * D;
        double* ck = a.ckpt + b * a.ck_slot;
        const double* th = a.theta + b * D;
        __syncthreads();
        if (!gwb_setup(s, a, th) || !isfinite(a.loglik[b]) || a.N == 0) {
            for (int j = tid; j < D; j += T) gout[j] = 0.0;
            continue;
        }
        bool scaled = a.flags[b] == 0;
        GwShare sh{0.0, 0.0, 0.0};
        for (;;) {   // the scaled frame, then (rarely) the unscaled one
            for (int i = tid; i < ne; i += T) s.Pb[i] = 0.0;
            for (int i = tid; i < n; i += T) s.mb[i] = 0.0;
            for (int i = tid; i < 5 * P; i += T) s.acc[i] = 0.0;
            for (int i = tid; i < P; i += T) s.sgb[i] = 0.0;
            sh = GwShare{0.0, 0.0, 0.0};
            if (!scaled) {   // the checkpoints again, unscaled
                __syncthreads();
                gwb_setup(s, a, th);
                double quad = 0.0;
                LogProd lp;
                for (int seg = 0; seg < a.nseg; ++seg) {
                    gwb_save(s, ck + seg * rec_len);
                    const int64_t k1 = min(int64_t(seg + 1) * a.L, a.N);
                    for (int64_t k = int64_t(seg) * a.L; k < k1; ++k) gwb_step<false>(s, a, a.rec[k], quad, lp);
                }
            }
            bool refold = false;
            for (int seg = a.nseg - 1; seg >= 0; --seg) {
                const int64_t k0 = int64_t(seg) * a.L, k1 = min(k0 + a.L, a.N);
                __syncthreads();
                for (int64_t i = tid; i < rec_len; i += T) s.Pm[i] = ck[seg * rec_len + i];
                if (tid == 0) s.gw[kGwRnAny] = 0.0;
                if (scaled) gwb_segment_coefs(s, a, k0, k1, tp, tl);
                __syncthreads();
                // re-run the segment, writing its tape
                for (int64_t k = k0; k < k1; ++k) {
                    if (scaled) gwb_tape_step_scaled(s, a, a.rec[k], tp + (k - k0) * tl);
                    else gwb_tape_step_unscaled(s, a, a.rec[k], tp + (k - k0) * tl);
                }
                if (scaled && s.gw[kGwRnAny] != 0.0) {   // a fold the likelihood pass did not flag
                    refold = true;
                    break;
                }
                // the adjoint steps, last first
                if (scaled) {
                    gwb_fetch_entry(Ebuf[(k1 - 1) & 1], tp + (k1 - 1 - k0) * tl, tl);
                    cp_async_wait_all();
                    __syncthreads();
                    for (int64_t k = k1 - 1; k >= k0; --k) {
                        const bool ahead = a.nbuf == 2 && k > k0;
                        const bool pend = a.nbuf == 2 && k < k1 - 1 && a.rec[k + 1].dt > 0.0;
                        gwb_adjoint_scaled(s, a, a.rec[k], Ebuf[k & 1], ahead ? Ebuf[(k - 1) & 1] : nullptr,
                                           ahead ? tp + (k - 1 - k0) * tl : nullptr,
                                           pend ? Ebuf[(k + 1) & 1] : nullptr, pend ? a.rec[k + 1].dt : 0.0, tl, sh);
                        if (a.nbuf == 1 || k == k0) {   // no buffer keeps this entry for the next step
                            __syncthreads();
                            if (a.rec[k].dt > 0.0)
                                for (int I = gwb_role_first(32); I < P; I += T)
                                    gwb_finish_pulsar(s, Ebuf[k & 1], a.rec[k].dt, I, sh);
                            if (a.nbuf == 1 && k > k0) {
                                __syncthreads();
                                gwb_fetch_entry(s.Pm, tp + (k - 1 - k0) * tl, tl);
                                cp_async_wait_all();
                                __syncthreads();
                            }
                        }
                    }
                } else {
                    for (int64_t k = k1 - 1; k >= k0; --k) {
                        __syncthreads();
                        for (int64_t i = tid; i < ne + n; i += T) s.Pm[i] = tp[(k - k0) * tl + i];
                        __syncthreads();
                        gwb_step_adjoint(s, a, a.rec[k]);
                    }
                }
            }
            if (!refold) break;
            scaled = false;
        }
        __syncthreads();
        // the stationary prior of the a block: h_a^2 G / (2 gamma_a)
        const double ha2 = s.gw[kGwHa2], ga = s.gw[kGwGa];
        for (int I = tid; I < P; I += T) {
            double h = 0.0;
            for (int J = 0; J < P; ++J) h = fma(psym(s.Pb, n, 3 * I + 2, 3 * J + 2), gwb_G(s, I, J), h);
            s.acc[5 * I + 3] += h / (2.0 * ga);
            s.acc[5 * I + 4] -= h * ha2 / (2.0 * ga * ga);
        }
        const double a3 = warp_sum(sh.a3), a4 = warp_sum(sh.a4);
        if (lane == 0) {
            s.red[2 * warp] = a3;
            s.red[2 * warp + 1] = a4;
        }
        __syncthreads();
        if (tid == 0) {
            double hb = 0.0, gb = 0.0;
            for (int I = 0; I < P; ++I) { hb += s.acc[5 * I + 3]; gb += s.acc[5 * I + 4]; }
            for (int w = 0; w < T / 32; ++w) { hb += s.red[2 * w]; gb += s.red[2 * w + 1]; }
            gout[0] = hb * 2.0 * kLn10Gwb * ha2;
            gout[1] = gb * kLn10Gwb * ga;
        }
        for (int p = tid; p < P; p += T) {
            gout[2 + 3 * p] = s.acc[5 * p] * 2.0 * kLn10Gwb * s.par[4 * p];
            gout[3 + 3 * p] = s.acc[5 * p + 1] * kLn10Gwb * s.par[4 * p + 1];
            gout[4 + 3 * p] = s.acc[5 * p + 2];
        }
    }
}

using GwbRevKernel = void (*)(GwbArgs);
struct GwbRevCand {
    GwbRevKernel k;
    int max_threads;
};
const GwbRevCand kGwbRevCands[] = {{k_gwb_reverse<128, 4>, 128}, {k_gwb_reverse<256, 1>, 256}};

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
    // gradient: per vector of a launch the segment-start states and the fold
    // flag; per resident reverse block one segment's tape
    double* d_ckpt = nullptr;
    int32_t* d_flags = nullptr;
    double* d_tape = nullptr;
    size_t cap_ckpt = 0, cap_flags = 0, cap_tape = 0;
    // reverse kernel's configuration (rev_threads 0: not chosen yet)
    GwbRevKernel rev_kernel = nullptr;
    int rev_threads = 0, rev_nbuf = 0, rev_per_sm = 0;
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
        const double dt = t - t_prev;
        rec[j] = GwbRec{dt, ps.r[loc[g]], ps.sigma[loc[g]] * ps.sigma[loc[g]], 0.5 * dt * dt, dt * dt * dt / 3.0,
                        dt * dt, psr_of[g], 0};
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
    // the kernels' dynamic shared memory limits, set for the largest array any
    // handle may hold (a per-function setting shared by all handles), and all
    // of the unified L1 as shared memory: blocks per SM are set by shared memory
    if ((e = cudaFuncSetAttribute(k_gwb_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(gwb_fwd_smem_bytes(kGwbMaxPulsars)))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_gwb_filter, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  int(cudaSharedmemCarveoutMaxShared))) != cudaSuccess)
        return bail(e, "cudaFuncSetAttribute");
    for (const GwbRevCand& c : kGwbRevCands) {
        const size_t most = std::min<size_t>(size_t(prop.sharedMemPerBlockOptin),
                                             gwb_rev_smem_bytes(kGwbGradMaxPulsars, 1, kGwbRevMaxThreads));
        if ((e = cudaFuncSetAttribute(c.k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(most))) != cudaSuccess ||
            (e = cudaFuncSetAttribute(c.k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      int(cudaSharedmemCarveoutMaxShared))) != cudaSuccess)
            return bail(e, "cudaFuncSetAttribute");
    }
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
    cudaFree(h->d_flags);
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
        const size_t smem = gwb_fwd_smem_bytes(h->P);
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
    const int P = h->P, D = 2 + 3 * P;
    const bool dev_in = gwb_is_device_ptr(theta), dev_ll = gwb_is_device_ptr(loglik),
               dev_g = gwb_is_device_ptr(grad);
    const double* th_d = theta;
    double *ll_d = loglik, *g_d = grad;
    cudaError_t e = cudaSuccess;
    argus_status st = ARGUS_OK;
    const int L = std::max(1, int(std::ceil(std::sqrt(double(std::max<int64_t>(h->N, 1))))));
    const int nseg = int((h->N + L - 1) / L);
    const int64_t rec_len = gwb_rec_len(P), tl = gwb_tape_len(P);
    const int64_t ck_slot = std::max<int64_t>(1, int64_t(nseg) * rec_len);
    const int64_t tape_slot = int64_t(L) * tl;
    int64_t chunk = 0, resident = 0;
    // reverse kernel: the most resident warps per SM; then two tape-entry
    // buffers over one, then fewer threads per block
    if (h->rev_threads == 0) {
        int best_w = 0;
        for (int nbuf = 2; nbuf >= 1; --nbuf)
            for (const GwbRevCand& c : kGwbRevCands)
                for (int t = 64; t <= c.max_threads; t *= 2) {
                    int per_sm = 0;
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c.k, t, gwb_rev_smem_bytes(P, nbuf, t)) !=
                        cudaSuccess) {
                        cudaGetLastError();
                        per_sm = 0;
                    }
                    if (per_sm * t / 32 > best_w) {
                        best_w = per_sm * t / 32;
                        h->rev_kernel = c.k;
                        h->rev_threads = t;
                        h->rev_nbuf = nbuf;
                        h->rev_per_sm = per_sm;
                    }
                }
        if (best_w == 0) {
            st = argus_status(gwb_fail(ARGUS_ERR_UNSUPPORTED, "the gradient kernel does not fit on this device"));
            goto done;
        }
    }
    // vectors per launch pair: every resident reverse block busy, checkpoints
    // within kGwbCkptBudget bytes where that allows more
    {
        constexpr int64_t kGwbCkptBudget = int64_t(4) << 30;
        resident = int64_t(h->n_sm) * h->rev_per_sm;
        const int64_t by_mem = kGwbCkptBudget / (ck_slot * int64_t(sizeof(double)));
        chunk = std::min<int64_t>(B, std::max<int64_t>(resident, by_mem - by_mem % resident));
    }
    if (size_t(chunk * ck_slot) > h->cap_ckpt) {
        cudaFree(h->d_ckpt);
        h->d_ckpt = nullptr;
        h->cap_ckpt = 0;
        if ((e = cudaMalloc(&h->d_ckpt, size_t(chunk * ck_slot) * sizeof(double))) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "cudaMalloc(gradient checkpoints)"));
            goto done;
        }
        h->cap_ckpt = size_t(chunk * ck_slot);
    }
    if (size_t(chunk) > h->cap_flags) {
        cudaFree(h->d_flags);
        h->d_flags = nullptr;
        h->cap_flags = 0;
        if ((e = cudaMalloc(&h->d_flags, size_t(chunk) * sizeof(int32_t))) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "cudaMalloc(gradient flags)"));
            goto done;
        }
        h->cap_flags = size_t(chunk);
    }
    {
        const size_t need = size_t(std::min(chunk, resident) * tape_slot);
        if (need > h->cap_tape) {
            cudaFree(h->d_tape);
            h->d_tape = nullptr;
            h->cap_tape = 0;
            if ((e = cudaMalloc(&h->d_tape, need * sizeof(double))) != cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMalloc(gradient tape)"));
                goto done;
            }
            h->cap_tape = need;
        }
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
    for (int64_t c0 = 0; c0 < B; c0 += chunk) {
        const int64_t bc = std::min(chunk, B - c0);
        GwbArgs a{};
        a.rec = h->d_rec; a.N = h->N; a.P = P; a.p0 = h->d_p0; a.equad2 = h->d_equad2; a.G = h->d_G;
        a.theta = th_d + c0 * D; a.B = bc; a.loglik = ll_d + c0; a.grad = g_d + c0 * D;
        a.ckpt = h->d_ckpt; a.flags = h->d_flags; a.tape = h->d_tape;
        a.ck_slot = ck_slot; a.tape_slot = tape_slot; a.L = L; a.nseg = nseg; a.nbuf = h->rev_nbuf;
        // the likelihood, the checkpoints and the fold flags; then the reverse sweep
        k_gwb_filter<<<int(std::min<int64_t>(bc, int64_t(h->n_sm) * 8)), kGwbFwdThreads, gwb_fwd_smem_bytes(P), s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "k_gwb_filter"));
            goto done;
        }
        h->rev_kernel<<<int(std::min(bc, resident)), h->rev_threads,
                        gwb_rev_smem_bytes(P, h->rev_nbuf, h->rev_threads), s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "k_gwb_reverse"));
            goto done;
        }
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
done:
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
