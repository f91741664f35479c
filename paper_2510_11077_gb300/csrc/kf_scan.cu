// Time-parallel Kalman-filter log-likelihood (associative scan), for the
// few-lane regime: one (walker, pulsar) lane's TOAs spread over many warps and
// SMs instead of one thread stepping through them in turn.
//
// Each TOA k defines an element (A, b, C, eta, J) of the parallel Bayesian
// filter of Sarkka & Garcia-Fernandez (2021, "Temporal parallelization of
// Bayesian smoothers"): given the previous state x_{k-1},
//   p(x_k | x_{k-1}, y_k) = N(x_k; A x_{k-1} + b, C),
//   p(y_k | x_{k-1}) oc N_info(x_{k-1}; eta, J).
// With y_k = r_k - s(t_k), predicted mean F x_{k-1}, covariance Q, H = (1, 0),
// S = Q00 + R, K = Q H^T / S:  A = (I - K H) F, b = K y_k, C = (I - K H) Q,
// eta = F^T H^T y_k / S, J = F^T H^T H F / S.  The first TOA's element holds
// the prior's update (A = 0).  The operator
//   (i) x (j):  M = I + C_i J_j,
//     A = A_j M^-1 A_i,  b = A_j M^-1 (b_i + C_i eta_j) + b_j,
//     C = A_j M^-1 C_i A_j^T + C_j,
//     eta = A_i^T M^-T (eta_j - J_j b_i) + eta_i,  J = A_i^T M^-T J_j A_i + J_i
// is associative, and the prefix of elements 0..k has b = filtered mean,
// C = filtered covariance at TOA k.
//
// Three passes, no block ever waits on another:
//   S1  one block of 4 warps per chunk of 32 E TOAs: warp 0's threads
//       combine their E elements in order, then the 4 warps scan the 32
//       partial products, each level's combines split by field group;
//   S2  one such block per lane: exclusive scan of the lane's chunk
//       aggregates (an empty lane's ll is set to 0 here);
//   S3  one warp per chunk: each thread's exact filtered state at the TOA
//       before its own (chunk prefix x thread prefix), then the ordinary
//       Kalman step of the sequential filter over its E TOAs, accumulating
//       e^2/S and ln S; warp sums per chunk.  The block that completes its
//       lane last (a per-lane counter) sums the lane's chunks in fixed
//       order -> ll;
//   S4  only when every lane is empty: their lls, 0.
// Work is O(N) per lane and depth O(E + log N).
#include <cmath>
#include <cstdint>

#include "kf_internal.cuh"
#include "kf_math.cuh"
#include "kf_model.cuh"
#include "kf_scan_grad.cuh"

namespace argus {

__global__ void k_fill_phase_table(double* tab) {
    fill_phase_table(PhaseTable{reinterpret_cast<longlong2*>(tab),
                                reinterpret_cast<float4*>(tab + 2 * kPhaseTable)});
}

void launch_fill_phase_table(double* tab, cudaStream_t s) { k_fill_phase_table<<<1, 256, 0, s>>>(tab); }

namespace {

constexpr double kLog2PiScan = 1.8378770664093454836;

struct SElem {
    double A00, A01, A10, A11, b0, b1, C00, C01, C11, e0, e1, J00, J01, J11;
};

__device__ __forceinline__ SElem scan_identity() {
    return SElem{1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
}

// The combine (i) x (j), restricted to one group of the output's fields:
// part 0 A, b; part 1 C; part 2 eta; part 3 J (field order of SElem: A00 A01
// A10 A11 b0 b1 C00 C01 C11 e0 e1 J00 J01 J11).  Every part forms the shared
// M^-1; scan_combine runs all four, so a split combine is bit for bit the
// whole one.
__host__ __device__ constexpr int part_begin(int p) { return p == 0 ? 0 : p == 1 ? 6 : p == 2 ? 9 : p == 3 ? 11 : 14; }

template <int kPart>
__device__ __forceinline__ void scan_combine_part(const SElem& i, const SElem& j, double* o) {
    // M = I + C_i J_j and X = M^-1
    const double M00 = 1.0 + fma(i.C00, j.J00, i.C01 * j.J01);
    const double M01 = fma(i.C00, j.J01, i.C01 * j.J11);
    const double M10 = fma(i.C01, j.J00, i.C11 * j.J01);
    const double M11 = 1.0 + fma(i.C01, j.J01, i.C11 * j.J11);
    // C_i, J_j are positive semi-definite, so det(I + C_i J_j) >= 1
    const double rdet = rcp_nr3(fma(M00, M11, -M01 * M10));
    const double X00 = M11 * rdet, X01 = -M01 * rdet, X10 = -M10 * rdet, X11 = M00 * rdet;
    if (kPart <= 1) {
        // G = A_j X
        const double G00 = fma(j.A00, X00, j.A01 * X10), G01 = fma(j.A00, X01, j.A01 * X11);
        const double G10 = fma(j.A10, X00, j.A11 * X10), G11 = fma(j.A10, X01, j.A11 * X11);
        if (kPart == 0) {
            o[0] = fma(G00, i.A00, G01 * i.A10);
            o[1] = fma(G00, i.A01, G01 * i.A11);
            o[2] = fma(G10, i.A00, G11 * i.A10);
            o[3] = fma(G10, i.A01, G11 * i.A11);
            const double u0 = i.b0 + fma(i.C00, j.e0, i.C01 * j.e1);
            const double u1 = i.b1 + fma(i.C01, j.e0, i.C11 * j.e1);
            o[4] = fma(G00, u0, fma(G01, u1, j.b0));
            o[5] = fma(G10, u0, fma(G11, u1, j.b1));
        } else {
            // C = (G C_i) A_j^T + C_j
            const double H00 = fma(G00, i.C00, G01 * i.C01), H01 = fma(G00, i.C01, G01 * i.C11);
            const double H10 = fma(G10, i.C00, G11 * i.C01), H11 = fma(G10, i.C01, G11 * i.C11);
            o[6] = fma(H00, j.A00, fma(H01, j.A01, j.C00));
            o[7] = fma(H00, j.A10, fma(H01, j.A11, j.C01));
            o[8] = fma(H10, j.A10, fma(H11, j.A11, j.C11));
        }
    } else {
        // Z = X A_i, so A_i^T M^-T = Z^T
        const double Z00 = fma(X00, i.A00, X01 * i.A10), Z01 = fma(X00, i.A01, X01 * i.A11);
        const double Z10 = fma(X10, i.A00, X11 * i.A10), Z11 = fma(X10, i.A01, X11 * i.A11);
        if (kPart == 2) {
            const double v0 = j.e0 - fma(j.J00, i.b0, j.J01 * i.b1);
            const double v1 = j.e1 - fma(j.J01, i.b0, j.J11 * i.b1);
            o[9] = fma(Z00, v0, fma(Z10, v1, i.e0));
            o[10] = fma(Z01, v0, fma(Z11, v1, i.e1));
        } else {
            // J = Z^T (J_j A_i) + J_i
            const double W00 = fma(j.J00, i.A00, j.J01 * i.A10), W01 = fma(j.J00, i.A01, j.J01 * i.A11);
            const double W10 = fma(j.J01, i.A00, j.J11 * i.A10), W11 = fma(j.J01, i.A01, j.J11 * i.A11);
            o[11] = fma(Z00, W00, fma(Z10, W10, i.J00));
            o[12] = fma(Z00, W01, fma(Z10, W11, i.J01));
            o[13] = fma(Z01, W01, fma(Z11, W11, i.J11));
        }
    }
}

__device__ __forceinline__ SElem scan_combine(const SElem& i, const SElem& j) {
    SElem o;
    double* p = &o.A00;
    scan_combine_part<0>(i, j, p);
    scan_combine_part<1>(i, j, p);
    scan_combine_part<2>(i, j, p);
    scan_combine_part<3>(i, j, p);
    return o;
}

__device__ __forceinline__ void store_elem(double* dst, const SElem& x) {
    const double* s = &x.A00;
#pragma unroll
    for (int q = 0; q < kScanElem; ++q) dst[q] = s[q];
}

__device__ __forceinline__ SElem load_elem(const double* src) {
    SElem x;
    double* d = &x.A00;
#pragma unroll
    for (int q = 0; q < kScanElem; ++q) d[q] = src[q];
    return x;
}

// The element of TOA k (record rec) of one lane.
template <bool kOU>
__device__ __forceinline__ SElem scan_element(int k, const double* __restrict__ rec, const Lane& L,
                                              PhaseTable tab, const PulsarDev& ps) {
    const double t = rec[0], dt = rec[1], h2 = rec[2], h3 = rec[3], r = rec[4], s2k = rec[5];
    double sn, cs;
    phase_sincos(fma(L.f, t, L.phc), tab, sn, cs);
    const double y = r - fma(L.A, sn, L.B * cs);
    const double R = fma(L.efac2, s2k, L.equad2);
    SElem E;
    if (k == 0) {
        // the prior N(0, P0) at the first TOA, updated by it
        const double p00 = ps.p0[0], p01 = ps.p0[1], p11 = ps.p0[2];
        const double rS = rcp_nr3(p00 + R);
        const double K1 = p01 * rS, w = R * rS;
        E = SElem{0.0, 0.0, 0.0, 0.0, p00 * rS * y, K1 * y, p00 * w, p01 * w, fma(-K1, p01, p11),
                  0.0, 0.0, 0.0, 0.0, 0.0};
    } else {
        double a = 1.0, b = dt, q00 = h3, q01 = h2, q11 = dt;
        if (kOU) {
            OuCoef c;
            ou_coef<false>(L.gam * dt, dt, h2, h3, rec[6], c);
            a = c.a; b = c.b; q00 = c.c00; q01 = c.c01; q11 = c.c11;
        }
        q00 *= L.sig2; q01 *= L.sig2; q11 *= L.sig2;
        const double rS = rcp_nr3(q00 + R);
        const double K1 = q01 * rS, w = R * rS;
        const double yr = y * rS;
        E.A00 = w; E.A01 = w * b; E.A10 = -K1; E.A11 = fma(-K1, b, a);
        E.b0 = q00 * yr; E.b1 = q01 * yr;
        E.C00 = q00 * w; E.C01 = q01 * w; E.C11 = fma(-K1, q01, q11);
        E.e0 = yr; E.e1 = b * yr;
        E.J00 = rS; E.J01 = b * rS; E.J11 = b * b * rS;
    }
    return E;
}

__device__ __forceinline__ Lane scan_lane(const ScanArgs& a, int lane, bool ou, double equad2) {
    const int64_t lanes = a.B * a.P;
    const double* o = a.lc + lane;
    Lane L;
    L.A = o[0 * lanes]; L.B = o[1 * lanes]; L.f = o[2 * lanes]; L.phc = o[3 * lanes];
    L.sig2 = o[4 * lanes]; L.efac2 = o[5 * lanes]; L.equad2 = equad2;
    L.gam = ou ? o[7 * lanes] : 0.0;
    return L;
}

// the handle's sin/cos table in global memory (filled once when the handle is
// built): a one-warp block would spend longer filling a shared copy than
// using it
__device__ __forceinline__ PhaseTable scan_table(const ScanArgs& a) {
    double* t = const_cast<double*>(a.phase_table);   // read only
    PhaseTable tab;
    tab.d = reinterpret_cast<longlong2*>(t);
    tab.f = reinterpret_cast<float4*>(t + 2 * kPhaseTable);
    return tab;
}

// Per-lane completion counters, one 8-byte slot per lane after the chunk
// sums (the handle allocates a.part with n_items * 2 + B P doubles).
__device__ __forceinline__ unsigned long long* lane_done(const ScanArgs& a) {
    return reinterpret_cast<unsigned long long*>(a.part + 2 * int64_t(a.n_items));
}

// ll of a lane from its chunk sums, in chunk order (reads bypass L1: other
// blocks wrote them)
__device__ __forceinline__ void lane_total(const ScanArgs& a, int64_t lane) {
    const int p = int(lane / a.B);
    const int n = a.psr[p].n;
    const int first = a.lane_first[lane], last = a.lane_first[lane + 1];
    double quad = 0.0, logdet = 0.0;
    for (int c = first; c < last; ++c) {
        quad += __ldcg(a.part + 2 * int64_t(c));
        logdet += __ldcg(a.part + 2 * int64_t(c) + 1);
    }
    double ll = (n == 0) ? 0.0 : -0.5 * (double(n) * kLog2PiScan + logdet + quad);
    if (!isfinite(ll)) ll = -INFINITY;
    a.lane_out[lane] = ll;
}

// Inclusive scan of 32 elements by a block's four warps, for a part whose
// FP64 units are split between its sub-partitions: a warp's 32-lane FP64
// instruction runs at a quarter of the SM's rate, so one warp alone spends
// ~95 of them per forward combine.  Here every level's 32 combines are shared
// out by field group (Op::part): in the forward scan warp w forms the common
// M^-1 and its own fields, ~50 FP64 instructions, and the four warps run on
// the four sub-partitions at once.  Element i starts in buf[0][i]; the
// result is in buf[returned index][i].  All kScanThreads threads call it.
// Op: the element (kN doubles, Elem, load), its combine split in four field
// groups (part<0..3>(earlier, later, out)) and the groups' first fields.
constexpr int kScanThreads = 128;

struct FwdScan {
    static constexpr int kN = kScanElem;
    using Elem = SElem;
    static __device__ __forceinline__ Elem load(const double* s) { return load_elem(s); }
    template <int kPart>
    static __device__ __forceinline__ void part(const Elem& i, const Elem& j, double* o) {
        scan_combine_part<kPart>(i, j, o);
    }
    static __host__ __device__ constexpr int begin(int p) { return part_begin(p); }
};

template <class Op>
__device__ __forceinline__ int coop_scan32(double (*buf)[32][Op::kN]) {
    const int lane = threadIdx.x & 31, part = threadIdx.x >> 5;
    int cur = 0;
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
        double* dst = buf[cur ^ 1][lane];
        const double* xs = buf[cur][lane];
        if (lane >= off) {
            const typename Op::Elem y = Op::load(buf[cur][lane - off]);
            const typename Op::Elem x = Op::load(xs);
            switch (part) {
                case 0: Op::template part<0>(y, x, dst); break;
                case 1: Op::template part<1>(y, x, dst); break;
                case 2: Op::template part<2>(y, x, dst); break;
                default: Op::template part<3>(y, x, dst); break;
            }
        } else {
            for (int f = Op::begin(part); f < Op::begin(part + 1); ++f) dst[f] = xs[f];
        }
        __syncthreads();
        cur ^= 1;
    }
    return cur;
}

// S1
template <bool kOU>
__global__ void __launch_bounds__(kScanThreads) k_scan_local(ScanArgs a) {
    __shared__ double buf[2][32][kScanElem];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        const PhaseTable tab = scan_table(a);
        const ScanItem it = a.items[blockIdx.x];
        if (threadIdx.x == 0 && it.k0 == 0) lane_done(a)[it.lane] = 0ull;   // before S3 (a later kernel)
        const int p = int(it.lane / a.B);
        const PulsarDev& ps = a.psr[p];
        const Lane L = scan_lane(a, it.lane, kOU, ps.equad2);
        const int k_lo = it.k0 + lane * a.E;
        const int k_hi = min(k_lo + a.E, ps.n);
        SElem agg = scan_identity();
        if (k_lo < k_hi) agg = scan_element<kOU>(k_lo, a.rec + (ps.off + k_lo) * kRecDoubles, L, tab, ps);
        for (int k = k_lo + 1; k < k_hi; ++k)
            agg = scan_combine(agg, scan_element<kOU>(k, a.rec + (ps.off + k) * kRecDoubles, L, tab, ps));
        store_elem(buf[0][lane], agg);
    }
    __syncthreads();
    const int res = coop_scan32<FwdScan>(buf);
    if (threadIdx.x < 32) {
        const SElem agg = load_elem(buf[res][lane]);
        store_elem(a.tpre + (int64_t(blockIdx.x) * 32 + lane) * kScanElem, agg);
        if (lane == 31) store_elem(a.bagg + int64_t(blockIdx.x) * kScanElem, agg);
    }
}

// S2
__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(ScanArgs a) {
    __shared__ double buf[2][32][kScanElem];
    const int lane = blockIdx.x, t = threadIdx.x & 31;
    const int first = a.lane_first[lane], cnt = a.lane_first[lane + 1] - first;
    if (cnt == 0) {   // the whole block: an empty lane's ll is 0
        if (threadIdx.x == 0) a.lane_out[lane] = 0.0;
        return;
    }
    const int q = (cnt + 31) / 32;
    const int c_lo = t * q, c_hi = min(c_lo + q, cnt);
    if (threadIdx.x < 32) {
        SElem agg = scan_identity();
        if (c_lo < c_hi) agg = load_elem(a.bagg + int64_t(first + c_lo) * kScanElem);
        for (int c = c_lo + 1; c < c_hi; ++c)
            agg = scan_combine(agg, load_elem(a.bagg + int64_t(first + c) * kScanElem));
        store_elem(buf[0][t], agg);
    }
    __syncthreads();
    const int res = coop_scan32<FwdScan>(buf);
    if (threadIdx.x < 32) {
        SElem pre = t == 0 ? scan_identity() : load_elem(buf[res][t - 1]);
        for (int c = c_lo; c < c_hi; ++c) {
            store_elem(a.bpre + int64_t(first + c) * kScanElem, pre);
            if (c + 1 < c_hi)   // the prefix after the thread's last chunk is not needed
                pre = scan_combine(pre, load_elem(a.bagg + int64_t(first + c) * kScanElem));
        }
    }
}

// Filtered state at TOA k_lo - 1 for thread t of a chunk whose TOAs start
// at k_lo > 0: the chunk's prefix x the earlier threads of the chunk (the
// lane's first chunk has no prefix).  Only the b and C fields of that
// combine are formed (parts 0 and 1; A is dead code), bit for bit those of
// the whole combine.
__device__ __forceinline__ State prefix_state(const ScanArgs& a, const ScanItem& it, int t) {
    if (t == 0) {
        const SElem pre = load_elem(a.bpre + int64_t(blockIdx.x) * kScanElem);
        return State{pre.b0, pre.b1, pre.C00, pre.C01, pre.C11};
    }
    const SElem th = load_elem(a.tpre + (int64_t(blockIdx.x) * 32 + t - 1) * kScanElem);
    if (it.k0 == 0) return State{th.b0, th.b1, th.C00, th.C01, th.C11};
    const SElem ch = load_elem(a.bpre + int64_t(blockIdx.x) * kScanElem);
    double o[kScanElem];
    scan_combine_part<0>(ch, th, o);
    scan_combine_part<1>(ch, th, o);
    return State{o[4], o[5], o[6], o[7], o[8]};
}

// The chunk's (sum e^2/S, sum ln S) by warp sums; the block that completes its
// lane last sums the lane's chunks (no block waits: the others just leave).
// Called by the block's first warp, all 32 threads.
__device__ __forceinline__ void finish_chunk_ll(const ScanArgs& a, const ScanItem& it, double quad,
                                                const LogProd& lp) {
    double logdet = lp.value();
    if (lp.bad) logdet = NAN;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        quad += __shfl_down_sync(0xffffffffu, quad, off);
        logdet += __shfl_down_sync(0xffffffffu, logdet, off);
    }
    if (threadIdx.x == 0) {
        a.part[2 * int64_t(blockIdx.x)] = quad;
        a.part[2 * int64_t(blockIdx.x) + 1] = logdet;
        __threadfence();
        const unsigned long long cnt = static_cast<unsigned long long>(a.lane_first[it.lane + 1] - a.lane_first[it.lane]);
        if (atomicAdd(lane_done(a) + it.lane, 1ull) == cnt - 1) {
            __threadfence();
            lane_total(a, it.lane);
        }
    }
}

// S3
template <bool kOU>
__global__ void __launch_bounds__(32) k_scan_finish(ScanArgs a) {
    const PhaseTable tab = scan_table(a);
    const ScanItem it = a.items[blockIdx.x];
    const int p = int(it.lane / a.B);
    const PulsarDev& ps = a.psr[p];
    const Lane L = scan_lane(a, it.lane, kOU, ps.equad2);
    const int k_lo = it.k0 + int(threadIdx.x) * a.E;
    const int k_hi = min(k_lo + a.E, ps.n);
    double quad = 0.0;
    LogProd lp;
    if (k_lo < k_hi) {
        State x{0.0, 0.0, ps.p0[0], ps.p0[1], ps.p0[2]};
        if (k_lo > 0) x = prefix_state(a, it, int(threadIdx.x));
        StepOut so;
        for (int k = k_lo; k < k_hi; ++k)
            kf_step<false, true, kOU, true>(x, a.rec + (ps.off + k) * kRecDoubles, L, tab, quad, lp, so);
    }
    finish_chunk_ll(a, it, quad, lp);
}

// S4
__global__ void k_scan_sum(ScanArgs a) {
    const int64_t lane = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (lane >= a.B * a.P) return;
    lane_total(a, lane);
}

// ---------------------------------------------------------------------------
// Time-parallel adjoint (plan mode SCAN with a gradient).
//
// The reverse sweep (adj_step below, the arithmetic of K3's adjoint step)
// takes the adjoint of TOA k's filtered state, a_k = (mu, Pi) with
// mu = dL/d(m0, m1) and Pi = [[pi00, pi01/2], [pi01/2, pi11]] (pi01 = dL/dP01
// of the one stored off-diagonal entry), to that of TOA k-1.  That map is
// affine:
//   mu_{k-1} = X mu_k + c,   Pi_{k-1} = X Pi_k X^T + mu0 Y0 + mu1 Y1 + Q,
// where X = A_k^T, the transpose of the filtered-state transition
// A_k = (I - K H) F = [[w, w b], [-K1, a - K1 b]] (w = R/S, K1 = M01/S,
// F = [[1, b], [0, a]]: b = dt and a = 1 for the random walk).  With
// g = e/S and s0 = -(1 - e g)/(2 S), in the packed symmetric form
// (00, 2 x 01, 11):
//   c = g (1, b),  Y0 = g w (1, 2b, b^2),  Y1 = g (-K1, a - 2 b K1, b (a - b K1)),
//   Q = s0 (1, 2b, b^2).
// (The covariance adjoint of the update is a congruence by [[w, -K1], [0, 1]]
// and that of the prediction one by [[1, 0], [b, a]]; their product is X.)
// Such maps are closed under composition: f then h (f x h, f the earlier in
// scan order) is
//   X = Xh Xf,  c = Xh cf + ch,
//   Yj = Xh Yfj Xh^T + sum_i Xf[i][j] Yhi,  Q = Xh Qf Xh^T + sum_i cf_i Yhi + Qh.
// The last TOA's adjoint is 0, so the adjoint at the end of a thread's TOAs
// is the (c, Q) of the composition of every later TOA's map, taken from the
// last TOA back: a suffix scan.  Each thread then runs the ordinary adjoint
// steps over its own TOAs from that exact start and sums its gradient terms.
// ---------------------------------------------------------------------------
struct AElem {
    double x00, x01, x10, x11, c0, c1;
    double y00, y01, y02, y10, y11, y12;
    double q0, q1, q2;
};

__device__ __forceinline__ AElem adj_identity() {
    return AElem{1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
}

__device__ __forceinline__ AElem adj_load(const double* src) {
    AElem x;
    double* d = &x.x00;
#pragma unroll
    for (int q = 0; q < kAdjElem; ++q) d[q] = src[q];
    return x;
}

__device__ __forceinline__ void adj_store(double* dst, const AElem& x) {
    const double* s = &x.x00;
#pragma unroll
    for (int q = 0; q < kAdjElem; ++q) dst[q] = s[q];
}

// X [[q0, q1/2], [q1/2, q2]] X^T in the packed form (00, 2 x 01, 11), X of h
__device__ __forceinline__ void congruence(const AElem& h, double q0, double q1, double q2,
                                           double& r0, double& r1, double& r2) {
    const double hq = 0.5 * q1;
    const double z00 = fma(h.x00, q0, h.x01 * hq), z01 = fma(h.x00, hq, h.x01 * q2);
    const double z10 = fma(h.x10, q0, h.x11 * hq), z11 = fma(h.x10, hq, h.x11 * q2);
    r0 = fma(z00, h.x00, z01 * h.x01);
    r1 = 2.0 * fma(z00, h.x10, z01 * h.x11);
    r2 = fma(z10, h.x10, z11 * h.x11);
}

// f x h restricted to one group of the output's fields (AElem order): part 0
// X and c; part 1 Y0; part 2 Y1; part 3 Q.  adj_combine runs all four.
template <int kPart>
__device__ __forceinline__ void adj_combine_part(const AElem& f, const AElem& h, double* o) {
    if (kPart == 0) {
        o[0] = fma(h.x00, f.x00, h.x01 * f.x10);
        o[1] = fma(h.x00, f.x01, h.x01 * f.x11);
        o[2] = fma(h.x10, f.x00, h.x11 * f.x10);
        o[3] = fma(h.x10, f.x01, h.x11 * f.x11);
        o[4] = fma(h.x00, f.c0, fma(h.x01, f.c1, h.c0));
        o[5] = fma(h.x10, f.c0, fma(h.x11, f.c1, h.c1));
    } else {
        // the congruence's argument and the weights (u, v) of Yh0, Yh1
        const double q0 = kPart == 1 ? f.y00 : kPart == 2 ? f.y10 : f.q0;
        const double q1 = kPart == 1 ? f.y01 : kPart == 2 ? f.y11 : f.q1;
        const double q2 = kPart == 1 ? f.y02 : kPart == 2 ? f.y12 : f.q2;
        const double u = kPart == 1 ? f.x00 : kPart == 2 ? f.x01 : f.c0;
        const double v = kPart == 1 ? f.x10 : kPart == 2 ? f.x11 : f.c1;
        double r0, r1, r2;
        congruence(h, q0, q1, q2, r0, r1, r2);
        if (kPart == 3) {
            r0 += h.q0;
            r1 += h.q1;
            r2 += h.q2;
        }
        constexpr int at = kPart == 1 ? 6 : kPart == 2 ? 9 : 12;
        o[at + 0] = fma(u, h.y00, fma(v, h.y10, r0));
        o[at + 1] = fma(u, h.y01, fma(v, h.y11, r1));
        o[at + 2] = fma(u, h.y02, fma(v, h.y12, r2));
    }
}

__device__ __forceinline__ AElem adj_combine(const AElem& f, const AElem& h) {
    AElem o;
    double* p = &o.x00;
    adj_combine_part<0>(f, h, p);
    adj_combine_part<1>(f, h, p);
    adj_combine_part<2>(f, h, p);
    adj_combine_part<3>(f, h, p);
    return o;
}

struct AdjScan {
    static constexpr int kN = kAdjElem;
    using Elem = AElem;
    static __device__ __forceinline__ Elem load(const double* s) { return adj_load(s); }
    template <int kPart>
    static __device__ __forceinline__ void part(const Elem& i, const Elem& j, double* o) {
        adj_combine_part<kPart>(i, j, o);
    }
    static __host__ __device__ constexpr int begin(int p) {
        return p == 0 ? 0 : p == 1 ? 6 : p == 2 ? 9 : p == 3 ? 12 : 15;
    }
};

// The reverse map of one TOA, from its forward step's quantities (rec: its
// record, whose dt is the random walk's b).
template <bool kOU>
__device__ __forceinline__ AElem adj_element(const StepOut& so, const double* __restrict__ rec) {
    const double a = kOU ? so.a : 1.0, b = kOU ? so.b : rec[1];
    const double g = so.g;
    const double s0 = 0.5 * so.h2;
    const double x11 = fma(-b, so.K1, a);
    const double twob = 2.0 * b, b2 = b * b, gw = g * so.w;
    AElem E;
    E.x00 = so.w; E.x01 = -so.K1; E.x10 = b * so.w; E.x11 = x11;
    E.c0 = g; E.c1 = b * g;
    E.y00 = gw; E.y01 = twob * gw; E.y02 = b2 * gw;
    E.y10 = -g * so.K1; E.y11 = g * fma(-twob, so.K1, a); E.y12 = g * (b * x11);
    E.q0 = s0; E.q1 = twob * s0; E.q2 = b2 * s0;
    return E;
}

struct AdjState {
    double mu0, mu1, pi00, pi01, pi11;   // adjoint of a TOA's filtered state
};

// Lane gradient sums, in the order of the lane output rows 1..7: dll/dA,
// dll/dB, the t-weighted sin and cos sums, dll/dsigma^2, the EFAC term and
// (Ornstein-Uhlenbeck) dll/dgamma.
struct GradSums {
    double A, B, At, Bt, s2, E, G;
};

// One reverse step: the adjoint of TOA k's filtered state -> that of TOA
// k-1, adding TOA k's gradient terms.  The same arithmetic as K3's step.
template <bool kOU>
__device__ __forceinline__ void adj_step(AdjState& a, const StepOut& so, const double* __restrict__ rec,
                                         const Lane& L, GradSums& g) {
    const double t = rec[0], dt = rec[1], h2 = rec[2], h3 = rec[3], s2k = rec[5], dt2 = rec[6];
    const double twodt = rec[7];
    const double w = so.w, K1 = so.K1, gg = so.g;
    const double t1 = fma(-a.mu0, w, fma(a.mu1, K1, a.mu0));    // mu0 K0 + mu1 K1, K0 = 1 - w
    const double ebar = t1 - gg;                                // dL/de
    const double u = fma(-a.pi00, w, fma(a.pi01, K1, a.pi00));  // pi00 K0 + pi01 K1
    const double v = a.pi11 * K1;
    const double ku = fma(-w, u, fma(v, K1, u));                // K0 u + K1 v
    const double Sbar = fma(0.5, so.h2, fma(-gg, t1, ku));
    const double a0 = a.mu0 - ebar;                             // dL/d(predicted m0)
    const double M00b = fma(a.mu0, gg, fma(a.pi00, fma(2.0, w, -1.0), fma(-a.pi01, K1, Sbar)));
    const double M01b = fma(a.mu1, gg, fma(a.pi01, w, -2.0 * v));
    const double M11b = a.pi11;
    g.E = fma(Sbar, s2k, g.E);
    g.A = fma(-ebar, so.sn, g.A);
    g.B = fma(-ebar, so.cs, g.B);
    const double st = -ebar * t;
    g.At = fma(st, so.sn, g.At);
    g.Bt = fma(st, so.cs, g.Bt);
    if (kOU) {
        g.s2 = fma(M00b, so.c00, fma(M01b, so.c01, fma(M11b, so.c11, g.s2)));
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

// A step's tape record in the chunk's field-major tape: field f at tk[f * st].
template <bool kOU>
__device__ __forceinline__ void stape_put(double* tk, int64_t st, const StepOut& so) {
    tk[0 * st] = so.w; tk[1 * st] = so.K1; tk[2 * st] = so.g;
    tk[3 * st] = so.h2; tk[4 * st] = so.sn; tk[5 * st] = so.cs;
    if (kOU) {
        tk[6 * st] = so.m1; tk[7 * st] = so.t1; tk[8 * st] = so.ap11;
        tk[9 * st] = so.a; tk[10 * st] = so.b; tk[11 * st] = so.c00; tk[12 * st] = so.c01;
        tk[13 * st] = so.c11; tk[14 * st] = so.db; tk[15 * st] = so.dc00; tk[16 * st] = so.dc01;
        tk[17 * st] = so.dc11;
    }
}

template <bool kOU>
__device__ __forceinline__ StepOut stape_get(const double* tk, int64_t st) {
    StepOut so{};
    so.w = tk[0 * st]; so.K1 = tk[1 * st]; so.g = tk[2 * st];
    so.h2 = tk[3 * st]; so.sn = tk[4 * st]; so.cs = tk[5 * st];
    if (kOU) {
        so.m1 = tk[6 * st]; so.t1 = tk[7 * st]; so.ap11 = tk[8 * st];
        so.a = tk[9 * st]; so.b = tk[10 * st]; so.c00 = tk[11 * st]; so.c01 = tk[12 * st];
        so.c11 = tk[13 * st]; so.db = tk[14 * st]; so.dc00 = tk[15 * st]; so.dc01 = tk[16 * st];
        so.dc11 = tk[17 * st];
    }
    return so;
}

// G3: S3 with the tape.  Warp 0 runs S3's forward steps, writes each step's
// tape record, composes the thread's reverse map (its latest TOA's applied
// first) and finishes the chunk's log-likelihood sums.  Then the four warps
// scan the 32 maps, thread t's stored at position 31 - t so that a prefix in
// that order is a suffix in TOA order: position 31 - t ends holding the map
// of thread t's TOAs and every later thread's.
template <bool kOU>
__global__ void __launch_bounds__(kScanThreads) k_scan_finish_grad(ScanGradArgs g) {
    constexpr int kTd = kOU ? kScanTapeDoublesOU : kScanTapeDoubles;
    __shared__ double buf[2][32][kAdjElem];
    const ScanArgs& a = g.s;
    const int t = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        const PhaseTable tab = scan_table(a);
        const ScanItem it = a.items[blockIdx.x];
        if (t == 0 && it.k0 == 0) g.rdone[it.lane] = 0ull;   // before R3 (a later kernel)
        const int p = int(it.lane / a.B);
        const PulsarDev& ps = a.psr[p];
        const Lane L = scan_lane(a, it.lane, kOU, ps.equad2);
        const int k_lo = it.k0 + t * a.E;
        const int k_hi = min(k_lo + a.E, ps.n);
        const int64_t span = int64_t(32) * a.E;
        double quad = 0.0;
        LogProd lp;
        AElem psi = adj_identity();
        if (k_lo < k_hi) {
            double* tp = g.tape + int64_t(blockIdx.x) * span * kTd + (k_lo - it.k0);
            State x{0.0, 0.0, ps.p0[0], ps.p0[1], ps.p0[2]};
            if (k_lo > 0) x = prefix_state(a, it, t);
            StepOut so;
            for (int k = k_lo; k < k_hi; ++k) {
                const double* rec = a.rec + (ps.off + k) * kRecDoubles;
                kf_step<true, true, kOU, true>(x, rec, L, tab, quad, lp, so);
                stape_put<kOU>(tp + (k - k_lo), span, so);
                const AElem f = adj_element<kOU>(so, rec);
                psi = (k == k_lo) ? f : adj_combine(f, psi);
            }
        }
        adj_store(buf[0][31 - t], psi);
        finish_chunk_ll(a, it, quad, lp);
    }
    __syncthreads();
    const int res = coop_scan32<AdjScan>(buf);
    if (threadIdx.x < 32) {
        adj_store(g.tsuf + (int64_t(blockIdx.x) * 32 + t) * kAdjElem, adj_load(buf[res][31 - t]));
        if (t == 0) adj_store(g.ragg + int64_t(blockIdx.x) * kAdjElem, adj_load(buf[res][31]));
    }
}

// R2: one block per lane.  For each chunk, the composition of every later
// chunk's map (an exclusive scan over the lane's chunks in reversed order:
// each thread composes its run of chunks, the four warps scan the 32 runs,
// then each thread walks its run).  An empty lane's gradient terms are 0.
__global__ void __launch_bounds__(kScanThreads) k_rscan_chunks(ScanGradArgs g) {
    __shared__ double buf[2][32][kAdjElem];
    const ScanArgs& a = g.s;
    const int lane = blockIdx.x, t = threadIdx.x & 31;
    const int first = a.lane_first[lane], cnt = a.lane_first[lane + 1] - first;
    if (cnt == 0) {   // the whole block
        if (threadIdx.x < kLaneGrads) a.lane_out[int64_t(1 + threadIdx.x) * a.B * a.P + lane] = 0.0;
        return;
    }
    const int q = (cnt + 31) / 32;
    const int r_lo = t * q, r_hi = min(r_lo + q, cnt);   // positions r: chunk first + cnt - 1 - r
    if (threadIdx.x < 32) {
        AElem agg = adj_identity();
        if (r_lo < r_hi) agg = adj_load(g.ragg + int64_t(first + cnt - 1 - r_lo) * kAdjElem);
        for (int r = r_lo + 1; r < r_hi; ++r)
            agg = adj_combine(agg, adj_load(g.ragg + int64_t(first + cnt - 1 - r) * kAdjElem));
        adj_store(buf[0][t], agg);
    }
    __syncthreads();
    const int res = coop_scan32<AdjScan>(buf);
    if (threadIdx.x < 32) {
        AElem pre = t == 0 ? adj_identity() : adj_load(buf[res][t - 1]);
        for (int r = r_lo; r < r_hi; ++r) {
            const int c = first + cnt - 1 - r;
            adj_store(g.rpre + int64_t(c) * kAdjElem, pre);
            if (r + 1 < r_hi)   // the composition past the thread's last chunk is not needed
                pre = adj_combine(pre, adj_load(g.ragg + int64_t(c) * kAdjElem));
        }
    }
}

// R3: one warp per chunk.  Thread t's adjoint at its last TOA is the (c, Q)
// of "later chunks, then threads t+1..31 of the chunk" (a_{N-1} = 0); from
// there it runs the adjoint steps over its own TOAs in reverse.  Warp sums
// per chunk; the block that completes its lane last sums the lane's chunks
// in chunk order into lane_out rows 1..7.
template <bool kOU>
__global__ void __launch_bounds__(32) k_rscan_finish(ScanGradArgs g) {
    constexpr int kTd = kOU ? kScanTapeDoublesOU : kScanTapeDoubles;
    const ScanArgs& a = g.s;
    const int t = threadIdx.x;
    const ScanItem it = a.items[blockIdx.x];
    const int p = int(it.lane / a.B);
    const PulsarDev& ps = a.psr[p];
    const int k_lo = it.k0 + t * a.E;
    const int k_hi = min(k_lo + a.E, ps.n);
    const int64_t span = int64_t(32) * a.E;
    GradSums gs{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (k_lo < k_hi) {
        const Lane L = scan_lane(a, it.lane, kOU, ps.equad2);
        const AElem om = adj_load(g.rpre + int64_t(blockIdx.x) * kAdjElem);
        AElem m = om;
        if (t < 31) {
            const AElem sf = adj_load(g.tsuf + (int64_t(blockIdx.x) * 32 + t + 1) * kAdjElem);
            adj_combine_part<0>(om, sf, &m.x00);   // c (and X)
            adj_combine_part<3>(om, sf, &m.x00);   // Q
        }
        AdjState adj{m.c0, m.c1, m.q0, m.q1, m.q2};
        const double* tp = g.tape + int64_t(blockIdx.x) * span * kTd + (k_lo - it.k0);
        for (int k = k_hi - 1; k >= k_lo; --k)
            adj_step<kOU>(adj, stape_get<kOU>(tp + (k - k_lo), span), a.rec + (ps.off + k) * kRecDoubles,
                          L, gs);
    }
    double* v = &gs.A;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int q = 0; q < kLaneGrads; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    }
    if (t == 0) {
        double* pg = g.partg + int64_t(blockIdx.x) * kLaneGrads;
#pragma unroll
        for (int q = 0; q < kLaneGrads; ++q) pg[q] = v[q];
        __threadfence();
        const int first = a.lane_first[it.lane], last = a.lane_first[it.lane + 1];
        const unsigned long long cnt = static_cast<unsigned long long>(last - first);
        if (atomicAdd(g.rdone + it.lane, 1ull) == cnt - 1) {
            __threadfence();
            double s[kLaneGrads];
#pragma unroll
            for (int q = 0; q < kLaneGrads; ++q) s[q] = 0.0;
            for (int c = first; c < last; ++c) {
#pragma unroll
                for (int q = 0; q < kLaneGrads; ++q) s[q] += __ldcg(g.partg + int64_t(c) * kLaneGrads + q);
            }
            const int64_t lanes = a.B * a.P;
            const int nout = kOU ? kLaneGrads : kLaneGrads - 1;
            for (int q = 0; q < nout; ++q) a.lane_out[int64_t(1 + q) * lanes + it.lane] = s[q];
        }
    }
}

}  // namespace

void launch_filter_scan(const ScanArgs& a, cudaStream_t s) {
    const size_t smem = 0;
    const bool ou = a.model == kOrnsteinUhlenbeck;
    const int lanes = int(a.B * a.P);
    if (a.n_items > 0) {
        if (ou) k_scan_local<true><<<a.n_items, kScanThreads, smem, s>>>(a);
        else k_scan_local<false><<<a.n_items, kScanThreads, smem, s>>>(a);
        k_scan_chunks<<<lanes, kScanThreads, 0, s>>>(a);
        if (ou) k_scan_finish<true><<<a.n_items, 32, smem, s>>>(a);
        else k_scan_finish<false><<<a.n_items, 32, smem, s>>>(a);
    } else {
        k_scan_sum<<<(lanes + 127) / 128, 128, 0, s>>>(a);   // every lane empty
    }
}

void launch_filter_scan_grad(const ScanGradArgs& g, cudaStream_t s) {
    const ScanArgs& a = g.s;
    const bool ou = a.model == kOrnsteinUhlenbeck;
    const int lanes = int(a.B * a.P);
    if (a.n_items > 0) {
        if (ou) k_scan_local<true><<<a.n_items, kScanThreads, 0, s>>>(a);
        else k_scan_local<false><<<a.n_items, kScanThreads, 0, s>>>(a);
        k_scan_chunks<<<lanes, kScanThreads, 0, s>>>(a);
        if (ou) k_scan_finish_grad<true><<<a.n_items, kScanThreads, 0, s>>>(g);
        else k_scan_finish_grad<false><<<a.n_items, kScanThreads, 0, s>>>(g);
        k_rscan_chunks<<<lanes, kScanThreads, 0, s>>>(g);
        if (ou) k_rscan_finish<true><<<a.n_items, 32, 0, s>>>(g);
        else k_rscan_finish<false><<<a.n_items, 32, 0, s>>>(g);
    } else {
        k_scan_sum<<<(lanes + 127) / 128, 128, 0, s>>>(a);   // every lane empty: ll 0
        k_rscan_chunks<<<lanes, kScanThreads, 0, s>>>(g);    // ... and gradient terms 0
    }
}

}  // namespace argus
