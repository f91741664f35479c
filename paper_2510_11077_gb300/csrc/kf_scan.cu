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

namespace argus {

__global__ void k_fill_phase_table(double* tab) {
    fill_phase_table(PhaseTable{reinterpret_cast<double2*>(tab),
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
    const double rdet = rcp_nr(fma(M00, M11, -M01 * M10));
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
        const double rS = rcp_nr(p00 + R);
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
        const double rS = rcp_nr(q00 + R);
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
    tab.d = reinterpret_cast<double2*>(t);
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
// ~95 of them per combine.  Here every level's 32 combines are shared out by
// field group (scan_combine_part): warp w forms the common M^-1 and its own
// fields, ~50 FP64 instructions, and the four warps run on the four
// sub-partitions at once.  Element i starts in buf[0][i]; the result is in
// buf[returned index][i].  All kScanThreads threads call it.
constexpr int kScanThreads = 128;

__device__ __forceinline__ int coop_scan32(double (*buf)[32][kScanElem]) {
    const int lane = threadIdx.x & 31, part = threadIdx.x >> 5;
    int cur = 0;
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
        double* dst = buf[cur ^ 1][lane];
        const double* xs = buf[cur][lane];
        if (lane >= off) {
            const SElem y = load_elem(buf[cur][lane - off]);
            const SElem x = load_elem(xs);
            switch (part) {
                case 0: scan_combine_part<0>(y, x, dst); break;
                case 1: scan_combine_part<1>(y, x, dst); break;
                case 2: scan_combine_part<2>(y, x, dst); break;
                default: scan_combine_part<3>(y, x, dst); break;
            }
        } else {
            for (int f = part_begin(part); f < part_begin(part + 1); ++f) dst[f] = xs[f];
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
    const int res = coop_scan32(buf);
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
    const int res = coop_scan32(buf);
    if (threadIdx.x < 32) {
        SElem pre = t == 0 ? scan_identity() : load_elem(buf[res][t - 1]);
        for (int c = c_lo; c < c_hi; ++c) {
            store_elem(a.bpre + int64_t(first + c) * kScanElem, pre);
            if (c + 1 < c_hi)   // the prefix after the thread's last chunk is not needed
                pre = scan_combine(pre, load_elem(a.bagg + int64_t(first + c) * kScanElem));
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
        if (k_lo > 0) {
            // filtered state at TOA k_lo - 1: chunk prefix x earlier threads of
            // the chunk (the lane's first chunk has no prefix)
            SElem pre;
            if (threadIdx.x == 0) {
                pre = load_elem(a.bpre + int64_t(blockIdx.x) * kScanElem);
            } else {
                pre = load_elem(a.tpre + (int64_t(blockIdx.x) * 32 + threadIdx.x - 1) * kScanElem);
                if (it.k0 > 0) pre = scan_combine(load_elem(a.bpre + int64_t(blockIdx.x) * kScanElem), pre);
            }
            x = State{pre.b0, pre.b1, pre.C00, pre.C01, pre.C11};
        }
        StepOut so;
        for (int k = k_lo; k < k_hi; ++k)
            kf_step<false, true, kOU>(x, a.rec + (ps.off + k) * kRecDoubles, L, tab, quad, lp, so);
    }
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
        // the block that completes its lane last sums the lane's chunks (no
        // block waits: the others just leave)
        __threadfence();
        const unsigned long long cnt = static_cast<unsigned long long>(a.lane_first[it.lane + 1] - a.lane_first[it.lane]);
        if (atomicAdd(lane_done(a) + it.lane, 1ull) == cnt - 1) {
            __threadfence();
            lane_total(a, it.lane);
        }
    }
}

// S4
__global__ void k_scan_sum(ScanArgs a) {
    const int64_t lane = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (lane >= a.B * a.P) return;
    lane_total(a, lane);
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

}  // namespace argus
