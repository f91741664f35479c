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
#include "kf_model.cuh"

namespace argus {

namespace {

constexpr double kLog2Pi = 1.8378770664093454836;
constexpr int kChunk = 128;  // TOA records per shared-memory chunk (forward kernel)

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
    const double w = so.w, K1 = so.K1, gg = so.g;
    const double t1 = fma(-a.mu0, w, fma(a.mu1, K1, a.mu0));    // mu0 K0 + mu1 K1
    const double ebar = t1 - gg;                                // dL/de
    const double u = fma(-a.pi00, w, fma(a.pi01, K1, a.pi00));  // pi00 K0 + pi01 K1
    const double v = a.pi11 * K1;
    const double ku = fma(-w, u, fma(v, K1, u));                // K0 u + K1 v
    // dL/dS: its own term -(1 - e^2/S)/(2S) = h2/2, and through g = e/S and K
    const double Sbar = fma(0.5, so.h2, fma(-gg, t1, ku));
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

// One step's tape record, field-major within the step: [field][W].  The
// signal's sin and cos are not stored: the record keeps the phase fraction F
// (8 bytes, bit pattern in a double slot) and tape_get forms them again with
// sincos_frac, which runs on the integer and FP32 pipes only -- in the
// shadow of the FP64 pipe, which bounds this kernel -- and gives the same
// bits as the forward step.
template <bool kOU>
__device__ __forceinline__ void tape_put(double* tk, int W, const StepOut& so) {
    tk[0 * W] = so.w; tk[1 * W] = so.K1; tk[2 * W] = so.g;
    tk[3 * W] = so.h2; tk[4 * W] = __longlong_as_double(static_cast<long long>(so.F));
    if (kOU) {
        tk[5 * W] = so.m1; tk[6 * W] = so.t1; tk[7 * W] = so.ap11;
        tk[8 * W] = so.a; tk[9 * W] = so.b; tk[10 * W] = so.c00; tk[11 * W] = so.c01;
        tk[12 * W] = so.c11; tk[13 * W] = so.db; tk[14 * W] = so.dc00; tk[15 * W] = so.dc01;
        tk[16 * W] = so.dc11;
    }
}

template <bool kOU>
__device__ __forceinline__ StepOut tape_get(const double* tk, int W, PhaseTable tab) {
    StepOut so{};
    so.w = tk[0 * W]; so.K1 = tk[1 * W]; so.g = tk[2 * W];
    so.h2 = tk[3 * W];
    so.F = static_cast<uint64_t>(__double_as_longlong(tk[4 * W]));
    if (kOU) {
        so.m1 = tk[5 * W]; so.t1 = tk[6 * W]; so.ap11 = tk[7 * W];
        so.a = tk[8 * W]; so.b = tk[9 * W]; so.c00 = tk[10 * W]; so.c01 = tk[11 * W];
        so.c11 = tk[12 * W]; so.db = tk[13 * W]; so.dc00 = tk[14 * W]; so.dc01 = tk[15 * W];
        so.dc11 = tk[16 * W];
    }
    sincos_frac(so.F, tab, so.sn, so.cs);
    return so;
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
    s.tab.d = reinterpret_cast<longlong2*>(smem_raw);
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
// recording (R/S, K1, e/S, (e/S)^2 - 1/S, phase fraction) per step in the
// block's tape, then run the adjoint steps in reverse.  Checkpoints and tape
// live in the block's own slot of global scratch ([..][field][W], so a warp's
// accesses coalesce).  With kCache the tape of every segment is written during
// pass 1 and kept in HBM (the slot holds the whole pulsar), so pass 2 skips the
// re-run and pass 1 writes no checkpoints: HBM traffic is traded for FP64
// work, which is the scarce resource here.
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
                if (!kCache) {   // the cached tape needs no checkpoints
                    double* cp = ck + int64_t(seg) * kCkptDoubles * W;
                    cp[0 * W] = x.m0; cp[1 * W] = x.m1; cp[2 * W] = x.p00; cp[3 * W] = x.p01;
                    cp[4 * W] = x.p11;
                }
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
                    const StepOut sk = tape_get<kOU>(ts + int64_t(k) * kTd * W, W, sm.tab);
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
