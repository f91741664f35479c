// Internal declarations shared by the C-ABI layer and the filter kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace argus {

constexpr int kNgw = 7;          // continuous-wave parameters at the head of theta
constexpr int kRecDoubles = 8;   // doubles per staged TOA record
constexpr int kCkptDoubles = 5;  // (m0, m1, p00, p01, p11) per checkpoint
constexpr int kTapeDoubles = 5;  // (R/S, K1, e/S, (e/S)^2 - 1/S, phase fraction) per step (K3)
constexpr int kTapeDoublesOU = 17; // ... plus (m1, p01 + b p11, a p11) before the step, the
                                   // transition a, b, Q / sigma^2 (3) and d/dgamma of b, Q (4)
// The time-parallel adjoint's tape keeps sin and cos themselves in place of
// the phase fraction (its steps are latency-bound, not FP64-bound).
constexpr int kScanTapeDoubles = 6;
constexpr int kScanTapeDoublesOU = 18;
constexpr int kMaxStride = 256;  // longest adjoint segment, in TOAs
constexpr int kLaneConsts = 8;   // A, B, f, Phi0/(2 pi), sigma^2, EFAC^2, EFAC, gamma
constexpr int kLaneGrads = 7;    // dll/dA, dB, t-weighted sin and cos sums, dsigma^2, EFAC term,
                                 // dll/dgamma

// Red-noise model of the frequency deviation y (argus.h: ARGUS_NOISE_*).
enum NoiseModel : int32_t { kRandomWalk = 0, kOrnsteinUhlenbeck = 1 };

// Model flags as in argus.h: bit 0 the noise model, bit 1 the wave's pulsar
// term.  Per pulsar theta holds (log10 sigma, [log10 gamma], EFAC, [d_kpc]).
constexpr int32_t kFlagOU = 1;
constexpr int32_t kFlagPulsarTerm = 2;
__host__ __device__ inline int params_per_pulsar(int32_t flags) {
    return 2 + (flags & kFlagOU) + ((flags & kFlagPulsarTerm) >> 1);
}
inline int tape_doubles(int32_t noise_model) {
    return noise_model == kOrnsteinUhlenbeck ? kTapeDoublesOU : kTapeDoubles;
}
inline int scan_tape_doubles(int32_t noise_model) {
    return noise_model == kOrnsteinUhlenbeck ? kScanTapeDoublesOU : kScanTapeDoubles;
}

// One staged TOA record (8 doubles = 64 bytes, 16-byte aligned):
//   [0] t  [1] dt  [2] dt^2/2  [3] dt^3/3  [4] r  [5] sigma^2  [6] dt^2  [7] 2 dt
struct PulsarDev {
    int64_t off;      // first record of this pulsar
    int32_t n;        // TOAs
    int32_t stride;   // adjoint checkpoint stride (TOAs per segment)
    int32_t nseg;     // ceil(n / stride)
    int32_t pad;
    double pos[3];    // unit vector
    double equad2;    // EQUAD^2
    double p0[3];     // prior covariance rr, ry, yy
};

struct WorkItem {
    int32_t p;        // pulsar
    int32_t b0;       // first walker of the tile
};

struct FilterArgs {
    const double* rec;        // [sum N][8]
    const PulsarDev* psr;     // [P]
    const WorkItem* items;    // [n_items], largest pulsars first
    int32_t n_items;
    int32_t P;
    int64_t B;
    const double* lc;         // lane constants [7][P][B]
    double* lane_out;         // [1 + 7][P][B]: ll, then the gradient terms
    double* ckpt;             // per block slot: [nseg_max][5][W]
    double* tape;             // per block slot: [stride_max or N_max][6][W]
    int64_t ckpt_slot;        // doubles per block slot in ckpt
    int64_t tape_slot;        // doubles per block slot in tape
    int32_t stride_max;       // longest segment of any pulsar (shared-memory records)
    int32_t tape_cache;       // 1: tape slot holds every segment of the pulsar (no re-run)
    int* counter;             // persistent work counter (nullptr: one item per block)
    int32_t model;            // NoiseModel (the pulsar term only changes K1 and K4)
    int32_t pad;
};

// K1: theta [B][D] -> lane constants [8][P][B] (flags: kFlagOU | kFlagPulsarTerm).
void launch_project(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                    double* lc, cudaStream_t s);
// K2: forward filter, ll per lane -> lane_out[0][P][B].
void launch_filter_fwd(const FilterArgs& a, int W, int grid, cudaStream_t s);
// K3: forward with checkpoints + reverse sweep -> lane_out[0..7][P][B].
void launch_filter_grad(const FilterArgs& a, int W, int grid, cudaStream_t s);
// Time-parallel (associative-scan) forward filter, for few lanes.  A lane's
// TOAs are cut into chunks of 32 x E; one warp per chunk.
constexpr int kScanElem = 14;   // doubles per scan element (A 4, b 2, C 3, eta 2, J 3)
struct ScanItem {
    int32_t lane;     // p * B + b
    int32_t k0;       // first TOA of the chunk
};
struct ScanArgs {
    const double* rec;
    const PulsarDev* psr;
    const double* lc;         // lane constants [8][P][B]
    int32_t P;
    int64_t B;
    const ScanItem* items;    // [n_items], lanes in order, chunks in order
    int32_t n_items;
    int32_t E;                // TOAs per thread
    const int32_t* lane_first;   // [B P + 1]: items of lane l are lane_first[l] .. [l + 1] - 1
    double* tpre;             // [n_items * 32][14]: inclusive prefix of each thread in its chunk
    double* bagg;             // [n_items][14]: chunk aggregates
    double* bpre;             // [n_items][14]: exclusive prefix of each chunk in its lane
    double* part;             // [n_items][2]: (sum e^2/S, sum ln S) of the chunk, NaN if invalid
    double* lane_out;         // [P][B]: ll per lane
    const double* phase_table;   // the handle's sin/cos(2 pi j / 256) table (kPhaseTableDoubles)
    int32_t model;            // NoiseModel
};
void launch_filter_scan(const ScanArgs& a, cudaStream_t s);
// the sin/cos table of phase_sincos in global memory: 256 longlong2 (the nodes in
// 2^-62 fixed point), then 256 float4 (the nodes as float pairs)
constexpr int kPhaseTableDoubles = 256 * 4;
void launch_fill_phase_table(double* tab, cudaStream_t s);

// K4: deterministic sum over pulsars (and chain rule through K1 for grad).
void launch_reduce(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                   const double* lane_out, double* loglik, double* grad, double* lane_ll,
                   cudaStream_t s);
// The model's continuous-wave residual at every TOA for one theta_gw [7] (device).
void launch_cw_signal(const double* theta_gw, int32_t P, const PulsarDev* psr, const double* rec,
                      int max_n, double* s, cudaStream_t st);
// shared-memory bytes a filter block needs
size_t filter_smem_bytes(bool grad, int stride_max);

}  // namespace argus
