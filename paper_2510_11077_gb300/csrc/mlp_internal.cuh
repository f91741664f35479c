// Internal declarations of the surrogate network's kernels (BF16 tensor cores).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace argus {

constexpr int kMlpLayers = 5;
constexpr int kMlpIn = 47, kMlpInPad = 64;
constexpr int kMlpOut = 48, kMlpOutPad = 64;
constexpr int kMlpHidden = 256;
constexpr int kGemmM = 128;      // rows per tile (tcgen05 M)
constexpr int kGemmKMax = 256;   // whole K of a tile is staged at once

// Epilogues of the tensor-core GEMM C[m][n] = sum_k A[m][k] B[n][k].
enum GemmEpi : int {
    kEpiF32 = 0,       // out_f32[m][n] = acc (+ bias[n] if bias)
    kEpiGelu = 1,      // z = acc + bias; out_f32 = z (if set); h = gelu(z): out_bf16, out_bf16_t
    kEpiGeluBwd = 2,   // d = acc * gelu'(zin[m][n]): out_f32 = d, out_bf16 = bf16(d), out_bf16_t
};

struct GemmEpiArgs {
    const float* bias;        // [N] or nullptr
    const float* zin;         // kEpiGeluBwd: saved pre-activation [M][ldz]
    int ldz;
    float* out_f32;           // [M][ldo] (+ blockIdx.z * chunk_stride)
    int ldo;
    int64_t chunk_stride;     // element offset between K-chunks of a split-K product
    __nv_bfloat16* out_bf16;  // [M][ldb]
    int ldb;
    __nv_bfloat16* out_bf16_t;  // transposed [N][ldt]
    int ldt;
};

// Launch one GEMM: M rows (multiple of 128), N columns (multiple of bn),
// K <= 256 per output tile; grid.z = number of K-chunks (split-K: chunk z
// reads K-coordinates [z K, (z+1) K) and writes out_f32 + z chunk_stride).
cudaError_t launch_gemm_tc(const CUtensorMap* ta, const CUtensorMap* tb, int M, int N, int K,
                           int bn, int chunks, int epi, const GemmEpiArgs& e, int* err,
                           cudaStream_t s);

// Fused evaluation of the whole network on one 128-row slab per cluster of 1,
// 2 or 4 CTAs (forward through the five layers and, in kFusedValueGrad, the
// value output's gradient back to the input), activations kept in shared
// memory; each CTA of a cluster computes its share of every layer's columns.
enum FusedMode : int {
    kFusedValue = 0,        // loglik only
    kFusedValueGrad = 1,    // loglik and the back-propagated gradient of the value output
    kFusedGradHead = 2,     // loglik and the gradient outputs of the network
};

struct MlpFusedMaps {
    CUtensorMap w[kMlpLayers];        // W_l [out][in] BF16, box rows = out / cluster size
    CUtensorMap wt[kMlpLayers - 1];   // W_l^T [in][out] BF16 for l = 0..3, box rows = in / cluster size
};

struct MlpFusedArgs {
    const float* theta;               // [n][47] raw inputs
    int64_t n;                        // rows of this launch
    float xm[kMlpInPad];              // input means (pad 0)
    float xs[kMlpInPad];              // input std devs (pad 1)
    float ym, ys;                     // value output mean and std
    const float* bias[kMlpLayers];    // [out] per layer
    const __nv_bfloat16* w4;          // W_4 [64][256] BF16 (row 0: the value output's weights)
    float* gscr[kMlpLayers - 1];      // [>= ceil(n/128)*128][256] scratch: gelu'(z) of layers 1..4
    const float* Hq;                  // [47][47] quadratic baseline or nullptr
    float* loglik;                    // [n]
    float* grad;                      // [n][47] or nullptr (kFusedValue)
    int mode;
    int* err;
    // FP64 input/output (z64 non-null): the network's input row is
    // float(z64[r] - zc), and loglik / grad go to ll64 / g64 as doubles, the
    // loglik plus off and -inf when not finite; theta, loglik, grad unused
    const double* z64;
    const double* zc;
    double off;
    double* ll64;
    double* g64;
    // optional trace of every GEMM stage (tests): tr_act + st * tr_stride + row * 256 gets
    // the stage's BF16 A operand row (as floats), tr_acc likewise its FP32 accumulator
    // row before any bias; nullptr = no trace
    float* tr_act;
    float* tr_acc;
    int64_t tr_stride;
};

// maps[0], [1], [2]: the weight maps for clusters of 1, 2 and 4 CTAs (boxes of
// N, N / 2 and N / 4 rows); cl = 1, 2 or 4 CTAs per 128-row slab, or 0 for the
// widest whose clusters all run at once.
cudaError_t launch_mlp_fused(const MlpFusedMaps* maps, const MlpFusedArgs& a, cudaStream_t s, int cl);
int fused_cluster_size(int64_t n);

// Make a 2-D BF16 tensor map over a row-major [rows][cols] array with a box of
// [box_rows][64] and 128-byte swizzle.  Returns false if the driver refuses.
bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                    uint32_t box_rows);

}  // namespace argus
