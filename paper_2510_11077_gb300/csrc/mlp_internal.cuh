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

// Make a 2-D BF16 tensor map over a row-major [rows][cols] array with a box of
// [box_rows][64] and 128-byte swizzle.  Returns false if the driver refuses.
bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                    uint32_t box_rows);

}  // namespace argus
