// Surrogate network of the array log-likelihood and its gradient:
// MLP 47 -> 256 -> 256 -> 256 -> 256 -> 48 (GELU), BF16 weights and
// activations, FP32 accumulation on the tensor cores (mlp_gemm.cu), FP32
// master weights and Adam.  C ABI in include/argus_surrogate.h.  Evaluation
// runs the fused kernel (every layer in one launch); training runs one GEMM
// launch per product, with the small reductions as parallel fixed-order
// kernels.
//
// Layer l computes z = x W_l^T + b_l.  Shapes are padded for the tensor
// cores: the input has 64 columns (47 used), the output 64 (48 used); padding
// weights are zero and get zero gradient.  Inputs are standardized
// (x_k - mean_k) / std_k; the value head predicts (ll - y_mean) / y_std and
// the gradient head predicts dll/dx_k * std_k / y_std.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/argus_selftest.h"
#include "../../include/argus_surrogate.h"
#include "mlp_internal.cuh"

using namespace argus;

namespace {

thread_local std::string g_sur_error;

argus_status sfail(argus_status st, const std::string& m) {
    g_sur_error = m;
    return st;
}

argus_status scuda(cudaError_t e, const char* what) {
    return sfail(e == cudaErrorMemoryAllocation ? ARGUS_ERR_OOM : ARGUS_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define SCK(call)                                          \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return scuda(_e, #call);    \
    } while (0)

constexpr int kIn[kMlpLayers] = {kMlpInPad, kMlpHidden, kMlpHidden, kMlpHidden, kMlpHidden};
constexpr int kOut[kMlpLayers] = {kMlpHidden, kMlpHidden, kMlpHidden, kMlpHidden, kMlpOutPad};

struct DeviceGuardS {
    int prev = -1;
    explicit DeviceGuardS(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuardS() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
struct Norm {
    float xm[kMlpInPad], xs[kMlpInPad];   // input mean / std (pad: 0 / 1)
    float ym, ys;                          // value mean / std
    float w[kMlpOut];                      // loss weights (value, then gradient components)
};

// X0[r][k] = bf16((theta[r][k] - xm_k) / xs_k) for k < 47, 0 otherwise; rows >= n are 0.
// xt (optional) is the transposed copy [64][pitch].
// One thread per (row, column): block (64 columns, 4 rows), grid rows / 4.
__global__ void k_standardize(const float* __restrict__ theta, int64_t n, int rows, Norm nm,
                              __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ xt,
                              int pitch) {
    const int k = threadIdx.x;
    const int r = blockIdx.x * blockDim.y + threadIdx.y;
    if (r >= rows || k >= kMlpInPad) return;
    float v = 0.0f;
    if (r < n && k < kMlpIn) v = (theta[int64_t(r) * kMlpIn + k] - nm.xm[k]) / nm.xs[k];
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    x[int64_t(r) * kMlpInPad + k] = b;
    if (xt) xt[int64_t(k) * pitch + r] = b;
}

constexpr int kRowsPerBlock = 4;   // rows per block of the (column, row) kernels
inline dim3 rc_grid(int rows) { return dim3(unsigned((rows + kRowsPerBlock - 1) / kRowsPerBlock)); }
inline dim3 rc_block() { return dim3(kMlpInPad, kRowsPerBlock); }

// Standardized targets (loglik ll[r ll_stride], gradient grad[r g_stride + k]),
// weighted squared error per row, and
// dY = bf16(2 w_j (y - t) / n) (+ its transpose); padding rows and columns get 0.
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ ll, int ll_stride,
                       const float* __restrict__ grad, int g_stride, const float* __restrict__ base,
                       const float* __restrict__ gbase, int64_t n, int rows, Norm nm,
                       __nv_bfloat16* __restrict__ dy, __nv_bfloat16* __restrict__ dyt, int pitch,
                       float* __restrict__ row_loss) {
    // one thread per (row, output j): block (64 outputs, 4 rows)
    __shared__ float term[kRowsPerBlock][kMlpOutPad];
    const int j = threadIdx.x, ty = threadIdx.y;
    const int r = blockIdx.x * blockDim.y + ty;
    const bool live = r < rows;
    float d = 0.0f, sq = 0.0f;
    if (live && r < n && j < kMlpOut) {
        const float b0 = base ? base[r] : 0.0f;
        const float bj = (gbase && j > 0) ? gbase[int64_t(r) * kMlpIn + (j - 1)] : 0.0f;
        const float t = (j == 0) ? (ll[int64_t(r) * ll_stride] - b0 - nm.ym) / nm.ys
                                 : (grad[int64_t(r) * g_stride + (j - 1)] - bj) * nm.xs[j - 1] / nm.ys;
        const float e = y[int64_t(r) * kMlpOutPad + j] - t;
        sq = nm.w[j] * e * e;
        d = 2.0f * nm.w[j] * e / float(n);
    }
    if (live) {
        const __nv_bfloat16 b = __float2bfloat16_rn(d);
        dy[int64_t(r) * kMlpOutPad + j] = b;
        dyt[int64_t(j) * pitch + r] = b;
    }
    term[ty][j] = sq;
    __syncthreads();
    if (live && j == 0) {   // the row's loss, summed over j in order
        float acc = 0.0f;
        for (int jj = 0; jj < kMlpOutPad; ++jj) acc += term[ty][jj];
        row_loss[r] = (r < n) ? acc : 0.0f;
    }
}

// loss = sum_r row_loss[r] / n in a fixed order: one block of 1024 threads,
// thread t sums rows t, t + 1024, ..., then a fixed binary tree.
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(kSumThreads) k_loss_sum(const float* __restrict__ row_loss, int rows,
                                                          int64_t n, float* __restrict__ out) {
    __shared__ float part[kSumThreads];
    float s = 0.0f;
    for (int r = threadIdx.x; r < rows; r += kSumThreads) s += row_loss[r];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0] / float(n);
}

// Column sums (bias gradients) in two fixed-order levels.  k_colsum_part:
// block (x, ch) takes 32 columns of row chunk ch (rows / kColChunks rows);
// thread (c, p) sums that chunk's rows p, p + 32, ... of column c and the 32
// phase sums are added in phase order into part[ch][c].  The optimizer adds
// the kColChunks chunk sums in chunk order.  Grid (cols / 32, kColChunks).
__device__ __forceinline__ float as_float(float v) { return v; }
__device__ __forceinline__ float as_float(__nv_bfloat16 v) { return __bfloat162float(v); }

constexpr int kColChunks = 16;   // rows is a multiple of 128, so every chunk has >= 8 rows

template <class T>
__global__ void __launch_bounds__(1024) k_colsum_part(const T* __restrict__ m, int rows, int cols,
                                                      float* __restrict__ part) {
    __shared__ float ph_sum[32][33];
    const int tx = threadIdx.x & 31, ph = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    const int rc = rows / kColChunks, r0 = blockIdx.y * rc;
    float s = 0.0f;
    if (c < cols)
        for (int r = ph; r < rc; r += 32) s += as_float(m[int64_t(r0 + r) * cols + c]);
    ph_sum[ph][tx] = s;
    __syncthreads();
    if (ph == 0 && c < cols) {
        float t = 0.0f;
        for (int k = 0; k < 32; ++k) t += ph_sum[k][tx];
        part[int64_t(blockIdx.y) * cols + c] = t;
    }
}

// Adam on every weight and bias of the network in one launch, one thread per
// parameter: weights first (layer by layer, row-major [N][K]), then biases.
// A weight's gradient is the fixed-order sum of its split-K partials
// (transposed partials for the last layer); a bias's, the fixed-order sum of
// its column's chunk sums (k_colsum_part), also kept in gb for inspection.
// The BF16 copies (and transposes) of the updated weights are written too.
struct AdamArgs {
    float* W[kMlpLayers];
    float* mW[kMlpLayers];
    float* vW[kMlpLayers];
    const float* part[kMlpLayers];
    __nv_bfloat16* w16[kMlpLayers];
    __nv_bfloat16* w16t[kMlpLayers];
    float* b[kMlpLayers];
    float* mb[kMlpLayers];
    float* vb[kMlpLayers];
    const float* bpart[kMlpLayers];
    float* gb[kMlpLayers];
    int N[kMlpLayers], K[kMlpLayers];   // layer l's outputs and inputs
    int64_t w_end[kMlpLayers];   // end of layer l's weights in the flat index
    int64_t b_end[kMlpLayers];   // end of layer l's biases (after all weights)
    int chunks;                  // split-K chunks of the weight gradients
    float lr, c1, c2;
};

__device__ __forceinline__ float adam_update(float& m, float& v, float g, float p, float lr, float c1,
                                             float c2) {
    const float mm = 0.9f * m + 0.1f * g;
    const float vv = 0.999f * v + 0.001f * g * g;
    m = mm;
    v = vv;
    return p - lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
}

__global__ void k_adam_all(AdamArgs a) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= a.b_end[kMlpLayers - 1]) return;
    if (idx < a.w_end[kMlpLayers - 1]) {
        int l = 0;
        while (idx >= a.w_end[l]) ++l;
        const int N = a.N[l], K = a.K[l];
        const int64_t j = idx - (l ? a.w_end[l - 1] : 0), stride = int64_t(N) * K;
        const int o = int(j / K), i = int(j % K);
        const int64_t pidx = (l == kMlpLayers - 1) ? int64_t(i) * N + o : j;
        float g = 0.0f;
        for (int c = 0; c < a.chunks; ++c) g += a.part[l][int64_t(c) * stride + pidx];
        float m = a.mW[l][j], v = a.vW[l][j];
        const float w = adam_update(m, v, g, a.W[l][j], a.lr, a.c1, a.c2);
        a.mW[l][j] = m;
        a.vW[l][j] = v;
        a.W[l][j] = w;
        const __nv_bfloat16 b16 = __float2bfloat16_rn(w);
        a.w16[l][j] = b16;
        a.w16t[l][int64_t(i) * N + o] = b16;
    } else {
        int l = 0;
        while (idx >= a.b_end[l]) ++l;
        const int N = a.N[l];
        const int i = int(idx - (l ? a.b_end[l - 1] : a.w_end[kMlpLayers - 1]));
        float g = 0.0f;
        for (int ch = 0; ch < kColChunks; ++ch) g += a.bpart[l][ch * N + i];
        a.gb[l][i] = g;
        float m = a.mb[l][i], v = a.vb[l][i];
        a.b[l][i] = adam_update(m, v, g, a.b[l][i], a.lr, a.c1, a.c2);
        a.mb[l][i] = m;
        a.vb[l][i] = v;
    }
}

// BF16 copies (and transposes) of the FP32 master weights.
__global__ void k_cast_w(const float* __restrict__ W, int N, int K, __nv_bfloat16* __restrict__ w16,
                         __nv_bfloat16* __restrict__ w16t) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * K) return;
    const int o = idx / K, i = idx % K;
    const __nv_bfloat16 b = __float2bfloat16_rn(W[idx]);
    w16[idx] = b;
    w16t[int64_t(i) * N + o] = b;
}

// dY = one-hot on the value output (1 in column 0 of real rows), for
// back-propagating the value head to the inputs.
__global__ void k_seed_value(int64_t n, int rows, __nv_bfloat16* __restrict__ dy) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int j = 0; j < kMlpOutPad; ++j)
        dy[int64_t(r) * kMlpOutPad + j] = __float2bfloat16_rn((j == 0 && r < n) ? 1.0f : 0.0f);
}

// Value and its exact input gradient: ll = y0 ys + ym (+ base),
// grad_k = dx0_k ys / xs_k (+ gbase), dx0 = d y0 / d(standardized input).
__global__ void k_destandardize_bp(const float* __restrict__ y, const float* __restrict__ dx0,
                                   int64_t n, Norm nm, const float* __restrict__ base,
                                   const float* __restrict__ gbase, float* __restrict__ ll,
                                   float* __restrict__ grad) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= n) return;
    ll[r] = y[r * kMlpOutPad] * nm.ys + nm.ym + (base ? base[r] : 0.0f);
    for (int k = 0; k < kMlpIn; ++k)
        grad[r * kMlpIn + k] = dx0[r * kMlpInPad + k] * nm.ys / nm.xs[k] +
                               (gbase ? gbase[r * kMlpIn + k] : 0.0f);
}

// Quadratic baseline of the log-likelihood in the network's input coordinates:
// base = -1/2 u^T H u, gbase = -H u (H symmetric [47][47]; all zero = no baseline).
// One thread per (row, i) forms (H u)_i; thread i == 0 then sums q over i in order.
// Block (64, 4 rows), grid ceil(n / 4).
__global__ void k_baseline(const float* __restrict__ u, int64_t n, const float* __restrict__ H,
                           float* __restrict__ base, float* __restrict__ gbase) {
    __shared__ float hus[4][kMlpInPad];
    const int i = threadIdx.x, ty = threadIdx.y;
    const int64_t r = int64_t(blockIdx.x) * blockDim.y + ty;
    const bool live = r < n;
    const float* ur = u + r * kMlpIn;
    float hu = 0.0f;
    if (live && i < kMlpIn) {
        for (int j = 0; j < kMlpIn; ++j) hu = fmaf(H[i * kMlpIn + j], ur[j], hu);
        gbase[r * kMlpIn + i] = -hu;
    }
    hus[ty][i] = hu;
    __syncthreads();
    if (live && i == 0) {
        float q = 0.0f;
        for (int k = 0; k < kMlpIn; ++k) q = fmaf(ur[k], hus[ty][k], q);
        base[r] = -0.5f * q;
    }
}

// De-standardize: ll = y0 ys + ym, grad_k = y_{1+k} ys / xs_k.
// (plus the baseline, if any: base [n], gbase [n][47]).
__global__ void k_destandardize(const float* __restrict__ y, int64_t n, Norm nm,
                                const float* __restrict__ base, const float* __restrict__ gbase,
                                float* __restrict__ ll, float* __restrict__ grad) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float* yr = y + r * kMlpOutPad;
    ll[r] = yr[0] * nm.ys + nm.ym + (base ? base[r] : 0.0f);
    if (grad)
        for (int k = 0; k < kMlpIn; ++k)
            grad[r * kMlpIn + k] = yr[1 + k] * nm.ys / nm.xs[k] + (gbase ? gbase[r * kMlpIn + k] : 0.0f);
}

template <class T>
argus_status dalloc(T** p, size_t n) {
    SCK(cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T)));
    return ARGUS_OK;
}

}  // namespace

struct argus_surrogate {
    int device = 0;
    int rows = 0;          // capacity (multiple of 128)
    int step = 0;
    Norm norm{};
    float* W[kMlpLayers] = {};
    float* b[kMlpLayers] = {};
    float* mW[kMlpLayers] = {};
    float* vW[kMlpLayers] = {};
    float* mb[kMlpLayers] = {};
    float* vb[kMlpLayers] = {};
    float* gb[kMlpLayers] = {};
    float* bpart[kMlpLayers] = {};   // [kColChunks][out]: the bias gradients' row-chunk sums
    float* part[kMlpLayers] = {};
    __nv_bfloat16* W16[kMlpLayers] = {};
    __nv_bfloat16* W16T[kMlpLayers] = {};
    // activations: H[0] = standardized input [rows][64], H[l] [rows][256]
    __nv_bfloat16* H[kMlpLayers] = {};
    __nv_bfloat16* HT[kMlpLayers] = {};
    float* Z[kMlpLayers] = {};      // Z[l] = pre-activation feeding H[l] (l = 1..4)
    float* Y = nullptr;
    __nv_bfloat16* dY = nullptr;
    __nv_bfloat16* dYT = nullptr;
    float* dZ32[2] = {};
    __nv_bfloat16* dZ16[2] = {};
    __nv_bfloat16* dZT[2] = {};
    float* row_loss = nullptr;
    float* Hq = nullptr;        // baseline precision matrix [47][47] (device)
    bool has_baseline = false;
    float* base = nullptr;      // [rows] baseline values of the current batch
    float* gbase = nullptr;     // [rows][47]
    int* err = nullptr;
    int last_chunks = 0;   // split-K chunks of the last training step
    // tensor maps
    CUtensorMap tmW[kMlpLayers], tmWT[kMlpLayers], tmH[kMlpLayers], tmHT[kMlpLayers];
    // the same with 64-row boxes: B operands of the training step's 64-column tiles
    CUtensorMap tmW64[kMlpLayers], tmWT64[kMlpLayers], tmHT64[kMlpLayers];
    CUtensorMap tmWT0_b64;   // W_0^T [64][256] with a 64-row box (B operand of dX0 = dZ1 W0)
    int grad_mode = 0;       // 0: gradient head; 1: back-propagated value head
    CUtensorMap tmdY, tmdYT, tmdZ16[2], tmdZT[2];
    MlpFusedMaps fmaps[3];   // weight maps of the fused kernel for clusters of 1, 2 and 4 CTAs
    int fused = 1;           // evaluate with the fused kernel (1) or layer by layer (0)
    int cluster = 0;         // fused kernel's CTAs per 128-row slab: 1, 2, 4 or 0 (automatic)
    // tests only (argus_selftest.h): the fused kernel's stage trace, and copies of
    // each layer's dZ that survive a training step (index l - 1 for dZ_l)
    float* tr_act = nullptr;
    float* tr_acc = nullptr;
    int64_t tr_rows = 0;
    float* keep_dz32[kMlpLayers - 1] = {};
    __nv_bfloat16* keep_dz16[kMlpLayers - 1] = {};
    int last_rows = 0;       // padded rows of the last training step
    float* loss_dev = nullptr;   // loss of the last argus_surrogate_train_step (packed form)
    // training: the weight-gradient GEMMs and bias sums of layer l run on a
    // side stream, forked after dZ_{l+1} is ready (ev_fork[l]) and joined
    // through ev_done[l], while the caller's stream goes on down the chain
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork[kMlpLayers] = {}, ev_done[kMlpLayers] = {};
};

namespace {

void free_all(argus_surrogate* s) {
    for (int l = 0; l < kMlpLayers; ++l) {
        cudaFree(s->W[l]); cudaFree(s->b[l]); cudaFree(s->mW[l]); cudaFree(s->vW[l]);
        cudaFree(s->mb[l]); cudaFree(s->vb[l]); cudaFree(s->gb[l]); cudaFree(s->part[l]);
        cudaFree(s->bpart[l]);
        cudaFree(s->W16[l]); cudaFree(s->W16T[l]); cudaFree(s->H[l]); cudaFree(s->HT[l]);
        cudaFree(s->Z[l]);
    }
    cudaFree(s->Y); cudaFree(s->dY); cudaFree(s->dYT); cudaFree(s->row_loss); cudaFree(s->err);
    cudaFree(s->Hq); cudaFree(s->base); cudaFree(s->gbase); cudaFree(s->loss_dev);
    for (int i = 0; i < 2; ++i) {
        cudaFree(s->dZ32[i]); cudaFree(s->dZ16[i]); cudaFree(s->dZT[i]);
    }
    for (int l = 0; l < kMlpLayers - 1; ++l) {
        cudaFree(s->keep_dz32[l]); cudaFree(s->keep_dz16[l]);
    }
    for (int l = 0; l < kMlpLayers; ++l) {
        if (s->ev_fork[l]) cudaEventDestroy(s->ev_fork[l]);
        if (s->ev_done[l]) cudaEventDestroy(s->ev_done[l]);
    }
    if (s->side) cudaStreamDestroy(s->side);
}

// Tests: copy dZ_l of the current training step (FP32 and BF16) to the kept buffers.
argus_status keep_dz(argus_surrogate* s, int l, int cur, int rows, cudaStream_t st) {
    if (!s->keep_dz32[0]) return ARGUS_OK;
    const size_t n = size_t(rows) * kMlpHidden;
    SCK(cudaMemcpyAsync(s->keep_dz32[l - 1], s->dZ32[cur], n * 4, cudaMemcpyDeviceToDevice, st));
    SCK(cudaMemcpyAsync(s->keep_dz16[l - 1], s->dZ16[cur], n * 2, cudaMemcpyDeviceToDevice, st));
    return ARGUS_OK;
}

argus_status build_maps(argus_surrogate* s) {
    const uint64_t R = uint64_t(s->rows);
    bool ok = true;
    for (int l = 0; l < kMlpLayers; ++l) {
        ok &= make_tmap_bf16(&s->tmW[l], s->W16[l], kOut[l], kIn[l], kOut[l] == 64 ? 64 : 128);
        ok &= make_tmap_bf16(&s->tmWT[l], s->W16T[l], kIn[l], kOut[l], 128);
        ok &= make_tmap_bf16(&s->tmH[l], s->H[l], R, kIn[l], 128);
        ok &= make_tmap_bf16(&s->tmHT[l], s->HT[l], kIn[l], R, kIn[l] == 64 ? 64 : 128);
        ok &= make_tmap_bf16(&s->tmW64[l], s->W16[l], kOut[l], kIn[l], 64);
        ok &= make_tmap_bf16(&s->tmWT64[l], s->W16T[l], kIn[l], kOut[l], 64);
        ok &= make_tmap_bf16(&s->tmHT64[l], s->HT[l], kIn[l], R, 64);
    }
    ok &= make_tmap_bf16(&s->tmWT0_b64, s->W16T[0], kIn[0], kOut[0], 64);
    for (int c = 0; c < 3; ++c) {   // cluster of 1 << c CTAs: each loads 1 / (1 << c) of the rows
        for (int l = 0; l < kMlpLayers; ++l)
            ok &= make_tmap_bf16(&s->fmaps[c].w[l], s->W16[l], kOut[l], kIn[l], kOut[l] >> c);
        for (int l = 0; l < kMlpLayers - 1; ++l)
            ok &= make_tmap_bf16(&s->fmaps[c].wt[l], s->W16T[l], kIn[l], kOut[l], kIn[l] >> c);
    }
    ok &= make_tmap_bf16(&s->tmdY, s->dY, R, kMlpOutPad, 128);
    ok &= make_tmap_bf16(&s->tmdYT, s->dYT, kMlpOutPad, R, 64);
    for (int i = 0; i < 2; ++i) {
        ok &= make_tmap_bf16(&s->tmdZ16[i], s->dZ16[i], R, kMlpHidden, 128);
        ok &= make_tmap_bf16(&s->tmdZT[i], s->dZT[i], kMlpHidden, R, 128);
    }
    return ok ? ARGUS_OK : sfail(ARGUS_ERR_CUDA, "cuTensorMapEncodeTiled refused a tensor map");
}

// Refresh BF16 copies from the FP32 master weights.
argus_status cast_weights(argus_surrogate* s, cudaStream_t st) {
    for (int l = 0; l < kMlpLayers; ++l) {
        const int n = kOut[l] * kIn[l];
        k_cast_w<<<(n + 255) / 256, 256, 0, st>>>(s->W[l], kOut[l], kIn[l], s->W16[l], s->W16T[l]);
    }
    SCK(cudaGetLastError());
    return ARGUS_OK;
}

// The fused kernel's arguments that come from the handle (rows and I/O are the caller's).
MlpFusedArgs fused_args(const argus_surrogate* s, bool with_grad) {
    MlpFusedArgs fa{};
    for (int k = 0; k < kMlpInPad; ++k) { fa.xm[k] = s->norm.xm[k]; fa.xs[k] = s->norm.xs[k]; }
    fa.ym = s->norm.ym;
    fa.ys = s->norm.ys;
    for (int l = 0; l < kMlpLayers; ++l) fa.bias[l] = s->b[l];
    for (int l = 0; l < kMlpLayers - 1; ++l) fa.gscr[l] = s->Z[l + 1];
    fa.w4 = s->W16[kMlpLayers - 1];
    fa.Hq = s->has_baseline ? s->Hq : nullptr;
    fa.mode = !with_grad ? kFusedValue : (s->grad_mode == 1 ? kFusedValueGrad : kFusedGradHead);
    fa.err = s->err;
    fa.tr_act = s->tr_act;
    fa.tr_acc = s->tr_acc;
    fa.tr_stride = s->tr_rows * kMlpHidden;
    return fa;
}

GemmEpiArgs epi_none() {
    GemmEpiArgs e{};
    return e;
}

// Forward over `rows` rows already standardized in H[0].  train: also save
// pre-activations and transposed activations for the backward pass.
argus_status forward(argus_surrogate* s, int rows, bool train, cudaStream_t st) {
    for (int l = 0; l < kMlpLayers; ++l) {
        GemmEpiArgs e = epi_none();
        e.bias = s->b[l];
        const int N = kOut[l], K = kIn[l];
        cudaError_t ce;   // 64-column tiles: 4 x more CTAs than 128-row slabs, each a quarter of the epilogue
        if (l < kMlpLayers - 1) {
            e.out_f32 = train ? s->Z[l + 1] : nullptr;
            e.ldo = N;
            e.out_bf16 = s->H[l + 1];
            e.ldb = N;
            e.out_bf16_t = train ? s->HT[l + 1] : nullptr;
            e.ldt = s->rows;
            ce = launch_gemm_tc(&s->tmH[l], &s->tmW64[l], rows, N, K, 64, 1, kEpiGelu, e, s->err, st);
        } else {
            e.out_f32 = s->Y;
            e.ldo = N;
            ce = launch_gemm_tc(&s->tmH[l], &s->tmW64[l], rows, N, K, 64, 1, kEpiF32, e, s->err, st);
        }
        if (ce != cudaSuccess) return scuda(ce, "forward GEMM");
    }
    return ARGUS_OK;
}

// d y0 / d(standardized input) for the rows of the last forward pass (which
// saved its pre-activations): back-propagate a one-hot dY on the value output
// through the four GELU layers and W_0.  Result in dZ32[1] as [rows][64].
argus_status value_input_grad(argus_surrogate* s, int64_t n, int rows, cudaStream_t st) {
    k_seed_value<<<(rows + 127) / 128, 128, 0, st>>>(n, rows, s->dY);
    GemmEpiArgs d = epi_none();
    d.zin = s->Z[4];
    d.ldz = kMlpHidden;
    d.out_bf16 = s->dZ16[0];
    d.ldb = kMlpHidden;
    cudaError_t ce = launch_gemm_tc(&s->tmdY, &s->tmWT64[4], rows, kMlpHidden, kMlpOutPad, 64, 1,
                                    kEpiGeluBwd, d, s->err, st);
    if (ce != cudaSuccess) return scuda(ce, "value backprop GEMM");
    int cur = 0;
    for (int l = kMlpLayers - 2; l >= 1; --l) {
        GemmEpiArgs g = epi_none();
        g.zin = s->Z[l];
        g.ldz = kMlpHidden;
        g.out_bf16 = s->dZ16[cur ^ 1];
        g.ldb = kMlpHidden;
        ce = launch_gemm_tc(&s->tmdZ16[cur], &s->tmWT64[l], rows, kMlpHidden, kMlpHidden, 64, 1,
                            kEpiGeluBwd, g, s->err, st);
        if (ce != cudaSuccess) return scuda(ce, "value backprop GEMM");
        cur ^= 1;
    }
    GemmEpiArgs x = epi_none();
    x.out_f32 = s->dZ32[1];
    x.ldo = kMlpInPad;
    ce = launch_gemm_tc(&s->tmdZ16[cur], &s->tmWT0_b64, rows, kMlpInPad, kMlpHidden, 64, 1, kEpiF32,
                        x, s->err, st);
    if (ce != cudaSuccess) return scuda(ce, "value backprop GEMM");
    return ARGUS_OK;
}

argus_status check_err(argus_surrogate* s) {
    int e = 0;
    SCK(cudaMemcpy(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        cudaMemset(s->err, 0, sizeof(int));
        return sfail(ARGUS_ERR_TIMEOUT, "a tensor-core GEMM wait timed out (code " + std::to_string(e) + ")");
    }
    return ARGUS_OK;
}

bool dev_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

argus_status train_step_impl(argus_surrogate* s, const float* theta, const float* loglik,
                             int ll_stride, const float* grad, int g_stride, int64_t n, float lr,
                             float* loss, cudaStream_t st);

}  // namespace

extern "C" {

int64_t argus_surrogate_param_count(void) {
    int64_t n = 0;
    for (int l = 0; l < kMlpLayers; ++l) n += int64_t(kOut[l]) * kIn[l] + kOut[l];
    return n;
}

argus_status argus_surrogate_create_ex(int32_t device, int32_t max_rows, uint64_t seed,
                                       argus_surrogate** out) {
    if (!out) return sfail(ARGUS_ERR_INVALID_ARG, "out is NULL");
    if (max_rows < 1 || max_rows > (1 << 20)) return sfail(ARGUS_ERR_INVALID_ARG, "max_rows out of range");
    int ndev = 0;
    SCK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return sfail(ARGUS_ERR_INVALID_ARG, "no such device");
    cudaDeviceProp prop{};
    SCK(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return sfail(ARGUS_ERR_UNSUPPORTED, std::string("built for sm_103a, device is ") + prop.name);
    DeviceGuardS guard(device);
    argus_surrogate* s = new argus_surrogate();
    s->device = device;
    s->rows = ((max_rows + 255) / 256) * 256;
    const size_t R = size_t(s->rows);
    const int max_chunks = s->rows / 128;
    argus_status st = ARGUS_OK;
    auto A = [&](argus_status x) { if (x && !st) st = x; };
    for (int l = 0; l < kMlpLayers; ++l) {
        const size_t nw = size_t(kOut[l]) * kIn[l];
        A(dalloc(&s->W[l], nw)); A(dalloc(&s->b[l], kOut[l]));
        A(dalloc(&s->mW[l], nw)); A(dalloc(&s->vW[l], nw));
        A(dalloc(&s->mb[l], kOut[l])); A(dalloc(&s->vb[l], kOut[l])); A(dalloc(&s->gb[l], kOut[l]));
        A(dalloc(&s->part[l], nw * max_chunks));
        A(dalloc(&s->bpart[l], size_t(kColChunks) * kOut[l]));
        A(dalloc(&s->W16[l], nw)); A(dalloc(&s->W16T[l], nw));
        A(dalloc(&s->H[l], R * kIn[l])); A(dalloc(&s->HT[l], R * kIn[l]));
        A(dalloc(&s->Z[l], R * kMlpHidden));
    }
    A(dalloc(&s->Y, R * kMlpOutPad));
    A(dalloc(&s->dY, R * kMlpOutPad)); A(dalloc(&s->dYT, R * kMlpOutPad));
    for (int i = 0; i < 2; ++i) {
        A(dalloc(&s->dZ32[i], R * kMlpHidden)); A(dalloc(&s->dZ16[i], R * kMlpHidden));
        A(dalloc(&s->dZT[i], R * kMlpHidden));
    }
    A(dalloc(&s->row_loss, R));
    A(dalloc(&s->Hq, size_t(kMlpIn) * kMlpIn));
    A(dalloc(&s->base, R));
    A(dalloc(&s->gbase, R * kMlpIn));
    A(dalloc(&s->err, 1));
    A(dalloc(&s->loss_dev, 1));
    if (!st) {
        // fan-in scaled normal weights from a seeded host generator (Box-Muller on splitmix64)
        std::vector<float> w;
        uint64_t x = seed ? seed : 0x9E3779B97F4A7C15ull;
        auto next = [&]() {
            x += 0x9E3779B97F4A7C15ull;
            uint64_t z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return double((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
        };
        for (int l = 0; l < kMlpLayers && !st; ++l) {
            const int N = kOut[l], K = kIn[l];
            const int fan_in = (l == 0) ? kMlpIn : K;
            const double sd = std::sqrt(2.0 / fan_in) * (l == kMlpLayers - 1 ? 0.5 : 1.0);
            w.assign(size_t(N) * K, 0.0f);
            for (int o = 0; o < N; ++o)
                for (int i = 0; i < K; ++i) {
                    const double u1 = std::max(next(), 1e-300), u2 = next();
                    const double g = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
                    const bool pad = (l == 0 && i >= kMlpIn) || (l == kMlpLayers - 1 && o >= kMlpOut);
                    w[size_t(o) * K + i] = pad ? 0.0f : float(g * sd);
                }
            if (cudaMemcpy(s->W[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemset(s->b[l], 0, N * 4) != cudaSuccess)
                st = sfail(ARGUS_ERR_CUDA, "initial weights");
        }
        for (int l = 0; l < kMlpLayers && !st; ++l) {
            const size_t nw = size_t(kOut[l]) * kIn[l];
            if (cudaMemset(s->mW[l], 0, nw * 4) || cudaMemset(s->vW[l], 0, nw * 4) ||
                cudaMemset(s->mb[l], 0, kOut[l] * 4) || cudaMemset(s->vb[l], 0, kOut[l] * 4))
                st = sfail(ARGUS_ERR_CUDA, "optimizer state");
        }
        if (!st && cudaMemset(s->err, 0, sizeof(int)) != cudaSuccess) st = sfail(ARGUS_ERR_CUDA, "err");
    }
    if (!st && cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess)
        st = sfail(ARGUS_ERR_CUDA, "side stream");
    for (int l = 0; l < kMlpLayers && !st; ++l)
        if (cudaEventCreateWithFlags(&s->ev_fork[l], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev_done[l], cudaEventDisableTiming) != cudaSuccess)
            st = sfail(ARGUS_ERR_CUDA, "training events");
    if (!st) st = build_maps(s);
    if (!st) st = cast_weights(s, nullptr);
    if (!st && cudaDeviceSynchronize() != cudaSuccess) st = sfail(ARGUS_ERR_CUDA, "create sync");
    if (st) {
        free_all(s);
        delete s;
        return st;
    }
    for (int k = 0; k < kMlpInPad; ++k) { s->norm.xm[k] = 0.0f; s->norm.xs[k] = 1.0f; }
    s->norm.ym = 0.0f; s->norm.ys = 1.0f;
    for (int j = 0; j < kMlpOut; ++j) s->norm.w[j] = 1.0f;
    *out = s;
    return ARGUS_OK;
}

void argus_surrogate_destroy(argus_surrogate* s) {
    if (!s) return;
    DeviceGuardS guard(s->device);
    cudaDeviceSynchronize();
    free_all(s);
    delete s;
}

argus_status argus_surrogate_set_normalizers(argus_surrogate* s, const float* x_mean,
                                             const float* x_std, float y_mean, float y_std,
                                             float value_weight, float grad_weight) {
    if (!s || !x_mean || !x_std) return sfail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < kMlpIn; ++k)
        if (!(x_std[k] > 0.0f) || !std::isfinite(x_mean[k]))
            return sfail(ARGUS_ERR_INVALID_ARG, "x_std must be > 0 and x_mean finite");
    if (!(y_std > 0.0f) || !std::isfinite(y_mean) || !(value_weight >= 0.0f) || !(grad_weight >= 0.0f))
        return sfail(ARGUS_ERR_INVALID_ARG, "bad value normalizer or loss weights");
    for (int k = 0; k < kMlpInPad; ++k) {
        s->norm.xm[k] = k < kMlpIn ? x_mean[k] : 0.0f;
        s->norm.xs[k] = k < kMlpIn ? x_std[k] : 1.0f;
    }
    s->norm.ym = y_mean;
    s->norm.ys = y_std;
    s->norm.w[0] = value_weight;
    for (int j = 1; j < kMlpOut; ++j) s->norm.w[j] = grad_weight;
    return ARGUS_OK;
}

argus_status argus_surrogate_set_baseline(argus_surrogate* s, const float* H) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    DeviceGuardS guard(s->device);
    if (!H) {
        s->has_baseline = false;
        return ARGUS_OK;
    }
    for (int i = 0; i < kMlpIn * kMlpIn; ++i)
        if (!std::isfinite(H[i])) return sfail(ARGUS_ERR_INVALID_ARG, "non-finite baseline matrix");
    SCK(cudaMemcpy(s->Hq, H, sizeof(float) * kMlpIn * kMlpIn, cudaMemcpyHostToDevice));
    s->has_baseline = true;
    return ARGUS_OK;
}

argus_status argus_surrogate_set_weights(argus_surrogate* s, const float* params) {
    if (!s || !params) return sfail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuardS guard(s->device);
    const float* p = params;
    for (int l = 0; l < kMlpLayers; ++l) {
        const size_t nw = size_t(kOut[l]) * kIn[l];
        SCK(cudaMemcpy(s->W[l], p, nw * 4, cudaMemcpyHostToDevice));
        p += nw;
        SCK(cudaMemcpy(s->b[l], p, kOut[l] * 4, cudaMemcpyHostToDevice));
        p += kOut[l];
        SCK(cudaMemset(s->mW[l], 0, nw * 4));
        SCK(cudaMemset(s->vW[l], 0, nw * 4));
        SCK(cudaMemset(s->mb[l], 0, kOut[l] * 4));
        SCK(cudaMemset(s->vb[l], 0, kOut[l] * 4));
    }
    s->step = 0;
    argus_status st = cast_weights(s, nullptr);
    if (st) return st;
    SCK(cudaDeviceSynchronize());
    return ARGUS_OK;
}

argus_status argus_surrogate_get_weights(argus_surrogate* s, float* params) {
    if (!s || !params) return sfail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuardS guard(s->device);
    SCK(cudaDeviceSynchronize());
    float* p = params;
    for (int l = 0; l < kMlpLayers; ++l) {
        const size_t nw = size_t(kOut[l]) * kIn[l];
        SCK(cudaMemcpy(p, s->W[l], nw * 4, cudaMemcpyDeviceToHost));
        p += nw;
        SCK(cudaMemcpy(p, s->b[l], kOut[l] * 4, cudaMemcpyDeviceToHost));
        p += kOut[l];
    }
    return ARGUS_OK;
}

argus_status argus_surrogate_eval(argus_surrogate* s, const float* theta, int64_t B, float* loglik,
                                  float* grad, void* stream) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    if (B < 0) return sfail(ARGUS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return ARGUS_OK;
    if (!theta || !loglik) return sfail(ARGUS_ERR_INVALID_ARG, "NULL theta or loglik");
    DeviceGuardS guard(s->device);
    if (!dev_ptr(theta) || !dev_ptr(loglik) || (grad && !dev_ptr(grad)))
        return sfail(ARGUS_ERR_INVALID_ARG, "argus_surrogate_eval needs device pointers");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (s->fused) {
        // one launch per max_rows rows: every layer (and the value output's
        // back-propagation) in one kernel; Z[1..4] hold gelu'(z) as scratch
        if (s->tr_act && B > s->tr_rows)
            return sfail(ARGUS_ERR_INVALID_ARG, "batch larger than the stage trace");
        MlpFusedArgs fa = fused_args(s, grad != nullptr);
        for (int64_t r0 = 0; r0 < B; r0 += s->rows) {
            fa.n = std::min<int64_t>(s->rows, B - r0);
            fa.theta = theta + r0 * kMlpIn;
            fa.loglik = loglik + r0;
            fa.grad = grad ? grad + r0 * kMlpIn : nullptr;
            if (s->tr_act) {
                fa.tr_act = s->tr_act + r0 * kMlpHidden;
                fa.tr_acc = s->tr_acc + r0 * kMlpHidden;
            }
            SCK(launch_mlp_fused(s->fmaps, fa, st, s->cluster));
        }
        return ARGUS_OK;
    }
    for (int64_t r0 = 0; r0 < B; r0 += s->rows) {
        const int64_t n = std::min<int64_t>(s->rows, B - r0);
        const int rows = int(((n + 127) / 128) * 128);
        k_standardize<<<rc_grid(rows), rc_block(), 0, st>>>(theta + r0 * kMlpIn, n, rows, s->norm,
                                                          s->H[0], nullptr, s->rows);
        const bool bp = grad && s->grad_mode == 1;
        argus_status e = forward(s, rows, bp, st);
        if (e) return e;
        if (s->has_baseline)
            k_baseline<<<rc_grid(int(n)), rc_block(), 0, st>>>(theta + r0 * kMlpIn, n, s->Hq,
                                                                 s->base, s->gbase);
        if (!bp) {
            k_destandardize<<<unsigned((n + 127) / 128), 128, 0, st>>>(
                s->Y, n, s->norm, s->has_baseline ? s->base : nullptr,
                s->has_baseline ? s->gbase : nullptr, loglik + r0, grad ? grad + r0 * kMlpIn : nullptr);
        } else {
            e = value_input_grad(s, n, rows, st);
            if (e) return e;
            k_destandardize_bp<<<unsigned((n + 127) / 128), 128, 0, st>>>(
                s->Y, s->dZ32[1], n, s->norm, s->has_baseline ? s->base : nullptr,
                s->has_baseline ? s->gbase : nullptr, loglik + r0, grad + r0 * kMlpIn);
        }
        SCK(cudaGetLastError());
    }
    return ARGUS_OK;
}

argus_status argus_surrogate_eval_f64(argus_surrogate* s, const double* z, const double* centre,
                                      double offset, int64_t B, double* loglik, double* grad,
                                      void* stream) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    if (B < 0) return sfail(ARGUS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return ARGUS_OK;
    if (!z || !centre || !loglik) return sfail(ARGUS_ERR_INVALID_ARG, "NULL z, centre or loglik");
    if (!std::isfinite(offset)) return sfail(ARGUS_ERR_INVALID_ARG, "offset must be finite");
    DeviceGuardS guard(s->device);
    if (!dev_ptr(z) || !dev_ptr(centre) || !dev_ptr(loglik) || (grad && !dev_ptr(grad)))
        return sfail(ARGUS_ERR_INVALID_ARG, "argus_surrogate_eval_f64 needs device pointers");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (s->tr_act && B > s->tr_rows)
        return sfail(ARGUS_ERR_INVALID_ARG, "batch larger than the stage trace");
    MlpFusedArgs fa = fused_args(s, grad != nullptr);
    fa.zc = centre;
    fa.off = offset;
    for (int64_t r0 = 0; r0 < B; r0 += s->rows) {
        fa.n = std::min<int64_t>(s->rows, B - r0);
        fa.z64 = z + r0 * kMlpIn;
        fa.ll64 = loglik + r0;
        fa.g64 = grad ? grad + r0 * kMlpIn : nullptr;
        if (s->tr_act) {
            fa.tr_act = s->tr_act + r0 * kMlpHidden;
            fa.tr_acc = s->tr_acc + r0 * kMlpHidden;
        }
        SCK(launch_mlp_fused(s->fmaps, fa, st, s->cluster));
    }
    return ARGUS_OK;
}

argus_status argus_surrogate_train_step_ex(argus_surrogate* s, const float* theta,
                                           const float* loglik, const float* grad, int64_t n,
                                           float lr, float* loss, void* stream) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    if (!theta || !loglik || !grad || !loss) return sfail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuardS guard(s->device);
    if (!dev_ptr(theta) || !dev_ptr(loglik) || !dev_ptr(grad) || !dev_ptr(loss))
        return sfail(ARGUS_ERR_INVALID_ARG, "argus_surrogate_train_step needs device pointers");
    return train_step_impl(s, theta, loglik, 1, grad, kMlpIn, n, lr, loss,
                           reinterpret_cast<cudaStream_t>(stream));
}

argus_status argus_surrogate_train_step(argus_surrogate* s, const float* x, const float* y, int64_t n,
                                        float lr, void* stream) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    if (!x || !y) return sfail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuardS guard(s->device);
    if (!dev_ptr(x) || !dev_ptr(y))
        return sfail(ARGUS_ERR_INVALID_ARG, "argus_surrogate_train_step needs device pointers");
    // y rows are (loglik, gradient[47]): strided views, no copy
    return train_step_impl(s, x, y, kMlpOut, y + 1, kMlpOut, n, lr, s->loss_dev,
                           reinterpret_cast<cudaStream_t>(stream));
}

argus_status argus_surrogate_last_loss(argus_surrogate* s, float* loss) {
    if (!s || !loss) return sfail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuardS guard(s->device);
    SCK(cudaDeviceSynchronize());
    SCK(cudaMemcpy(loss, s->loss_dev, sizeof(float), cudaMemcpyDeviceToHost));
    return ARGUS_OK;
}

}  // extern "C"

namespace {

argus_status train_step_impl(argus_surrogate* s, const float* theta, const float* loglik,
                             int ll_stride, const float* grad, int g_stride, int64_t n, float lr,
                             float* loss, cudaStream_t st) {
    if (n < 1 || n > s->rows)
        return sfail(ARGUS_ERR_INVALID_ARG, "n must be in 1..max_rows (rounded up to 256)");
    if (!(lr > 0.0f) || !std::isfinite(lr)) return sfail(ARGUS_ERR_INVALID_ARG, "lr must be > 0");
    const int rows = int(((n + 127) / 128) * 128);
    const int ck = (rows % 256 == 0) ? 256 : 128;   // K per split-K chunk over the batch
    const int chunks = rows / ck;
    k_standardize<<<rc_grid(rows), rc_block(), 0, st>>>(theta, n, rows, s->norm, s->H[0], s->HT[0],
                                                      s->rows);
    argus_status e = forward(s, rows, true, st);
    if (e) return e;
    if (s->has_baseline)
        k_baseline<<<rc_grid(int(n)), rc_block(), 0, st>>>(theta, n, s->Hq, s->base, s->gbase);
    k_loss<<<rc_grid(rows), rc_block(), 0, st>>>(s->Y, loglik, ll_stride, grad, g_stride,
                                               s->has_baseline ? s->base : nullptr,
                                               s->has_baseline ? s->gbase : nullptr, n, rows, s->norm,
                                               s->dY, s->dYT, s->rows, s->row_loss);
    k_loss_sum<<<1, kSumThreads, 0, st>>>(s->row_loss, rows, n, loss);
    // Layer l's weight gradient (split-K GEMM) and bias sums only read dZ_{l+1}
    // (dY for l = 4) and H_l, so they run on the side stream while this stream
    // forms dZ_l; dH_l may overwrite a ping-pong buffer only once the side
    // stream's reads of it (layer l + 2's) are done, and Adam joins them all.
    cudaStream_t sd = s->side;
    // If a call below fails after the fork, the caller's stream still waits
    // for whatever the side stream was given, so that no later work on it
    // overwrites buffers the side stream reads (the normal path joins below).
    struct SideJoin {
        cudaStream_t main, side;
        cudaEvent_t ev;
        bool pending = true;
        ~SideJoin() {
            if (pending && cudaEventRecord(ev, side) == cudaSuccess) cudaStreamWaitEvent(main, ev, 0);
        }
    } side_join{st, sd, s->ev_done[0]};
    // output layer: dW4^T = H4^T dY (split-K over rows), db4 = sum_r dY, dH4 = dY W4 -> dZ4
    {
        SCK(cudaEventRecord(s->ev_fork[4], st));
        SCK(cudaStreamWaitEvent(sd, s->ev_fork[4], 0));
        GemmEpiArgs g = epi_none();
        g.out_f32 = s->part[4];
        g.ldo = kMlpOutPad;
        g.chunk_stride = int64_t(kMlpHidden) * kMlpOutPad;
        cudaError_t ce = launch_gemm_tc(&s->tmHT[4], &s->tmdYT, kMlpHidden, kMlpOutPad, ck, 64, chunks,
                                        kEpiF32, g, s->err, sd);
        if (ce != cudaSuccess) return scuda(ce, "dW4 GEMM");
        k_colsum_part<__nv_bfloat16><<<dim3(kMlpOutPad / 32, kColChunks), 1024, 0, sd>>>(s->dY, rows, kMlpOutPad,
                                                                                      s->bpart[4]);
        SCK(cudaEventRecord(s->ev_done[4], sd));
        GemmEpiArgs d = epi_none();
        d.zin = s->Z[4];
        d.ldz = kMlpHidden;
        d.out_f32 = s->dZ32[0];
        d.ldo = kMlpHidden;
        d.out_bf16 = s->dZ16[0];
        d.ldb = kMlpHidden;
        d.out_bf16_t = s->dZT[0];
        d.ldt = s->rows;
        ce = launch_gemm_tc(&s->tmdY, &s->tmWT64[4], rows, kMlpHidden, kMlpOutPad, 64, 1, kEpiGeluBwd, d,
                            s->err, st);
        if (ce != cudaSuccess) return scuda(ce, "dH4 GEMM");
        if ((e = keep_dz(s, 4, 0, rows, st))) return e;
    }
    // hidden layers l = 3..0: cur holds dZ_{l+1}
    int cur = 0;
    for (int l = kMlpLayers - 2; l >= 0; --l) {
        const int K = kIn[l];
        GemmEpiArgs g = epi_none();
        g.out_f32 = s->part[l];
        g.ldo = K;
        g.chunk_stride = int64_t(kMlpHidden) * K;
        SCK(cudaEventRecord(s->ev_fork[l], st));
        SCK(cudaStreamWaitEvent(sd, s->ev_fork[l], 0));
        cudaError_t ce = launch_gemm_tc(&s->tmdZT[cur], &s->tmHT64[l], kMlpHidden, K, ck, 64,
                                        chunks, kEpiF32, g, s->err, sd);
        if (ce != cudaSuccess) return scuda(ce, "dW GEMM");
        k_colsum_part<float><<<dim3(kMlpHidden / 32, kColChunks), 1024, 0, sd>>>(s->dZ32[cur], rows, kMlpHidden,
                                                                              s->bpart[l]);
        SCK(cudaEventRecord(s->ev_done[l], sd));
        if (l > 0) {
            // buffer cur ^ 1 last held dZ_{l+2}, which layer l + 1's side work read
            if (l + 1 < kMlpLayers - 1) SCK(cudaStreamWaitEvent(st, s->ev_done[l + 1], 0));
            GemmEpiArgs d = epi_none();
            d.zin = s->Z[l];
            d.ldz = kMlpHidden;
            d.out_f32 = s->dZ32[cur ^ 1];
            d.ldo = kMlpHidden;
            d.out_bf16 = s->dZ16[cur ^ 1];
            d.ldb = kMlpHidden;
            d.out_bf16_t = s->dZT[cur ^ 1];
            d.ldt = s->rows;
            ce = launch_gemm_tc(&s->tmdZ16[cur], &s->tmWT64[l], rows, kMlpHidden, kMlpHidden, 64, 1,
                                kEpiGeluBwd, d, s->err, st);
            if (ce != cudaSuccess) return scuda(ce, "dH GEMM");
            cur ^= 1;
            if ((e = keep_dz(s, l, cur, rows, st))) return e;
        }
    }
    SCK(cudaStreamWaitEvent(st, s->ev_done[0], 0));   // the side stream ran layer 0's work last
    side_join.pending = false;
    s->last_chunks = chunks;
    s->last_rows = rows;
    // Adam
    s->step += 1;
    const float c1 = float(1.0 - std::pow(0.9, s->step));
    const float c2 = float(1.0 - std::pow(0.999, s->step));
    AdamArgs aa{};
    int64_t off = 0;
    for (int l = 0; l < kMlpLayers; ++l) {
        aa.W[l] = s->W[l]; aa.mW[l] = s->mW[l]; aa.vW[l] = s->vW[l]; aa.part[l] = s->part[l];
        aa.w16[l] = s->W16[l]; aa.w16t[l] = s->W16T[l];
        aa.b[l] = s->b[l]; aa.mb[l] = s->mb[l]; aa.vb[l] = s->vb[l]; aa.bpart[l] = s->bpart[l];
        aa.gb[l] = s->gb[l];
        aa.N[l] = kOut[l];
        aa.K[l] = kIn[l];
        off += int64_t(kOut[l]) * kIn[l];
        aa.w_end[l] = off;
    }
    for (int l = 0; l < kMlpLayers; ++l) {
        off += kOut[l];
        aa.b_end[l] = off;
    }
    aa.chunks = chunks; aa.lr = lr; aa.c1 = c1; aa.c2 = c2;
    k_adam_all<<<unsigned((off + 255) / 256), 256, 0, st>>>(aa);
    SCK(cudaGetLastError());
    return ARGUS_OK;
}

}  // namespace

extern "C" {

argus_status argus_surrogate_set_grad_mode(argus_surrogate* s, int32_t mode) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    if (mode != 0 && mode != 1) return sfail(ARGUS_ERR_INVALID_ARG, "mode must be 0 or 1");
    s->grad_mode = mode;
    return ARGUS_OK;
}

argus_status argus_surrogate_set_fused(argus_surrogate* s, int32_t on) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    if (on != 0 && on != 1) return sfail(ARGUS_ERR_INVALID_ARG, "on must be 0 or 1");
    s->fused = on;
    return ARGUS_OK;
}

argus_status argus_surrogate_set_cluster(argus_surrogate* s, int32_t ctas) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    if (ctas != 0 && ctas != 1 && ctas != 2 && ctas != 4)
        return sfail(ARGUS_ERR_INVALID_ARG, "ctas must be 0, 1, 2 or 4");
    s->cluster = ctas;
    return ARGUS_OK;
}

argus_status argus_surrogate_check(argus_surrogate* s) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    DeviceGuardS guard(s->device);
    SCK(cudaDeviceSynchronize());
    return check_err(s);
}

const char* argus_surrogate_last_error(void) { return g_sur_error.c_str(); }

// ---------------------------------------------------------------------------
// The surrogate of one array's log-likelihood, and its weights file.
// File layout (little-endian): 8 bytes "ARGUSNN1"; int32 version (1), number
// of parameters, input width (47), has_baseline; FP32 parameters (flat
// layout), x_mean[47], x_std[47], y_mean, y_std, value weight, gradient
// weight; FP32 H[47][47] if has_baseline.
// ---------------------------------------------------------------------------
namespace {

constexpr char kMagic[8] = {'A', 'R', 'G', 'U', 'S', 'N', 'N', '1'};
constexpr int32_t kFileVersion = 1;
constexpr int32_t kDefaultRows = 4096;
constexpr uint64_t kDefaultSeed = 20251013ull;

struct FileCloser {
    FILE* f;
    ~FileCloser() { if (f) fclose(f); }
};

}  // namespace

argus_status argus_surrogate_create(const argus_array* array, const char* weights_path_or_null,
                                    argus_surrogate** out) {
    if (!array || !out) return sfail(ARGUS_ERR_INVALID_ARG, "NULL array or out");
    const int32_t dim = argus_array_dim(array);
    if (dim != kMlpIn)
        return sfail(ARGUS_ERR_UNSUPPORTED,
                     "the network takes 47 inputs: a 20-pulsar array with random-walk red noise, "
                     "no pulsar term (this array has D = " + std::to_string(dim) + ")");
    std::vector<float> params, tail, H;
    int32_t has_baseline = 0;
    if (weights_path_or_null) {
        FileCloser fc{fopen(weights_path_or_null, "rb")};
        if (!fc.f) return sfail(ARGUS_ERR_INVALID_ARG, std::string("cannot open ") + weights_path_or_null);
        char magic[8];
        int32_t hdr[4];
        if (fread(magic, 1, 8, fc.f) != 8 || memcmp(magic, kMagic, 8) != 0 ||
            fread(hdr, sizeof(int32_t), 4, fc.f) != 4)
            return sfail(ARGUS_ERR_INVALID_ARG, "not an argus surrogate weights file");
        if (hdr[0] != kFileVersion || hdr[1] != argus_surrogate_param_count() || hdr[2] != kMlpIn ||
            (hdr[3] != 0 && hdr[3] != 1))
            return sfail(ARGUS_ERR_INVALID_ARG, "weights file: unsupported version or shape");
        has_baseline = hdr[3];
        params.resize(size_t(hdr[1]));
        tail.resize(2 * kMlpIn + 4);
        if (fread(params.data(), 4, params.size(), fc.f) != params.size() ||
            fread(tail.data(), 4, tail.size(), fc.f) != tail.size())
            return sfail(ARGUS_ERR_INVALID_ARG, "weights file is truncated");
        if (has_baseline) {
            H.resize(size_t(kMlpIn) * kMlpIn);
            if (fread(H.data(), 4, H.size(), fc.f) != H.size())
                return sfail(ARGUS_ERR_INVALID_ARG, "weights file is truncated");
        }
        for (float v : params)
            if (!std::isfinite(v)) return sfail(ARGUS_ERR_INVALID_ARG, "weights file holds a non-finite weight");
    }
    argus_surrogate* s = nullptr;
    argus_status st = argus_surrogate_create_ex(argus_array_device(array), kDefaultRows, kDefaultSeed, &s);
    if (st) return st;
    if (weights_path_or_null) {
        const float* t = tail.data();
        if (!st) st = argus_surrogate_set_weights(s, params.data());
        if (!st) st = argus_surrogate_set_normalizers(s, t, t + kMlpIn, t[2 * kMlpIn], t[2 * kMlpIn + 1],
                                                      t[2 * kMlpIn + 2], t[2 * kMlpIn + 3]);
        if (!st && has_baseline) st = argus_surrogate_set_baseline(s, H.data());
        if (st) {
            argus_surrogate_destroy(s);
            return st;
        }
    }
    *out = s;
    return ARGUS_OK;
}

argus_status argus_surrogate_save(argus_surrogate* s, const char* path) {
    if (!s || !path) return sfail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    std::vector<float> params(static_cast<size_t>(argus_surrogate_param_count()), 0.0f);
    argus_status st = argus_surrogate_get_weights(s, params.data());
    if (st) return st;
    std::vector<float> H;
    if (s->has_baseline) {
        DeviceGuardS guard(s->device);
        H.resize(size_t(kMlpIn) * kMlpIn);
        SCK(cudaMemcpy(H.data(), s->Hq, H.size() * 4, cudaMemcpyDeviceToHost));
    }
    std::vector<float> tail(2 * kMlpIn + 4);
    for (int k = 0; k < kMlpIn; ++k) {
        tail[k] = s->norm.xm[k];
        tail[kMlpIn + k] = s->norm.xs[k];
    }
    tail[2 * kMlpIn] = s->norm.ym;
    tail[2 * kMlpIn + 1] = s->norm.ys;
    tail[2 * kMlpIn + 2] = s->norm.w[0];
    tail[2 * kMlpIn + 3] = s->norm.w[1];
    const int32_t hdr[4] = {kFileVersion, int32_t(params.size()), kMlpIn, s->has_baseline ? 1 : 0};
    FileCloser fc{fopen(path, "wb")};
    if (!fc.f) return sfail(ARGUS_ERR_INVALID_ARG, std::string("cannot write ") + path);
    bool ok = fwrite(kMagic, 1, 8, fc.f) == 8 && fwrite(hdr, 4, 4, fc.f) == 4 &&
              fwrite(params.data(), 4, params.size(), fc.f) == params.size() &&
              fwrite(tail.data(), 4, tail.size(), fc.f) == tail.size() &&
              (H.empty() || fwrite(H.data(), 4, H.size(), fc.f) == H.size());
    ok = (fclose(fc.f) == 0) && ok;
    fc.f = nullptr;
    return ok ? ARGUS_OK : sfail(ARGUS_ERR_CUDA, std::string("write failed: ") + path);
}

argus_status argus_selftest_surrogate_trace(argus_surrogate* s, float* act, float* acc, int64_t rows) {
    if (!s) return sfail(ARGUS_ERR_INVALID_ARG, "surrogate handle is NULL");
    if (!act != !acc || (act && rows < 1)) return sfail(ARGUS_ERR_INVALID_ARG, "bad trace buffers");
    DeviceGuardS guard(s->device);
    if (act && (!dev_ptr(act) || !dev_ptr(acc)))
        return sfail(ARGUS_ERR_INVALID_ARG, "trace buffers must be device memory");
    s->tr_act = act;
    s->tr_acc = acc;
    s->tr_rows = act ? rows : 0;
    return ARGUS_OK;
}

argus_status argus_selftest_surrogate_keep(argus_surrogate* s, int32_t on) {
    if (!s || (on != 0 && on != 1)) return sfail(ARGUS_ERR_INVALID_ARG, "bad argument");
    DeviceGuardS guard(s->device);
    SCK(cudaDeviceSynchronize());
    for (int l = 0; l < kMlpLayers - 1; ++l) {
        cudaFree(s->keep_dz32[l]); cudaFree(s->keep_dz16[l]);
        s->keep_dz32[l] = nullptr; s->keep_dz16[l] = nullptr;
    }
    if (on) {
        const size_t n = size_t(s->rows) * kMlpHidden;
        for (int l = 0; l < kMlpLayers - 1; ++l) {
            argus_status st = dalloc(&s->keep_dz32[l], n);
            if (!st) st = dalloc(&s->keep_dz16[l], n);
            if (st) return st;
        }
    }
    return ARGUS_OK;
}

argus_status argus_selftest_surrogate_buffer(argus_surrogate* s, int32_t which, int32_t layer,
                                             void* host, int64_t bytes) {
    if (!s || !host) return sfail(ARGUS_ERR_INVALID_ARG, "NULL argument");
    if (s->last_rows < 1) return sfail(ARGUS_ERR_INVALID_ARG, "no training step yet");
    const size_t R = size_t(s->last_rows);
    const void* src = nullptr;
    size_t n = 0;
    switch (which) {
        case 0:
            if (layer < 0 || layer >= kMlpLayers) break;
            src = s->H[layer]; n = R * kIn[layer] * 2; break;
        case 1:
            if (layer < 1 || layer >= kMlpLayers) break;
            src = s->Z[layer]; n = R * kMlpHidden * 4; break;
        case 2: src = s->Y; n = R * kMlpOutPad * 4; break;
        case 3: src = s->dY; n = R * kMlpOutPad * 2; break;
        case 4:
            if (layer < 1 || layer >= kMlpLayers) break;
            src = s->keep_dz32[layer - 1]; n = R * kMlpHidden * 4; break;
        case 5:
            if (layer < 1 || layer >= kMlpLayers) break;
            src = s->keep_dz16[layer - 1]; n = R * kMlpHidden * 2; break;
        default: break;
    }
    if (!src) return sfail(ARGUS_ERR_INVALID_ARG, "no such buffer (or dZ not kept)");
    if (bytes != int64_t(n)) return sfail(ARGUS_ERR_INVALID_ARG, "byte count does not match");
    DeviceGuardS guard(s->device);
    SCK(cudaDeviceSynchronize());
    SCK(cudaMemcpy(host, src, n, cudaMemcpyDeviceToHost));
    return ARGUS_OK;
}

argus_status argus_selftest_surrogate_grads(argus_surrogate* s, float* grads) {
    if (!s || !grads || s->last_chunks < 1) return sfail(ARGUS_ERR_INVALID_ARG, "no training step yet");
    DeviceGuardS guard(s->device);
    SCK(cudaDeviceSynchronize());
    float* p = grads;
    for (int l = 0; l < kMlpLayers; ++l) {
        const int N = kOut[l], K = kIn[l];
        const size_t nw = size_t(N) * K;
        std::vector<float> part(nw * s->last_chunks);
        SCK(cudaMemcpy(part.data(), s->part[l], part.size() * 4, cudaMemcpyDeviceToHost));
        for (int o = 0; o < N; ++o)
            for (int i = 0; i < K; ++i) {
                const size_t pidx = (l == kMlpLayers - 1) ? size_t(i) * N + o : size_t(o) * K + i;
                float g = 0.0f;
                for (int c = 0; c < s->last_chunks; ++c) g += part[size_t(c) * nw + pidx];
                p[size_t(o) * K + i] = g;
            }
        p += nw;
        SCK(cudaMemcpy(p, s->gb[l], N * 4, cudaMemcpyDeviceToHost));
        p += N;
    }
    return ARGUS_OK;
}

}  // extern "C"
