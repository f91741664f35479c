// Self-check entry points of the device arithmetic helpers (argus_selftest.h).
#include <algorithm>
#include <string>

#include <cuda_runtime.h>

#include "../../include/argus_selftest.h"
#include "kf_math.cuh"
#include "mlp_internal.cuh"

namespace {

using namespace argus;

__global__ void k_phase(const double* x, int64_t n, double* s, double* c, double* rs, double* rc) {
    __shared__ longlong2 tabd[kPhaseTable];
    __shared__ float4 tabf[kPhaseTable];
    const PhaseTable tab{tabd, tabf};
    fill_phase_table(tab);
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        phase_sincos(x[i], tab, s[i], c[i]);
        sincospi(2.0 * x[i], &rs[i], &rc[i]);
    }
}

template <bool kShort>
__global__ void k_rcp(const double* S, int64_t n, double* out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = kShort ? rcp_nr3(S[i]) : rcp_nr(S[i]);
}

__global__ void k_logsum(const double* S, int64_t n, double* out, int* bad) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    LogProd lp;
    for (int64_t i = 0; i < n; ++i) lp.add(S[i]);
    *out = lp.value();
    *bad = int(lp.bad);
}

// FP64 FMA throughput probe: every thread runs C independent chains
// a <- a x + y (|x| < 1, so the values stay bounded) for `iters` rounds and
// stores the sum, so nothing is dead code.  With kRegOps the multiplier and
// addend are per-thread registers loaded from memory (the compiler cannot
// treat them as uniform constants); otherwise they are kernel parameters.
template <int C, bool kRegOps>
__global__ void __launch_bounds__(256) k_dfma(int64_t iters, double x, double y, double* out) {
    double a[C];
#pragma unroll
    for (int j = 0; j < C; ++j) a[j] = double(threadIdx.x + j);
    double xr = x, yr = y;
    if (kRegOps) {
        xr = out[threadIdx.x] * 0.0 + x;    // out is zeroed before the probe
        yr = out[threadIdx.x + 256] * 0.0 + y;
    }
#pragma unroll 4
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < C; ++j) a[j] = fma(a[j], xr, yr);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < C; ++j) s += a[j];
    out[int64_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

argus_status cuda_status(cudaError_t e) {
    return e == cudaSuccess ? ARGUS_OK
                            : (e == cudaErrorMemoryAllocation ? ARGUS_ERR_OOM : ARGUS_ERR_CUDA);
}

#define TRY(call)                                        \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_status(_e);   \
    } while (0)

}  // namespace

namespace {
template <bool kShort>
argus_status selftest_rcp(const double* S, int64_t n, double* out) {
    if (n < 0 || (n > 0 && (!S || !out))) return ARGUS_ERR_INVALID_ARG;
    if (n == 0) return ARGUS_OK;
    const size_t bytes = size_t(n) * sizeof(double);
    DevBuf b;
    TRY(cudaMalloc(&b.p, 2 * bytes));
    double* d = static_cast<double*>(b.p);
    TRY(cudaMemcpy(d, S, bytes, cudaMemcpyHostToDevice));
    k_rcp<kShort><<<152, 256>>>(d, n, d + n);
    TRY(cudaGetLastError());
    TRY(cudaDeviceSynchronize());
    TRY(cudaMemcpy(out, d + n, bytes, cudaMemcpyDeviceToHost));
    return ARGUS_OK;
}
}  // namespace

extern "C" {

argus_status argus_selftest_phase(const double* x, int64_t n, double* sin_out, double* cos_out,
                                  double* ref_sin, double* ref_cos) {
    if (n < 0 || (n > 0 && (!x || !sin_out || !cos_out || !ref_sin || !ref_cos)))
        return ARGUS_ERR_INVALID_ARG;
    if (n == 0) return ARGUS_OK;
    const size_t bytes = size_t(n) * sizeof(double);
    DevBuf b;
    TRY(cudaMalloc(&b.p, 5 * bytes));
    double* d = static_cast<double*>(b.p);
    TRY(cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice));
    k_phase<<<152, 256>>>(d, n, d + n, d + 2 * n, d + 3 * n, d + 4 * n);
    TRY(cudaGetLastError());
    TRY(cudaDeviceSynchronize());
    TRY(cudaMemcpy(sin_out, d + n, bytes, cudaMemcpyDeviceToHost));
    TRY(cudaMemcpy(cos_out, d + 2 * n, bytes, cudaMemcpyDeviceToHost));
    TRY(cudaMemcpy(ref_sin, d + 3 * n, bytes, cudaMemcpyDeviceToHost));
    TRY(cudaMemcpy(ref_cos, d + 4 * n, bytes, cudaMemcpyDeviceToHost));
    return ARGUS_OK;
}


argus_status argus_selftest_rcp(const double* S, int64_t n, double* out) {
    return selftest_rcp<false>(S, n, out);
}

argus_status argus_selftest_rcp3(const double* S, int64_t n, double* out) {
    return selftest_rcp<true>(S, n, out);
}

argus_status argus_selftest_logsum(const double* S, int64_t n, double* out, int32_t* bad) {
    if (n < 0 || !out || !bad || (n > 0 && !S)) return ARGUS_ERR_INVALID_ARG;
    const size_t bytes = size_t(n > 0 ? n : 1) * sizeof(double);
    DevBuf b;
    TRY(cudaMalloc(&b.p, bytes + 16));
    double* d = static_cast<double*>(b.p);
    if (n > 0) TRY(cudaMemcpy(d, S, size_t(n) * sizeof(double), cudaMemcpyHostToDevice));
    double* dout = reinterpret_cast<double*>(reinterpret_cast<char*>(b.p) + bytes);
    int* dbad = reinterpret_cast<int*>(dout + 1);
    k_logsum<<<1, 32>>>(d, n, dout, dbad);
    TRY(cudaGetLastError());
    TRY(cudaDeviceSynchronize());
    TRY(cudaMemcpy(out, dout, sizeof(double), cudaMemcpyDeviceToHost));
    int hb = 0;
    TRY(cudaMemcpy(&hb, dbad, sizeof(int), cudaMemcpyDeviceToHost));
    *bad = hb;
    return ARGUS_OK;
}

argus_status argus_selftest_dfma_rate(int64_t iters, int32_t launches, int32_t variant,
                                      double* dfma_per_s, float* ms) {
    if (iters < 1 || launches < 1 || variant < 0 || variant > 3 || !dfma_per_s || !ms)
        return ARGUS_ERR_INVALID_ARG;
    int dev = 0, n_sm = 0;
    TRY(cudaGetDevice(&dev));
    TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256;
    const int chains[4] = {8, 8, 4, 16};
    // one full wave: as many blocks per SM as the variant's registers allow
    int per_sm = 0;
    switch (variant) {
        case 0: TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma<8, false>, threads, 0)); break;
        case 1: TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma<8, true>, threads, 0)); break;
        case 2: TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma<4, false>, threads, 0)); break;
        default: TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma<16, false>, threads, 0)); break;
    }
    const int grid = n_sm * std::max(per_sm, 1);
    DevBuf b;
    TRY(cudaMalloc(&b.p, size_t(std::max(grid, 2)) * threads * sizeof(double)));
    TRY(cudaMemset(b.p, 0, size_t(std::max(grid, 2)) * threads * sizeof(double)));
    double* out = static_cast<double*>(b.p);
    // the same FMA count for every variant: rounds scale inversely with the chains
    const int64_t rounds = iters * 8 / chains[variant];
    auto launch = [&](int64_t r) {
        switch (variant) {
            case 0: k_dfma<8, false><<<grid, threads>>>(r, 0.999, 1e-3, out); break;
            case 1: k_dfma<8, true><<<grid, threads>>>(r, 0.999, 1e-3, out); break;
            case 2: k_dfma<4, false><<<grid, threads>>>(r, 0.999, 1e-3, out); break;
            default: k_dfma<16, false><<<grid, threads>>>(r, 0.999, 1e-3, out); break;
        }
    };
    launch(rounds / 8 + 1);   // warm-up
    TRY(cudaGetLastError());
    TRY(cudaDeviceSynchronize());
    TRY(cudaMemset(b.p, 0, size_t(std::max(grid, 2)) * threads * sizeof(double)));
    cudaEvent_t e0, e1;
    TRY(cudaEventCreate(&e0));
    TRY(cudaEventCreate(&e1));
    const double fmas = double(grid) * threads * double(chains[variant]) * double(rounds);
    for (int l = 0; l < launches; ++l) {
        cudaEventRecord(e0);
        launch(rounds);
        cudaEventRecord(e1);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_status(e);
        }
        ms[l] = t;
        dfma_per_s[l] = fmas / (double(t) * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ARGUS_OK;
}

argus_status argus_selftest_gemm(const uint16_t* A, const uint16_t* B, int32_t M, int32_t N,
                                 int32_t k_total, int32_t bn, int32_t chunks, float* C) {
    if (!A || !B || !C || M <= 0 || N <= 0 || chunks < 1 || k_total <= 0 || k_total % chunks ||
        M % 128 || (bn != 64 && bn != 128) || N % bn)
        return ARGUS_ERR_INVALID_ARG;
    const int K = k_total / chunks;
    if (K % 64 || K > 256) return ARGUS_ERR_INVALID_ARG;
    const size_t na = size_t(M) * k_total, nb = size_t(N) * k_total, nc = size_t(chunks) * M * N;
    DevBuf bufA, bufB, bufC, bufE;
    TRY(cudaMalloc(&bufA.p, na * 2));
    TRY(cudaMalloc(&bufB.p, nb * 2));
    TRY(cudaMalloc(&bufC.p, nc * 4));
    TRY(cudaMalloc(&bufE.p, sizeof(int)));
    TRY(cudaMemcpy(bufA.p, A, na * 2, cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(bufB.p, B, nb * 2, cudaMemcpyHostToDevice));
    TRY(cudaMemset(bufC.p, 0, nc * 4));
    TRY(cudaMemset(bufE.p, 0, sizeof(int)));
    CUtensorMap ta, tb;
    if (!make_tmap_bf16(&ta, bufA.p, uint64_t(M), uint64_t(k_total), 128) ||
        !make_tmap_bf16(&tb, bufB.p, uint64_t(N), uint64_t(k_total), uint32_t(bn)))
        return ARGUS_ERR_CUDA;
    GemmEpiArgs e{};
    e.out_f32 = static_cast<float*>(bufC.p);
    e.ldo = N;
    e.chunk_stride = int64_t(M) * N;
    TRY(launch_gemm_tc(&ta, &tb, M, N, K, bn, chunks, kEpiF32, e, static_cast<int*>(bufE.p), nullptr));
    TRY(cudaDeviceSynchronize());
    int err = 0;
    TRY(cudaMemcpy(&err, bufE.p, sizeof(int), cudaMemcpyDeviceToHost));
    TRY(cudaMemcpy(C, bufC.p, nc * 4, cudaMemcpyDeviceToHost));
    return err ? ARGUS_ERR_TIMEOUT : ARGUS_OK;
}

}  // extern "C"
