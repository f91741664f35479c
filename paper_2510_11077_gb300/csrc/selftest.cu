// Self-check entry points of the device arithmetic helpers (argus_selftest.h).
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

__global__ void k_rcp(const double* S, int64_t n, double* out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = rcp_nr(S[i]);
}

__global__ void k_logsum(const double* S, int64_t n, double* out, int* bad) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    LogProd lp;
    for (int64_t i = 0; i < n; ++i) lp.add(S[i]);
    *out = lp.value();
    *bad = int(lp.bad);
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
    if (n < 0 || (n > 0 && (!S || !out))) return ARGUS_ERR_INVALID_ARG;
    if (n == 0) return ARGUS_OK;
    const size_t bytes = size_t(n) * sizeof(double);
    DevBuf b;
    TRY(cudaMalloc(&b.p, 2 * bytes));
    double* d = static_cast<double*>(b.p);
    TRY(cudaMemcpy(d, S, bytes, cudaMemcpyHostToDevice));
    k_rcp<<<152, 256>>>(d, n, d + n);
    TRY(cudaGetLastError());
    TRY(cudaDeviceSynchronize());
    TRY(cudaMemcpy(out, d + n, bytes, cudaMemcpyDeviceToHost));
    return ARGUS_OK;
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
