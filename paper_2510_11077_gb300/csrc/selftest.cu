// Self-check entry points of the device arithmetic helpers (argus_selftest.h).
#include <string>

#include <cuda_runtime.h>

#include "../../include/argus_selftest.h"
#include "kf_math.cuh"

namespace {

using namespace argus;

__global__ void k_phase(const double* x, int64_t n, double* s, double* c, double* rs, double* rc) {
    __shared__ double2 tabd[kPhaseTable];
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

}  // extern "C"
