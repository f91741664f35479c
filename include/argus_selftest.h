/*
 * argus_selftest.h -- self-checks of the device arithmetic helpers used by
 * the filter kernels.  The paper has no counterpart: these expose, for tests
 * only, the GPU routines that replace FP64 transcendentals on the hot path so
 * that their accuracy can be measured against CUDA's own functions and
 * high-precision references.  All pointers are HOST memory; each call
 * allocates its own device buffers, runs on the legacy stream and
 * synchronises.  Errors: ARGUS_ERR_INVALID_ARG for NULL or n < 0,
 * ARGUS_ERR_CUDA / ARGUS_ERR_OOM from CUDA.
 */
#ifndef ARGUS_SELFTEST_H
#define ARGUS_SELFTEST_H

#include <stdint.h>

#include "argus.h"

#ifdef __cplusplus
extern "C" {
#endif

/* For each phase x[i] (cycles): the filter's sin/cos of 2 pi x (table node +
 * double-float correction, summed in 2^-62 fixed point) (sin_out, cos_out)
 * and CUDA's sincospi(2 x) (ref_sin, ref_cos), all [n]. */
argus_status argus_selftest_phase(const double* x, int64_t n, double* sin_out, double* cos_out,
                                  double* ref_sin, double* ref_cos);

/* out[i] = 1 / S[i] by the approximate reciprocal refined by one third-order
 * step r (1 + e + e^2), e = 1 - S r (the filter's 1/S); S[i] must be positive
 * and normal. */
argus_status argus_selftest_rcp(const double* S, int64_t n, double* out);

/* *out = sum_i ln S[i] by the running mantissa product; *bad = 1 if some S[i]
 * is not a positive, normal, finite number. */
argus_status argus_selftest_logsum(const double* S, int64_t n, double* out, int32_t* bad);

/* The tensor-core GEMM of the surrogate network, plain FP32 epilogue:
 * for each K-chunk z < chunks, C[z][m][n] = sum_k A[m][zK + k] B[n][zK + k]
 * with K = k_total / chunks.  A [M][k_total], B [N][k_total] as BF16 bit
 * patterns (uint16), C [chunks][M][N] FP32; M a multiple of 128, K a multiple
 * of 64 and <= 256, bn (64 or 128) divides N.  Returns ARGUS_ERR_TIMEOUT if a
 * bounded device-side wait gave up. */
argus_status argus_selftest_gemm(const uint16_t* A, const uint16_t* B, int32_t M, int32_t N,
                                 int32_t k_total, int32_t bn, int32_t chunks, float* C);

/* Gradient of the loss of the last argus_surrogate_train_step, in the flat
 * parameter layout of argus_surrogate.h (host array of
 * argus_surrogate_param_count() floats): the fixed-order sum of the split-K
 * weight partials and the bias column sums that the Adam update consumed. */
struct argus_surrogate;
argus_status argus_selftest_surrogate_grads(struct argus_surrogate* s, float* grads);

#ifdef __cplusplus
}
#endif

#endif /* ARGUS_SELFTEST_H */
