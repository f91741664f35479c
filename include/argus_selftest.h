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

/* out[i] = 1 / S[i] by the filter kernels' reciprocal: a double-float seed
 * formed on the FP32 and integer pipes, refined by one FP64 Newton-Raphson
 * step; S[i] must be normal. */
argus_status argus_selftest_rcp(const double* S, int64_t n, double* out);

/* out[i] = 1 / S[i] by the short-latency reciprocal of the time-parallel
 * scan and the joint filter: the FP64 approximate reciprocal refined by one
 * third-order step r (1 + e + e^2), e = 1 - S r; S[i] must be positive and
 * normal. */
argus_status argus_selftest_rcp3(const double* S, int64_t n, double* out);

/* *out = sum_i ln S[i] by the running mantissa product; *bad = 1 if some S[i]
 * is not a positive, normal, finite number. */
argus_status argus_selftest_logsum(const double* S, int64_t n, double* out, int32_t* bad);

/* Measured FP64 FMA issue rate of the current device: `launches` timed
 * launches (after one untimed warm-up) of one full wave of 256-thread blocks
 * (as many per SM as the variant's registers allow) whose threads each run
 * independent FMA chains a <- a x + y; variant 0: 8 chains, x and y
 * kernel parameters; 1: 8 chains, x and y per-thread registers; 2: 4 chains;
 * 3: 16 chains.  Every variant runs 8 x iters FMAs per thread.  dfma_per_s[l]
 * gets launch l's FMA instructions (thread-level) per second and ms[l] its
 * CUDA-event duration; a FLOP/s peak is 2 x that.  This is the FP64 roofline
 * the filter kernels are compared against. */
argus_status argus_selftest_dfma_rate(int64_t iters, int32_t launches, int32_t variant,
                                      double* dfma_per_s, float* ms);

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

/* Stage trace of the fused surrogate evaluation, for layer-by-layer parity
 * tests.  With device buffers act and acc of 9 x rows x 256 floats set, every
 * later fused evaluation of at most `rows` rows writes, for each of its nine
 * tensor-core GEMM stages st (0..3 hidden layers, 4 output layer, 5..8 the
 * value output's back-propagation, which runs only with the gradient in
 * mode 1): act[st][r][0..K) = the stage's BF16 A operand (the activations it
 * multiplies, as floats) and acc[st][r][0..N) = its FP32 accumulator before
 * any bias, N = 256, or 48 for stages 4 and 8.  NULL buffers switch the trace
 * off.  A batch of more than `rows` rows is then rejected. */
argus_status argus_selftest_surrogate_trace(struct argus_surrogate* s, float* act, float* acc,
                                            int64_t rows);

/* on = 1: later training steps keep each layer's dZ (FP32 and its BF16
 * rounding), which the step's ping-pong buffers would overwrite; on = 0 frees
 * the copies. */
argus_status argus_selftest_surrogate_keep(struct argus_surrogate* s, int32_t on);

/* Copy one buffer of the last training step to host memory; `bytes` must be its
 * exact size, with R = the step's rows padded to a multiple of 128:
 *   which 0: H_l, the BF16 input activations of layer l (0..4) as uint16 bit
 *            patterns [R][K_l] (K = 64 for l = 0, else 256);
 *   which 1: Z_l, the FP32 pre-activations feeding H_l (l = 1..4) [R][256];
 *   which 2: Y, the FP32 outputs [R][64];
 *   which 3: dY, the BF16 loss gradient of the outputs, uint16 [R][64];
 *   which 4: dZ_l = dL/dZ_l in FP32 [R][256] (l = 1..4; needs keep);
 *   which 5: the BF16 rounding of dZ_l, uint16 [R][256] (l = 1..4; needs keep). */
argus_status argus_selftest_surrogate_buffer(struct argus_surrogate* s, int32_t which, int32_t layer,
                                             void* host, int64_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* ARGUS_SELFTEST_H */
