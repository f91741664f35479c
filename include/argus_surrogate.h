/*
 * argus_surrogate.h -- C ABI of the learned surrogate of the array
 * log-likelihood and its gradient.
 *
 * The target path pairs the exact filter with a small network trained on the
 * exact filter's own evaluations and used as the first stage of a
 * delayed-acceptance sampler whose second stage, fallback and arbiter is the
 * exact FP64 filter (argus.h).  The paper's own sampler integration
 * (Functionality, "Sampler Integration") calls a likelihood and its gradient
 * at every step; the surrogate supplies a cheap approximation of both.
 *
 * Network: 47 -> 256 -> 256 -> 256 -> 256 -> 48, GELU (exact erf form) after
 * each hidden layer; BF16 weights and activations, FP32 accumulation on the
 * tensor cores (tcgen05, TMA-staged operands), FP32 master weights and Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  The 47 inputs are a 20-pulsar array's
 * parameter vector (7 source + 2 x 20 noise); the 48 outputs are the
 * log-likelihood and its 47 derivatives.  Inputs are standardized by
 * (x - x_mean) / x_std; the value output is (ll - y_mean) / y_std and output
 * 1 + k is dll/dx_k * x_std_k / y_std (the gradient in standardized units).
 *
 * Parameters, as one flat FP32 array of argus_surrogate_param_count() values:
 * for each layer l = 0..4, W_l row-major [N_l][K_l] then b_l [N_l], with
 * (K_l, N_l) = (64, 256), (256, 256), (256, 256), (256, 256), (256, 64); the
 * padding (input columns 47..63 of W_0, output rows 48..63 of W_4 and b_4) is
 * zero and stays zero.
 *
 * Device pointers throughout (ARGUS_ERR_INVALID_ARG otherwise); calls are
 * asynchronous on `stream` except create/destroy/set/get, which synchronise.
 */
#ifndef ARGUS_SURROGATE_H
#define ARGUS_SURROGATE_H

#include <stdint.h>

#include "argus.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct argus_surrogate argus_surrogate;

/* Number of FP32 parameters in the flat layout above. */
int64_t argus_surrogate_param_count(void);

/* The surrogate of one array's log-likelihood (the target path's call: a
 * network whose inputs are that array's parameter vectors): allocated on the
 * array's device for batches of up to 4096 rows.  The array must have
 * D = 47 (20 pulsars, random-walk red noise, no pulsar term), else
 * ARGUS_ERR_UNSUPPORTED.  weights_path_or_null: a file written by
 * argus_surrogate_save (weights, normalizers, loss weights and baseline),
 * or NULL for fan-in scaled normal weights from a fixed seed, zero biases and
 * identity normalizers.  ARGUS_ERR_INVALID_ARG for an unreadable, foreign,
 * truncated or non-finite file.  *out is set only on success; the array
 * handle is not retained. */
argus_status argus_surrogate_create(const argus_array* array, const char* weights_path_or_null,
                                    argus_surrogate** out);

/* The same with the device, the batch capacity (max_rows, rounded up to a
 * multiple of 256) and the initial weights' seed given directly.
 * ARGUS_ERR_UNSUPPORTED if the device is not sm_103. */
argus_status argus_surrogate_create_ex(int32_t device, int32_t max_rows, uint64_t seed,
                                       argus_surrogate** out);
void argus_surrogate_destroy(argus_surrogate* s);

/* Write the network (parameters, normalizers, loss weights and baseline) to
 * `path` in the format argus_surrogate_create reads: 8 bytes "ARGUSNN1",
 * int32 version 1, parameter count, input width 47, has_baseline, then FP32
 * parameters (flat layout), x_mean[47], x_std[47], y_mean, y_std, value
 * weight, gradient weight, and H[47][47] when has_baseline; little-endian.
 * Synchronises. */
argus_status argus_surrogate_save(argus_surrogate* s, const char* path);

/* Host arrays x_mean[47], x_std[47] (> 0); value mean/std (> 0); loss
 * weights of the value output and of each gradient output (>= 0). */
argus_status argus_surrogate_set_normalizers(argus_surrogate* s, const float* x_mean,
                                             const float* x_std, float y_mean, float y_std,
                                             float value_weight, float grad_weight);

/* Optional quadratic baseline in the network's input coordinates x:
 * ll(x) ~ net(x) - 1/2 x^T H x, grad ~ net_grad(x) - H x, with H a host
 * [47][47] row-major FP32 matrix (e.g. the inverse posterior covariance of a
 * Gaussian approximation, with x the offset from its mean).  The network then
 * only learns the residual: training targets have the baseline subtracted and
 * eval adds it back.  NULL removes the baseline. */
argus_status argus_surrogate_set_baseline(argus_surrogate* s, const float* H);

/* Copy all parameters from / to a host array in the flat layout.  set_weights
 * also resets the Adam state and step count. */
argus_status argus_surrogate_set_weights(argus_surrogate* s, const float* params);
argus_status argus_surrogate_get_weights(argus_surrogate* s, float* params);

/* Surrogate log-likelihood and gradient of B parameter vectors:
 * theta [B][47], loglik [B], grad [B][47] or NULL (FP32, device).  By default
 * one fused kernel evaluates every max_rows rows: each cluster of thread
 * blocks (argus_surrogate_set_cluster) takes 128 rows through all five layers,
 * and in grad mode 1 back through them to the input, with the activations in
 * shared memory and the weights streamed in by TMA layer by layer.  Its results equal the layer-by-layer path's up to
 * the rounding order of a few FP32 operations. */
argus_status argus_surrogate_eval(argus_surrogate* s, const float* theta, int64_t B, float* loglik,
                                  float* grad, void* stream);

/* argus_surrogate_eval in a sampler's FP64 coordinates, with no conversion
 * kernels around it: the network's input row is float(z[b] - centre) (z
 * [B][47], centre [47], FP64), loglik[b] = (double) surrogate loglik + offset
 * (-inf when not finite), grad [B][47] FP64 = the surrogate gradient
 * converted to double, or NULL.  Device pointers.  Always the fused kernel;
 * the same rounding as argus_surrogate_eval on float(z - centre) followed by
 * the conversions. */
argus_status argus_surrogate_eval_f64(argus_surrogate* s, const double* z, const double* centre,
                                      double offset, int64_t B, double* loglik, double* grad,
                                      void* stream);

/* Selects how argus_surrogate_eval runs: on = 1 (default) the fused kernel,
 * on = 0 one tensor-core GEMM launch per layer (the kernels training uses).
 * For comparison and measurement; both compute the same network. */
argus_status argus_surrogate_set_fused(argus_surrogate* s, int32_t on);

/* CTAs of the fused kernel per 128-row slab: 1, 2 or 4 (a thread-block
 * cluster whose CTAs each compute 1/ctas of every layer's columns and share
 * the activations through distributed shared memory), or 0 (default) for the
 * widest whose clusters all run at once -- 4 up to a few thousand rows, 1 for
 * batches that fill the GPU with single-CTA slabs.  For comparison and
 * measurement; the results differ only in the rounding order of the
 * quadratic baseline's sum. */
argus_status argus_surrogate_set_cluster(argus_surrogate* s, int32_t ctas);

/* One Adam step on a minibatch of n <= max_rows exact evaluations:
 * x [n][47] parameter vectors and y [n][1 + 47] their exact log-likelihood
 * followed by its gradient (FP32, device; the layout the exact filter's
 * outputs pack into).  The loss is the weighted mean squared error of the
 * standardized outputs; argus_surrogate_last_loss reads its value before the
 * step.  The step is ordered on `stream`: its weight-gradient products run on
 * a stream the handle owns, forked from `stream` after the work they read and
 * joined back into it before the weights change. */
argus_status argus_surrogate_train_step(argus_surrogate* s, const float* x, const float* y, int64_t n,
                                        float lr, void* stream);

/* The same with the targets in separate arrays, theta [n][47], loglik [n],
 * grad [n][47], and the loss written to *loss (device FP32) on the stream. */
argus_status argus_surrogate_train_step_ex(argus_surrogate* s, const float* theta,
                                           const float* loglik, const float* grad, int64_t n,
                                           float lr, float* loss, void* stream);

/* Synchronise and copy the loss of the last argus_surrogate_train_step to *loss (host). */
argus_status argus_surrogate_last_loss(argus_surrogate* s, float* loss);

/* Which gradient argus_surrogate_eval returns: mode 0 (default) = the 47
 * gradient outputs of the network; mode 1 = the exact input gradient of the
 * value output, by back-propagation through the network (one backward pass
 * per eval).  Mode 1 makes the surrogate a conservative field -- the gradient
 * of the density it reports -- which a Hamiltonian integrator needs to
 * conserve the surrogate's energy. */
argus_status argus_surrogate_set_grad_mode(argus_surrogate* s, int32_t mode);

/* Synchronise and report whether a bounded device-side wait of the tensor-core
 * kernels gave up since the last check (ARGUS_ERR_TIMEOUT; the flag is then
 * cleared).  Message of the last surrogate error on this host thread. */
argus_status argus_surrogate_check(argus_surrogate* s);
const char* argus_surrogate_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ARGUS_SURROGATE_H */
