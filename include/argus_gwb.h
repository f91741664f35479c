/*
 * argus_gwb.h -- C ABI of the joint likelihood of a pulsar timing array with a
 * stochastic gravitational-wave background (GWB) whose per-pulsar signals are
 * coupled by the Hellings-Downs correlation, on the GB300 (sm_103a).
 *
 * Model (paper, Functionality: OU red noise and the GWB specified as linear
 * SDEs and compiled into one state-space model, Hellings-Downs correlations
 * in the covariance that couples the processes across pulsars; the corner
 * plot's parameters h_a, gamma_a, sigma_p, gamma_p, EFAC).  Per pulsar n the
 * state is (rho_n, y_n, a_n):
 *   d rho_n = (y_n + a_n) dt,
 *   d y_n = -gamma_p,n y_n dt + sigma_p,n dW_n       (independent per pulsar),
 *   d a_n = -gamma_a a_n dt + h_a dB_n,  <dB_n dB_m> = G_nm dt,
 *   G_nm = 3/2 x ln x - x/4 + 1/2, x = (1 - c_n.c_m)/2 (n != m),  G_nn = 1,
 *   r_k = rho_{n_k}(t_k) + eps_k,  eps_k ~ N(0, EFAC_n^2 sigma_k^2 + EQUAD_n^2).
 * At the array's earliest TOA (rho_n, y_n) ~ N(0, P0_n) and the a block is
 * stationary, N(0, h_a^2 G / (2 gamma_a)).  Every TOA of every pulsar updates
 * the joint 3P-dimensional state, in time order (ties: pulsar order, then TOA
 * order); the likelihood is the prediction-error decomposition.  The work per
 * TOA is O(P^2), so the likelihood is O(N P^2), not data-parallel over
 * pulsars: the kernel runs one thread block per parameter vector, with the
 * joint covariance in shared memory.
 *
 * Parameter vector theta (D = 2 + 3P doubles, row-major [B][D]):
 *   [log10 h_a [s^-1/2], log10 gamma_a [1/s], (log10 sigma_p, log10 gamma_p, EFAC_p) per pulsar].
 * Out-of-domain vectors (a non-finite entry, EFAC <= 0) and filters that meet
 * a non-positive or non-finite innovation variance give loglik = -inf.
 * theta and loglik may be device or host memory, as in argus.h.
 */
#ifndef ARGUS_GWB_H
#define ARGUS_GWB_H

#include <stdint.h>

#include "argus.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct argus_gwb argus_gwb;

/* Copy the pulsars (argus.h's argus_pulsar, validated the same way) to device
 * `device` and build the handle: the merged, time-ordered TOA stream and the
 * Hellings-Downs matrix of the pulsar positions.  ARGUS_ERR_UNSUPPORTED for
 * more than 64 pulsars or a device that is not sm_103. */
argus_status argus_gwb_create(const argus_pulsar* pulsars, int32_t n_pulsars, int32_t device,
                              argus_gwb** out);

/* Free the handle.  NULL is allowed. */
void argus_gwb_destroy(argus_gwb* gwb);

/* D = 2 + 3P; -1 for NULL. */
int32_t argus_gwb_dim(const argus_gwb* gwb);

/* Joint log-likelihood of B parameter vectors theta [B][D] -> loglik [B].
 * B = 0 is a no-op.  stream: a cudaStream_t, or NULL for the legacy stream. */
argus_status argus_gwb_loglik(argus_gwb* gwb, const double* theta, int64_t B, double* loglik,
                              void* stream);

/* The joint log-likelihood and its gradient d loglik / d theta [B][D], by a
 * reverse-mode adjoint sweep through the joint filter.  The likelihood pass
 * (the same kernel as argus_gwb_loglik, so loglik is identical) saves the
 * state (upper triangle of the covariance, mean and scale factors) every
 * L = ceil(sqrt(N)) TOAs; the reverse pass then takes one thread block per
 * vector and, segment by segment from the last, re-runs the segment writing
 * a tape entry per TOA (the state before it, the step's transition
 * coefficients with their gamma-derivatives and its predicted column) and
 * runs the adjoint steps backwards through it.  At most 48 pulsars (the
 * adjoint and two tape entries stay in shared memory; ARGUS_ERR_UNSUPPORTED
 * beyond).  Device scratch: per vector of a launch the checkpoints,
 * ceil(N / L) x (3P(3P+1)/2 + 4P + 1) doubles; per resident block one
 * segment's tape, L x (3P(3P+1)/2 + 21P + 18) doubles at most; vectors are
 * processed in launches of at most about 4 GB of checkpoints.  Out-of-domain
 * vectors get loglik = -inf and a zero gradient. */
argus_status argus_gwb_loglik_grad(argus_gwb* gwb, const double* theta, int64_t B, double* loglik,
                                   double* grad, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ARGUS_GWB_H */
