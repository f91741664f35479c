/*
 * argus.h -- C ABI of the GB300 (sm_103a) batched Kalman-filter likelihood of
 * pulsar-timing-array data.
 *
 * The paper (Functionality: "Kalman filter likelihood evaluation" and
 * "Sampler Integration") makes one call the core of the method: the
 * log-likelihood of the TOA data under a linear Gaussian state-space model,
 * evaluated by a Kalman filter in O(N), and its gradient, called by a
 * gradient-based sampler at every step.  This library evaluates that call for
 * a batch of B parameter vectors ("walkers") at once, one (walker, pulsar)
 * lane per CUDA thread, in FP64.
 *
 * Model, per pulsar p (paper, Functionality: "State-space model
 * construction"; the continuous-wave source of Future Directions):
 *   state x = (rho, y): timing residual [s] and fractional frequency deviation;
 *   d rho/dt = y,  dy/dt = xi(t),  <xi(t) xi(t')> = sigma_p^2 delta(t - t');
 *   r_k = rho(t_k) + s_p(t_k) + eps_k,  eps_k ~ N(0, EFAC_p^2 sigma_k^2 + EQUAD_p^2);
 *   x(t_1) ~ N(0, P0_p);
 *   s_p(t) = A sin(W t + Phi0) + B cos(W t + Phi0), the Earth term of a
 *   monochromatic gravitational wave projected on the pulsar direction.
 * ll(theta) = sum_p sum_k -1/2 (ln 2 pi + ln S_k + e_k^2 / S_k).
 * With Ornstein-Uhlenbeck red noise (ARGUS_NOISE_OU; paper, Functionality:
 * OU processes for pulsar-intrinsic red noise) the frequency deviation obeys
 * dy/dt = -gamma_p y + xi(t) instead, with one more parameter per pulsar.
 * With the wave's pulsar term (ARGUS_PULSAR_TERM; the source model of the
 * paper's cited prior work on pulsar terms) s_p(t) also subtracts the same
 * wave at the retarded time t - d_p (1 - n.c)/c, d_p the pulsar's distance:
 *   s_p(t) = A sin Phi + B cos Phi - A sin(Phi - L_p) - B cos(Phi - L_p),
 *   L_p = W d_p (1 - n.c) / c,  1 kpc / c = 1e3 (648000/pi) au / c.
 *
 * Parameter vector theta (row-major [B][D]):
 *   [log10 f_gw (Hz), Phi0 (rad), psi (rad), cos iota, sin delta, alpha (rad),
 *    log10 h0, then per pulsar (log10 sigma_p, EFAC_p)]  (D = 7 + 2P), or
 *   per pulsar (log10 sigma_p, log10 gamma_p [1/s], EFAC_p) with
 *   ARGUS_NOISE_OU (D = 7 + 3P); ARGUS_PULSAR_TERM appends d_p [kpc] to each
 *   pulsar's block (D = 7 + 3P or 7 + 4P).
 * Out-of-domain vectors (a non-finite entry, EFAC <= 0, d_p <= 0, |cos iota| > 1,
 * |sin delta| > 1) and filters that meet a non-positive or non-finite
 * innovation variance give loglik = -inf and a zero gradient for that walker.
 * -inf is the per-walker flag a sampler's accept test needs; argus_walker_flags
 * tells the two causes apart.  An out-of-domain vector is an ordinary
 * rejection (status ARGUS_OK); a filter failure in a call whose loglik is host
 * memory (which synchronises anyway) returns ARGUS_ERR_NONFINITE after writing
 * every output.
 *
 * Pointers: theta, loglik and grad may each be device memory or host memory
 * (pinned or pageable); the library asks CUDA which.  With device pointers a
 * call only enqueues work on `stream` and returns.  With any host pointer the
 * call stages through device buffers owned by the handle, and returns after
 * the stream has finished and the host outputs are written.  The caller owns
 * theta and the outputs; the handle owns the staged TOA data and all scratch.
 * Calls on one handle must not run concurrently from several host threads.
 */
#ifndef ARGUS_H
#define ARGUS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum argus_status {
    ARGUS_OK = 0,
    ARGUS_ERR_INVALID_ARG = 1,   /* rejected on the host before any launch */
    ARGUS_ERR_CUDA = 2,          /* a CUDA call failed; see argus_last_error() */
    ARGUS_ERR_OOM = 3,           /* device allocation failed */
    ARGUS_ERR_NONFINITE = 4,     /* a call with host outputs: some walker's filter met an
                                    innovation variance S_k that is not a positive normal
                                    finite number; its loglik is -inf, its gradient 0, and
                                    the other walkers' results are valid (asynchronous
                                    device-pointer calls: see argus_walker_flags) */
    ARGUS_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    ARGUS_ERR_UNSUPPORTED = 6    /* no sm_103a device, or a size beyond a documented limit */
} argus_status;

/* One pulsar as handed to argus_array_create (all host memory, copied). */
typedef struct argus_pulsar {
    int64_t n_toa;          /* >= 0 TOAs */
    const double* t;        /* [n_toa] TOA times, s from the array epoch, non-decreasing */
    const double* r;        /* [n_toa] timing residuals, s */
    const double* sigma;    /* [n_toa] TOA errors, s, finite and > 0 */
    double pos[3];          /* unit vector towards the pulsar (|pos| = 1 within 1e-6) */
    double equad;           /* EQUAD, s, >= 0 */
    double p0[3];           /* prior covariance of (rho, y): {rr, ry, yy}, positive semi-definite */
} argus_pulsar;

/* Opaque handle: device copies of the TOA data, scratch, plans, graphs. */
typedef struct argus_array argus_array;

/* How a batch is scheduled (paper: none -- this is the GPU's own choice).
 * mode ARGUS_MODE_BATCHED: all B x P lanes in one persistent launch fed by an
 *   atomic work counter over (pulsar, walker-tile) items sorted by TOA count,
 *   largest first; optionally replayed from a captured CUDA graph.
 * mode ARGUS_MODE_PLAIN: the same kernels launched once per parameter vector
 *   (B launches of P lanes each); the comparison point.
 * mode ARGUS_MODE_SCAN: for few lanes (a single parameter vector, a few
 *   pulsars), argus_loglik and argus_lane_loglik run the time-parallel
 *   filter: each lane's TOAs are cut into chunks of 32 x scan_elems, one warp
 *   per chunk, combined by an associative scan (Sarkka & Garcia-Fernandez
 *   2021) and finished by ordinary Kalman steps; O(N) work, O(scan_elems +
 *   log N) depth.  It costs ~10x the sequential filter's FP64 work, so it
 *   pays only while the sequential filter leaves the GPU idle.
 *   argus_loglik_grad in this mode runs the time-parallel adjoint: the
 *   reverse sweep's step is an affine map of the adjoint state, so the
 *   adjoint at the end of each thread's TOAs is a suffix scan of those maps
 *   (chunks as above), after which each thread runs the ordinary adjoint
 *   steps over its own TOAs.  Scratch: 48 B per TOA per lane for the tape
 *   (144 B with ARGUS_NOISE_OU), plus ~4 KB per chunk. */
enum { ARGUS_MODE_BATCHED = 0, ARGUS_MODE_PLAIN = 1, ARGUS_MODE_SCAN = 2 };
typedef struct argus_plan {
    int32_t mode;             /* ARGUS_MODE_BATCHED, ARGUS_MODE_PLAIN or ARGUS_MODE_SCAN */
    int32_t walkers_per_cta;  /* lanes of one pulsar per thread block: 32, 64, 128 or 256 */
    int32_t ctas_per_sm;      /* resident blocks per SM of the persistent grid, 1..16 */
    int32_t ckpt_stride;      /* adjoint checkpoint stride in TOAs; 0 = ceil(sqrt(N_p)) */
    int32_t use_graph;        /* 1: capture each (theta, B, outputs) call once, then replay */
    int32_t tape_cache;       /* adjoint: 0 = re-run each segment from its checkpoint (memory
                                 O(sqrt N) per lane); 1 = also keep every segment's tape in HBM
                                 during the forward pass and skip the re-run (memory O(N) per
                                 lane: 40 B per TOA per resident lane, 136 B with
                                 ARGUS_NOISE_OU) */
    int32_t scan_elems;       /* ARGUS_MODE_SCAN: TOAs per thread, 1..4096; 0 = chosen from the
                                 batch (about 4 warps per SM, at most the longest
                                 pulsar's TOAs / 32) */
    int32_t reserved;         /* must be 0 */
} argus_plan;

/* Copy n_pulsars pulsars to device `device` and build the handle.
 * Precomputes per TOA: dt_k = t_k - t_{k-1} (dt_1 = 0), dt^2/2, dt^3/3,
 * sigma_k^2.  Returns ARGUS_ERR_INVALID_ARG for unsorted times, non-positive
 * or non-finite errors, a non-unit position, a negative EQUAD, a prior that is
 * not positive semi-definite, or n_pulsars < 1; ARGUS_ERR_UNSUPPORTED if the
 * device is not sm_103; *out is set only on success. */
argus_status argus_array_create(const argus_pulsar* pulsars, int32_t n_pulsars, int32_t device,
                                argus_array** out);

/* Model flags: the red-noise model of the frequency deviation y, optionally
 * OR-ed with the wave's pulsar term. */
enum { ARGUS_NOISE_RANDOM_WALK = 0, ARGUS_NOISE_OU = 1, ARGUS_PULSAR_TERM = 2 };

/* argus_array_create with a choice of model.  ARGUS_NOISE_RANDOM_WALK is what
 * argus_array_create builds; with ARGUS_NOISE_OU the state transition over a
 * step dt is F = [[1, (1 - e^{-gamma dt})/gamma], [0, e^{-gamma dt}]] and the
 * process noise the exact covariance of the integrated OU increment;
 * | ARGUS_PULSAR_TERM adds the pulsar term.  ARGUS_ERR_INVALID_ARG for any
 * other bit; otherwise as argus_array_create. */
argus_status argus_array_create_ex(const argus_pulsar* pulsars, int32_t n_pulsars, int32_t device,
                                   int32_t model, argus_array** out);

/* Free everything the handle owns.  NULL is allowed.  Synchronises the device. */
void argus_array_destroy(argus_array* array);

/* D = 7 + kP, k = 2 (random walk) or 3 (OU), plus 1 with the pulsar term:
 * the length of one parameter vector; -1 for NULL. */
int32_t argus_array_dim(const argus_array* array);

/* The handle's model flags (ARGUS_NOISE_* | ARGUS_PULSAR_TERM); -1 for NULL. */
int32_t argus_array_model(const argus_array* array);

/* The CUDA device ordinal the handle lives on; -1 for NULL. */
int32_t argus_array_device(const argus_array* array);

/* Replace / read the scheduling plan.  set_plan validates every field and
 * drops captured graphs; get_plan copies the current plan into *plan. */
argus_status argus_array_set_plan(argus_array* array, const argus_plan* plan);
argus_status argus_array_get_plan(const argus_array* array, argus_plan* plan);

/* Array log-likelihood of B parameter vectors.
 * theta [B][D] doubles, loglik [B] doubles (device or host, see above).
 * B = 0 is a no-op.  stream: a cudaStream_t, or NULL for the legacy stream. */
argus_status argus_loglik(argus_array* array, const double* theta, int64_t B,
                          double* loglik, void* stream);

/* Log-likelihood and its gradient d loglik / d theta, [B][D] doubles, by a
 * reverse-mode adjoint sweep through the filter with forward states
 * checkpointed every ckpt_stride TOAs (default ceil(sqrt(N_p))). */
argus_status argus_loglik_grad(argus_array* array, const double* theta, int64_t B,
                               double* loglik, double* grad, void* stream);

/* Allocation-free variant of argus_loglik_grad.  The paper has no
 * counterpart: this exists for callers that must not allocate device memory
 * while they run -- e.g. code inside a framework that has already reserved
 * (nearly) all GPU memory for its own pool, where a cudaMalloc from this
 * library would fail or fragment that pool, or a sampler's hot loop where a
 * cudaMalloc/cudaFree (which may synchronise the device) is unacceptable.
 * Create the handle beforehand with argus_array_create (which does allocate);
 * this call then allocates nothing: all of its scratch (work counter and
 * items, lane constants, per-lane results, adjoint checkpoints and tape)
 * comes from one file-scope device array of 64 MiB that every GPU which
 * loads the library holds until the process exits.
 * theta [B][D], loglik [B] and grad [B][D] must be device memory (otherwise
 * ARGUS_ERR_INVALID_ARG); results equal argus_loglik_grad's.  A batch whose
 * scratch does not fit in 64 MiB (about 128 bytes per walker x pulsar lane,
 * plus at least one block's checkpoint and tape slot) is rejected with
 * ARGUS_ERR_UNSUPPORTED and a message giving the bytes needed.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current, and again after the device's context has
 * changed, e.g. after a device reset); make that first call before any stream
 * capture.  Every call shares the one array and leaves its contents behind;
 * calls whose work overlaps on the GPU (other streams, other host threads,
 * other handles on the same device) race on it and must be serialised by
 * the caller. */
argus_status argus_loglik_grad_noalloc(argus_array* array, const double* theta, int64_t B,
                                       double* loglik, double* grad, void* stream);

/* The model's continuous-wave timing residual, Earth term only,
 * s_p(t_k) = A sin(W t_k + Phi0) + B cos(W t_k + Phi0), at every TOA of the
 * array (whatever the handle's model flags), for one set of source
 * parameters theta_gw = [log10 f_gw, Phi0, psi, cos iota, sin delta, alpha,
 * log10 h0] (host, 7 doubles).  s: host array of sum_p N_p doubles in the
 * pulsars' order.  Synchronous.  For simulating or subtracting a source. */
argus_status argus_cw_signal(argus_array* array, const double* theta_gw, double* s);

/* Per-walker status of a finished call, for asynchronous callers (device
 * pointers theta [B][D], loglik [B] as the call wrote it, flags [B] int32):
 * flags[b] = 0 if loglik[b] is finite, 1 if theta_b lies outside the domain
 * above, 2 if theta_b is in the domain but the filter met an innovation
 * variance that is not a positive normal finite number (the
 * ARGUS_ERR_NONFINITE condition).  Enqueued on `stream`. */
argus_status argus_walker_flags(argus_array* array, const double* theta, int64_t B,
                                const double* loglik, int32_t* flags, void* stream);

/* Per-(walker, pulsar) terms, for inspection: lane_ll [B][P] doubles (device
 * or host) receives ll_p(theta_b).  Same rules as argus_loglik. */
argus_status argus_lane_loglik(argus_array* array, const double* theta, int64_t B,
                               double* lane_ll, void* stream);

/* Kernel timing, for measurement.  With timing enabled (default off) every
 * batched call records CUDA events around its three stages on its stream
 * (captured graphs include them); argus_array_get_timing waits for the last
 * call and writes its stage durations in milliseconds to ms[3] =
 * {projection (K1), filter (K2 or K3), reduction (K4)}.  Enabling or
 * disabling drops captured graphs.  ARGUS_ERR_INVALID_ARG if no timed call
 * has run since timing was enabled. */
argus_status argus_array_set_timing(argus_array* array, int32_t enable);
argus_status argus_array_get_timing(argus_array* array, float* ms);

/* Human-readable name of a status, and the message of the last error raised
 * on the calling host thread ("" if none). */
const char* argus_status_string(argus_status status);
const char* argus_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ARGUS_H */
