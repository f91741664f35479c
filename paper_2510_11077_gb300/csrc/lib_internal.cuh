// Host-side declarations shared by the library's entry points (not by the
// filter kernels): the last-error record, pulsar validation, the size limit
// of the joint filter, and the per-walker status launcher.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

struct argus_pulsar;

namespace argus {

// Stores msg as the calling thread's argus_last_error() and returns status.
int record_error(int status, const char* msg);

// Host validation of argus_pulsar data (argus_array_create's rules); returns
// an argus_status and the total TOA count.
int validate_pulsars(const argus_pulsar* psrs, int32_t n_pulsars, int64_t* total);

// Joint filter with a Hellings-Downs correlated GW background (gwb.cu):
// pulsars at most kGwbMaxPulsars (the 3P x 3P covariance lives in shared memory).
constexpr int kGwbMaxPulsars = 64;

// Per-walker status after a call (kf_project.cu): 0 finite log-likelihood,
// 1 theta outside the domain, 2 the filter met an innovation variance that is
// not a positive normal finite number; *any2 |= 1 if some walker has status 2.
// out and any2 may each be nullptr.
void launch_walker_flags(const double* theta, int64_t B, int32_t P, int32_t flags, const double* loglik,
                         int32_t* out, int* any2, cudaStream_t s);

}  // namespace argus
