// Host-side declarations shared by the library's entry points (not by the
// filter kernels): the last-error record, pulsar validation, and the size
// limit of the joint filter.
#pragma once

#include <cstdint>

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

}  // namespace argus
