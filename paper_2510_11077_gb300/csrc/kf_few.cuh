// K1 and K4 for batches of a few walkers (the time-parallel plan's): one
// block of four warps per walker, so that a walker's transcendentals run on
// the SM's four sub-partitions at once.  Declarations shared by the C-ABI
// layer and kf_project.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kf_internal.cuh"

namespace argus {

constexpr int64_t kFewMaxWalkers = 8;
constexpr int32_t kFewMaxPulsars = 256;   // shared memory: 96 B per pulsar

// Whether a batch is small enough for the few-walker kernels.
bool few_walkers(int64_t B, int32_t P);
// launch_project with the same arguments and outputs.
void launch_project_few(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                        double* lc, cudaStream_t s);
// launch_reduce with a gradient (grad != nullptr), the same arguments and outputs.
void launch_reduce_few(const double* theta, int64_t B, int32_t P, int32_t flags, const PulsarDev* psr,
                       const double* lane_out, double* loglik, double* grad, double* lane_ll,
                       cudaStream_t s);

}  // namespace argus
