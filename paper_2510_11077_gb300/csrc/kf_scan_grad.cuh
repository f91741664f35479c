// Time-parallel adjoint (the gradient in plan mode ARGUS_MODE_SCAN):
// declarations shared by the C-ABI layer and kf_scan.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kf_internal.cuh"

namespace argus {

// doubles per element of the reverse scan: X (4), c (2), Y0 (3), Y1 (3), Q (3)
constexpr int kAdjElem = 15;

struct ScanGradArgs {
    ScanArgs s;                  // the forward scan; s.lane_out is [1 + 7][P][B] here
    double* tape;                // [n_items][tape fields][32 E]: each step's quantities for
                                 // its adjoint (kScanTapeDoubles, or kScanTapeDoublesOU)
    double* tsuf;                // [n_items * 32][15]: each thread's inclusive suffix map
                                 // within its chunk (its own TOAs and every later thread's)
    double* ragg;                // [n_items][15]: each chunk's composed reverse map
    double* rpre;                // [n_items][15]: composition of all later chunks of the lane
    double* partg;               // [n_items][7]: the chunk's gradient sums
    unsigned long long* rdone;   // [B P]: per-lane counters of the last pass
};

// S1, S2 (as the log-likelihood), then G3 (forward steps with their tape, the
// log-likelihood, each thread's reverse map and the chunk's suffix scan), R2
// (suffix scan over the chunks of a lane) and R3 (each thread's adjoint
// steps from its exact end-of-segment adjoint; fixed-order sums) ->
// s.lane_out[0..7][P][B], the layout of K3.
void launch_filter_scan_grad(const ScanGradArgs& a, cudaStream_t s);

}  // namespace argus
