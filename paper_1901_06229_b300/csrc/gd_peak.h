// Pipe-peak microbenchmarks (gd_peak.cu).
#pragma once
#include <cuda_runtime.h>

namespace gd {
// Throughput microbenchmarks of the FP32 FMA pipe and of shared-memory byte loads on
// the current device, in lane operations per second (either pointer may be null).
cudaError_t measure_peaks(cudaStream_t s, double* ffma_per_s, double* lds_per_s);
}  // namespace gd
