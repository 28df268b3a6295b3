// Throughput microbenchmarks for the search kernel's roofline denominators.
//
// The search path is bound by plain arithmetic and on-chip loads, not by HBM or the
// tensor cores, so its peaks are those of the FP32 FMA pipe (lane FFMAs per second) and
// of shared-memory byte loads (lane loads per second).  Each kernel fills every SM with
// 256-thread blocks and gives every warp enough independent work to hide the pipe's
// latency; the rate is the best of three timed launches (CUDA events on the caller's
// stream).  Neither kernel writes memory in practice: each keeps its work live through
// a store guarded by a comparison the values never meet (in bounds either way).
#include <cuda_runtime.h>

#include <cstdint>

#include "gd_peak.h"

namespace gd {
namespace {

constexpr int kThreads = 256;
constexpr int kChains = 16;  // independent FMA chains per thread (latency 4, 4 schedulers)
constexpr int kUnroll = 8;   // FMA rounds per loop iteration: loop control < 2 % of issue

// x <- a x + b on kChains chains; with 0 < a < 1, b > 0 and positive starts every value
// stays in (0, b / (1 - a)], so the guard (negative) is never met.
__global__ void __launch_bounds__(kThreads) ffma_peak_kernel(float a, float b, int rounds, float guard,
                                                              float* out) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = __fmaf_rn((float)(threadIdx.x + j), 1.0e-3f, 1.0e-3f);
  for (int i = 0; i < rounds; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = __fmaf_rn(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s = __fadd_rn(s, x[j]);
  if (s == guard) out[0] = s;
}

constexpr int kLdsBytes = 4096;
constexpr int kLdsPerIter = 32;  // byte loads per thread per iteration, 32 B apart

// Lane t of a warp reads byte base + 32 u + t: the warp's 32 bytes sit in 8 banks, one
// wavefront per load.  base cycles through [0, 2048), so every address is below
// 2048 + 31 * 32 + 31 < kLdsBytes.  The byte sum stays below 2^32 for rounds < 2^19, so
// the guard (0xFFFFFFFF) is never met.
__global__ void __launch_bounds__(kThreads) lds_peak_kernel(int rounds, unsigned guard, unsigned* out) {
  __shared__ uint8_t buf[kLdsBytes];
  for (int i = threadIdx.x; i < kLdsBytes; i += kThreads) buf[i] = (uint8_t)(i * 7 + 3);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  unsigned acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
  for (int i = 0; i < rounds; ++i) {
    const uint8_t* p = buf + ((i * 64 + (threadIdx.x >> 5) * 256) & 2047) + lane;
#pragma unroll
    for (int u = 0; u < kLdsPerIter; u += 4) {
      acc0 += p[(u + 0) * 32];
      acc1 += p[(u + 1) * 32];
      acc2 += p[(u + 2) * 32];
      acc3 += p[(u + 3) * 32];
    }
  }
  if (acc0 + acc1 + acc2 + acc3 == guard) out[0] = acc0;
}

template <typename Launch>
cudaError_t best_of_three(cudaStream_t s, Launch launch, float* best_ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  *best_ms = 3.0e38f;
  launch();  // warm-up (clocks up, code loaded)
  for (int t = 0; t < 3 && e == cudaSuccess; ++t) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < *best_ms) *best_ms = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

cudaError_t measure_peaks(cudaStream_t s, double* ffma_per_s, double* lds_per_s) {
  int dev = 0, sms = 0, per_f = 0, per_l = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f, ffma_peak_kernel, kThreads, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_l, lds_peak_kernel, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_f < 1 || per_l < 1 || sms < 1) return cudaErrorInvalidConfiguration;
  void* out = nullptr;
  e = cudaMalloc(&out, 16);
  if (e != cudaSuccess) return e;
  const unsigned bf = (unsigned)(per_f * sms), bl = (unsigned)(per_l * sms);
  const int f_rounds = 8192, l_rounds = 8192;  // about 7 ms each on a 148-SM part at 2 GHz
  float ms = 0.f;
  e = best_of_three(s, [&] {
    ffma_peak_kernel<<<bf, kThreads, 0, s>>>(0.9999f, 1.0e-4f, f_rounds, -1.0f, static_cast<float*>(out));
  }, &ms);
  if (e == cudaSuccess && ffma_per_s)
    *ffma_per_s = (double)bf * kThreads * kChains * kUnroll * f_rounds / (ms * 1.0e-3);
  if (e == cudaSuccess)
    e = best_of_three(s, [&] {
      lds_peak_kernel<<<bl, kThreads, 0, s>>>(l_rounds, 0xFFFFFFFFu, static_cast<unsigned*>(out));
    }, &ms);
  if (e == cudaSuccess && lds_per_s) *lds_per_s = (double)bl * kThreads * kLdsPerIter * l_rounds / (ms * 1.0e-3);
  const cudaError_t ef = cudaFree(out);
  return e != cudaSuccess ? e : ef;
}

}  // namespace gd
