// Calibration: the FP32 FMA throughput of the current device, measured.  The
// edge kernels are bound by the FP32 pipe, and their roofline is quoted
// against SMs x 128 lanes x 2 flops x the maximum clock; this kernel shows
// how much of that figure a pure FMA stream reaches on the machine at hand
// (its clocks and power state).  It has no counterpart in the paper.
#include <cuda_runtime.h>

#include "../../include/gtmp.h"

namespace {

constexpr int kCalThreads = 256;
constexpr int kChains = 8;   // independent FMA chains per thread (hide the pipe latency)
constexpr int kUnroll = 16;  // FMAs per chain per loop trip

__device__ float g_calib_sink;

__global__ void __launch_bounds__(kCalThreads) ffma_throughput_kernel(int trips, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = static_cast<float>(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) g_calib_sink = s;  // keeps every chain live; the values stay positive
}

}  // namespace

extern "C" {

GTMP_API gtmp_status gtmp_fp32_fma_peak(void* cuda_stream, double* tflops) {
  if (!tflops) return GTMP_ERR_INVALID_ARG;
  *tflops = 0.0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ffma_throughput_kernel, kCalThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return GTMP_ERR_CUDA;
  const int grid = sms * per_sm;
  const int trips = 2048;
  const double flops = 2.0 * kChains * kUnroll * static_cast<double>(trips) * kCalThreads * grid;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GTMP_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GTMP_ERR_CUDA;
  }
  const float a = 0.999999f, b = 1e-6f;  // x -> b / (1 - a) = 1: bounded, positive
  double best = 0.0;
  gtmp_status status = GTMP_OK;
  for (int rep = 0; rep < 8 && status == GTMP_OK; ++rep) {
    cudaEventRecord(e0, st);
    ffma_throughput_kernel<<<grid, kCalThreads, 0, st>>>(trips, a, b);
    cudaEventRecord(e1, st);
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      status = GTMP_ERR_CUDA;
      break;
    }
    if (rep >= 2 && ms > 0.0f) {  // the first launches warm the clocks up
      const double r = flops / (ms * 1e-3) / 1e12;
      best = r > best ? r : best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return status;
}

}  // extern "C"
