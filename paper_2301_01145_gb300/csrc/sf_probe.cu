// sf_probe.cu -- measured FP32 FMA throughput of the current device.
//
// The register fast path of the solver is bound by FP32 instruction issue, so
// its roofline is quoted against the FP32 peak.  The nominal peak follows from
// the unit counts (SMs x 128 FP32 lanes x 2 flop per FMA x clock); this probe
// measures what a plain FMA stream reaches under the clocks and power limit
// of the moment: every thread runs 8 independent FMA chains, the grid fills
// every SM with 8 CTAs of 256 threads, and the launch is timed with CUDA
// events on the caller's stream.
#include <cuda_runtime.h>

#include "../../include/sailfish_gb300.h"

namespace {

__device__ float sf_probe_sink;

__global__ void __launch_bounds__(256) k_fma_probe(int iters, float seed) {
  float a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + (float)(threadIdx.x + c);
  const float m = 0.999999f, d = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fmaf(a[c], m, d);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == 1234.5f) sf_probe_sink = s;  // keeps the chains alive; practically never taken
}

}  // namespace

extern "C" sf_status sf_probe_fp32_fma(double *tflops, void *cuda_stream) {
  if (!tflops) return SF_ERR_ARG;
  *tflops = 0.0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SF_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SF_ERR_CUDA;
  const int grid = nsm * 8, threads = 256, iters = 1 << 19;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return SF_ERR_CUDA;
  }
  sf_status r = SF_OK;
  float ms = 0.f;
  k_fma_probe<<<grid, threads, 0, st>>>(iters / 8, 1.0f);  // warm-up
  if (cudaEventRecord(e0, st) != cudaSuccess) r = SF_ERR_CUDA;
  k_fma_probe<<<grid, threads, 0, st>>>(iters, 1.0f);
  if (r == SF_OK && cudaEventRecord(e1, st) != cudaSuccess) r = SF_ERR_CUDA;
  if (r == SF_OK && cudaGetLastError() != cudaSuccess) r = SF_ERR_CUDA;
  if (r == SF_OK && cudaEventSynchronize(e1) != cudaSuccess) r = SF_ERR_CUDA;
  if (r == SF_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = SF_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != SF_OK) return r;
  if (ms <= 0.f) return SF_ERR_CUDA;
  const double flops = 2.0 * 8.0 * (double)iters * (double)grid * (double)threads;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return SF_OK;
}
