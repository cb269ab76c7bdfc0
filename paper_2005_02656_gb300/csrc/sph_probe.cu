// sph_measure_fp32_peak: the FP32 fused-multiply-add rate this GPU sustains,
// measured by the library's own kernel, as the denominator of the FP32-pipe
// roofline of the pair sums (the paper has no counterpart; it is a
// measurement utility).
//
// Every thread of a grid of (SMs x 8) blocks of 256 threads runs kChains
// independent chains of dependent FFMAs (enough independent work per warp to
// cover the pipeline latency) for `iters` iterations; the rate is
// 2 kChains iters threads / time, timed with CUDA events around the launch
// after one untimed launch.
#include <cuda_runtime.h>

#include "sph_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__device__ float g_probe_sink;  // written only if the chains reach a value they cannot reach

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, float seed) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed + 0.001f * (threadIdx.x + c);
  const float a = 0.9999f, b = 1.0e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == 12345.678f) g_probe_sink = s;  // keeps the chains live (they converge to ~8e-3)
}

}  // namespace

extern "C" int sph_measure_fp32_peak(double* tflops, sph_stream_t stream) {
  if (!tflops) return SPH_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return SPH_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = sms * 8, iters = 1 << 16;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fma_probe<<<blocks, kProbeThreads, 0, st>>>(iters, 1.0f);  // warm-up
    e = cudaEventRecord(e0, st);
  }
  if (e == cudaSuccess) {
    k_fma_probe<<<blocks, kProbeThreads, 0, st>>>(iters, 1.0f);
    e = cudaEventRecord(e1, st);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.0f) return SPH_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kProbeThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SPH_OK;
}
