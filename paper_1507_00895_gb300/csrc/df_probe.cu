// Arithmetic peaks of the GPU that runs libdf, measured by FMA loops: the
// denominators of the roofline fractions of the ladder kernels (the FP64 LU
// runs on the FP64 pipe, the mixed-precision Gauss-Jordan sweeps on the FP32
// pipe).  Every thread runs kChains independent multiply-add chains so that
// the pipe, not the chain latency, bounds the loop; the grid fills every SM
// with 8 blocks of 256 threads.
#include <cstdio>

#include "df_internal.cuh"

namespace df {

constexpr int kChains = 8;
constexpr int kProbeIters = 4096;

template <int KIND>
__global__ void __launch_bounds__(256) peak_probe_kernel(float seed, float* __restrict__ sink) {
  if constexpr (KIND == 2) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (double)seed + c + threadIdx.x;
    const double m = 0.999999, b = 1e-7;
#pragma unroll 4
    for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678) sink[0] = (float)s;      // never true: keeps the loop
  } else if constexpr (KIND == 1) {
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + c, seed - c + threadIdx.x);
    const float2 m = make_float2(0.999999f, 0.999998f), b = make_float2(1e-7f, 2e-7f);
#pragma unroll 4
    for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = x2_fma(a[c], m, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
    if (s == 12345.678f) sink[0] = s;
  } else {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + c + threadIdx.x;
    const float m = 0.999999f, b = 1e-7f;
#pragma unroll 4
    for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678f) sink[0] = s;
  }
}

template <int KIND>
static cudaError_t time_probe(int blocks, float* sink, double* gflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) return e;
  peak_probe_kernel<KIND><<<blocks, 256>>>(1.0f, sink);   // warm-up (clocks up)
  float best = 1e30f;
  for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0);
    peak_probe_kernel<KIND><<<blocks, 256>>>(1.0f + rep, sink);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double per_fma = (KIND == 1) ? 4.0 : 2.0;   // flops per instruction: f32x2 holds two FMAs
  const double flops = (double)blocks * 256 * kProbeIters * kChains * per_fma;
  if (e == cudaSuccess) *gflops = flops / (best * 1e-3) / 1e9;
  return e;
}

}  // namespace df

extern "C" df_status df_peak_probe(int kind, double* gflops) {
  if (!gflops || kind < 0 || kind > 2) return DF_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DF_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DF_ERR_CUDA;
  float* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return DF_ERR_OOM;
  const int blocks = sms * 8;
  cudaError_t e;
  if (kind == 0) e = df::time_probe<0>(blocks, sink, gflops);
  else if (kind == 1) e = df::time_probe<1>(blocks, sink, gflops);
  else e = df::time_probe<2>(blocks, sink, gflops);
  cudaFree(sink);
  if (e != cudaSuccess) {
    fprintf(stderr, "libdf: df_peak_probe: %s\n", cudaGetErrorString(e));
    return DF_ERR_CUDA;
  }
  return DF_OK;
}
