// FMA throughput microbenchmark: the measured denominator of the ALU roofline.
// Every thread runs NACC independent FMA chains (enough to cover the pipe latency)
// for `iters` rounds; the grid fills every SM several times over.  The result is
// stored only when it is impossible in practice (a value no chain reaches), so the
// compiler keeps the arithmetic.  binary32 uses the packed two-lane FMA, the form the
// objective kernels issue; binary64 the plain one.
#include "host.h"

namespace chisao {

constexpr int PEAK_NT = 256, PEAK_NACC = 8;

__global__ void __launch_bounds__(PEAK_NT) k_peak_f32(int iters, float seed, float* sink) {
  float2 acc[PEAK_NACC];
#pragma unroll
  for (int k = 0; k < PEAK_NACC; ++k) acc[k] = make_float2(seed + k, seed - k);
  const float2 a = make_float2(0.999999f, 1.000001f), b = make_float2(1e-7f, -1e-7f);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < PEAK_NACC; ++k) acc[k] = __ffma2_rn(acc[k], a, b);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PEAK_NACC; ++k) s += acc[k].x + acc[k].y;
  if (s == 1234.5678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_NT) k_peak_f64(int iters, double seed, double* sink) {
  double acc[PEAK_NACC];
#pragma unroll
  for (int k = 0; k < PEAK_NACC; ++k) acc[k] = seed + k;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < PEAK_NACC; ++k) acc[k] = fma(acc[k], 0.999999, 1e-7);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PEAK_NACC; ++k) s += acc[k];
  if (s == 1234.5678) sink[threadIdx.x] = s;
}

// FLOP/s (2 per FMA) of the chosen precision, timed with CUDA events on `st` after
// one untimed launch; blocks = 8 x the SM count.
cudaError_t measure_fma_peak(int f64, double* flops, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blocks = 8 * sms, iters = f64 ? 2000 : 40000;
  void* sink = nullptr;
  if ((e = cudaMalloc(&sink, PEAK_NT * sizeof(double))) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {         // the first launch is untimed
    if (rep == 1 && (e = cudaEventRecord(e0, st)) != cudaSuccess) break;
    if (f64)
      k_peak_f64<<<blocks, PEAK_NT, 0, st>>>(iters, 1.0, static_cast<double*>(sink));
    else
      k_peak_f32<<<blocks, PEAK_NT, 0, st>>>(iters, 1.0f, static_cast<float*>(sink));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return e;
  const double fmas = (double)blocks * PEAK_NT * iters * PEAK_NACC * (f64 ? 1.0 : 2.0);
  *flops = 2.0 * fmas / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace chisao
