// peak.cu -- FMA-rate microbenchmark for the roofline of the ALU-bound kernels (not from the
// paper).  Every thread runs 16 independent chains of fused multiply-adds whose values stay
// bounded (x <- x * a + b with |a| < 1), so the pipe never waits on a dependency; the grid
// covers every SM several times.  The rate is 2 flop per FMA over the CUDA-event time, the
// best of three runs.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/pnmcc.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T a, T b, T* __restrict__ sink) {
  T x[16];
#pragma unroll
  for (int k = 0; k < 16; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) s += x[k];
  if (s == (T)-12345) sink[0] = s;  // keeps the chains live; never true for these inputs
}

template <typename T>
int measure(void* stream, double* tflops) {
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PNM_ECUDA;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return PNM_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = nsm * 8, threads = 256, iters = sizeof(T) == 8 ? 2048 : 32768;
  k_fma_peak<T><<<blocks, threads, 0, s>>>(iters, (T)0.999, (T)1e-3, sink);  // warm-up
  int rc = PNM_OK;
  double best = 0.0;
  for (int rep = 0; rep < 3 && rc == PNM_OK; rep++) {
    cudaEventRecord(e0, s);
    k_fma_peak<T><<<blocks, threads, 0, s>>>(iters, (T)0.999, (T)1e-3, sink);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = PNM_ECUDA;
    } else {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      double flop = 2.0 * 16.0 * (double)iters * (double)blocks * threads;
      best = std::max(best, flop / (ms * 1e-3) / 1e12);
    }
  }
  *tflops = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return rc;
}

}  // namespace

extern "C" int pnm_measure_fma_peak(int fp64, void* stream, double* tflops) {
  if (!tflops) return PNM_EINVAL;
  return fp64 ? measure<double>(stream, tflops) : measure<float>(stream, tflops);
}
