// Arithmetic peaks of the device, measured: the FP32 and FP64 fused
// multiply-add rates that bound the pair and level-stencil kernels (their
// roofline denominators).  Not part of the method; a measurement tool.
#include <cuda_runtime.h>

#include "mls6_internal.h"

namespace mls6 {

constexpr int kPeakChains = 8;    // independent FMA chains per thread
constexpr int kPeakUnroll = 16;   // FMAs per chain per loop trip

// Each thread runs kPeakChains independent chains x <- x * m + b; m < 1 and
// b > 0 keep every value bounded and away from denormals, and the final
// comparison keeps the chains live without a store on the timed path.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ out, int trips, T m, T b) {
  T x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = T(threadIdx.x & 7) + T(k);
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) x[k] = fma(x[k], m, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += x[k];
  if (s == T(-1)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T> static int fma_peak(double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MLS6_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T* out = nullptr;
  const int blocks = sms * 8, threads = 256;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return MLS6_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // trips sized for ~20 ms at the nominal rate of each type
  const int trips = sizeof(T) == 8 ? 200 : 8000;
  const T m = T(0.999999), b = T(1e-3);
  k_fma_peak<T><<<blocks, threads>>>(out, trips, m, b);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_fma_peak<T><<<blocks, threads>>>(out, trips, m, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return MLS6_ERR_CUDA;
  const double flop = 2.0 * kPeakChains * kPeakUnroll * (double)trips * blocks * threads;
  *tflops = flop / (best * 1e-3) / 1e12;
  return MLS6_OK;
}

}  // namespace mls6

extern "C" int mls6_fma_peak(int precision, double* tflops) {
  if (!tflops) return MLS6_ERR_ARG;
  if (precision == MLS6_FP64) return mls6::fma_peak<double>(tflops);
  if (precision == MLS6_FP32) return mls6::fma_peak<float>(tflops);
  return MLS6_ERR_ARG;
}
