// Measurement helper for the roofline denominators of the CUDA-core kernels (no counterpart
// in the paper): the fused multiply-add throughput of this GPU in FP64 or FP32.  Every
// thread runs eight independent FMA chains (enough to cover the FMA latency at full
// occupancy); eight blocks of 256 threads per SM.
#include <cuda_runtime.h>

#include "../../include/td.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  T s = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == T(-1)) out[blockIdx.x] = s;   // never true; keeps the chains live
}

template <typename T>
cudaError_t time_fma(int iters, cudaStream_t st, double* tflops) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  T* out = nullptr;
  if ((e = cudaMalloc(&out, sizeof(T) * 8 * nsm)) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = 8 * nsm, threads = 256;
  k_fma_peak<T><<<blocks, threads, 0, st>>>(out, iters, T(0.999999), T(1e-7));   // warm-up
  cudaEventRecord(e0, st);
  k_fma_peak<T><<<blocks, threads, 0, st>>>(out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e == cudaSuccess) *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  return e;
}

}  // namespace

extern "C" td_status td_measure_fma_peak(int32_t fp64, int32_t iters, double* tflops, void* stream) {
  if (!tflops || iters < 1) return TD_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t e = fp64 ? time_fma<double>(iters, st, tflops) : time_fma<float>(iters, st, tflops);
  return e == cudaSuccess ? TD_OK : TD_ERR_CUDA;
}
