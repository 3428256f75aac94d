// Gradient of the mean total log-probability from the virtual shots of the gradient pass.
//
// P(m) = sum_L p_{m,L} is affine in every mechanism rate (Sec. 2.4: each mechanism is one
// factor p^x (1-p)^(1-x) of the sum), so d log P / d p_j = (P_{x_j=1} - P_{x_j=0}) / P.
// Virtual shot (b, 0) decodes shot b at the given rates; (b, 1 + 2a + x) decodes it with
// the parameter object of the a-th mechanism forced to x.  All three are the decoder's
// (truncated) values; without truncation the result is the exact gradient.
#include <cmath>

#include "sweep.cuh"

namespace td {

__device__ __forceinline__ double total_of(const double* lp) {
  const double a = lp[0], c = lp[1];
  const double m = fmax(a, c);
  if (!(m > -INFINITY)) return -INFINITY;
  return m + log(exp(a - m) + exp(c - m));
}

// One thread per mechanism (gradient) and per shot (log P); shots summed in order.
__global__ void k_grad_combine(const double* __restrict__ vlogp, int64_t B, int32_t NV,
                               const int32_t* __restrict__ act, int32_t n_mech, double* __restrict__ logP,
                               double* __restrict__ grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) logP[i] = total_of(vlogp + i * NV * 2);
  if (i >= n_mech) return;
  const int a = act[i];
  double acc = 0.0;
  if (a >= 0)
    for (int64_t b = 0; b < B; ++b) {
      const double* v = vlogp + b * NV * 2;
      const double t = total_of(v);
      if (!(t > -INFINITY)) continue;   // a shot of probability 0 contributes nothing
      const double t0 = total_of(v + 2 * (1 + 2 * a));
      const double t1 = total_of(v + 2 * (2 + 2 * a));
      acc += exp(t1 - t) - exp(t0 - t);
    }
  grad[i] = B > 0 ? acc / (double)B : 0.0;
}

cudaError_t launch_grad_combine(const double* vlogp, int64_t B, int32_t NV, const int32_t* act, int32_t n_mech,
                                double* logP, double* grad, cudaStream_t st) {
  const int64_t n = B > n_mech ? B : n_mech;
  if (n == 0) return cudaSuccess;
  k_grad_combine<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(vlogp, B, NV, act, n_mech, logP, grad);
  return cudaGetLastError();
}

// Checkpoints of the reverse sweep: copies, for every shot b and site s, len[s] doubles from
// src + b * src_stride + src_off[s] to dst + b * dst_stride + dst_off[s] (the tables in device
// memory, [S] each).  One block per (site, shot).
__global__ void k_copy_sites(const double* __restrict__ src, int64_t src_stride, const int64_t* __restrict__ src_off,
                             double* __restrict__ dst, int64_t dst_stride, const int64_t* __restrict__ dst_off,
                             const int64_t* __restrict__ len) {
  const int s = blockIdx.x, b = blockIdx.y;
  const double* a = src + (int64_t)b * src_stride + src_off[s];
  double* c = dst + (int64_t)b * dst_stride + dst_off[s];
  for (int64_t i = threadIdx.x; i < len[s]; i += blockDim.x) c[i] = a[i];
}

// For every shot b, n doubles from src + b * src_stride + src_off to dst + b * dst_stride + dst_off.
__global__ void k_copy_rows(const double* __restrict__ src, int64_t src_stride, int64_t src_off,
                            double* __restrict__ dst, int64_t dst_stride, int64_t dst_off, int64_t n) {
  const int b = blockIdx.x;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dst[(int64_t)b * dst_stride + dst_off + i] =
      src[(int64_t)b * src_stride + src_off + i];
}

cudaError_t launch_copy_sites(const double* src, int64_t src_stride, const int64_t* src_off, double* dst,
                              int64_t dst_stride, const int64_t* dst_off, const int64_t* len, int S, int B,
                              cudaStream_t st) {
  if (S <= 0 || B <= 0) return cudaSuccess;
  k_copy_sites<<<dim3(S, B), 256, 0, st>>>(src, src_stride, src_off, dst, dst_stride, dst_off, len);
  return cudaGetLastError();
}

cudaError_t launch_copy_rows(const double* src, int64_t src_stride, int64_t src_off, double* dst, int64_t dst_stride,
                             int64_t dst_off, int64_t n, int B, cudaStream_t st) {
  if (n <= 0 || B <= 0) return cudaSuccess;
  k_copy_rows<<<B, 256, 0, st>>>(src, src_stride, src_off, dst, dst_stride, dst_off, n);
  return cudaGetLastError();
}

}  // namespace td
