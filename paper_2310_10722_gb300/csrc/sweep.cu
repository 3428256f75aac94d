// Layer absorption of the boundary sweep (Sec. 4) on the GPU: site-local operators, and
// for every two-site gate (1-p) I x I + p X x X on a bond (the natural split of Sec. 5.1)
// the simple-update truncation of that bond back to chi (Sec. 4): Gram pass (absorb.cu),
// truncation core (core.cu), update pass (absorb.cu).
//
// Gate as bond doubling: with k the gate's bit, Gamma'_X[sigma; ..., (b, k)] =
// Gamma_X[sigma ^ k mask_X; ..., b] and lambda'_(b,k) = lambda_b w_k, w = (1-p, p).  In the
// basis kappa = (k=0 +- k=1)/sqrt2 the Gram matrix of M'_X (Gamma'_X with the other bonds'
// lambdas absorbed) is block diagonal: G+ = sum Y Y^T, G- = sum Z Z^T over rows, where
// Y = M[sigma_lo] + M[sigma_hi], Z = M[sigma_lo] - M[sigma_hi] for each pair
// sigma_hi = sigma_lo ^ mask.  The core kernel turns the four blocks into R factors,
// forms the 2D x 2D core theta = R_A Lambda' R_B^T, takes its SVD and keeps <= chi values;
// the update applies Gamma_new[lo] = Y T+ + Z T-, Gamma_new[hi] = Y T+ - Z T-.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "sweep.cuh"

namespace td {

template <typename T>
__global__ void k_init(SweepArgs a, const LocalDesc* __restrict__ locals0, int S) {
  const int b = blockIdx.x;
  T* g = reinterpret_cast<T*>(a.gamma) + (int64_t)b * a.shot_elems;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const LocalDesc& d = locals0[s];
    for (int k = 0; k < d.P; ++k) g[d.off + k] = (k == 0) ? T(1) : T(0);
  }
  double* lam = a.lam + (int64_t)b * a.nbonds * a.chi;
  for (int w = threadIdx.x; w < a.nbonds * a.chi; w += blockDim.x) lam[w] = (w % a.chi == 0) ? 1.0 : 0.0;
  double* la = a.logacc + (int64_t)b * a.nslots;
  for (int w = threadIdx.x; w < a.nslots; w += blockDim.x) la[w] = 0.0;
}

template <typename R>
__device__ R block_max(R v, R* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : R(0);
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  return red[0];
}

// psi_s <- X^{m(s,t)} K psi_s on the physical leg, then divide by the power of two at or
// above the largest magnitude (an exact scaling; its log goes to the site's log-scale
// slot).  The mixing is computed in FP64 whatever the storage type: psi has entries of both
// signs, and a rounded FP32 sum would be an additive perturbation of the state.  One block
// per (site, shot); in place.
template <typename T>
__global__ void k_local(SweepArgs a, const LocalDesc* __restrict__ locals) {
  const int s = blockIdx.x, b = blockIdx.y;
  const LocalDesc d = locals[s];
  __shared__ double K[kMaxPhys * kMaxPhys];
  __shared__ double red[32];
  const int m = a.det[(int64_t)vshot_row(a.vs, a.wave_first, b) * a.n_det + d.det] & 1;
  const Override* o = vshot_ovr(a.vs, a.ovr, a.wave_first, b, kOvrLocal, a.layer * (int)gridDim.x + s);
  const double* Ksrc = o ? o->val : d.K;
  if (threadIdx.x < d.P * d.P) {
    const int row = threadIdx.x / d.P, col = threadIdx.x % d.P;
    K[threadIdx.x] = Ksrc[(row ^ m) * d.P + col];     // rows of X^m K
  }
  __syncthreads();
  const T* g = reinterpret_cast<const T*>(a.gamma) + (int64_t)b * a.shot_elems + d.off;
  T* go = reinterpret_cast<T*>(a.gamma) + (int64_t)b * a.shot_elems + d.out_off;
  double mx = 0.0;
  for (int r = threadIdx.x; r < d.rest; r += blockDim.x) {
    double v[kMaxPhys];
    for (int k = 0; k < d.P; ++k) v[k] = double(g[(int64_t)k * d.rest + r]);
    for (int i = 0; i < d.P; ++i) {
      double acc = 0.0;
      for (int k = 0; k < d.P; ++k) acc += K[i * d.P + k] * v[k];
      mx = fmax(mx, fabs(acc));
    }
  }
  mx = block_max<double>(mx, red);
  int e2 = 0;
  if (mx > 0.0) frexp(mx, &e2);             // mx = f 2^e2, f in [1/2, 1)
  const double sc = ldexp(1.0, -e2);        // exact
  for (int r = threadIdx.x; r < d.rest; r += blockDim.x) {
    double v[kMaxPhys];
    for (int k = 0; k < d.P; ++k) v[k] = double(g[(int64_t)k * d.rest + r]);
    for (int i = 0; i < d.P; ++i) {
      double acc = 0.0;
      for (int k = 0; k < d.P; ++k) acc += K[i * d.P + k] * v[k];
      go[(int64_t)i * d.rest + r] = T(acc * sc);
    }
  }
  if (threadIdx.x == 0) {
    double* la = a.logacc + (int64_t)b * a.nslots + s;
    *la += (mx > 0.0) ? double(e2) * 0.69314718055994530942 : -INFINITY;
    if (a.rec_sc) a.rec_sc[(int64_t)b * gridDim.x + s] = sc;
  }
}

// ---- launchers ---------------------------------------------------------------------------
template <typename T, typename R>
cudaError_t launch_sweep_init(const SweepArgs& a, const LocalDesc* locals0, int S, cudaStream_t st) {
  k_init<T><<<a.B, 256, 0, st>>>(a, locals0, S);
  return cudaGetLastError();
}

template <typename T, typename R>
cudaError_t launch_local(const SweepArgs& a, const LocalDesc* locals, int S, cudaStream_t st) {
  k_local<T><<<dim3(S, a.B), 256, 0, st>>>(a, locals);
  return cudaGetLastError();
}

template <typename T, typename R>
cudaError_t launch_round(const SweepArgs& a0, const GateDesc* gates, const Round& rd, double* gram, double* tbuf, int S,
                         cudaStream_t st, Prof* prof) {
  const GateDesc* g = gates + rd.first;
  const int D = std::max(rd.maxD, rd.maxDn);
  SweepArgs a = a0;
  const int cr = a0.chunk_rows > 0 ? a0.chunk_rows : kChunkRows;
  a.gram_chunks = absorb_chunks(rd.max_rows, cr);
  a.gate_base = rd.first;
  auto B = [&](int k) { if (prof) prof->begin(k); };
  auto E = [&](int k) { if (prof) prof->end(k); };
  B(TD_K_GRAM);
  cudaError_t e = (a.tc && gram_tc_supported(rd.maxD))
                      ? launch_gram_tc<T>(a, g, rd.count, rd.maxD, gram, a.gram_chunks, cr, st)
                      : launch_gram2<T>(a, g, rd.count, D, gram, a.gram_chunks, cr, st);
  E(TD_K_GRAM);
  if (e != cudaSuccess) return e;
  B(TD_K_CORE);
  e = launch_core2<R>(a, g, rd.count, rd.maxD, gram, tbuf, S, a.precond != 0, st);
  E(TD_K_CORE);
  if (e != cudaSuccess) return e;
  B(TD_K_UPDATE);
  e = launch_update2<T>(a, g, rd.count, D, tbuf, a.gram_chunks, cr, st);
  E(TD_K_UPDATE);
  return e;
}

template cudaError_t launch_sweep_init<double, double>(const SweepArgs&, const LocalDesc*, int, cudaStream_t);
template cudaError_t launch_sweep_init<float, float>(const SweepArgs&, const LocalDesc*, int, cudaStream_t);
template cudaError_t launch_local<double, double>(const SweepArgs&, const LocalDesc*, int, cudaStream_t);
template cudaError_t launch_local<float, float>(const SweepArgs&, const LocalDesc*, int, cudaStream_t);
template cudaError_t launch_round<double, double>(const SweepArgs&, const GateDesc*, const Round&, double*, double*,
                                                  int, cudaStream_t, Prof*);
template cudaError_t launch_round<float, float>(const SweepArgs&, const GateDesc*, const Round&, double*, double*, int,
                                                cudaStream_t, Prof*);

}  // namespace td
