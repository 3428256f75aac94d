// Layer absorption of the boundary sweep (Sec. 4) on the GPU: site-local operators, and
// for every two-site gate (1-p) I x I + p X x X on a bond (the natural split of Sec. 5.1)
// the simple-update truncation of that bond back to chi (Sec. 4).
//
// Gate as bond doubling: with k the gate's bit, Gamma'_X[sigma; ..., (b, k)] =
// Gamma_X[sigma ^ k mask_X; ..., b] and lambda'_(b,k) = lambda_b w_k, w = (1-p, p).  In the
// basis kappa = (k=0 +- k=1)/sqrt2 the Gram matrix of M'_X (Gamma'_X with the other bonds'
// lambdas absorbed) is block diagonal: G+ = sum Y Y^T, G- = sum Z Z^T over rows, where
// Y = M[sigma_lo] + M[sigma_hi], Z = M[sigma_lo] - M[sigma_hi] for each pair
// sigma_hi = sigma_lo ^ mask.  The core kernel turns the four blocks into R factors,
// forms the 2D x 2D core theta = R_A Lambda' R_B^T, takes its SVD and keeps <= chi values;
// the update applies Gamma_new[lo] = Y T+ + Z T-, Gamma_new[hi] = Y T+ - Z T-.
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

// psi_s <- X^{m(s,t)} K psi_s on the physical leg, then divide by the largest magnitude
// (its log goes to the site's log-scale slot).  One block per (site, shot); in place.
template <typename T>
__global__ void k_local(SweepArgs a, const LocalDesc* __restrict__ locals) {
  const int s = blockIdx.x, b = blockIdx.y;
  const LocalDesc d = locals[s];
  __shared__ T K[kMaxPhys * kMaxPhys];
  __shared__ T red[32];
  const int m = a.det[(int64_t)(a.wave_first + b) * a.n_det + d.det] & 1;
  if (threadIdx.x < d.P * d.P) {
    const int row = threadIdx.x / d.P, col = threadIdx.x % d.P;
    K[threadIdx.x] = T(d.K[(row ^ m) * d.P + col]);     // rows of X^m K
  }
  __syncthreads();
  T* g = reinterpret_cast<T*>(a.gamma) + (int64_t)b * a.shot_elems + d.off;
  T mx = T(0);
  for (int r = threadIdx.x; r < d.rest; r += blockDim.x) {
    T v[kMaxPhys], o[kMaxPhys];
    for (int k = 0; k < d.P; ++k) v[k] = g[(int64_t)k * d.rest + r];
    for (int i = 0; i < d.P; ++i) {
      T acc = T(0);
      for (int k = 0; k < d.P; ++k) acc += K[i * d.P + k] * v[k];
      o[i] = acc;
      mx = fmax(mx, fabs(acc));
    }
    for (int i = 0; i < d.P; ++i) g[(int64_t)i * d.rest + r] = o[i];
  }
  mx = block_max<T>(mx, red);
  if (mx > T(0)) {
    const T inv = T(1) / mx;
    for (int w = threadIdx.x; w < d.P * d.rest; w += blockDim.x) g[w] *= inv;
  }
  if (threadIdx.x == 0) {
    double* la = a.logacc + (int64_t)b * a.nslots + s;
    *la += (mx > T(0)) ? log((double)mx) : -INFINITY;
  }
}

// Decompose row r of a side into (sigma_lo, sigma_hi, o, i) and its environment weight
// prod over the other bonds of lambda[digit].
struct RowGeom {
  int lo[2], hi[2];
  int npairs;
};

__device__ __forceinline__ RowGeom make_pairs(int P, int mask) {
  RowGeom g;
  g.npairs = 0;
  for (int sg = 0; sg < P; ++sg)
    if (sg < (sg ^ mask)) {
      g.lo[g.npairs] = sg;
      g.hi[g.npairs] = sg ^ mask;
      ++g.npairs;
    }
  return g;
}

template <typename R>
__device__ __forceinline__ R env_weight(const SideDesc& sd, int o, int i, const double* lamv, int chi) {
  // lamv: [kMaxBonds][chi] lambdas of the site's bonds (shared)
  R w = R(1);
  for (int k = sd.nb - 1; k > sd.pos; --k) {
    const int dk = sd.dims[k];
    w *= R(lamv[k * chi + i % dk]);
    i /= dk;
  }
  for (int k = sd.pos - 1; k >= 0; --k) {
    const int dk = sd.dims[k];
    w *= R(lamv[k * chi + o % dk]);
    o /= dk;
  }
  return w;
}

constexpr int kGramRows = 32;

// Gram blocks G+ = sum_rows Y Y^T and G- = sum_rows Z Z^T (D x D each) of one gate side.
// With t1buf (refinement pass) each staged row is first multiplied by the side's T1 block:
// the Gram of Q1 = Y T1+ (resp. Z T1-), where T1 = W Sigma^-1 comes from the first Gram.
template <typename T, typename R>
__global__ void k_gram(SweepArgs a, const GateDesc* __restrict__ gates, R* __restrict__ gram,
                       const double* __restrict__ t1buf) {
  const int gi = blockIdx.x >> 1, side = blockIdx.x & 1, b = blockIdx.y;
  const GateDesc& gd = gates[gi];
  const SideDesc sd = gd.side[side];
  const int D = gd.D, chi = a.chi;
  extern __shared__ unsigned char smem_raw[];
  R* Ys = reinterpret_cast<R*>(smem_raw);                 // [kGramRows][D]
  R* Zs = Ys + kGramRows * D;
  R* Yq = Zs + kGramRows * D;                             // transformed rows (refinement)
  R* Zq = Yq + kGramRows * D;
  R* T1p = Zq + kGramRows * D;                            // [D][D]
  R* T1m = T1p + D * D;
  R* wrow = T1m + D * D;                                  // [kGramRows]
  double* lamv = reinterpret_cast<double*>(wrow + kGramRows + 2);
  lamv = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(lamv) + 7) & ~uintptr_t(7));
  const double* lamb = a.lam + (int64_t)b * a.nbonds * chi;
  for (int w = threadIdx.x; w < kMaxBonds * chi; w += blockDim.x) {
    const int k = w / chi;
    lamv[w] = (k < sd.nb) ? lamb[sd.bond[k] * chi + (w % chi)] : 1.0;
  }
  const bool refine = t1buf != nullptr;
  if (refine) {
    const double* t1 = t1buf + ((int64_t)(gi * a.B + b) * 4 + 2 * side) * 2 * chi * chi;
    for (int w = threadIdx.x; w < D * D; w += blockDim.x) {
      T1p[w] = R(t1[w]);
      T1m[w] = R(t1[2 * chi * chi + w]);
    }
  }
  const RowGeom pg = make_pairs(sd.P, sd.mask);
  const int OI = sd.outer * sd.inner;
  const int rows = pg.npairs * OI;
  const int64_t SZ = (int64_t)OI * D;
  const T* gin = reinterpret_cast<const T*>(a.gamma) + (int64_t)b * a.shot_elems + sd.in_off;
  const int nent = D * D;
  const R* Yu = refine ? Yq : Ys;
  const R* Zu = refine ? Zq : Zs;
  constexpr int kMaxEnt = 4;                               // entries per thread (D <= 32, 256 threads)
  R accP[kMaxEnt], accM[kMaxEnt];
  for (int e = 0; e < kMaxEnt; ++e) { accP[e] = R(0); accM[e] = R(0); }
  const bool rows_fast = sd.inner >= 8;
  for (int r0 = 0; r0 < rows; r0 += kGramRows) {
    __syncthreads();
    for (int rr = threadIdx.x; rr < kGramRows; rr += blockDim.x) {
      const int r = r0 + rr;
      R w = R(0);
      if (r < rows) {
        const int oi = r % OI;
        w = env_weight<R>(sd, oi / sd.inner, oi % sd.inner, lamv, chi);
      }
      wrow[rr] = w;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < kGramRows * D; w += blockDim.x) {
      int rr, bc;
      if (rows_fast) { rr = w % kGramRows; bc = w / kGramRows; } else { rr = w / D; bc = w % D; }
      const int r = r0 + rr;
      R y = R(0), z = R(0);
      if (r < rows) {
        const int pr = r / OI, oi = r % OI, o = oi / sd.inner, i = oi % sd.inner;
        const int64_t base = (int64_t)o * D * sd.inner + (int64_t)bc * sd.inner + i;
        const R lo = R(gin[pg.lo[pr] * SZ + base]), hi = R(gin[pg.hi[pr] * SZ + base]);
        const R wr = wrow[rr];
        y = (lo + hi) * wr;
        z = (lo - hi) * wr;
      }
      Ys[rr * D + bc] = y;
      Zs[rr * D + bc] = z;
    }
    __syncthreads();
    const int nr = min(kGramRows, rows - r0);
    if (refine) {
      for (int w = threadIdx.x; w < nr * D; w += blockDim.x) {
        const int rr = w / D, j = w % D;
        R qy = R(0), qz = R(0);
        for (int q = 0; q < D; ++q) {
          qy += Ys[rr * D + q] * T1p[q * D + j];
          qz += Zs[rr * D + q] * T1m[q * D + j];
        }
        Yq[rr * D + j] = qy;
        Zq[rr * D + j] = qz;
      }
      __syncthreads();
    }
    for (int e = 0; e < kMaxEnt; ++e) {
      const int ent = threadIdx.x + e * blockDim.x;
      if (ent >= nent) break;
      const int b1 = ent / D, b2 = ent % D;
      R sp = R(0), sm = R(0);
      for (int rr = 0; rr < nr; ++rr) {
        sp += Yu[rr * D + b1] * Yu[rr * D + b2];
        sm += Zu[rr * D + b1] * Zu[rr * D + b2];
      }
      accP[e] += sp;
      accM[e] += sm;
    }
  }
  R* out = gram + ((int64_t)(gi * a.B + b) * 2 + side) * 2 * chi * chi;
  for (int e = 0; e < kMaxEnt; ++e) {
    const int ent = threadIdx.x + e * blockDim.x;
    if (ent >= nent) break;
    out[ent] = accP[e];
    out[chi * chi + ent] = accM[e];
  }
}

constexpr int kUpdRows = 32;

// Gamma_new[lo] = Y T+ + Z T-, Gamma_new[hi] = Y T+ - Z T- for a tile of rows of one side.
template <typename T, typename R>
__global__ void k_update(SweepArgs a, const GateDesc* __restrict__ gates, const double* __restrict__ tbuf,
                         int tiles) {
  const int gi = blockIdx.x / (2 * tiles), side = (blockIdx.x / tiles) & 1, tile = blockIdx.x % tiles;
  const int b = blockIdx.y;
  const GateDesc& gd = gates[gi];
  const SideDesc sd = gd.side[side];
  const int D = gd.D, Dn = gd.Dn, chi = a.chi;
  const RowGeom pg = make_pairs(sd.P, sd.mask);
  const int OI = sd.outer * sd.inner;
  const int rows = pg.npairs * OI;
  const int r0 = tile * kUpdRows;
  if (r0 >= rows) return;
  extern __shared__ unsigned char smem_raw[];
  R* Tp = reinterpret_cast<R*>(smem_raw);   // [D][Dn]
  R* Tm = Tp + D * Dn;
  R* Ys = Tm + D * Dn;                      // [kUpdRows][D]
  R* Zs = Ys + kUpdRows * D;
  const double* tsrc = tbuf + (int64_t)(gi * a.B + b) * 4 * chi * chi + (int64_t)side * 2 * chi * chi;
  for (int w = threadIdx.x; w < D * Dn; w += blockDim.x) {
    Tp[w] = R(tsrc[w]);
    Tm[w] = R(tsrc[chi * chi + w]);
  }
  const T* gin = reinterpret_cast<const T*>(a.gamma) + (int64_t)b * a.shot_elems + sd.in_off;
  T* gout = reinterpret_cast<T*>(a.gamma) + (int64_t)b * a.shot_elems + sd.out_off;
  const int64_t SZ = (int64_t)OI * D, SZn = (int64_t)OI * Dn;
  const bool rows_fast = sd.inner >= 8;
  for (int w = threadIdx.x; w < kUpdRows * D; w += blockDim.x) {
    int rr, bc;
    if (rows_fast) { rr = w % kUpdRows; bc = w / kUpdRows; } else { rr = w / D; bc = w % D; }
    const int r = r0 + rr;
    R y = R(0), z = R(0);
    if (r < rows) {
      const int pr = r / OI, oi = r % OI, o = oi / sd.inner, i = oi % sd.inner;
      const int64_t base = (int64_t)o * D * sd.inner + (int64_t)bc * sd.inner + i;
      const R lo = R(gin[pg.lo[pr] * SZ + base]), hi = R(gin[pg.hi[pr] * SZ + base]);
      y = lo + hi;
      z = lo - hi;
    }
    Ys[rr * D + bc] = y;
    Zs[rr * D + bc] = z;
  }
  __syncthreads();
  for (int w = threadIdx.x; w < kUpdRows * Dn; w += blockDim.x) {
    int rr, j;
    if (rows_fast) { rr = w % kUpdRows; j = w / kUpdRows; } else { rr = w / Dn; j = w % Dn; }
    const int r = r0 + rr;
    if (r >= rows) continue;
    R u1 = R(0), u2 = R(0);
    for (int q = 0; q < D; ++q) {
      u1 += Ys[rr * D + q] * Tp[q * Dn + j];
      u2 += Zs[rr * D + q] * Tm[q * Dn + j];
    }
    const int pr = r / OI, oi = r % OI, o = oi / sd.inner, i = oi % sd.inner;
    const int64_t base = (int64_t)o * Dn * sd.inner + (int64_t)j * sd.inner + i;
    gout[pg.lo[pr] * SZn + base] = T(u1 + u2);
    gout[pg.hi[pr] * SZn + base] = T(u1 - u2);
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
cudaError_t launch_round(const SweepArgs& a, const GateDesc* gates, const Round& rd, void* gram, double* tbuf,
                         double* t1buf, int S, cudaStream_t st, Prof* prof) {
  const GateDesc* g = gates + rd.first;
  const int D = rd.maxD, Dn = rd.maxDn;
  const size_t smem_g = sizeof(R) * (4 * kGramRows * D + 2 * D * D + kGramRows + 2) +
                        sizeof(double) * (kMaxBonds * a.chi + 1) + 16;
  auto B = [&](int k) { if (prof) prof->begin(k); };
  auto E = [&](int k) { if (prof) prof->end(k); };
  B(TD_K_GRAM);
  k_gram<T, R><<<dim3(2 * rd.count, a.B), 256, smem_g, st>>>(a, g, reinterpret_cast<R*>(gram), nullptr);
  E(TD_K_GRAM);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool refine = t1buf != nullptr;
  if (refine) {
    B(TD_K_PRE);
    e = launch_pre2<R>(a, g, rd.count, D, gram, t1buf, st);
    E(TD_K_PRE);
    if (e != cudaSuccess) return e;
    B(TD_K_GRAM);
    k_gram<T, R><<<dim3(2 * rd.count, a.B), 256, smem_g, st>>>(a, g, reinterpret_cast<R*>(gram), t1buf);
    E(TD_K_GRAM);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  B(TD_K_CORE);
  e = launch_core2<R>(a, g, rd.count, D, gram, tbuf, t1buf, S, /*precond=*/sizeof(R) == 4, st);
  E(TD_K_CORE);
  if (e != cudaSuccess) return e;
  const int tiles = (rd.max_rows + kUpdRows - 1) / kUpdRows;
  const size_t smem_u = sizeof(R) * (2 * D * Dn + 2 * kUpdRows * D);
  B(TD_K_UPDATE);
  k_update<T, R><<<dim3(2 * rd.count * tiles, a.B), 256, smem_u, st>>>(a, g, tbuf, tiles);
  E(TD_K_UPDATE);
  return cudaGetLastError();
}

template cudaError_t launch_sweep_init<double, double>(const SweepArgs&, const LocalDesc*, int, cudaStream_t);
template cudaError_t launch_sweep_init<float, float>(const SweepArgs&, const LocalDesc*, int, cudaStream_t);
template cudaError_t launch_local<double, double>(const SweepArgs&, const LocalDesc*, int, cudaStream_t);
template cudaError_t launch_local<float, float>(const SweepArgs&, const LocalDesc*, int, cudaStream_t);
template cudaError_t launch_round<double, double>(const SweepArgs&, const GateDesc*, const Round&, void*, double*,
                                                  double*, int, cudaStream_t, Prof*);
template cudaError_t launch_round<float, float>(const SweepArgs&, const GateDesc*, const Round&, void*, double*,
                                                double*, int, cudaStream_t, Prof*);

}  // namespace td
