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

#include "linalg.cuh"
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

// Refinement step 1 (FP32 storage): eigen-decompose the four first-pass Gram blocks in FP64
// and emit T1 = W Sigma^-1 and T1^-1 = Sigma W^T per block.  Eigenvalues are floored at
// kPreFloor of the side's largest -- the rounding level of an FP32 Gram -- so T1 stays
// invertible, no direction is dropped here, and every column of Q1 = M T1 has norm O(1)
// or less (a floored direction is resolved by the second Gram instead).
constexpr double kPreFloor = 1e-6;
template <typename R>
__global__ void k_pre(SweepArgs a, const GateDesc* __restrict__ gates, const R* __restrict__ gram,
                      double* __restrict__ t1buf) {
  const int gi = blockIdx.x, b = blockIdx.y;
  const int D = gates[gi].D, chi = a.chi;
  extern __shared__ double sm[];
  double* G = sm;                 // [4][D*D]
  double* V = G + 4 * D * D;      // [4][D*D]
  double* rot = V + 4 * D * D;    // [D + 2]
  int* flag = reinterpret_cast<int*>(rot + D + 2);
  const R* gsrc = gram + (int64_t)(gi * a.B + b) * 4 * chi * chi;
  for (int w = threadIdx.x; w < 4 * D * D; w += blockDim.x)
    G[w] = double(gsrc[(int64_t)(w / (D * D)) * chi * chi + w % (D * D)]);
  __syncthreads();
  for (int blk = 0; blk < 4; ++blk) block_sym_eig<double>(G + blk * D * D, D, V + blk * D * D, D, D, rot, flag);
  __syncthreads();
  double* out = t1buf + (int64_t)(gi * a.B + b) * 4 * 2 * chi * chi;
  for (int w = threadIdx.x; w < 4 * D * D; w += blockDim.x) {
    const int blk = w / (D * D), q = (w / D) % D, j = w % D;
    const int side = blk / 2;
    double emax = 0;
    for (int bb = 2 * side; bb < 2 * side + 2; ++bb)
      for (int i = 0; i < D; ++i) emax = fmax(emax, G[bb * D * D + i * D + i]);
    double* o = out + (int64_t)blk * 2 * chi * chi;
    if (emax <= 0) {
      o[q * D + j] = (q == j) ? 1.0 : 0.0;
      o[chi * chi + q * D + j] = (q == j) ? 1.0 : 0.0;
      continue;
    }
    const double e = fmax(G[blk * D * D + j * D + j], kPreFloor * emax);
    const double s = sqrt(e);
    o[q * D + j] = V[blk * D * D + q * D + j] / s;                     // T1[q][j]
    const double ej = fmax(G[blk * D * D + q * D + q], kPreFloor * emax);
    o[chi * chi + q * D + j] = sqrt(ej) * V[blk * D * D + j * D + q];  // T1^-1[q][j] = s_q W[j][q]
  }
}

// Simple-update core of one gate (FP64): eigen-decompose the four Gram blocks, build theta,
// SVD it, truncate, emit T+- for both sides and the new lambda of the bond.
// With t1buf the Gram blocks are those of Q1 = M T1: the R factor of a block is
// Sigma W^T T1^-1 and the update transform T1 W Sigma^-1 U.
template <typename R>
__global__ void k_core(SweepArgs a, const GateDesc* __restrict__ gates, const R* __restrict__ gram,
                       double* __restrict__ tbuf, int S, const double* __restrict__ t1buf) {
  const int gi = blockIdx.x, b = blockIdx.y;
  const GateDesc& gd = gates[gi];
  const int D = gd.D, Dn = gd.Dn, chi = a.chi;
  const int D2 = 2 * D;
  extern __shared__ double sm[];
  double* G = sm;                       // [4][D*D]
  double* V = G + 4 * D * D;            // [4][D*D]
  double* th = V + 4 * D * D;           // [D2][D2]
  double* Vt = th + D2 * D2;            // [D2][D2]
  double* sA = Vt + D2 * D2;            // [D2] kept sigma of A
  double* sB = sA + D2;                 // [D2]
  double* sv = sB + D2;                 // [D2] singular values (unsorted)
  double* lamb = sv + D2;               // [D]
  double* rot = lamb + D + 1;           // [D2 + 2]
  int* iA = reinterpret_cast<int*>(rot + D2 + 2);   // [D2] kept index (block*D + j)
  int* iB = iA + D2;
  int* order = iB + D2;                 // [D2]
  int* meta = order + D2;               // [8]
  double* Wt = reinterpret_cast<double*>(meta + 8);   // [4][D*D] (refinement only)
  double* Wf = Wt + 4 * D * D;                        // [4][D*D]
  const int tid = threadIdx.x, nt = blockDim.x;
  const R* gsrc = gram + (int64_t)(gi * a.B + b) * 4 * chi * chi;
  for (int w = tid; w < 4 * D * D; w += nt) {
    const int blk = w / (D * D), e = w % (D * D);
    G[w] = double(gsrc[(int64_t)blk * chi * chi + e]);
  }
  double* lamg = a.lam + ((int64_t)b * a.nbonds + gd.bond) * chi;
  for (int w = tid; w < D; w += nt) lamb[w] = lamg[w];
  __syncthreads();
  for (int blk = 0; blk < 4; ++blk)
    block_sym_eig<double>(G + blk * D * D, D, V + blk * D * D, D, D, rot, meta + 7);
  __syncthreads();
  const double* WtU = V;   // rows of R = Sigma (W^T T1^-1): WtU[q][j] = (T1^-T W)[q][j]
  const double* WfU = V;   // columns of the update transform: WfU = T1 W
  if (t1buf) {
    const double* t1 = t1buf + (int64_t)(gi * a.B + b) * 4 * 2 * chi * chi;
    for (int w = tid; w < 4 * D * D; w += nt) {
      const int blk = w / (D * D), q = (w / D) % D, j = w % D;
      const double* T1 = t1 + (int64_t)blk * 2 * chi * chi;
      const double* Ti = T1 + chi * chi;
      const double* W = V + blk * D * D;
      double at = 0, af = 0;
      for (int r = 0; r < D; ++r) {
        at += Ti[r * D + q] * W[r * D + j];
        af += T1[q * D + r] * W[r * D + j];
      }
      Wt[w] = at;
      Wf[w] = af;
    }
    __syncthreads();
    WtU = Wt;
    WfU = Wf;
  }
  if (tid == 0) {
    // keep Gram eigen-directions above gram_cutoff * largest eigenvalue of that side
    for (int side = 0; side < 2; ++side) {
      double emax = 0;
      for (int blk = 0; blk < 2; ++blk)
        for (int j = 0; j < D; ++j) emax = fmax(emax, G[(2 * side + blk) * D * D + j * D + j]);
      int r = 0;
      for (int blk = 0; blk < 2; ++blk)
        for (int j = 0; j < D; ++j) {
          const double e = G[(2 * side + blk) * D * D + j * D + j];
          if (emax > 0 && e > a.gram_cutoff * emax) {
            (side ? iB : iA)[r] = blk * D + j;
            (side ? sB : sA)[r] = sqrt(e);
            ++r;
          }
        }
      meta[side] = r;
    }
  }
  __syncthreads();
  const int rA = meta[0], rB = meta[1];
  const double p = gd.p;
  const double cpp = 0.5, cpm = 0.5 * (1.0 - 2.0 * p);
  double* tout = tbuf + (int64_t)(gi * a.B + b) * 4 * chi * chi;
  if (rA == 0 || rB == 0) {                  // zero state: this shot has probability 0
    for (int w = tid; w < 4 * chi * chi; w += nt) tout[w] = 0.0;
    for (int w = tid; w < Dn; w += nt) lamg[w] = 0.0;
    if (tid == 0) a.logacc[(int64_t)b * a.nslots + S + gd.bond] = -INFINITY;
    return;
  }
  // theta[i][j] = sA_i sB_j c(ki,kj) sum_b W_A[b][i'] lambda_b W_B[b][j']
  for (int w = tid; w < rA * rB; w += nt) {
    const int i = w / rB, j = w % rB;
    const int ba = iA[i] / D, ja = iA[i] % D, bb = iB[j] / D, jb = iB[j] % D;
    const double* WA = WtU + ba * D * D;
    const double* WB = WtU + (2 + bb) * D * D;
    double acc = 0;
    for (int q = 0; q < D; ++q) acc += WA[q * D + ja] * lamb[q] * WB[q * D + jb];
    th[i * rB + j] = sA[i] * sB[j] * (ba == bb ? cpp : cpm) * acc;
  }
  __syncthreads();
  block_svd_onesided<double>(th, rB, rA, rB, Vt, rB, rot, meta + 7);
  for (int j = tid; j < rB; j += nt) {
    double s2 = 0;
    for (int i = 0; i < rA; ++i) s2 += th[i * rB + j] * th[i * rB + j];
    sv[j] = sqrt(s2);
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < rB; ++j) order[j] = j;
    for (int j = 1; j < rB; ++j) {           // insertion sort, descending
      int x = order[j], k = j - 1;
      while (k >= 0 && sv[order[k]] < sv[x]) { order[k + 1] = order[k]; --k; }
      order[k + 1] = x;
    }
    double srt[2 * kMaxChi];
    for (int j = 0; j < rB; ++j) srt[j] = sv[order[j]];
    int k = 0;
    if (srt[0] > 0) k = keep_count<double>(srt, rB < rA ? rB : rA, Dn, a.svd_cutoff, a.multiplet_rtol);
    meta[2] = k;
  }
  __syncthreads();
  const int k = meta[2];
  const double s0 = sv[order[0]];
  if (k == 0 || !(s0 > 0)) {
    for (int w = tid; w < 4 * chi * chi; w += nt) tout[w] = 0.0;
    for (int w = tid; w < Dn; w += nt) lamg[w] = 0.0;
    if (tid == 0) a.logacc[(int64_t)b * a.nslots + S + gd.bond] = -INFINITY;
    return;
  }
  const double rs2 = 0.70710678118654752440;
  // T_A(kappa)[q][j] = sum_{i in A kappa} W_A[q][i'] / sA_i * U[i][j] / sqrt2, U[:, j] = th[:, order j] / s_j
  for (int w = tid; w < 2 * D * Dn; w += nt) {
    const int kap = w / (D * Dn), q = (w / Dn) % D, j = w % Dn;
    double acc = 0;
    if (j < k) {
      const int cj = order[j];
      const double inv = 1.0 / sv[cj];
      for (int i = 0; i < rA; ++i) {
        if (iA[i] / D != kap) continue;
        acc += WfU[kap * D * D + q * D + (iA[i] % D)] / sA[i] * th[i * rB + cj] * inv;
      }
    }
    tout[(int64_t)kap * chi * chi + q * Dn + j] = acc * rs2;
  }
  for (int w = tid; w < 2 * D * Dn; w += nt) {
    const int kap = w / (D * Dn), q = (w / Dn) % D, j = w % Dn;
    double acc = 0;
    if (j < k) {
      const int cj = order[j];
      for (int i = 0; i < rB; ++i) {
        if (iB[i] / D != kap) continue;
        acc += WfU[(2 + kap) * D * D + q * D + (iB[i] % D)] / sB[i] * Vt[i * rB + cj];
      }
    }
    tout[(int64_t)(2 + kap) * chi * chi + q * Dn + j] = acc * rs2;
  }
  __syncthreads();
  for (int j = tid; j < Dn; j += nt) lamg[j] = (j < k) ? sv[order[j]] / s0 : 0.0;
  if (tid == 0) a.logacc[(int64_t)b * a.nslots + S + gd.bond] += log(s0);
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

size_t core_smem_bytes(int D) {
  const int D2 = 2 * D;
  return sizeof(double) * (8 * D * D + 2 * D2 * D2 + 3 * D2 + D + 1 + D2 + 2) + sizeof(int) * (4 * D2 + 8) +
         sizeof(double) * 8 * D * D + 64;
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
    const size_t smem_p = sizeof(double) * (8 * D * D + D + 2) + 16;
    if (smem_p > 48 * 1024) {
      e = cudaFuncSetAttribute(k_pre<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p);
      if (e != cudaSuccess) return e;
    }
    B(TD_K_PRE);
    k_pre<R><<<dim3(rd.count, a.B), 128, smem_p, st>>>(a, g, reinterpret_cast<const R*>(gram), t1buf);
    E(TD_K_PRE);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    B(TD_K_GRAM);
    k_gram<T, R><<<dim3(2 * rd.count, a.B), 256, smem_g, st>>>(a, g, reinterpret_cast<R*>(gram), t1buf);
    E(TD_K_GRAM);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem_c = core_smem_bytes(D);
  if (smem_c > 48 * 1024) {
    e = cudaFuncSetAttribute(k_core<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
    if (e != cudaSuccess) return e;
  }
  B(TD_K_CORE);
  k_core<R><<<dim3(rd.count, a.B), 128, smem_c, st>>>(a, g, reinterpret_cast<const R*>(gram), tbuf, S, t1buf);
  E(TD_K_CORE);
  e = cudaGetLastError();
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
