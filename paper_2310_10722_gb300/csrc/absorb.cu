// Gate absorption passes of the sweep (Sec. 4): the Gram pass and the update pass of the
// simple update, one warp per (gate side, shot, row chunk).
//
// The two-site gate (1-p) I x I + p X x X is applied by doubling its bond (see sweep.cu):
// with Y = M[sigma_lo] + M[sigma_hi] and Z = M[sigma_lo] - M[sigma_hi] for each physical
// pair sigma_hi = sigma_lo ^ mask, the Gram of the doubled side matrix is block diagonal,
// G+ = sum_rows Y^T Y and G- = sum_rows Z^T Z (rows weighted by the other bonds' lambda), and
// the update is Gamma_new[lo] = Y T+ + Z T-, Gamma_new[hi] = Y T+ - Z T-.
//
// A side tensor is [phys][outer][D][inner]; a row is (pair, outer index o, inner index i)
// and holds D values at stride `inner`.  Each row is handled by LPR lanes; lane `sub` of a
// row loads BPL = DMAX/LPR of its columns, and the full row is assembled in every lane of
// the row by shuffles.  The Gram lane accumulates its BPL x DMAX block of G+ and of G- in
// registers, summed over the warp at the end; the update lane produces BPL output columns.
// No shared-memory staging of the data and no block-wide barrier.  Chunks of a long side
// write separate partial Grams, summed in a fixed order by the core kernel (deterministic).
//
// Precision.  Both passes compute in FP64 for both storage types (FP32 storage is read,
// widened, and the update's result rounded back): the Gram's small eigenvalues come from
// cancellation, the update applies an ill-conditioned transform (T = R^+ U), and the simple
// update keeps directions down to its cutoff, to which its result is sensitive.  Measured
// against the FP64 oracle at chi = 16 (rotated d = 9), FP32 Grams moved log p by up to 0.3;
// FP64 Grams with an FP32 update still by 0.2 on one shot in eight; FP64 arithmetic on FP32
// storage stays within 2e-4.  Forming Y = lo + hi and Z = lo - hi in FP32 alone cost 1e-3.
#include <algorithm>
#include <cmath>

#include "sweep.cuh"

namespace td {

namespace {

// Physical index pairs (lo, hi = lo ^ mask) of a side, as scalars (no local arrays).
struct Pairs {
  int lo0, hi0, lo1, hi1;
  int npairs;
  __device__ __forceinline__ int lo(int pr) const { return pr ? lo1 : lo0; }
  __device__ __forceinline__ int hi(int pr) const { return pr ? hi1 : hi0; }
};

__device__ __forceinline__ Pairs side_pairs(int P, int mask) {
  Pairs g;
  g.lo0 = g.hi0 = g.lo1 = g.hi1 = 0;
  g.npairs = 0;
  for (int sg = 0; sg < P; ++sg)
    if (sg < (sg ^ mask)) {
      if (g.npairs == 0) {
        g.lo0 = sg;
        g.hi0 = sg ^ mask;
      } else {
        g.lo1 = sg;
        g.hi1 = sg ^ mask;
      }
      ++g.npairs;
    }
  return g;
}

// Environment weight of row (o, i): product over the side's other bonds of lambda[digit]
// (loops unrolled over the four bond slots so the descriptor stays in registers).
template <typename R>
__device__ __forceinline__ R row_weight(const SideDesc& sd, int o, int i, const R* lamv, int chi) {
  R w = R(1);
#pragma unroll
  for (int k = kMaxBonds - 1; k >= 0; --k)
    if (k < sd.nb && k > sd.pos) {
      const int dk = sd.dims[k];
      w *= lamv[k * chi + i % dk];
      i /= dk;
    }
#pragma unroll
  for (int k = kMaxBonds - 1; k >= 0; --k)
    if (k < sd.pos) {
      const int dk = sd.dims[k];
      w *= lamv[k * chi + o % dk];
      o /= dk;
    }
  return w;
}

template <int DMAX>
struct Shape;   // lanes per row
template <>
struct Shape<8> { static constexpr int LPR = 2; };
template <>
struct Shape<16> { static constexpr int LPR = 8; };
template <>
struct Shape<32> { static constexpr int LPR = 32; };

struct Job {
  int ch, side, gi, b;
  int64_t gb;   // gate * B + shot
};

__device__ __forceinline__ Job decode_job(int64_t job, int nchunk, int B) {
  Job j;
  j.ch = (int)(job % nchunk);
  const int64_t gs = job / nchunk;
  j.side = (int)(gs & 1);
  j.gb = gs >> 1;
  j.gi = (int)(j.gb / B);
  j.b = (int)(j.gb % B);
  return j;
}

}  // namespace

// Gram pass.  T: storage type; accumulation in FP64.  One warp per job =
// ((gate * B + shot) * 2 + side) * nchunk + chunk.
// gram: [(gate * B + shot) * nchunk + chunk][4][chi * chi], block 2 * side + kappa.
template <typename T, int DMAX>
__global__ void __launch_bounds__(256) k_gram(SweepArgs a, const GateDesc* __restrict__ gates,
                                              double* __restrict__ gram, int64_t n_jobs, int nchunk, int chunk_rows) {
  constexpr int LPR = Shape<DMAX>::LPR, BPL = DMAX / LPR, RPW = 32 / LPR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int64_t job = (int64_t)blockIdx.x * wpb + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int chi = a.chi;
  double* lamv = reinterpret_cast<double*>(smem_raw) + (size_t)warp * kMaxBonds * chi;
  if (job >= n_jobs) return;
  const Job jb = decode_job(job, nchunk, a.B);
  const GateDesc& gd = gates[jb.gi];
  const SideDesc sd = gd.side[jb.side];
  const int D = gd.D;
  const double* lamb = a.lam + (int64_t)jb.b * a.nbonds * chi;
  for (int w = lane; w < kMaxBonds * chi; w += 32) {
    const int k = w / chi;
    lamv[w] = (k < sd.nb) ? lamb[sd.bond[k] * chi + (w % chi)] : 1.0;
  }
  __syncwarp();
  const Pairs pg = side_pairs(sd.P, sd.mask);
  const int OI = sd.outer * sd.inner;
  const int rows = pg.npairs * OI;
  const int r_begin = jb.ch * chunk_rows;
  const int r_end = min(rows, r_begin + chunk_rows);
  const int64_t SZ = (int64_t)OI * D;
  const T* gin = reinterpret_cast<const T*>(a.gamma) + (int64_t)jb.b * a.shot_elems + sd.in_off;
  const int slot = lane / LPR, sub = lane % LPR, row0 = slot * LPR;
  const int base = sub * BPL;
  double accp[BPL][DMAX], accm[BPL][DMAX];
#pragma unroll
  for (int k = 0; k < BPL; ++k)
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
      accp[k][j] = 0.0;
      accm[k][j] = 0.0;
    }
  for (int r0 = r_begin; r0 < r_end; r0 += RPW) {
    const int r = r0 + slot;
    const bool live = r < r_end;
    double yo[BPL], zo[BPL];
    {
      int pr = 0, o = 0, i = 0;
      double w = 0.0;
      if (live) {
        pr = r / OI;
        const int oi = r % OI;
        o = oi / sd.inner;
        i = oi % sd.inner;
        w = row_weight<double>(sd, o, i, lamv, chi);
      }
      const T* plo = gin + pg.lo(pr) * SZ + (int64_t)o * D * sd.inner + i;
      const T* phi = gin + pg.hi(pr) * SZ + (int64_t)o * D * sd.inner + i;
#pragma unroll
      for (int k = 0; k < BPL; ++k) {
        const int q = base + k;
        double lo = 0.0, hi = 0.0;
        if (live && q < D) {
          lo = double(plo[(int64_t)q * sd.inner]);
          hi = double(phi[(int64_t)q * sd.inner]);
        }
        yo[k] = (lo + hi) * w;
        zo[k] = (lo - hi) * w;
      }
    }
    double y[DMAX], z[DMAX];
#pragma unroll
    for (int q = 0; q < DMAX; ++q) {
      y[q] = __shfl_sync(0xffffffffu, yo[q % BPL], row0 + q / BPL);
      z[q] = __shfl_sync(0xffffffffu, zo[q % BPL], row0 + q / BPL);
    }
#pragma unroll
    for (int k = 0; k < BPL; ++k)
#pragma unroll
      for (int j = 0; j < DMAX; ++j) {
        accp[k][j] += yo[k] * y[j];
        accm[k][j] += zo[k] * z[j];
      }
  }
  // sum over the row slots of the warp (lanes with equal sub)
#pragma unroll
  for (int k = 0; k < BPL; ++k)
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
#pragma unroll
      for (int o = 16; o >= LPR; o >>= 1) {
        accp[k][j] += __shfl_xor_sync(0xffffffffu, accp[k][j], o);
        accm[k][j] += __shfl_xor_sync(0xffffffffu, accm[k][j], o);
      }
  if (slot == 0) {
    double* out = gram + (jb.gb * nchunk + jb.ch) * 4 * chi * chi + (int64_t)(2 * jb.side) * chi * chi;
#pragma unroll
    for (int k = 0; k < BPL; ++k)
#pragma unroll
      for (int j = 0; j < DMAX; ++j) {
        const int b1 = base + k;
        if (b1 < D && j < D) {
          out[b1 * D + j] = accp[k][j];
          out[chi * chi + b1 * D + j] = accm[k][j];
        }
      }
  }
}

// Gram pass for bond dimensions <= 8 using the symmetry of G+ and G-.  Two lanes per row;
// lane sub of a row holds the row with its halves swapped when sub = 1 (column q of the
// lane's copy is column q ^ 4*sub of the row), assembled by shuffles.  Both lanes accumulate
// the same fixed list of 20 entries (i, j) of their copy; lane sub's entry (i, j) is entry
// (i ^ 4 sub, j ^ 4 sub) of the Gram.  The list holds one entry of each orbit of the 36
// entries i <= j under i -> i ^ 4 (the four self-paired entries (i, i ^ 4) are computed by
// both lanes, with identical results): 20 products per row and Gram instead of 32.
namespace {
__device__ constexpr int kSymI[20] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3};
__device__ constexpr int kSymJ[20] = {0, 1, 2, 3, 4, 5, 6, 7, 1, 2, 3, 5, 6, 7, 2, 3, 6, 7, 3, 7};
}  // namespace

template <typename T>
__global__ void __launch_bounds__(256) k_gram_sym8(SweepArgs a, const GateDesc* __restrict__ gates,
                                                   double* __restrict__ gram, int64_t n_jobs, int nchunk,
                                                   int chunk_rows) {
  constexpr int LPR = 2, BPL = 4, RPW = 16, NE = 20;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int64_t job = (int64_t)blockIdx.x * wpb + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int chi = a.chi;
  double* lamv = reinterpret_cast<double*>(smem_raw) + (size_t)warp * kMaxBonds * chi;
  if (job >= n_jobs) return;
  const Job jb = decode_job(job, nchunk, a.B);
  const GateDesc& gd = gates[jb.gi];
  const SideDesc sd = gd.side[jb.side];
  const int D = gd.D;
  const double* lamb = a.lam + (int64_t)jb.b * a.nbonds * chi;
  for (int w = lane; w < kMaxBonds * chi; w += 32) {
    const int k = w / chi;
    lamv[w] = (k < sd.nb) ? lamb[sd.bond[k] * chi + (w % chi)] : 1.0;
  }
  __syncwarp();
  const Pairs pg = side_pairs(sd.P, sd.mask);
  const int OI = sd.outer * sd.inner;
  const int rows = pg.npairs * OI;
  const int r_begin = jb.ch * chunk_rows;
  const int r_end = min(rows, r_begin + chunk_rows);
  const int64_t SZ = (int64_t)OI * D;
  const T* gin = reinterpret_cast<const T*>(a.gamma) + (int64_t)jb.b * a.shot_elems + sd.in_off;
  const int slot = lane / LPR, sub = lane % LPR, row0 = slot * LPR;
  double accp[NE], accm[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    accp[e] = 0.0;
    accm[e] = 0.0;
  }
  for (int r0 = r_begin; r0 < r_end; r0 += RPW) {
    const int r = r0 + slot;
    const bool live = r < r_end;
    double yo[BPL], zo[BPL];
    {
      int pr = 0, o = 0, i = 0;
      double w = 0.0;
      if (live) {
        pr = r / OI;
        const int oi = r % OI;
        o = oi / sd.inner;
        i = oi % sd.inner;
        w = row_weight<double>(sd, o, i, lamv, chi);
      }
      const T* plo = gin + pg.lo(pr) * SZ + (int64_t)o * D * sd.inner + i;
      const T* phi = gin + pg.hi(pr) * SZ + (int64_t)o * D * sd.inner + i;
#pragma unroll
      for (int k = 0; k < BPL; ++k) {
        const int q = sub * BPL + k;
        double lo = 0.0, hi = 0.0;
        if (live && q < D) {
          lo = double(plo[(int64_t)q * sd.inner]);
          hi = double(phi[(int64_t)q * sd.inner]);
        }
        yo[k] = (lo + hi) * w;
        zo[k] = (lo - hi) * w;
      }
    }
    double y[8], z[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int src = row0 + ((q / BPL) ^ sub);
      y[q] = __shfl_sync(0xffffffffu, yo[q % BPL], src);
      z[q] = __shfl_sync(0xffffffffu, zo[q % BPL], src);
    }
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      accp[e] += y[kSymI[e]] * y[kSymJ[e]];
      accm[e] += z[kSymI[e]] * z[kSymJ[e]];
    }
  }
#pragma unroll
  for (int e = 0; e < NE; ++e)
#pragma unroll
    for (int o = 16; o >= LPR; o >>= 1) {
      accp[e] += __shfl_xor_sync(0xffffffffu, accp[e], o);
      accm[e] += __shfl_xor_sync(0xffffffffu, accm[e], o);
    }
  if (slot == 0) {
    double* out = gram + (jb.gb * nchunk + jb.ch) * 4 * chi * chi + (int64_t)(2 * jb.side) * chi * chi;
    const int sw = 4 * sub;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const int i = kSymI[e] ^ sw, j = kSymJ[e] ^ sw;
      if (i < D && j < D) {
        out[i * D + j] = accp[e];
        out[j * D + i] = accp[e];
        out[chi * chi + i * D + j] = accm[e];
        out[chi * chi + j * D + i] = accm[e];
      }
    }
  }
}

// Gram pass for bond dimensions 9..16 using the symmetry of G+ and G-.  Eight lanes per row;
// lane sub holds the row with its index permuted by q -> q ^ 2 sub (assembled by shuffles),
// and every lane accumulates the same list of 24 entries (i, j) of its copy, which is entry
// (i ^ 2 sub, j ^ 2 sub) of the Gram.  The list holds one entry of each orbit of the 136
// entries i <= j under the eight maps q -> q ^ 2s: (0, j) for every j and (1, j) for odd j;
// the orbits of the entries (i, i ^ 2s) have four elements and are computed twice, with
// identical results.  24 products per row and Gram instead of 32.
namespace {
__device__ constexpr int kSym16I[24] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1};
__device__ constexpr int kSym16J[24] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 1, 3, 5, 7, 9, 11, 13, 15};
}  // namespace

template <typename T>
__global__ void __launch_bounds__(256) k_gram_sym16(SweepArgs a, const GateDesc* __restrict__ gates,
                                                    double* __restrict__ gram, int64_t n_jobs, int nchunk,
                                                    int chunk_rows) {
  constexpr int LPR = 8, BPL = 2, RPW = 4, NE = 24;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int64_t job = (int64_t)blockIdx.x * wpb + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int chi = a.chi;
  double* lamv = reinterpret_cast<double*>(smem_raw) + (size_t)warp * kMaxBonds * chi;
  if (job >= n_jobs) return;
  const Job jb = decode_job(job, nchunk, a.B);
  const GateDesc& gd = gates[jb.gi];
  const SideDesc sd = gd.side[jb.side];
  const int D = gd.D;
  const double* lamb = a.lam + (int64_t)jb.b * a.nbonds * chi;
  for (int w = lane; w < kMaxBonds * chi; w += 32) {
    const int k = w / chi;
    lamv[w] = (k < sd.nb) ? lamb[sd.bond[k] * chi + (w % chi)] : 1.0;
  }
  __syncwarp();
  const Pairs pg = side_pairs(sd.P, sd.mask);
  const int OI = sd.outer * sd.inner;
  const int rows = pg.npairs * OI;
  const int r_begin = jb.ch * chunk_rows;
  const int r_end = min(rows, r_begin + chunk_rows);
  const int64_t SZ = (int64_t)OI * D;
  const T* gin = reinterpret_cast<const T*>(a.gamma) + (int64_t)jb.b * a.shot_elems + sd.in_off;
  const int slot = lane / LPR, sub = lane % LPR, row0 = slot * LPR;
  double accp[NE], accm[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    accp[e] = 0.0;
    accm[e] = 0.0;
  }
  for (int r0 = r_begin; r0 < r_end; r0 += RPW) {
    const int r = r0 + slot;
    const bool live = r < r_end;
    double yo[BPL], zo[BPL];
    {
      int pr = 0, o = 0, i = 0;
      double w = 0.0;
      if (live) {
        pr = r / OI;
        const int oi = r % OI;
        o = oi / sd.inner;
        i = oi % sd.inner;
        w = row_weight<double>(sd, o, i, lamv, chi);
      }
      const T* plo = gin + pg.lo(pr) * SZ + (int64_t)o * D * sd.inner + i;
      const T* phi = gin + pg.hi(pr) * SZ + (int64_t)o * D * sd.inner + i;
#pragma unroll
      for (int k = 0; k < BPL; ++k) {
        const int q = sub * BPL + k;
        double lo = 0.0, hi = 0.0;
        if (live && q < D) {
          lo = double(plo[(int64_t)q * sd.inner]);
          hi = double(phi[(int64_t)q * sd.inner]);
        }
        yo[k] = (lo + hi) * w;
        zo[k] = (lo - hi) * w;
      }
    }
    double y[16], z[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int src = row0 + ((q >> 1) ^ sub);   // element q of the copy is element q ^ 2 sub of the row
      y[q] = __shfl_sync(0xffffffffu, yo[q & 1], src);
      z[q] = __shfl_sync(0xffffffffu, zo[q & 1], src);
    }
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      accp[e] += y[kSym16I[e]] * y[kSym16J[e]];
      accm[e] += z[kSym16I[e]] * z[kSym16J[e]];
    }
  }
#pragma unroll
  for (int e = 0; e < NE; ++e)
#pragma unroll
    for (int o = 16; o >= LPR; o >>= 1) {
      accp[e] += __shfl_xor_sync(0xffffffffu, accp[e], o);
      accm[e] += __shfl_xor_sync(0xffffffffu, accm[e], o);
    }
  if (slot == 0) {
    double* out = gram + (jb.gb * nchunk + jb.ch) * 4 * chi * chi + (int64_t)(2 * jb.side) * chi * chi;
    const int sw = 2 * sub;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const int i = kSym16I[e] ^ sw, j = kSym16J[e] ^ sw;
      if (i < D && j < D) {
        out[i * D + j] = accp[e];
        out[j * D + i] = accp[e];
        out[chi * chi + i * D + j] = accm[e];
        out[chi * chi + j * D + i] = accm[e];
      }
    }
  }
}

// Update pass: Gamma_new[lo] = Y T+ + Z T-, Gamma_new[hi] = Y T+ - Z T-, in FP64 arithmetic
// for both storage types (T), the result rounded to the storage type.
template <typename T, int DMAX>
__global__ void __launch_bounds__(256) k_update(SweepArgs a, const GateDesc* __restrict__ gates,
                                                    const double* __restrict__ tbuf, int64_t n_jobs, int nchunk,
                                                    int chunk_rows) {
  constexpr int LPR = Shape<DMAX>::LPR, BPL = DMAX / LPR, RPW = 32 / LPR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int64_t job = (int64_t)blockIdx.x * wpb + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int chi = a.chi;
  double* Tp = reinterpret_cast<double*>(smem_raw) + (size_t)warp * 2 * DMAX * DMAX;   // [DMAX][DMAX]
  double* Tm = Tp + DMAX * DMAX;
  if (job >= n_jobs) return;
  const Job jb = decode_job(job, nchunk, a.B);
  const GateDesc& gd = gates[jb.gi];
  const SideDesc sd = gd.side[jb.side];
  const int D = gd.D, Dn = gd.Dn;
  const double* tsrc = tbuf + jb.gb * 4 * chi * chi + (int64_t)jb.side * 2 * chi * chi;
  for (int w = lane; w < DMAX * DMAX; w += 32) {
    const int q = w / DMAX, j = w % DMAX;
    const bool in = q < D && j < Dn;
    Tp[w] = in ? tsrc[q * Dn + j] : 0.0;
    Tm[w] = in ? tsrc[chi * chi + q * Dn + j] : 0.0;
  }
  __syncwarp();
  const Pairs pg = side_pairs(sd.P, sd.mask);
  const int OI = sd.outer * sd.inner;
  const int rows = pg.npairs * OI;
  const int r_begin = jb.ch * chunk_rows;
  const int r_end = min(rows, r_begin + chunk_rows);
  const int64_t SZ = (int64_t)OI * D, SZn = (int64_t)OI * Dn;
  const T* gin = reinterpret_cast<const T*>(a.gamma) + (int64_t)jb.b * a.shot_elems + sd.in_off;
  T* gout = reinterpret_cast<T*>(a.gamma) + (int64_t)jb.b * a.shot_elems + sd.out_off;
  const int slot = lane / LPR, sub = lane % LPR, row0 = slot * LPR;
  const int base = sub * BPL;
  for (int r0 = r_begin; r0 < r_end; r0 += RPW) {
    const int r = r0 + slot;
    const bool live = r < r_end;
    int pr = 0, o = 0, i = 0;
    if (live) {
      pr = r / OI;
      const int oi = r % OI;
      o = oi / sd.inner;
      i = oi % sd.inner;
    }
    double yo[BPL], zo[BPL];
    {
      const T* plo = gin + pg.lo(pr) * SZ + (int64_t)o * D * sd.inner + i;
      const T* phi = gin + pg.hi(pr) * SZ + (int64_t)o * D * sd.inner + i;
#pragma unroll
      for (int k = 0; k < BPL; ++k) {
        const int q = base + k;
        double lo = 0.0, hi = 0.0;
        if (live && q < D) {
          lo = double(plo[(int64_t)q * sd.inner]);
          hi = double(phi[(int64_t)q * sd.inner]);
        }
        yo[k] = lo + hi;
        zo[k] = lo - hi;
      }
    }
    double y[DMAX], z[DMAX];
#pragma unroll
    for (int q = 0; q < DMAX; ++q) {
      y[q] = __shfl_sync(0xffffffffu, yo[q % BPL], row0 + q / BPL);
      z[q] = __shfl_sync(0xffffffffu, zo[q % BPL], row0 + q / BPL);
    }
    T* qlo = gout + pg.lo(pr) * SZn + (int64_t)o * Dn * sd.inner + i;
    T* qhi = gout + pg.hi(pr) * SZn + (int64_t)o * Dn * sd.inner + i;
#pragma unroll
    for (int k = 0; k < BPL; ++k) {
      const int j = base + k;
      double u1 = 0.0, u2 = 0.0;
#pragma unroll
      for (int q = 0; q < DMAX; ++q) {
        u1 += y[q] * Tp[q * DMAX + j];
        u2 += z[q] * Tm[q * DMAX + j];
      }
      if (live && j < Dn) {
        qlo[(int64_t)j * sd.inner] = T(u1 + u2);
        qhi[(int64_t)j * sd.inner] = T(u1 - u2);
      }
    }
  }
}

// ---- launchers -----------------------------------------------------------------------------
int absorb_dmax(int D) { return D <= 8 ? 8 : (D <= 16 ? 16 : 32); }

int absorb_chunks(int max_rows, int chunk_rows) { return std::max(1, (max_rows + chunk_rows - 1) / chunk_rows); }

template <typename T, int DMAX>
static cudaError_t gram_launch(const SweepArgs& a, const GateDesc* g, int count, double* gram, int nchunk,
                               int chunk_rows, cudaStream_t st) {
  const int wpb = DMAX >= 32 ? 4 : 8;
  const int64_t n_jobs = (int64_t)count * a.B * 2 * nchunk;
  const unsigned blocks = (unsigned)((n_jobs + wpb - 1) / wpb);
  const size_t smem = (size_t)wpb * kMaxBonds * a.chi * sizeof(double);
  if constexpr (DMAX == 8) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_sym8<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_sym8<T><<<blocks, wpb * 32, smem, st>>>(a, g, gram, n_jobs, nchunk, chunk_rows);
  } else if constexpr (DMAX == 16) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_sym16<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_sym16<T><<<blocks, wpb * 32, smem, st>>>(a, g, gram, n_jobs, nchunk, chunk_rows);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_gram<T, DMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram<T, DMAX><<<blocks, wpb * 32, smem, st>>>(a, g, gram, n_jobs, nchunk, chunk_rows);
  }
  return cudaGetLastError();
}

template <typename T, int DMAX>
static cudaError_t update_launch(const SweepArgs& a, const GateDesc* g, int count, const double* tbuf, int nchunk,
                                 int chunk_rows, cudaStream_t st) {
  const int wpb = DMAX >= 32 ? 4 : 8;
  const int64_t n_jobs = (int64_t)count * a.B * 2 * nchunk;
  const unsigned blocks = (unsigned)((n_jobs + wpb - 1) / wpb);
  const size_t smem = (size_t)wpb * 2 * DMAX * DMAX * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_update<T, DMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_update<T, DMAX><<<blocks, wpb * 32, smem, st>>>(a, g, tbuf, n_jobs, nchunk, chunk_rows);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram2(const SweepArgs& a, const GateDesc* g, int count, int Dm, double* gram, int nchunk,
                         int chunk_rows, cudaStream_t st) {
  switch (absorb_dmax(Dm)) {
    case 8: return gram_launch<T, 8>(a, g, count, gram, nchunk, chunk_rows, st);
    case 16: return gram_launch<T, 16>(a, g, count, gram, nchunk, chunk_rows, st);
    default: return gram_launch<T, 32>(a, g, count, gram, nchunk, chunk_rows, st);
  }
}

template <typename T>
cudaError_t launch_update2(const SweepArgs& a, const GateDesc* g, int count, int Dm, const double* tbuf, int nchunk,
                           int chunk_rows, cudaStream_t st) {
  switch (absorb_dmax(Dm)) {
    case 8: return update_launch<T, 8>(a, g, count, tbuf, nchunk, chunk_rows, st);
    case 16: return update_launch<T, 16>(a, g, count, tbuf, nchunk, chunk_rows, st);
    default: return update_launch<T, 32>(a, g, count, tbuf, nchunk, chunk_rows, st);
  }
}

template cudaError_t launch_gram2<float>(const SweepArgs&, const GateDesc*, int, int, double*, int, int, cudaStream_t);
template cudaError_t launch_gram2<double>(const SweepArgs&, const GateDesc*, int, int, double*, int, int,
                                          cudaStream_t);
template cudaError_t launch_update2<float>(const SweepArgs&, const GateDesc*, int, int, const double*, int, int,
                                           cudaStream_t);
template cudaError_t launch_update2<double>(const SweepArgs&, const GateDesc*, int, int, const double*, int, int,
                                            cudaStream_t);

}  // namespace td
