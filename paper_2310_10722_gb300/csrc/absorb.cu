// Gate absorption passes of the sweep (Sec. 4): the Gram pass and the update pass of the
// simple update, one warp per (gate side, shot, row chunk).
//
// The two-site gate (1-p) I x I + p X x X is applied by doubling its bond (see sweep.cu):
// with Y = M[sigma_lo] + M[sigma_hi] and Z = M[sigma_lo] - M[sigma_hi] for each physical
// pair sigma_hi = sigma_lo ^ mask, the Gram of the doubled side matrix is block diagonal,
// G+ = sum_rows Y^T Y and G- = sum_rows Z^T Z (rows weighted by the other bonds' lambda), and
// the update is Gamma_new[lo] = Y T+ + Z T-, Gamma_new[hi] = Y T+ - Z T-.  The diagonal gate
// diag(w(r + s_a + s_b)) of the generator picture (Sec. 3.2; GateDesc.diag) doubles its bond
// with kappa = the physical bit: Y = M[sigma_lo], Z = M[sigma_hi], and the update is
// Gamma_new[lo] = Y T0, Gamma_new[hi] = Z T1.
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
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "sweep.cuh"
#include "tc.cuh"

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
  const bool dg = gd.diag != 0;   // diagonal gate: the blocks are lo and hi themselves
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
        yo[k] = (dg ? lo : lo + hi) * w;
        zo[k] = (dg ? hi : lo - hi) * w;
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
  const bool dg = gd.diag != 0;   // diagonal gate: the blocks are lo and hi themselves
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
        yo[k] = (dg ? lo : lo + hi) * w;
        zo[k] = (dg ? hi : lo - hi) * w;
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
  const bool dg = gd.diag != 0;   // diagonal gate: the blocks are lo and hi themselves
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
        yo[k] = (dg ? lo : lo + hi) * w;
        zo[k] = (dg ? hi : lo - hi) * w;
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
  const bool dg = gd.diag != 0;   // diagonal gate: the blocks are lo and hi themselves
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
        yo[k] = dg ? lo : lo + hi;
        zo[k] = dg ? hi : lo - hi;
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
        qlo[(int64_t)j * sd.inner] = T(dg ? u1 : u1 + u2);
        qhi[(int64_t)j * sd.inner] = T(dg ? u2 : u1 - u2);
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


// ---- Gram pass on the tensor cores (tcgen05), exact BF16 slices ------------------------------
// G+ = Y^T Y and G- = Z^T Z of one job (gate side, shot, row chunk) as products of BF16 slices
// on the tensor cores (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", 2012: split the operands
// into slices whose pairwise products are summed without rounding, then add the slice
// products in higher precision).
//   1. Column bound: b_q = max over the chunk's rows of (|lo| + |hi|) w, and a power of two
//      2^E_q > b_q with one bit of margin, so every |y|, |z| of column q is below 2^E_q.
//   2. Per block of KB rows, y = (lo + hi) w and z = (lo - hi) w are cut into kTcSlices
//      integer slices t_i below the bound: y 2^-E = sum_i t_i 2^(-BITS (i+1)) up to the last
//      slice.  FP64 storage: y, z in FP64, the slices read off the 63-bit fixed-point value
//      |y| 2^(63-E) (BITS = 7, |t_i| <= 127, 56 bits kept).  FP32 storage: y, z as exact FP32
//      pairs (TwoSum of lo, hi; TwoProduct with w = w1 + w2; the dropped term is below 2^-47
//      |y|), each part sliced by 6 bits and the slices added (BITS = 6, |t_i| <= 126, 48
//      bits).  Every slice is an integer below 2^8, exact in BF16.
//   3. The slices of a block form the K-major operand S (row a = (slice i, column q), K = the
//      block's rows) and one MMA chain accumulates S S^T in TMEM (FP32).  Its entries sum
//      products of integers below 2^14 over at most kTcGroupRows = 1024 rows: every partial
//      sum is an integer below 2^24, exact.
//   4. Every 1024 rows the accumulator is read (tcgen05.ld) and combined in FP64:
//      G[q][q'] = 2^(E_q + E_q') sum_(i,j) 2^(-BITS (i+j+2)) (S S^T)[(i,q),(j,q')].
// DPAD = 16 (bond dimensions 9..16): two operands (Y, Z) of 128 rows, two 128-column
// accumulators.  DPAD = 8 (bond dimensions 4..8): one operand with Y's 64 rows above Z's.
namespace {
constexpr int kTcSlices = 8;
constexpr int kTcGroupRows = 1024;
constexpr int kTcThreads = 256;
constexpr int kTcMaxPolls = 1 << 22;   // bounded MMA-completion wait, then TD_ERR_TIMEOUT
template <int DPAD>
struct TcCfg;
template <>
struct TcCfg<8> { static constexpr int KB = 256, NACC = 1, NCOL = 128; };
template <>
struct TcCfg<16> { static constexpr int KB = 128, NACC = 2, NCOL = 256; };
template <typename T>
struct TcBits;
template <>
struct TcBits<float> { static constexpr int BITS = 6; };
template <>
struct TcBits<double> { static constexpr int BITS = 7; };

template <int DPAD>
constexpr size_t tc_operand_bytes() { return (size_t)TcCfg<DPAD>::NACC * 128 * TcCfg<DPAD>::KB * 2; }
// dynamic shared memory: operands, the block's row weights [KB] (8 bytes each), the
// environment lambdas [kMaxBonds][chi] (FP64); padded so that at most two blocks share an SM
// (two 256-column TMEM accumulators fill the SM's 512 columns)
template <int DPAD>
size_t tc_smem_bytes(int chi) {
  const size_t need = tc_operand_bytes<DPAD>() + (size_t)TcCfg<DPAD>::KB * 8 + (size_t)kMaxBonds * chi * 8;
  return std::max<size_t>(need, 100 * 1024);
}

// 2^e as a double for -1022 <= e <= 1023 (exact, integer operations only).
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// FP32 storage: slices of v = x1 + x2 (x1, x2 already scaled into (-1, 1)), six bits of
// each part per slice, summed.
__device__ __forceinline__ void tc_slices32(float x1, float x2, float (&t)[kTcSlices]) {
#pragma unroll
  for (int i = 0; i < kTcSlices; ++i) {
    x1 *= 64.f;
    x2 *= 64.f;
    const float a1 = truncf(x1), a2 = truncf(x2);
    x1 -= a1;
    x2 -= a2;
    t[i] = a1 + a2;
  }
}

// (lo + hi) w as an FP32 pair: exact sum, then the product with w1 + w2.
__device__ __forceinline__ void tc_pair(float lo, float hi, float w1, float w2, float& y1, float& y2) {
  const float s1 = lo + hi;
  const float bb = s1 - lo;
  const float s2 = (lo - (s1 - bb)) + (hi - bb);
  const float p = s1 * w1;
  const float e = fmaf(s1, w1, -p);
  y1 = p;
  y2 = e + fmaf(s1, w2, s2 * w1);
}

// FP64 storage: slices of v with |v| < 2^E from its bit pattern: F = floor(|v| 2^(63-E)) < 2^63,
// slice i = bits 62-7i .. 56-7i of F (as an exact float, with v's sign).
__device__ __forceinline__ void tc_slices64(double v, int E, float (&t)[kTcSlices]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int ev = (int)((bits >> 52) & 0x7FFull);
  unsigned long long F = 0ull;
  if (ev != 0) {
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = (ev - 1075) + 63 - E;
    if (sh >= 0)
      F = mant << sh;
    else if (sh > -64)
      F = mant >> (-sh);
  }
  const unsigned sgn = (unsigned)(bits >> 63) << 31;
#pragma unroll
  for (int i = 0; i < kTcSlices; ++i) {
    const unsigned u = (unsigned)(F >> (56 - 7 * i)) & 0x7Fu;
    t[i] = __uint_as_float(__float_as_uint(__int_as_float(0x4B000000 | (int)u) - 8388608.f) | sgn);
  }
}
}  // namespace

template <typename T, int DPAD>
__global__ void __launch_bounds__(kTcThreads, 2) k_gram_tc(SweepArgs a, const GateDesc* __restrict__ gates,
                                                        double* __restrict__ gram, int64_t n_jobs, int nchunk,
                                                        int chunk_rows) {
  using Cfg = TcCfg<DPAD>;
  constexpr int KB = Cfg::KB, NACC = Cfg::NACC, NCOL = Cfg::NCOL, BITS = TcBits<T>::BITS;
  constexpr uint32_t IDESC = tc::idesc_bf16(128, 128);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_holder;
  __shared__ unsigned int colbits[DPAD];
  __shared__ int colexp[DPAD];
  __shared__ float colscale[DPAD];
  unsigned char* opnd = smem_raw;
  double* wt = reinterpret_cast<double*>(smem_raw + tc_operand_bytes<DPAD>());   // [KB] row weights
  double* lamv = wt + KB;
  double* red = reinterpret_cast<double*>(smem_raw);   // end-of-job reduction (aliases the operands)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int chi = a.chi;
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tmem_holder, NCOL);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  uint32_t phase = 0;
  bool failed = false;
  const int qi = tid % DPAD, kg = tid / DPAD;   // slicing item: column qi, rows 8 kg .. 8 kg + 7
  for (int64_t job = blockIdx.x; job < n_jobs && !failed; job += gridDim.x) {
    const Job jb = decode_job(job, nchunk, a.B);
    const GateDesc& gd = gates[jb.gi];
    const SideDesc sd = gd.side[jb.side];
    const bool dg = gd.diag != 0;   // diagonal gate: the blocks are lo and hi themselves
    const int D = gd.D;
    const double* lamb = a.lam + (int64_t)jb.b * a.nbonds * chi;
    for (int w = tid; w < kMaxBonds * chi; w += kTcThreads) {
      const int k = w / chi;
      lamv[w] = (k < sd.nb) ? lamb[sd.bond[k] * chi + (w % chi)] : 1.0;
    }
    if (tid < DPAD) colbits[tid] = 0u;
    __syncthreads();
    const Pairs pg = side_pairs(sd.P, sd.mask);
    const int OI = sd.outer * sd.inner;
    const int rows = pg.npairs * OI;
    const int r_begin = jb.ch * chunk_rows;
    const int r_end = min(rows, r_begin + chunk_rows);
    const int64_t SZ = (int64_t)OI * D;
    const int inner = sd.inner;
    const T* gin = reinterpret_cast<const T*>(a.gamma) + (int64_t)jb.b * a.shot_elems + sd.in_off;
    // 1. column bounds (the FP32 value of each bound; the exponent below has a bit of margin)
    {
      float cm[DPAD];
#pragma unroll
      for (int c = 0; c < DPAD; ++c) cm[c] = 0.f;
      for (int r = r_begin + tid; r < r_end; r += kTcThreads) {
        const int pr = r / OI, oi = r % OI, o = oi / inner, i = oi % inner;
        const T w = T(row_weight<double>(sd, o, i, lamv, chi));
        const T* plo = gin + pg.lo(pr) * SZ + (int64_t)o * D * inner + i;
        const T* phi = gin + pg.hi(pr) * SZ + (int64_t)o * D * inner + i;
#pragma unroll
        for (int c = 0; c < DPAD; ++c)
          if (c < D) cm[c] = fmaxf(cm[c], float((fabs(plo[(int64_t)c * inner]) + fabs(phi[(int64_t)c * inner])) * w));
      }
#pragma unroll
      for (int c = 0; c < DPAD; ++c) {
        float v = cm[c];
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0 && v > 0.f) atomicMax(&colbits[c], __float_as_uint(v));
      }
    }
    __syncthreads();
    if (tid < DPAD) {
      const float bnd = __uint_as_float(colbits[tid]);
      int e = -100;
      if (bnd > 0.f) {
        frexpf(bnd, &e);   // bnd < 2^e
        e = min(max(e + 1, -100), 100);
      }
      colexp[tid] = e;
      colscale[tid] = ldexpf(1.f, -e);
    }
    double part[DPAD];
#pragma unroll
    for (int c = 0; c < DPAD; ++c) part[c] = 0.0;
    int grp_rows = 0;
    const int nblk = (r_end - r_begin + KB - 1) / KB;
    for (int blk = 0; blk < nblk; ++blk) {
      const int rb = r_begin + blk * KB;
      // 2. row weights of the block
      for (int k = tid; k < KB; k += kTcThreads) {
        const int r = rb + k;
        double w = 0.0;
        if (r < r_end) {
          const int oi = r % OI;
          w = row_weight<double>(sd, oi / inner, oi % inner, lamv, chi);
        }
        wt[k] = w;
      }
      __syncthreads();
      {
        T lo8[8], hi8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int r = rb + kg * 8 + u;
          lo8[u] = T(0);
          hi8[u] = T(0);
          if (qi < D && r < r_end) {
            const int pr = r / OI, oi = r % OI, o = oi / inner, i = oi % inner;
            const int64_t off = (int64_t)o * D * inner + (int64_t)qi * inner + i;
            lo8[u] = gin[pg.lo(pr) * SZ + off];
            hi8[u] = gin[pg.hi(pr) * SZ + off];
          }
        }
        const float sc = colscale[qi];
        const int E = colexp[qi];
#pragma unroll
        for (int pt = 0; pt < 2; ++pt) {
          uint32_t pk[kTcSlices][4];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float t0[kTcSlices], t1[kTcSlices];
            const int k0 = kg * 8 + 2 * v;
            if constexpr (sizeof(T) == 4) {
              float y1, y2;
              const double w0 = wt[k0], w1 = wt[k0 + 1];
              const float w0a = (float)w0, w1a = (float)w1;
              // X x X gate: (lo + hi) w, (lo - hi) w; diagonal gate: lo w, hi w
              const float a0 = dg ? (pt ? 0.f : lo8[2 * v]) : lo8[2 * v];
              const float b0 = dg ? (pt ? hi8[2 * v] : 0.f) : (pt ? -hi8[2 * v] : hi8[2 * v]);
              const float a1 = dg ? (pt ? 0.f : lo8[2 * v + 1]) : lo8[2 * v + 1];
              const float b1 = dg ? (pt ? hi8[2 * v + 1] : 0.f) : (pt ? -hi8[2 * v + 1] : hi8[2 * v + 1]);
              tc_pair(a0, b0, w0a, (float)(w0 - (double)w0a), y1, y2);
              tc_slices32(y1 * sc, y2 * sc, t0);
              tc_pair(a1, b1, w1a, (float)(w1 - (double)w1a), y1, y2);
              tc_slices32(y1 * sc, y2 * sc, t1);
            } else {
              // X x X gate: (lo + hi) w, (lo - hi) w; diagonal gate: lo w, hi w
              const double y0 = dg ? (pt ? hi8[2 * v] : lo8[2 * v]) : (pt ? lo8[2 * v] - hi8[2 * v] : lo8[2 * v] + hi8[2 * v]);
              const double y1v = dg ? (pt ? hi8[2 * v + 1] : lo8[2 * v + 1])
                                    : (pt ? lo8[2 * v + 1] - hi8[2 * v + 1] : lo8[2 * v + 1] + hi8[2 * v + 1]);
              tc_slices64(y0 * wt[k0], E, t0);
              tc_slices64(y1v * wt[k0 + 1], E, t1);
            }
#pragma unroll
            for (int i = 0; i < kTcSlices; ++i) {
              const __nv_bfloat162 h = __floats2bfloat162_rn(t0[i], t1[i]);
              pk[i][v] = *reinterpret_cast<const uint32_t*>(&h);
            }
          }
          unsigned char* base = opnd + (NACC == 2 ? (size_t)pt * 128 * KB * 2 : 0);
          const int row_off = (NACC == 2) ? 0 : pt * 64;
#pragma unroll
          for (int i = 0; i < kTcSlices; ++i) {
            const int arow = row_off + i * DPAD + qi;
            *reinterpret_cast<uint4*>(base + tc::kmajor_off(arow, kg * 8, KB)) =
                make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
          }
        }
      }
      // 3. one MMA chain over the block
      tc::fence_smem_async();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t b0 = tc::smem_u32(opnd);
#pragma unroll 1
        for (int ks = 0; ks < KB / 16; ++ks)
#pragma unroll
          for (int p = 0; p < NACC; ++p) {
            const uint64_t d = tc::sdesc(b0 + (uint32_t)(p * 128 * KB * 2 + ks * 256), 128, (KB / 8) * 128);
            tc::mma_bf16(tmem + (uint32_t)(p * 128), d, d, IDESC, (grp_rows > 0 || ks > 0) ? 1u : 0u);
          }
        tc::commit(&mbar);
      }
      const bool ok = tc::mbar_wait(&mbar, phase, kTcMaxPolls);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc::fence_after_sync();
      grp_rows += KB;
      if (grp_rows >= kTcGroupRows || blk == nblk - 1) {
        // 4. read the accumulator(s) and add the slice products in FP64
        if (NACC == 2) {
          const int sub = warp & 3, sel = warp >> 2;
          const int ia = (sub * 32 + lane) / DPAD;
#pragma unroll 1
          for (int j = 0; j < kTcSlices; ++j) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(sel * 128 + j * 16), v);
            const double scl = pow2d(-BITS * (ia + j + 2));
#pragma unroll
            for (int c = 0; c < DPAD; ++c) part[c] += (double)v[c] * scl;
          }
        } else if (warp < 4) {
          const int arow = warp * 32 + lane;
          const int pa = arow / 64, ia = (arow % 64) / DPAD;
#pragma unroll 1
          for (int jj = 0; jj < kTcSlices / 2; ++jj) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(pa * 64 + jj * 16), v);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const double scl = pow2d(-BITS * (ia + 2 * jj + h + 2));
#pragma unroll
              for (int c = 0; c < DPAD; ++c) part[c] += (double)v[h * DPAD + c] * scl;
            }
          }
        }
        grp_rows = 0;
        tc::fence_before_sync();
      }
      __syncthreads();
    }
    if (failed) break;
    // end of job: sum the partials of the slice lanes (i) of every (part, q)
    if (NACC == 2) {
      const int row = (warp >> 2) * 128 + (warp & 3) * 32 + lane;
#pragma unroll
      for (int c = 0; c < DPAD; ++c) red[row * DPAD + c] = part[c];
    } else if (warp < 4) {
      const int row = warp * 32 + lane;
#pragma unroll
      for (int c = 0; c < DPAD; ++c) red[row * DPAD + c] = part[c];
    }
    __syncthreads();
    double* out = gram + (jb.gb * nchunk + jb.ch) * 4 * chi * chi + (int64_t)(2 * jb.side) * chi * chi;
    for (int w = tid; w < 2 * D * D; w += kTcThreads) {
      const int pt = w / (D * D), qa = (w / D) % D, qb = w % D;
      const int rbase = (NACC == 2) ? pt * 128 : pt * 64;
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < kTcSlices; ++i) s += red[(rbase + i * DPAD + qa) * DPAD + qb];
      out[(int64_t)pt * chi * chi + qa * D + qb] = ldexp(s, colexp[qa] + colexp[qb]);
    }
    __syncthreads();
  }
  if (failed && tid == 0 && a.status) atomicExch(a.status, (int)TD_ERR_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, NCOL);
}

template <typename T, int DPAD>
static cudaError_t gram_tc_launch(const SweepArgs& a, const GateDesc* g, int count, double* gram, int nchunk,
                                  int chunk_rows, cudaStream_t st) {
  const int64_t n_jobs = (int64_t)count * a.B * 2 * nchunk;
  if (n_jobs == 0) return cudaSuccess;
  const size_t smem = tc_smem_bytes<DPAD>(a.chi);
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc<T, DPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(n_jobs, 2LL * nsm);
  k_gram_tc<T, DPAD><<<(unsigned)grid, kTcThreads, smem, st>>>(a, g, gram, n_jobs, nchunk, chunk_rows);
  return cudaGetLastError();
}

bool gram_tc_supported(int maxD) { return maxD >= 4 && maxD <= 16; }

template <typename T>
cudaError_t launch_gram_tc(const SweepArgs& a, const GateDesc* g, int count, int maxD, double* gram, int nchunk,
                           int chunk_rows, cudaStream_t st) {
  return maxD <= 8 ? gram_tc_launch<T, 8>(a, g, count, gram, nchunk, chunk_rows, st)
                   : gram_tc_launch<T, 16>(a, g, count, gram, nchunk, chunk_rows, st);
}
template cudaError_t launch_gram_tc<float>(const SweepArgs&, const GateDesc*, int, int, double*, int, int, cudaStream_t);
template cudaError_t launch_gram_tc<double>(const SweepArgs&, const GateDesc*, int, int, double*, int, int,
                                            cudaStream_t);

template cudaError_t launch_gram2<float>(const SweepArgs&, const GateDesc*, int, int, double*, int, int, cudaStream_t);
template cudaError_t launch_gram2<double>(const SweepArgs&, const GateDesc*, int, int, double*, int, int,
                                          cudaStream_t);
template cudaError_t launch_update2<float>(const SweepArgs&, const GateDesc*, int, int, const double*, int, int,
                                           cudaStream_t);
template cudaError_t launch_update2<double>(const SweepArgs&, const GateDesc*, int, int, const double*, int, int,
                                            cudaStream_t);

}  // namespace td
