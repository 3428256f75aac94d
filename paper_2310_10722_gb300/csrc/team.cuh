// Team-cooperative dense linear algebra for the small FP64/FP32 factorisations of the
// sweep (Sec. 4 simple-update truncation) and of the final boundary-MPS contraction.
//
// A team is a group of nt threads of one block (nt = 32: one warp, synchronised with
// __syncwarp; nt a larger multiple of 32: its own named barrier).  Several teams share a
// block, each working on an independent problem, so no step waits on a block-wide barrier.
//
// Methods (textbook, written for this layout):
//   * pivoted Cholesky of a positive semi-definite Gram matrix (Golub & Van Loan,
//     Matrix Computations, 4th ed., Alg. 4.2.4 with diagonal pivoting, Sec. 4.2.8), stopped
//     at the first pivot below a tolerance: a rank-revealing R factor of the Gram's matrix;
//   * the inverse of the triangular part by back substitution (ibid. Sec. 3.1);
//   * the one-sided (Hestenes) Jacobi SVD with the round-robin parallel ordering
//     (ibid. Sec. 8.6.3 and 8.5.5): the n/2 column pairs of one step are disjoint, so each
//     pair is handled by its own group of g lanes, which computes the pair's three inner
//     products (lane partial sums combined by shuffles), the rotation (the symmetric 2x2
//     Schur rotation, ibid. Alg. 8.5.1), and applies it to both columns of A and of V.
//     One barrier per step.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace td {

struct Team {
  int tid;   // thread index inside the team
  int nt;    // team size: 32, or a multiple of 32 using named barrier `bar`
  int bar;   // named barrier id (1..15), unused for nt == 32
  __device__ __forceinline__ void sync() const {
    if (nt == 32)
      __syncwarp();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
  }
};

template <typename R>
struct TeamTol;
template <>
struct TeamTol<double> {
  static __device__ __forceinline__ double rel() { return 1e-15; }
  static __device__ __forceinline__ double tiny() { return 1e-290; }
};
template <>
struct TeamTol<float> {
  static __device__ __forceinline__ float rel() { return 1e-7f; }
  static __device__ __forceinline__ float tiny() { return 1e-30f; }
};

// Pair i of step k of the round-robin ("circle") ordering of ne (even) players; player
// ne-1 stays in place.  p < q on return.
__device__ __forceinline__ void team_rr_pair(int k, int i, int ne, int& p, int& q) {
  const int m = ne - 1;
  if (i == 0) {
    p = k;
    q = m;
  } else {
    p = (k + i) % m;
    q = (k - i + m) % m;
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// Pivoted Cholesky of the symmetric positive semi-definite D x D matrix G (row-major,
// leading dimension ldg; destroyed), D <= 32.  Pivot k is the largest remaining diagonal
// entry; the factorisation stops when it is <= tol.  On return rows 0..r-1 of Rf (ld ldr)
// hold the factor in the original column order -- G ~= Rf^T Rf, Rf[i][piv[j]] = 0 for
// j < i -- and piv[0..r) the pivot columns.  `shr` is 2 ints of team-shared scratch.
// Returns the rank r.
template <typename R>
__device__ int team_pchol(const Team& tm, R* G, int ldg, int D, R tol, R* Rf, int ldr, int* piv, int* shr) {
  uint32_t done = 0;
  int r = 0;
  for (int k = 0; k < D; ++k) {
    if (tm.tid < 32) {
      const int lane = tm.tid;
      R v = (lane < D && !((done >> lane) & 1u)) ? G[lane * ldg + lane] : R(-1);
      int idx = lane;
      for (int o = 16; o > 0; o >>= 1) {
        const R v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (v2 > v || (v2 == v && i2 < idx)) {
          v = v2;
          idx = i2;
        }
      }
      if (lane == 0) {
        shr[0] = idx;
        shr[1] = (v > tol) ? 1 : 0;
      }
    }
    tm.sync();
    const int p = shr[0];
    if (!shr[1]) break;
    const R rkk = sqrt(G[p * ldg + p]);
    const R inv = R(1) / rkk;
    for (int c = tm.tid; c < D; c += tm.nt) {
      R v;
      if (c == p)
        v = rkk;
      else if ((done >> c) & 1u)
        v = R(0);
      else
        v = G[p * ldg + c] * inv;
      Rf[k * ldr + c] = v;
    }
    if (tm.tid == 0) piv[k] = p;
    done |= 1u << p;
    tm.sync();
    for (int w = tm.tid; w < D * D; w += tm.nt) {
      const int a = w / D, c = w % D;
      if (((done >> a) & 1u) || ((done >> c) & 1u)) continue;
      G[a * ldg + c] -= Rf[k * ldr + a] * Rf[k * ldr + c];
    }
    tm.sync();
    r = k + 1;
  }
  return r;
}

// Right inverse of the pivoted factor: Ri (D x r, ld ldi) with Rf Ri = I_r, nonzero only
// in the pivot rows: Ri[piv[i]][j] = (R11^-1)[i][j], R11[i][j] = Rf[i][piv[j]] upper
// triangular.  One column of R11^-1 per thread, by back substitution.
template <typename R>
__device__ void team_pchol_rinv(const Team& tm, const R* Rf, int ldr, const int* piv, int r, int D, R* Ri,
                                int ldi) {
  for (int w = tm.tid; w < D * r; w += tm.nt) Ri[(w / r) * ldi + (w % r)] = R(0);
  tm.sync();
  for (int j = tm.tid; j < r; j += tm.nt) {
    Ri[piv[j] * ldi + j] = R(1) / Rf[j * ldr + piv[j]];
    for (int i = j - 1; i >= 0; --i) {
      R s = R(0);
      for (int l = i + 1; l <= j; ++l) s += Rf[i * ldr + piv[l]] * Ri[piv[l] * ldi + j];
      Ri[piv[i] * ldi + j] = -s / Rf[i * ldr + piv[i]];
    }
  }
  tm.sync();
}

// Four independent pivoted Cholesky factorisations (as team_pchol) run concurrently: the
// team is split into four lane segments of seg = nt/4 lanes (D <= seg <= 32); segment b
// factors the D x D block G + b*bstride into Rf + b*bstride (ld D), with its pivots and the
// reciprocals of R11's diagonal (from one rsqrt per pivot) in piv/dinv + b*pstride and its
// rank in rank[b] (team-shared).  tol[b] < 0 marks an empty block (rank 0).  Pivot
// candidates are compared as bit patterns: non-negative doubles order as integers, and a
// negative rounding residue loses to any admissible pivot.
__device__ __forceinline__ void team_pchol4(const Team& tm, double* G, int D, int bstride, const double* tol,
                                            double* Rf, int* piv, double* dinv, int pstride, int* rank) {
  const int seg = tm.nt / 4;
  const int blk = tm.tid / seg, sl = tm.tid % seg;
  double* Gb = G + blk * bstride;
  double* Rb = Rf + blk * bstride;
  const double tl = tol[blk];
  const long long tbits = __double_as_longlong(tl);
  bool active = tl >= 0.0;
  uint32_t done = 0;
  int r = 0;
  for (int k = 0; k < D; ++k) {
    long long key = -1;
    int idx = sl;
    if (active && sl < D && !((done >> sl) & 1u)) key = __double_as_longlong(Gb[sl * D + sl]);
    for (int o = seg >> 1; o > 0; o >>= 1) {
      const long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (k2 > key || (k2 == key && i2 < idx)) {
        key = k2;
        idx = i2;
      }
    }
    const bool ok = active && key > tbits;
    const int p = idx;
    if (ok) {
      const double dpp = Gb[p * D + p];
      const double inv = rsqrt(dpp);
      const double rkk = dpp * inv;
      for (int c = sl; c < D; c += seg) {
        double v;
        if (c == p)
          v = rkk;
        else if ((done >> c) & 1u)
          v = 0.0;
        else
          v = Gb[p * D + c] * inv;
        Rb[k * D + c] = v;
      }
      if (sl == 0) {
        piv[blk * pstride + k] = p;
        dinv[blk * pstride + k] = inv;
      }
      done |= 1u << p;
      r = k + 1;
    } else {
      active = false;
    }
    tm.sync();
    if (ok)
      for (int w = sl; w < D * D; w += seg) {
        const int a = w / D, c = w % D;
        if (((done >> a) & 1u) || ((done >> c) & 1u)) continue;
        Gb[a * D + c] -= Rb[k * D + a] * Rb[k * D + c];
      }
    tm.sync();
  }
  if (sl == 0) rank[blk] = r;
  tm.sync();
}

// Right inverses of the four factors of team_pchol4 (as team_pchol_rinv, multiplying by
// the stored reciprocal diagonals): Ri + b*bstride is D x r_b (ld D); one (block, column)
// per thread.
__device__ __forceinline__ void team_pchol_rinv4(const Team& tm, const double* Rf, int D, int bstride, const int* piv,
                                                 const double* dinv, int pstride, const int* rank, double* Ri) {
  for (int w = tm.tid; w < 4 * D * D; w += tm.nt) Ri[(w / (D * D)) * bstride + w % (D * D)] = 0.0;
  tm.sync();
  const int seg = tm.nt / 4;
  const int blk = tm.tid / seg, j = tm.tid % seg;
  const int r = rank[blk];
  if (j < r) {
    const double* Rb = Rf + blk * bstride;
    double* Ib = Ri + blk * bstride;
    const int* pb = piv + blk * pstride;
    const double* db = dinv + blk * pstride;
    Ib[pb[j] * D + j] = db[j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= j; ++l) s += Rb[i * D + pb[l]] * Ib[pb[l] * D + j];
      Ib[pb[i] * D + j] = -s * db[i];
    }
  }
  tm.sync();
}

// Rotation (c, s) of the one-sided Jacobi step for columns with squared norms al, be and
// inner product ga; false when the pair is already orthogonal to working precision
// (ga^2 <= tol^2 al be), or when a column is negligible (squared norm below tiny(); FP32
// solves run on matrices scaled to a largest entry of 1).
template <typename R>
__device__ __forceinline__ bool jacobi_rot(R al, R be, R ga, R tol, R& c, R& s) {
  if (ga == R(0) || al <= TeamTol<R>::tiny() || be <= TeamTol<R>::tiny() || ga * ga <= tol * tol * (al * be)) {
    c = R(1);
    s = R(0);
    return false;
  }
  const R zeta = (be - al) / (R(2) * ga);
  const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
  c = rsqrt(R(1) + t * t);
  s = t * c;
  return true;
}

// Largest power of two <= x (x >= 1).
__device__ __forceinline__ int team_pow2_floor(int x) {
  int g = 1;
  while (2 * g <= x) g *= 2;
  return g;
}

// One-sided Jacobi SVD of the m x n matrix A, stored column-major (element (r, c) at
// A[c * lda + r]; an odd lda keeps the lanes of different column pairs on different shared
// memory banks): on return the columns of A are mutually orthogonal, A_out = A_in V, with
// V (n x n, column-major, ldv) orthogonal -- so the singular values are the column norms
// of A_out and its normalised columns the left singular vectors.  With init_V false, V
// holds an orthogonal matrix on entry and is updated as V <- V J.  `flag` is one int of
// team-shared scratch.  Returns the number of sweeps.
// `tol`: convergence tolerance (<= 0: TeamTol<R>::rel()).
template <typename R>
__device__ int team_svd_onesided(const Team& tm, R* A, int lda, int m, int n, R* V, int ldv, int* flag,
                                 int max_sweeps, bool init_V = true, R tol = R(0)) {
  if (!(tol > R(0))) tol = TeamTol<R>::rel();
  if (init_V)
    for (int w = tm.tid; w < n * n; w += tm.nt) V[(w / n) * ldv + (w % n)] = (w / n == w % n) ? R(1) : R(0);
  tm.sync();
  if (n < 2) return 0;
  const int ne = n + (n & 1), half = ne / 2;
  int g = tm.nt / half;
  g = g < 1 ? 1 : (g > 32 ? 32 : team_pow2_floor(g));
  const int rows_max = m > n ? m : n;
  while (g > 1 && g > rows_max) g >>= 1;
  const int ngroups = tm.nt / g;
  const int grp = tm.tid / g, gl = tm.tid % g;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tm.tid == 0) *flag = 0;
    tm.sync();
    for (int k = 0; k < ne - 1; ++k) {
      for (int i0 = 0; i0 < half; i0 += ngroups) {
        const int i = i0 + grp;
        int p = 0, q = 0;
        bool active = i < half;
        if (active) {
          team_rr_pair(k, i, ne, p, q);
          active = q < n;
        }
        R* ap_ = A + (size_t)p * lda;
        R* aq_ = A + (size_t)q * lda;
        R al = R(0), be = R(0), ga = R(0);
        if (active)
          for (int r = gl; r < m; r += g) {
            const R ap = ap_[r], aq = aq_[r];
            al += ap * ap;
            be += aq * aq;
            ga += ap * aq;
          }
        for (int o = g >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        R c, s;
        if (active && jacobi_rot(al, be, ga, tol, c, s)) {
          if (gl == 0) *flag = 1;
          for (int r = gl; r < m; r += g) {
            const R ap = ap_[r], aq = aq_[r];
            ap_[r] = c * ap - s * aq;
            aq_[r] = s * ap + c * aq;
          }
          R* vp_ = V + (size_t)p * ldv;
          R* vq_ = V + (size_t)q * ldv;
          for (int r = gl; r < n; r += g) {
            const R vp = vp_[r], vq = vq_[r];
            vp_[r] = c * vp - s * vq;
            vq_[r] = s * vp + c * vq;
          }
        }
      }
      tm.sync();
    }
    const int any = *flag;
    tm.sync();
    if (!any) break;
  }
  return sweep;
}

// Column norms of A (m x n, column-major, lda): out[j] = ||A[:, j]||.
template <typename R>
__device__ void team_col_norms(const Team& tm, const R* A, int lda, int m, int n, R* out) {
  for (int j = tm.tid; j < n; j += tm.nt) {
    const R* a = A + (size_t)j * lda;
    R s = R(0);
    for (int r = 0; r < m; ++r) s += a[r] * a[r];
    out[j] = sqrt(s);
  }
  tm.sync();
}

// Odd leading dimension >= rows (column-major storage without bank-aligned columns).
__host__ __device__ __forceinline__ int odd_ld(int rows) { return rows | 1; }

// Lanes per column pair used by team_svd_onesided for a team of nt threads and an m x n
// matrix, and a leading dimension for 4-byte elements that puts the g-lane windows of
// consecutive columns on disjoint shared-memory banks (ld = g mod 32).
__host__ __device__ __forceinline__ int team_svd_group(int nt, int m, int n) {
  const int half = (n + (n & 1)) / 2;
  int g = half > 0 ? nt / half : 32;
  if (g < 1) g = 1;
  if (g > 32) g = 32;
  int p2 = 1;
  while (2 * p2 <= g) p2 *= 2;
  g = p2;
  const int rows_max = m > n ? m : n;
  while (g > 1 && g > rows_max) g >>= 1;
  return g;
}
__host__ __device__ __forceinline__ int bank_ld32(int rows, int g) { return (rows + 31) / 32 * 32 + (g & 31); }

// Descending order of n non-negative values (ties: lower index first): order[rank] = j.
// Ranks are counted on the bit patterns, which order non-negative IEEE values exactly.
template <typename R>
__device__ void team_sort_desc(const Team& tm, const R* v, int n, int* order) {
  for (int j = tm.tid; j < n; j += tm.nt) {
    const double vj = double(v[j]);
    const long long bj = __double_as_longlong(vj);
    int rank = 0;
    for (int i = 0; i < n; ++i) {
      const long long bi = __double_as_longlong(double(v[i]));
      rank += (bi > bj || (bi == bj && i < j)) ? 1 : 0;
    }
    order[rank] = j;
  }
  tm.sync();
}

// Number of singular values kept: s (descending, s[0] > 0); at most chi, only those above
// cutoff * s[0]; a cut inside a multiplet (s[k-1] - s[k] <= rtol * s[0]) drops it whole
// unless that leaves nothing.
template <typename R>
__device__ __forceinline__ int team_keep_count(const R* s, int n, int chi, double cutoff, double rtol) {
  int r = 0;
  while (r < n && double(s[r]) > cutoff * double(s[0])) ++r;
  int k = r < chi ? r : chi;
  if (k < r) {
    int kk = k;
    while (kk > 0 && double(s[kk - 1]) - double(s[kk]) <= rtol * double(s[0])) --kk;
    if (kk > 0) k = kk;
  }
  return k;
}

// FP64 (or FP32) one-sided Jacobi sweeps restricted to the column pairs that involve one of
// the first ktop columns of A (m x n, column-major, lda), V (n x n, ldv) rotated alongside;
// sweeps until one passes without a rotation.  In step k of the round-robin ordering each of
// the first ktop columns x meets one partner (k for the fixed player, the fixed player for k,
// 2k - x mod (ne - 1) otherwise); the pair is handled by the g-lane group of its smaller top
// member, so each step has at most ktop pairs and every group gets nt / ktop lanes.  On
// return the first ktop columns are orthogonal to each other and to every other column (the
// others keep whatever mutual orthogonality they had).  Returns the number of sweeps.
template <typename R>
__device__ int team_jacobi_topk(const Team& tm, R* A, int lda, int m, int n, R* V, int ldv, int ktop, int* flag,
                                int max_sweeps) {
  tm.sync();
  if (n < 2 || ktop < 1) return 0;
  if (ktop > n) ktop = n;
  const R tol = TeamTol<R>::rel();
  const int ne = n + (n & 1), mm = ne - 1;
  int g = tm.nt / ktop;
  g = g < 1 ? 1 : (g > 32 ? 32 : team_pow2_floor(g));
  const int rows_max = m > n ? m : n;
  while (g > 1 && g > rows_max) g >>= 1;
  const int ngroups = tm.nt / g;
  const int grp = tm.tid / g, gl = tm.tid % g;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tm.tid == 0) *flag = 0;
    tm.sync();
    for (int k = 0; k < ne - 1; ++k) {
      for (int x0 = 0; x0 < ktop; x0 += ngroups) {
        const int x = x0 + grp;
        int y = -1;
        if (x < ktop) {
          y = (x == mm) ? k : (x == k ? mm : (2 * k - x + 2 * mm) % mm);
          if ((y < ktop && y < x) || y >= n) y = -1;
        }
        const bool active = y >= 0;
        const int p = active ? (x < y ? x : y) : 0, q = active ? (x < y ? y : x) : 0;
        R* ap_ = A + (size_t)p * lda;
        R* aq_ = A + (size_t)q * lda;
        R al = R(0), be = R(0), ga = R(0);
        if (active)
          for (int r = gl; r < m; r += g) {
            const R ap = ap_[r], aq = aq_[r];
            al += ap * ap;
            be += aq * aq;
            ga += ap * aq;
          }
        for (int o = g >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        R c, s;
        if (active && jacobi_rot(al, be, ga, tol, c, s)) {
          if (gl == 0) *flag = 1;
          for (int r = gl; r < m; r += g) {
            const R ap = ap_[r], aq = aq_[r];
            ap_[r] = c * ap - s * aq;
            aq_[r] = s * ap + c * aq;
          }
          R* vp_ = V + (size_t)p * ldv;
          R* vq_ = V + (size_t)q * ldv;
          for (int r = gl; r < n; r += g) {
            const R vp = vp_[r], vq = vq_[r];
            vp_[r] = c * vp - s * vq;
            vq_[r] = s * vp + c * vq;
          }
        }
      }
      tm.sync();
    }
    const int any = *flag;
    tm.sync();
    if (!any) break;
  }
  return sweep;
}

// Max |x| over the m x n column-major matrix x (ld), through a shared double slot.
__device__ inline double team_absmax(const Team& tm, const double* x, int ld, int m, int n, double* slot) {
  double v = 0.0;
  for (int w = tm.tid; w < m * n; w += tm.nt) v = fmax(v, fabs(x[(w / m) * ld + (w % m)]));
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (tm.tid == 0) *slot = 0.0;
  tm.sync();
  if ((tm.tid & 31) == 0) {
    // benign max via compare-and-swap on the bit pattern (non-negative doubles order as integers)
    unsigned long long* p = reinterpret_cast<unsigned long long*>(slot);
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
  }
  tm.sync();
  const double r = *slot;
  tm.sync();
  return r;
}

// C (m x n) = A (m x k) B (k x n), all row-major with the given leading dimensions.
template <typename R>
__device__ __forceinline__ void team_gemm(const Team& tm, const R* A, int lda, const R* B, int ldb, R* C, int ldc,
                                          int m, int n, int k) {
  for (int w = tm.tid; w < m * n; w += tm.nt) {
    const int i = w / n, j = w % n;
    R s = R(0);
    for (int l = 0; l < k; ++l) s += A[i * lda + l] * B[l * ldb + j];
    C[i * ldc + j] = s;
  }
}

// One-sided Jacobi SVD of A (m x n, column-major, lda; as team_svd_onesided) preconditioned
// by an FP32 solve (mixed-precision Jacobi): the FP32 Jacobi runs on a copy scaled to a
// largest entry of 1; its right factor, re-orthogonalised in FP64 by one Newton-Schulz step
// V <- V (3I - V^T V) / 2, is applied to A in FP64, and FP64 Jacobi sweeps then run to
// convergence from it.  The FP32 solve cannot resolve singular values below ~1e-7 of the
// largest, so the FP64 sweeps are never cut short.  V column-major (ldv).  F: scratch of
// >= max(m, n) * (max(m, n) + 1) doubles (it also holds the two FP32 matrices); Tt: >= n*n
// doubles; flag: one team-shared int; slot: one team-shared double.
// With 0 < ktop < n only the ktop columns of largest norm after the FP32 start are needed to
// FP64 accuracy (a truncation keeps at most ktop - 2 of them): the columns of A and V are
// reordered by decreasing norm (nrm: n doubles, ord: n ints of scratch) and the FP64 sweeps
// rotate only pairs that involve one of the first ktop columns (team_jacobi_topk).  Those
// columns come out orthogonal to every column; the others, mutually orthogonal to FP32
// accuracy, give the remaining singular values to FP32 relative accuracy.
__device__ inline void svd_precond(const Team& tm, double* A, int lda, int m, int n, double* V, int ldv, double* F,
                                   double* Tt, int* flag, double* slot, int ktop = 0, double* nrm = nullptr,
                                   int* ord = nullptr, bool upper = false) {
  const double amax = team_absmax(tm, A, lda, m, n, slot);
  if (!(amax > 0.0) || n < 2) {
    team_svd_onesided<double>(tm, A, lda, m, n, V, ldv, flag, 40, true);
    return;
  }
  const int la32 = odd_ld(m), lv32 = odd_ld(n);
  float* A32 = reinterpret_cast<float*>(F);
  float* V32 = A32 + la32 * n;
  const double sc = 1.0 / amax;
  for (int w = tm.tid; w < m * n; w += tm.nt) {
    const int c = w / m, r = w % m;
    A32[c * la32 + r] = float(A[c * lda + r] * sc);
  }
  tm.sync();
  team_svd_onesided<float>(tm, A32, la32, m, n, V32, lv32, flag, 30, true);
  for (int w = tm.tid; w < n * n; w += tm.nt) {
    const int c = w / n, r = w % n;
    V[c * ldv + r] = double(V32[c * lv32 + r]);
  }
  tm.sync();
  // Newton-Schulz: V <- V (3I - V^T V) / 2   (Tt, F: column-major, ld n); V^T V is
  // symmetric: the entries i <= j are computed and mirrored (the same products in the same
  // order, so the mirror is exact)
  for (int w = tm.tid; w < n * (n + 1) / 2; w += tm.nt) {
    int j = (int)((sqrt(8.0 * w + 1.0) - 1.0) * 0.5);
    while ((j + 1) * (j + 2) / 2 <= w) ++j;
    while (j * (j + 1) / 2 > w) --j;
    const int i = w - j * (j + 1) / 2;   // 0 <= i <= j
    const double* vi = V + i * ldv;
    const double* vj = V + j * ldv;
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += vi[l] * vj[l];
    const double t = (i == j ? 1.5 : 0.0) - 0.5 * s;
    Tt[j * n + i] = t;
    Tt[i * n + j] = t;
  }
  tm.sync();
  for (int w = tm.tid; w < n * n; w += tm.nt) {
    const int j = w / n, i = w % n;
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += V[l * ldv + i] * Tt[j * n + l];
    F[j * n + i] = s;
  }
  tm.sync();
  for (int w = tm.tid; w < n * n; w += tm.nt) V[(w / n) * ldv + (w % n)] = F[w];
  tm.sync();
  // A <- A V   (F: column-major, ld m); an upper-triangular A (row i zero in columns < i)
  // skips the zero products
  for (int w = tm.tid; w < m * n; w += tm.nt) {
    const int j = w / m, i = w % m;
    double s = 0.0;
    for (int l = upper ? i : 0; l < n; ++l) s += A[l * lda + i] * V[j * ldv + l];
    F[j * m + i] = s;
  }
  tm.sync();
  for (int w = tm.tid; w < m * n; w += tm.nt) A[(w / m) * lda + (w % m)] = F[w];
  if (ktop > 0 && ktop < n && nrm && ord) {
    tm.sync();
    team_col_norms<double>(tm, A, lda, m, n, nrm);
    team_sort_desc<double>(tm, nrm, n, ord);
    for (int w = tm.tid; w < m * n; w += tm.nt) F[w] = A[ord[w / m] * lda + (w % m)];
    for (int w = tm.tid; w < n * n; w += tm.nt) Tt[w] = V[ord[w / n] * ldv + (w % n)];
    tm.sync();
    for (int w = tm.tid; w < m * n; w += tm.nt) A[(w / m) * lda + (w % m)] = F[w];
    for (int w = tm.tid; w < n * n; w += tm.nt) V[(w / n) * ldv + (w % n)] = Tt[w];
    team_jacobi_topk<double>(tm, A, lda, m, n, V, ldv, ktop, flag, 40);
    return;
  }
  team_svd_onesided<double>(tm, A, lda, m, n, V, ldv, flag, 40, false);
}


// Householder QR (Golub & Van Loan, Alg. 5.2.1): A (m x n, column-major, lda, m >= n) is
// overwritten; on return its upper triangle A[0:n, 0:n] holds R of A = Q R (the reflector
// vectors below the diagonal are not kept; the diagonal of R may be negative).  Each
// column norm is summed by one warp (a fixed order, so the factor is reproducible), and
// the reflector is applied to the remaining columns by groups of g lanes per column.
// `red`: 2 values of team-shared scratch.
template <typename R>
__device__ void team_qr_r(const Team& tm, R* A, int lda, int m, int n, R* red) {
  int g = tm.nt / (n > 1 ? n - 1 : 1);
  g = g < 1 ? 1 : (g > 32 ? 32 : team_pow2_floor(g));
  while (g > 1 && g > m) g >>= 1;
  const int ngroups = tm.nt / g;
  const int grp = tm.tid / g, gl = tm.tid % g;
  for (int j = 0; j < n; ++j) {
    R* a = A + (size_t)j * lda;
    if (tm.tid < 32) {
      R s = R(0);
      for (int r = j + 1 + tm.tid; r < m; r += 32) s += a[r] * a[r];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (tm.tid == 0) {
        const R x0 = a[j];
        const R nrm = sqrt(x0 * x0 + s);
        if (!(s > R(0))) {
          red[0] = R(0);            // nothing below the diagonal: no reflection
        } else {
          const R alpha = x0 >= R(0) ? -nrm : nrm;
          const R v0 = x0 - alpha;  // |v0| = nrm + |x0|: no cancellation
          red[0] = R(2) / (s + v0 * v0);
          red[1] = alpha;
          a[j] = v0;                // v = (v0, a[j+1:m])
        }
      }
    }
    tm.sync();
    const R tau = red[0];
    if (tau != R(0)) {
      for (int c0 = j + 1; c0 < n; c0 += ngroups) {
        const int c = c0 + grp;
        R* ac = A + (size_t)c * lda;
        R w = R(0);
        if (c < n)
          for (int r = j + gl; r < m; r += g) w += a[r] * ac[r];
        for (int o = g >> 1; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (c < n) {
          const R f = tau * w;
          for (int r = j + gl; r < m; r += g) ac[r] -= f * a[r];
        }
      }
      tm.sync();
      if (tm.tid == 0) a[j] = red[1];
    }
    tm.sync();
  }
}

}  // namespace td
