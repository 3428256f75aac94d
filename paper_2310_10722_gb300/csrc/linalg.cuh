// Block-cooperative dense linear algebra for small matrices (n <= a few hundred).
//
// Symmetric eigendecomposition by the cyclic Jacobi method and SVD by the one-sided
// (Hestenes) Jacobi method, both with the round-robin ("circle") parallel ordering: in each
// of the n-1 steps of a sweep the n/2 index pairs are disjoint, so their rotations are
// computed and applied concurrently (Golub & Van Loan, Matrix Computations, Sec. 8.5 and
// 8.6.3; the 2x2 symmetric Schur rotation of their Algorithm 8.5.1).  Every call is made by
// all threads of the block; matrices live in shared or global memory, row-major.
#pragma once

#include <cuda_runtime.h>

namespace td {

template <typename R>
struct JacobiTol;
template <>
struct JacobiTol<double> {
  static __device__ __forceinline__ double rel() { return 1e-15; }
};
template <>
struct JacobiTol<float> {
  static __device__ __forceinline__ float rel() { return 1e-7f; }
};

// Pair i of step k for `ne` (even) players; player ne-1 stays fixed.
__device__ __forceinline__ void rr_pair(int k, int i, int ne, int& p, int& q) {
  const int m = ne - 1;
  if (i == 0) {
    p = k;
    q = m;
  } else {
    p = (k + i) % m;
    q = (k - i + m) % m;
  }
  if (p > q) {
    int t = p; p = q; q = t;
  }
}

// Symmetric 2x2 Schur rotation zeroing a_pq: returns (c, s) with
// [a_pp a_pq; a_pq a_qq] -> J^T A J diagonal, J = [c s; -s c].
template <typename R>
__device__ __forceinline__ bool schur2(R app, R aqq, R apq, R& c, R& s) {
  const R thresh = JacobiTol<R>::rel() * sqrt(fabs(app * aqq));
  if (apq == R(0) || fabs(apq) <= thresh) {
    c = R(1); s = R(0);
    return false;
  }
  const R tau = (aqq - app) / (R(2) * apq);
  const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
  c = R(1) / sqrt(R(1) + t * t);
  s = t * c;
  return true;
}

// Eigendecomposition of the symmetric n x n matrix A (leading dimension lda).  On return
// the diagonal of A holds the eigenvalues and column j of V (n x n, ldv) the eigenvector
// of A[j][j].  `rot` is scratch of at least 2 * ((n+1)/2) elements of R, `flag` one int,
// both in shared memory.  Returns the number of sweeps.
template <typename R>
__device__ int block_sym_eig(R* A, int lda, R* V, int ldv, int n, R* rot, int* flag, int max_sweeps = 40) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int w = tid; w < n * n; w += nt) V[(w / n) * ldv + (w % n)] = (w / n == w % n) ? R(1) : R(0);
  const int ne = n + (n & 1);
  const int half = ne / 2;
  int sweep = 0;
  __syncthreads();
  for (; sweep < max_sweeps && n > 1; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int k = 0; k < ne - 1; ++k) {
      for (int i = tid; i < half; i += nt) {
        int p, q;
        rr_pair(k, i, ne, p, q);
        R c = R(1), s = R(0);
        if (q < n && schur2(A[p * lda + p], A[q * lda + q], A[p * lda + q], c, s)) *flag = 1;
        rot[2 * i] = c;
        rot[2 * i + 1] = s;
      }
      __syncthreads();
      for (int w = tid; w < half * n; w += nt) {        // rows p, q
        const int i = w / n, col = w % n;
        const R s = rot[2 * i + 1];
        if (s == R(0)) continue;
        const R c = rot[2 * i];
        int p, q;
        rr_pair(k, i, ne, p, q);
        const R ap = A[p * lda + col], aq = A[q * lda + col];
        A[p * lda + col] = c * ap - s * aq;
        A[q * lda + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int w = tid; w < half * n; w += nt) {        // columns p, q of A and V
        const int i = w / n, row = w % n;
        const R s = rot[2 * i + 1];
        if (s == R(0)) continue;
        const R c = rot[2 * i];
        int p, q;
        rr_pair(k, i, ne, p, q);
        const R ap = A[row * lda + p], aq = A[row * lda + q];
        A[row * lda + p] = c * ap - s * aq;
        A[row * lda + q] = s * ap + c * aq;
        const R vp = V[row * ldv + p], vq = V[row * ldv + q];
        V[row * ldv + p] = c * vp - s * vq;
        V[row * ldv + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

// One-sided Jacobi SVD of the m x n matrix A (row-major, lda): on return the columns of A
// are mutually orthogonal (A_out = A_in V) and V (n x n, ldv) is orthogonal, so the
// singular values are the column norms of A_out and the left singular vectors its
// normalised columns.  `rot` holds 2 * ((n+1)/2) elements, `flag` one int (shared).
template <typename R>
__device__ int block_svd_onesided(R* A, int lda, int m, int n, R* V, int ldv, R* rot, int* flag,
                                  int max_sweeps = 40) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int w = tid; w < n * n; w += nt) V[(w / n) * ldv + (w % n)] = (w / n == w % n) ? R(1) : R(0);
  const int ne = n + (n & 1);
  const int half = ne / 2;
  int sweep = 0;
  __syncthreads();
  for (; sweep < max_sweeps && n > 1; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int k = 0; k < ne - 1; ++k) {
      for (int i = tid; i < half; i += nt) {
        int p, q;
        rr_pair(k, i, ne, p, q);
        R c = R(1), s = R(0);
        if (q < n) {
          R al = 0, be = 0, ga = 0;
          for (int r = 0; r < m; ++r) {
            const R ap = A[r * lda + p], aq = A[r * lda + q];
            al += ap * ap;
            be += aq * aq;
            ga += ap * aq;
          }
          if (schur2(al, be, ga, c, s)) *flag = 1;
        }
        rot[2 * i] = c;
        rot[2 * i + 1] = s;
      }
      __syncthreads();
      const int rows = m > n ? m : n;
      for (int w = tid; w < half * rows; w += nt) {
        const int i = w / rows, r = w % rows;
        const R s = rot[2 * i + 1];
        if (s == R(0)) continue;
        const R c = rot[2 * i];
        int p, q;
        rr_pair(k, i, ne, p, q);
        if (r < m) {
          const R ap = A[r * lda + p], aq = A[r * lda + q];
          A[r * lda + p] = c * ap - s * aq;
          A[r * lda + q] = s * ap + c * aq;
        }
        if (r < n) {
          const R vp = V[r * ldv + p], vq = V[r * ldv + q];
          V[r * ldv + p] = c * vp - s * vq;
          V[r * ldv + q] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

// Number of singular values kept: s (descending, s[0] > 0); at most chi, only those above
// cutoff * s[0]; a cut inside a multiplet (s[k-1] - s[k] <= rtol * s[0]) drops it whole
// unless that leaves nothing.
template <typename R>
__device__ __forceinline__ int keep_count(const R* s, int n, int chi, double cutoff, double rtol) {
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

}  // namespace td
