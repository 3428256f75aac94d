// Final 2D contraction (Sec. 4: "the remaining two-dimensional network is contracted by
// sweeping an MPS across it"; chi_MPS of Sec. 5) and the coset log-sum / decision.
//
// Site tensor of the final network: F[c][l][r][d][u] = sum_phys R[phys][c] Gamma[phys][..]
// with sqrt(lambda) absorbed on every bond; c is the site's class bit.  Rows y = 0..ny-1 are
// absorbed into a boundary MPS A_x[a][d][b] by zip-up: a carry C[j][a][l][p] runs left to
// right, T[j][u][b][r][q] = sum C A F~ with F~[l,p; r,q] = F[p^q], and (j,u) x (b,r,q) is
// truncated to chi_mps by its leading singular vectors.  The class parity p flows along
// each row into a two-valued output leg of the last MPS tensor.  The last row is contracted
// exactly.
//
// Arithmetic.  The contraction computes in FP64 on both paths (T is the storage type of the
// site tensors it reads): the class-parity leg carries both cosets through one MPS, so FP32
// sums and FP32 singular vectors err by ~eps32 times the majority coset's weight, a relative
// error of ~eps32 exp(margin) on the minority coset.  Each cut's left singular vectors come
// from a one-sided Jacobi SVD; when M^T (n x m) has at least as many rows as columns it is
// first reduced by a Householder QR, M^T = Q R, and the Jacobi orthogonalises the m columns
// of the m x m factor R (half-length columns; R V has orthogonal columns exactly when M^T V
// has).  The carry is then (M^T V_k)^T from the unreduced M^T.  On the mixed path the
// Jacobi of R is preconditioned by an FP32 solve and finished by FP64 sweeps run to
// convergence (svd_precond), and only for the chi_mps + 2 columns of largest norm, the only
// ones a cut can keep (and the one after them, for the multiplet rule): the FP64 sweeps rotate
// just the pairs that involve one of them.  The gradient pass's recorded forward keeps the
// unreduced Jacobi on M^T (its records are M^T V and V).
#include <cmath>
#include <mutex>

#include "sweep.cuh"
#include "team.cuh"

namespace td {

// F[c][l][r][d][u] of site (x, y) into F (dims into fd: L, R, D, U; fd[4] = 1 when the
// class-1 half F[1] can be nonzero, 0 when it is exactly zero -- the readout has no class
// flip).  sqrt(lambda) of the site's bonds is staged in slam[4][chi] first.
template <typename T, typename R>
__device__ void build_F(const Team& tm, const FinalArgs& fa, int b, int x, int y, R* F, int* fd, R* slam) {
  const int s = fa.grid_site[y * fa.nx + x];
  if (s < 0) {
    if (tm.tid == 0) { F[0] = R(1); F[1] = R(0); fd[4] = 0; }
    if (tm.tid < 4) fd[tm.tid] = 1;
    tm.sync();
    return;
  }
  const FinalSite& fs = fa.sites[s];
  const Override* ov = vshot_ovr(fa.vs, fa.ovr, fa.wave_first, b, kOvrRead, s);
  const double* Rv = ov ? ov->val : fs.R;
  const double* lam = fa.lam + (int64_t)b * fa.nbonds * fa.chi;
  for (int w = tm.tid; w < 4 * fa.chi; w += tm.nt) {
    const int dir = w / fa.chi, i = w % fa.chi;
    slam[w] = (fs.dir_pos[dir] >= 0 && i < fs.dir_dim[dir]) ? R(sqrt(lam[fs.dir_bond[dir] * fa.chi + i])) : R(1);
  }
  const int dL = fs.dir_dim[0], dR = fs.dir_dim[1], dD = fs.dir_dim[2], dU = fs.dir_dim[3];
  int stride[4];   // stride of each direction's index in the site tensor (0 if absent)
  {
    int st[kMaxBonds];
    int acc = 1;
    for (int k = fs.nb - 1; k >= 0; --k) {
      st[k] = acc;
      int dk = 1;
      for (int dir = 0; dir < 4; ++dir)
        if (fs.dir_pos[dir] == k) dk = fs.dir_dim[dir];
      acc *= dk;
    }
    for (int dir = 0; dir < 4; ++dir) stride[dir] = fs.dir_pos[dir] >= 0 ? st[fs.dir_pos[dir]] : 0;
  }
  const int rest = dL * dR * dD * dU;
  const T* g = reinterpret_cast<const T*>(fa.gamma) + (int64_t)b * fa.shot_elems + fs.off;
  tm.sync();
  for (int w = tm.tid; w < rest; w += tm.nt) {
    int e = w;
    const int iu = e % dU; e /= dU;
    const int id = e % dD; e /= dD;
    const int ir = e % dR; e /= dR;
    const int il = e;
    const int off = il * stride[0] + ir * stride[1] + id * stride[2] + iu * stride[3];
    const R wgt = slam[il] * slam[fa.chi + ir] * slam[2 * fa.chi + id] * slam[3 * fa.chi + iu];
    R a0 = R(0), a1 = R(0);
    for (int ph = 0; ph < fs.P; ++ph) {
      const R gv = R(g[(int64_t)ph * rest + off]);
      a0 += R(Rv[ph * 2 + 0]) * gv;
      a1 += R(Rv[ph * 2 + 1]) * gv;
    }
    F[w] = a0 * wgt;
    F[rest + w] = a1 * wgt;
  }
  if (tm.tid == 0) {
    fd[0] = dL; fd[1] = dR; fd[2] = dD; fd[3] = dU;
    int c1 = 0;
    for (int ph = 0; ph < fs.P; ++ph) c1 |= (Rv[ph * 2 + 1] != 0.0);
    fd[4] = c1;
  }
  tm.sync();
}

// One block per shot.  The work region (site tensor F, T1 / V, M^T, carries) lives in
// shared memory when it fits, otherwise in the shot's global scratch; the boundary MPS is
// always in global scratch.
template <typename T, typename R>
__global__ void __launch_bounds__(1024) k_final(FinalArgs fa) {
  const int b = blockIdx.x;
  const Team tm{(int)threadIdx.x, (int)blockDim.x, 1};
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* scr = reinterpret_cast<R*>(fa.scratch) + (int64_t)b * fa.scratch_elems;
  R* work = fa.use_smem ? reinterpret_cast<R*>(smem_raw) : scr + fa.off_work;
  R* mps[2] = {scr + fa.off_mps0, scr + fa.off_mps1};
  R* F = work + fa.w_F;
  R* W = work + fa.w_W;        // T1, then V of the SVD
  R* MT = work + fa.w_MT;      // M^T (n x m)
  R* Cb[2] = {work + fa.w_C0, work + fa.w_C1};
  R* sv = work + fa.w_s;
  int* ord = reinterpret_cast<int*>(work + fa.w_ord);
  __shared__ int mdim[2][kMaxGridX][3];   // per column: (left, down, right) of the MPS tensors
  __shared__ int fd[5];
  __shared__ int meta[8];
  __shared__ R slam[4 * kMaxChi];
  __shared__ double logsum_s;
  __shared__ double trunc_s[2];   // largest and summed discarded fraction of the cuts
  __shared__ R red_s[2];
  __shared__ double slot_s;
  const int nx = fa.nx, ny = fa.ny;
  if (tm.tid == 0) { logsum_s = 0.0; trunc_s[0] = 0.0; trunc_s[1] = 0.0; }
  for (int x = tm.tid; x < nx; x += tm.nt) {
    mdim[0][x][0] = 1; mdim[0][x][1] = 1; mdim[0][x][2] = (x == nx - 1) ? 2 : 1;
    R* A = mps[0] + (int64_t)x * fa.mps_stride;
    A[0] = R(1);
    if (x == nx - 1) A[1] = R(0);
  }
  tm.sync();
  int cur = 0;
  for (int y = 0; y < ny; ++y) {
    int cc = 0;
    if (tm.tid == 0) { Cb[0][0] = R(1); Cb[0][1] = R(0); }
    int cJ = 1, cA = 1, cL = 1;
    tm.sync();
    for (int x = 0; x < nx; ++x) {
      build_F<T, R>(tm, fa, b, x, y, F, fd, slam);
      const int L = fd[0], Rr = fd[1], U = fd[3];
      const R* A = mps[cur] + (int64_t)x * fa.mps_stride;
      const int aL = mdim[cur][x][0], aD = mdim[cur][x][1], aR = mdim[cur][x][2];
      const R* C = Cb[cc];
      (void)cA;
      // T1[l][p][d][bb][j] = sum_a C[j][a][l][p] A[a][d][bb]  (j fastest: the lanes of one
      // warp below read four j values of the same (l, p, d, bb) from distinct banks)
      double* rs = nullptr;    // this column's record slot (reverse sweep)
      if constexpr (sizeof(R) == 8) {
        if (fa.rec) {
          rs = fa.rec + (int64_t)b * fa.rec_stride + (int64_t)(y * nx + x) * fa.rec_slot;
          const FinRecSlot ly(fa.rec_mC, fa.rec_mA, fa.rec_m, fa.rec_n);
          for (int w = tm.tid; w < cJ * aL * cL * 2; w += tm.nt) rs[ly.C + w] = double(C[w]);
          for (int w = tm.tid; w < aL * aD * aR; w += tm.nt) rs[ly.A + w] = double(A[w]);
          if (tm.tid == 0) {
            rs[1] = cJ; rs[2] = aL; rs[3] = cL; rs[4] = aD; rs[5] = aR;
            rs[6] = L; rs[7] = Rr; rs[8] = U;
            rs[0] = (x == nx - 1) ? 2 : (y == ny - 1 ? 1 : 0);
          }
        }
      }
      R* T1 = W;
      const int n1 = cJ * L * 2 * aD * aR;
      for (int w = tm.tid; w < n1; w += tm.nt) {
        int e = w;
        const int j = e % cJ; e /= cJ;
        const int bb = e % aR; e /= aR;
        const int d = e % aD; e /= aD;
        const int p = e % 2; e /= 2;
        const int l = e;
        R acc = R(0);
        for (int a = 0; a < aL; ++a) acc += C[((j * aL + a) * cL + l) * 2 + p] * A[(a * aD + d) * aR + bb];
        T1[w] = acc;
      }
      tm.sync();
      // MT[(bb, r, q)][(j, u)] = sum_{l,p,d} T1[l][p][d][bb][j] F[p^q][l][r][d][u], stored
      // column-major: column (j, u) of MT is row (j, u) of M; leading dimensions chosen so
      // the Jacobi lane groups of consecutive columns fall on disjoint banks
      const int nF = L * Rr * aD * U;
      const int m = cJ * U, n = aR * Rr * 2;
      const int pc = fd[4];   // 0: F[1] is zero, so only p = q contributes (half the products)
      const int ldm = bank_ld32(n, team_svd_group(tm.nt, n, m));
      const int ldv = bank_ld32(m, team_svd_group(tm.nt, n, m));
      for (int w = tm.tid; w < m * n; w += tm.nt) {
        const int c = w / m, ju = w % m;      // consecutive lanes: consecutive u (F) and ju (MT)
        const int q = c % 2, r = (c / 2) % Rr, bb = c / (2 * Rr);
        const int j = ju / U, u = ju % U;
        R acc = R(0);
        const int p_lo = pc ? 0 : q, p_hi = pc ? 2 : q + 1;
        for (int l = 0; l < L; ++l)
          for (int p = p_lo; p < p_hi; ++p) {
            const R* t1 = T1 + (((l * 2 + p) * aD) * aR + bb) * cJ + j;
            const R* f = F + (p ^ q) * nF + ((l * Rr + r) * aD) * U + u;
            for (int d = 0; d < aD; ++d) acc += t1[d * aR * cJ] * f[d * U];
          }
        MT[ju * ldm + c] = acc;
      }
      tm.sync();
      R* An = mps[cur ^ 1] + (int64_t)x * fa.mps_stride;
      R* Cn = Cb[cc ^ 1];
      if (x < nx - 1 && y < ny - 1) {
        // left singular vectors of M = MT^T: one-sided Jacobi on the m columns of MT, or on
        // the columns of the triangular factor of MT's QR (see the file comment)
        R* V = W;
        const bool qr = !rs && m >= 2 && n >= m;
        // a wide cut (n < m: the first row, where the incoming MPS has bond 1) has rank <= n:
        // one-sided Jacobi on the n columns of M (not the m columns of M^T); the left singular
        // vectors are M's rotated columns, normalised
        const bool wide = !rs && n < m;
        const int nc = wide ? n : m;   // singular values computed
        R* Mt = work + fa.w_Q;
        const int ldt = bank_ld32(m, team_svd_group(tm.nt, m, n));
        int ldvv = ldv;
        if (wide) {
          for (int w = tm.tid; w < m * n; w += tm.nt) {
            const int c = w / m, ju = w % m;
            Mt[c * ldt + ju] = MT[ju * ldm + c];
          }
          tm.sync();
          ldvv = bank_ld32(n, team_svd_group(tm.nt, m, n));
          team_svd_onesided<R>(tm, Mt, ldt, m, n, V, ldvv, meta + 7, 40, true);
          team_col_norms<R>(tm, Mt, ldt, m, n, sv);
        } else if (qr) {
          R* Qw = work + fa.w_Q;
          R* Rk = work + fa.w_R;
          const int ldr = bank_ld32(m, team_svd_group(tm.nt, m, m));
          ldvv = bank_ld32(m, team_svd_group(tm.nt, m, m));
          for (int w = tm.tid; w < m * n; w += tm.nt) Qw[(w / n) * n + w % n] = MT[(w / n) * ldm + w % n];
          tm.sync();
          team_qr_r<R>(tm, Qw, n, n, m, red_s);
          for (int w = tm.tid; w < m * m; w += tm.nt) {
            const int c = w / m, r = w % m;
            Rk[c * ldr + r] = (r <= c) ? Qw[c * n + r] : R(0);
          }
          tm.sync();
          if constexpr (sizeof(R) == 8) {
            if (fa.precond)
              svd_precond(tm, Rk, ldr, m, m, V, ldvv, work + fa.w_P, work + fa.w_T, meta + 7, &slot_s,
                          fa.chi_mps + 2 < m ? fa.chi_mps + 2 : 0, sv, ord, true);
            else
              team_svd_onesided<R>(tm, Rk, ldr, m, m, V, ldvv, meta + 7, 40, true);
          } else {
            team_svd_onesided<R>(tm, Rk, ldr, m, m, V, ldvv, meta + 7, 40, true);
          }
          team_col_norms<R>(tm, Rk, ldr, m, m, sv);
        } else {
          team_svd_onesided<R>(tm, MT, ldm, n, m, V, ldv, meta + 7, 40, true);
          team_col_norms<R>(tm, MT, ldm, n, m, sv);
        }
        team_sort_desc<R>(tm, sv, nc, ord);
        if (tm.tid == 0) {
          int k = 0;
          const R s0 = sv[ord[0]];
          if (s0 > R(0)) {
            R* srt = sv + m;   // the second half of the singular-value region
            const int nsv = m < n ? m : n;
            for (int i = 0; i < nsv; ++i) srt[i] = sv[ord[i]];
            k = team_keep_count<R>(srt, nsv, fa.chi_mps, fa.svd_cutoff, fa.multiplet_rtol);
            if (fa.stats) {   // discarded fraction sum_{i >= k} s_i^2 / sum_i s_i^2
              double tot = 0.0, disc = 0.0;
              for (int i = 0; i < nsv; ++i) {
                const double q = double(srt[i]) * double(srt[i]);
                tot += q;
                if (i >= k) disc += q;
              }
              const double f = tot > 0.0 ? disc / tot : 0.0;
              trunc_s[0] = fmax(trunc_s[0], f);
              trunc_s[1] += f;
            }
          }
          meta[0] = k;
        }
        tm.sync();
        const int k = meta[0];
        if constexpr (sizeof(R) == 8) {
          if (rs) {
            const FinRecSlot ly(fa.rec_mC, fa.rec_mA, fa.rec_m, fa.rec_n);
            for (int w = tm.tid; w < m * m; w += tm.nt) rs[ly.V + w] = double(V[(w / m) * ldv + w % m]);
            for (int w = tm.tid; w < n * m; w += tm.nt) rs[ly.MT + w] = double(MT[(w / n) * ldm + w % n]);
            for (int w = tm.tid; w < m; w += tm.nt) { rs[ly.sv + w] = double(sv[w]); rs[ly.ord + w] = ord[w]; }
            if (tm.tid == 0) {
              int e2r = 0;
              if (k > 0) frexp(double(sv[ord[0]]), &e2r);
              rs[9] = m; rs[10] = n; rs[11] = k; rs[12] = e2r;
            }
          }
        }
        if (k == 0) {
          if (tm.tid == 0) logsum_s = -INFINITY;
          for (int w = tm.tid; w < m; w += tm.nt) An[w] = R(0);
          for (int w = tm.tid; w < n; w += tm.nt) Cn[w] = R(0);
          if (tm.tid == 0) { mdim[cur ^ 1][x][0] = cJ; mdim[cur ^ 1][x][1] = U; mdim[cur ^ 1][x][2] = 1; }
          cJ = 1;
        } else {
          // exact power-of-two normalisation of the carry (its log to the log-scale)
          int e2 = 0;
          frexp(double(sv[ord[0]]), &e2);
          const R inv0 = R(ldexp(1.0, -e2));
          if (wide) {
            for (int w = tm.tid; w < m * k; w += tm.nt) {
              const int ju = w / k, kk = w % k;
              An[w] = Mt[ord[kk] * ldt + ju] / sv[ord[kk]];
            }
            tm.sync();
            // carry = (M^T U_k)^T from the unrotated M^T
            for (int w = tm.tid; w < k * n; w += tm.nt) {
              const int kk = w / n, c = w % n;
              R acc = R(0);
              for (int j = 0; j < m; ++j) acc += MT[j * ldm + c] * An[j * k + kk];
              Cn[w] = acc * inv0;
            }
          } else {
            for (int w = tm.tid; w < m * k; w += tm.nt) {
              const int ju = w / k, kk = w % k;
              An[w] = V[ord[kk] * ldvv + ju];
            }
            if (qr) {
              // carry = (M^T V_k)^T from the unreduced M^T
              for (int w = tm.tid; w < k * n; w += tm.nt) {
                const int kk = w / n, c = w % n;
                const R* vk = V + ord[kk] * ldvv;
                R acc = R(0);
                for (int j = 0; j < m; ++j) acc += MT[j * ldm + c] * vk[j];
                Cn[w] = acc * inv0;
              }
            } else {
              for (int w = tm.tid; w < k * n; w += tm.nt) {
                const int kk = w / n, c = w % n;
                Cn[w] = MT[ord[kk] * ldm + c] * inv0;
              }
            }
          }
          if (tm.tid == 0) {
            logsum_s += double(e2) * 0.69314718055994530942;
            mdim[cur ^ 1][x][0] = cJ; mdim[cur ^ 1][x][1] = U; mdim[cur ^ 1][x][2] = k;
          }
          cJ = k;
        }
        cA = aR; cL = Rr;
        cc ^= 1;
        tm.sync();
      } else if (x < nx - 1) {
        // last row: U == 1, no truncation; the carry takes the whole contraction
        if (rs && tm.tid == 0) { rs[9] = m; rs[10] = n; }
        for (int w = tm.tid; w < m * n; w += tm.nt) {
          const int ju = w / n, c = w % n;
          Cn[w] = MT[ju * ldm + c];
        }
        for (int w = tm.tid; w < m * m; w += tm.nt) An[w] = (w / m == w % m) ? R(1) : R(0);
        if (tm.tid == 0) { mdim[cur ^ 1][x][0] = cJ; mdim[cur ^ 1][x][1] = U; mdim[cur ^ 1][x][2] = m; }
        cJ = m; cA = aR; cL = Rr;
        cc ^= 1;
        tm.sync();
      } else {
        // last column (Rr == 1): merge the old class leg bb and the row parity q into bb ^ q
        for (int w = tm.tid; w < m * 2; w += tm.nt) {
          const int ju = w / 2, c2 = w % 2;
          R acc = R(0);
          for (int bb = 0; bb < aR; ++bb) acc += MT[ju * ldm + bb * 2 + (bb ^ c2)];
          An[w] = acc;
        }
        tm.sync();
        if (tm.tid < 32) {
          R mx = R(0);
          for (int w = tm.tid; w < m * 2; w += 32) mx = fmax(mx, fabs(An[w]));
          for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          if (tm.tid == 0) {
            meta[1] = 0;
            int e2 = 0;
            if (mx > R(0)) {
              frexp(double(mx), &e2);
              logsum_s += double(e2) * 0.69314718055994530942;
            } else {
              logsum_s = -INFINITY;
            }
            slam[0] = mx > R(0) ? R(ldexp(1.0, -e2)) : R(0);
            if (rs) { rs[9] = m; rs[10] = n; rs[12] = e2; }
            mdim[cur ^ 1][x][0] = cJ; mdim[cur ^ 1][x][1] = U; mdim[cur ^ 1][x][2] = 2;
          }
        }
        tm.sync();
        const R inv = slam[0];
        if (inv > R(0))
          for (int w = tm.tid; w < m * 2; w += tm.nt) An[w] *= inv;
        tm.sync();
      }
    }
    cur ^= 1;
    tm.sync();
  }
  // contract the last MPS (vertical legs are trivial): v <- v A_x, the vectors in the two
  // carry buffers (each holds at least chi_mps * final bond dimension values)
  {
    R* v = Cb[0];
    R* vn = Cb[1];
    if (tm.tid == 0) v[0] = R(1);
    int dv = 1;
    tm.sync();
    for (int x = 0; x < nx; ++x) {
      const R* A = mps[cur] + (int64_t)x * fa.mps_stride;
      const int aL = mdim[cur][x][0], aR = mdim[cur][x][2];
      const int na = aL < dv ? aL : dv;
      for (int bb = tm.tid; bb < aR; bb += tm.nt) {
        R acc = R(0);
        for (int a = 0; a < na; ++a) acc += v[a] * A[a * aR + bb];
        vn[bb] = acc;
      }
      tm.sync();
      R* t = v; v = vn; vn = t;
      dv = aR;
    }
    if (tm.tid == 0) {
      fa.Z[(int64_t)b * 2 + 0] = double(v[0]);
      fa.Z[(int64_t)b * 2 + 1] = double(v[1]);
      fa.logacc[(int64_t)b * fa.nslots + fa.slot] = logsum_s;
      if (fa.stats) {
        fa.stats[(int64_t)(fa.wave_first + b) * 4 + 2] = trunc_s[0];
        fa.stats[(int64_t)(fa.wave_first + b) * 4 + 3] = trunc_s[1];
      }
    }
  }
}

__global__ void k_finalize(FinalizeArgs f) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= f.B) return;
  double ls = 0.0;
  for (int k = 0; k < f.nslots; ++k) ls += f.logacc[(int64_t)b * f.nslots + k];
  const double z0 = f.Z[2 * b], z1 = f.Z[2 * b + 1];
  double zz[2] = {f.mix[0] * z0 + f.mix[1] * z1, f.mix[2] * z0 + f.mix[3] * z1};
  int off = 0;
  if (f.offset_all) {
    const uint8_t* m = f.det + (int64_t)vshot_row(f.vs, f.wave_first, b) * f.n_det;
    for (int i = 0; i < f.n_det; ++i) off ^= m[i] & 1;
  }
  double lp[2];
  for (int c = 0; c < 2; ++c) {
    const double z = zz[c ^ off];
    lp[c] = (z > 0.0 && ls > -INFINITY) ? log(z) + ls : -INFINITY;
  }
  // a non-finite intermediate (NaN in a log-scale or in the final contraction, or an
  // infinite weight) makes the shot's result NaN and is reported by td_network_check
  if (isnan(ls) || isnan(z0) || isnan(z1) || ls == INFINITY || isinf(z0) || isinf(z1)) {
    lp[0] = lp[1] = NAN;
    if (f.status) atomicExch(f.status, (int)TD_ERR_NUMERIC);
  }
  const int64_t gb = f.wave_first + b;
  if (f.logp) {
    f.logp[2 * gb] = lp[0];
    f.logp[2 * gb + 1] = lp[1];
  }
  const int dec = (lp[1] > lp[0]) ? 1 : 0;
  if (f.decision) f.decision[gb] = dec;
  if (f.margin) f.margin[gb] = lp[dec] - lp[dec ^ 1];
}

template <typename T, typename R>
cudaError_t launch_final(const FinalArgs& f, cudaStream_t st) {
  size_t smem = 0;
  if (f.use_smem) {
    smem = (size_t)f.work_elems * sizeof(R);
    cudaError_t e = cudaFuncSetAttribute(k_final<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_final<T, R><<<f.B, f.threads, smem, st>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& f, cudaStream_t st) {
  k_finalize<<<(f.B + 127) / 128, 128, 0, st>>>(f);
  return cudaGetLastError();
}

// ---- final contraction with scratch in a static device array ----------------------------
// For callers that cannot call cudaMalloc: the scratch of k_final comes from this
// file-scope array instead of the network workspace.  Every GPU that loads the library holds
// it until the process exits.  Host code must not use the symbol as an address; the device
// address is looked up once per device (cudaGetSymbolAddress) with that device current.
static __device__ __align__(256) unsigned char g_final_scratch[kStaticFinalScratchBytes];

namespace {
std::mutex g_static_mu;
void* g_static_ptr[kMaxStaticDevices] = {};
}  // namespace

cudaError_t static_final_scratch(void** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxStaticDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_final_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *ptr = g_static_ptr[dev];
  return cudaSuccess;
}

template cudaError_t launch_final<double, double>(const FinalArgs&, cudaStream_t);
template cudaError_t launch_final<float, double>(const FinalArgs&, cudaStream_t);

}  // namespace td
