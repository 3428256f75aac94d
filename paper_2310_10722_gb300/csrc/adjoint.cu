// Reverse sweep: d log P(m) / d (parameter objects) of the decoder, truncations included.
//
// The forward sweep (Sec. 4) is run once in the versioned layout with its truncation
// cores and zip-up cuts recorded (sweep.cu, core.cu, final.cu); this file walks it
// backwards, one block of threads per shot, in FP64:
//   * final contraction: every zip-up cut keeps U_k (the new MPS tensor) and passes
//     U_k^T M (times an exact power of two) on as the carry; the adjoint of the truncated
//     SVD of M is the textbook one (the thin SVD over the nonzero singular values,
//     F_ij = 1 / (s_j^2 - s_i^2), plus the projection of U-bar off the kept space);
//   * gate: the simple update is the truncated SVD of Theta = M_A Lambda' M_B^T, with M_X
//     the doubled side matrix (environment weights absorbed) and Lambda' = c(p) (x) lambda
//     in the kappa basis.  With Q_X = M_X R_X^+ the recorded R factors, the adjoint is
//       theta-bar = SVD adjoint of the core theta = R_A Lambda' R_B^T (U-bar = R_A^+T M_A^T X-bar,
//                   V-bar likewise, S-bar = lambda-bar / s_1),
//       M_A-bar = M_A R_A^+ (theta-bar - U-bar S^-1 V_k^T) R_B Lambda' + X-bar S^-1 V_k^T R_B Lambda',
//       Lambda'-bar = R_A^T theta-bar R_B   (-> lambda-bar of the bond, p-bar of the gate),
//     and the environment weights' adjoints go to the other bonds' lambda-bar;
//   * site-local operator psi <- sc K' psi: K'-bar = sc psi-bar psi_in^T, psi_in-bar = sc K'^T psi-bar.
// Every normalisation of the forward sweep (powers of two, s_1, the zip-up divisors) is
// held fixed: log P does not depend on them (each is a gauge of the representation).
// The parameter objects are the site-local matrices K (per layer and site), the gates'
// p and the readouts R; their adjoints are written per shot and mapped to the rates on
// the host.
#include <cmath>

#include "sweep.cuh"

namespace td {

namespace {

constexpr double kRs2 = 0.70710678118654752440;

__device__ __forceinline__ void bsync() { __syncthreads(); }

// Sum of v over the block (fixed order: per-warp shuffles, then warp 0), broadcast.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bsync();
  if (lane == 0) red[warp] = v;
  bsync();
  if (warp == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[32] = v;
  }
  bsync();
  const double r = red[32];
  bsync();
  return r;
}

// Environment weight of row (o, i) of a side and the digit of each bond slot.
__device__ __forceinline__ double env_weight(const SideDesc& sd, int o, int i, const double* lam, int chi, int* dig) {
  double w = 1.0;
  for (int k = kMaxBonds - 1; k >= 0; --k) {
    dig[k] = -1;
    if (k < sd.nb && k > sd.pos) {
      const int dk = sd.dims[k];
      dig[k] = i % dk;
      w *= lam[sd.bond[k] * chi + dig[k]];
      i /= dk;
    }
  }
  for (int k = kMaxBonds - 1; k >= 0; --k)
    if (k < sd.pos) {
      const int dk = sd.dims[k];
      dig[k] = o % dk;
      w *= lam[sd.bond[k] * chi + dig[k]];
      o /= dk;
    }
  return w;
}

// Adds sum over rows (o, i) of r[o * inner + i] / lambda to lambda-bar of every other bond
// of the side, at the row's digit.  A row index oi = o * inner + i is a mixed-radix number
// over the side's other bonds (in slot order, the last fastest), so the rows of digit d of
// slot k are oi = h * (dim_k * stride_k) + d * stride_k + l.  Every (slot, digit) gets
// blockDim / n_out threads; their partial sums are added in a fixed order (red: >= blockDim
// doubles of shared memory).
__device__ void env_lambar(const SideDesc& sd, const double* r, const double* lam, double* lambar, int chi,
                           double sign, double* red) {
  const int OI = sd.outer * sd.inner;
  int stride[kMaxBonds], first[kMaxBonds + 1];
  int n_out = 0;
  {
    int acc = 1;
    for (int k = kMaxBonds - 1; k >= 0; --k) {
      stride[k] = acc;
      if (k < sd.nb && k != sd.pos) acc *= sd.dims[k];
    }
    for (int k = 0; k < kMaxBonds; ++k) {
      first[k] = n_out;
      if (k < sd.nb && k != sd.pos) n_out += sd.dims[k];
    }
    first[kMaxBonds] = n_out;
  }
  if (n_out == 0) return;
  const int parts = (int)blockDim.x / n_out;   // >= 1: n_out <= 3 * chi <= 96 < blockDim
  const int t = threadIdx.x;
  double acc = 0.0;
  int k = -1, d = 0;
  if (t < parts * n_out) {
    const int o = t % n_out, part = t / n_out;
    for (int kk = 0; kk < kMaxBonds; ++kk)
      if (kk < sd.nb && kk != sd.pos && o >= first[kk] && o < first[kk] + sd.dims[kk]) { k = kk; d = o - first[kk]; }
    const int dk = sd.dims[k], sk = stride[k];
    const int cnt = OI / dk;
    for (int e = part; e < cnt; e += parts) {
      const int h = e / sk, l = e % sk;
      acc += r[h * dk * sk + d * sk + l];
    }
  }
  __syncthreads();
  red[t] = acc;
  __syncthreads();
  if (t < n_out) {
    double tot = 0.0;
    for (int part = 0; part < parts; ++part) tot += red[part * n_out + t];
    int kk = 0;
    while (!(kk < sd.nb && kk != sd.pos && t >= first[kk] && t < first[kk] + sd.dims[kk])) ++kk;
    const int dd = t - first[kk];
    const double l2 = lam[sd.bond[kk] * chi + dd];
    if (l2 > 0.0) lambar[sd.bond[kk] * chi + dd] += sign * tot / l2;
  }
  __syncthreads();
}

// Strides of a final site's tensor per direction (left, right, down, up); 0 if absent.
__device__ void site_strides(const FinalSite& fs, int* stride) {
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

__device__ __forceinline__ double dir_weight(const FinalSite& fs, const double* lam, int chi, int dir, int idx) {
  return fs.dir_pos[dir] >= 0 ? sqrt(lam[fs.dir_bond[dir] * chi + idx]) : 1.0;
}

// Adjoint of the final contraction (the zip-up of final.cu): fills gbar[s] (adjoint of each
// site's last tensor), adds to lambar (sqrt(lambda) on both sides of every bond) and writes
// the readouts' adjoints.
__device__ void final_bwd(const AdjArgs& a, int b, double* scr, double* gbar, double* lambar, double* Rbar,
                          double* red, double* red2) {
  const int nx = a.nx, ny = a.ny, chi = a.chi;
  const double* rec = a.rec_fin + (int64_t)b * a.fin_stride;
  const FinRecSlot ly(a.fin_mC, a.fin_mA, a.fin_m, a.fin_n);
  const double* lam = a.lam + (int64_t)b * a.nbonds * chi;
  const double* hist = a.hist + (int64_t)b * a.hist_elems;
  double* F = scr + a.fo_F;
  double* Fb = scr + a.fo_Fb;
  double* T1 = scr + a.fo_T1;
  double* T1b = scr + a.fo_T1b;
  double* M = scr + a.fo_M;
  double* Mb = scr + a.fo_Mb;
  double* Cb[2] = {scr + a.fo_C0, scr + a.fo_C1};
  double* Aout = scr + a.fo_A0;   // adjoints of this row's output MPS tensors
  double* Ain = scr + a.fo_A1;    // adjoints of its input tensors (the previous row's outputs)
  double* Ub = scr + a.fo_Ub;
  double* W = scr + a.fo_W;
  double* J = scr + a.fo_J;
  double* In = scr + a.fo_In;     // F_ij (J_ij - J_ji) s_j of a cut
  double* wg = scr + a.fo_wg;     // per entry of a site: weight, then F-bar . F
  int* offs = reinterpret_cast<int*>(scr + a.fo_off);
  const int mA = a.mps_stride;
  const double z = a.Z[2 * b] + a.Z[2 * b + 1];
  for (int w = threadIdx.x; w < nx * mA; w += blockDim.x) Aout[w] = 0.0;
  bsync();
  if (threadIdx.x < 2) Aout[(nx - 1) * mA + threadIdx.x] = 1.0 / z;   // v = last tensor [0][0][c]
  bsync();
  for (int y = ny - 1; y >= 0; --y) {
    for (int w = threadIdx.x; w < nx * mA; w += blockDim.x) Ain[w] = 0.0;
    int cb = 0;
    for (int x = nx - 1; x >= 0; --x) {
      const double* sl = rec + (int64_t)(y * nx + x) * a.fin_slot;
      const int kind = (int)sl[0], cJ = (int)sl[1], aL = (int)sl[2], cL = (int)sl[3], aD = (int)sl[4],
                aR = (int)sl[5], L = (int)sl[6], Rr = (int)sl[7], U = (int)sl[8], m = (int)sl[9], n = (int)sl[10],
                k = (int)sl[11], e2 = (int)sl[12];
      const double* C = sl + ly.C;
      const double* A = sl + ly.A;
      const int s = a.grid_site[y * nx + x];
      // F[c][l][r][d][u] of the site (trivial tensor if no site)
      const int nF = L * Rr * aD * U;
      int stride[4] = {0, 0, 0, 0};
      const double* g = nullptr;
      if (s >= 0) {
        const FinalSite& fs = a.finals[s];
        site_strides(fs, stride);
        g = hist + fs.off;
        for (int e = threadIdx.x; e < nF; e += blockDim.x) {
          int q = e;
          const int iu = q % U; q /= U;
          const int id = q % aD; q /= aD;
          const int ir = q % Rr; q /= Rr;
          const int il = q;
          const int off = il * stride[0] + ir * stride[1] + id * stride[2] + iu * stride[3];
          const double wgt = dir_weight(fs, lam, chi, 0, il) * dir_weight(fs, lam, chi, 1, ir) *
                             dir_weight(fs, lam, chi, 2, id) * dir_weight(fs, lam, chi, 3, iu);
          wg[e] = wgt;
          offs[e] = off;
          double a0 = 0.0, a1 = 0.0;
          for (int ph = 0; ph < fs.P; ++ph) {
            const double gv = g[(int64_t)ph * nF + off];
            a0 += fs.R[ph * 2 + 0] * gv;
            a1 += fs.R[ph * 2 + 1] * gv;
          }
          F[e] = a0 * wgt;
          F[nF + e] = a1 * wgt;
        }
      } else if (threadIdx.x == 0) {
        F[0] = 1.0;
        F[1] = 0.0;
      }
      // T1[l][p][d][bb][j] = sum_a C[j][a][l][p] A[a][d][bb]
      const int n1 = L * 2 * aD * aR * cJ;
      for (int w = threadIdx.x; w < n1; w += blockDim.x) {
        int q = w;
        const int j = q % cJ; q /= cJ;
        const int bb = q % aR; q /= aR;
        const int d = q % aD; q /= aD;
        const int pp = q % 2; q /= 2;
        const int l = q;
        double acc = 0.0;
        for (int aa = 0; aa < aL; ++aa) acc += C[((j * aL + aa) * cL + l) * 2 + pp] * A[(aa * aD + d) * aR + bb];
        T1[w] = acc;
      }
      bsync();
      // M[(j,u)][(bb,r,q)] = sum_{l,p,d} T1[l][p][d][bb][j] F[p^q][l][r][d][u]
      for (int w = threadIdx.x; w < m * n; w += blockDim.x) {
        const int ju = w / n, c = w % n;
        const int q = c % 2, r = (c / 2) % Rr, bb = c / (2 * Rr);
        const int j = ju / U, u = ju % U;
        double acc = 0.0;
        for (int l = 0; l < L; ++l)
          for (int pp = 0; pp < 2; ++pp)
            for (int d = 0; d < aD; ++d)
              acc += T1[(((l * 2 + pp) * aD + d) * aR + bb) * cJ + j] *
                     F[(pp ^ q) * nF + ((l * Rr + r) * aD + d) * U + u];
        M[w] = acc;
      }
      bsync();
      // M-bar
      const double* Cbar = Cb[cb];
      if (kind == 2) {
        const double inv = ldexp(1.0, -e2);
        const double* ob = Aout + (int64_t)x * mA;
        for (int w = threadIdx.x; w < m * n; w += blockDim.x) {
          const int ju = w / n, c = w % n;
          const int q = c % 2, bb = c / 2;
          Mb[w] = ob[ju * 2 + (bb ^ q)] * inv;
        }
      } else if (kind == 1) {
        for (int w = threadIdx.x; w < m * n; w += blockDim.x) Mb[w] = Cbar[w];
      } else {
        const double inv0 = ldexp(1.0, -e2);
        const double* V = sl + ly.V;
        const double* MT = sl + ly.MT;
        const double* sv = sl + ly.sv;
        const double* ordd = sl + ly.ord;
        const double* Ab = Aout + (int64_t)x * mA;
        // U-bar[ju][kk] = A-bar[ju][kk] + inv0 sum_c M[ju][c] C-bar[kk][c]
        for (int w = threadIdx.x; w < m * k; w += blockDim.x) {
          const int ju = w / k, kk = w % k;
          double acc = 0.0;
          for (int c = 0; c < n; ++c) acc += M[ju * n + c] * Cbar[kk * n + c];
          Ub[w] = Ab[ju * k + kk] + inv0 * acc;
        }
        bsync();
        int rr = 0;   // nonzero singular values (sorted)
        {
          const double s0 = sv[(int)ordd[0]];
          const int rmax = m < n ? m : n;
          while (rr < rmax && sv[(int)ordd[rr]] > 1e-13 * s0) ++rr;
        }
        // J[i][j] = U_i . U-bar_j  (i < rr, j < k)
        for (int w = threadIdx.x; w < rr * k; w += blockDim.x) {
          const int i = w / k, j = w % k;
          const double* ui = V + (int64_t)(int)ordd[i] * m;
          double acc = 0.0;
          for (int ju = 0; ju < m; ++ju) acc += ui[ju] * Ub[ju * k + j];
          J[w] = acc;
        }
        bsync();
        // In[i][j] = F_ij (J_ij - J_ji) s_j  (i, j < rr; J_ij = 0 for j >= k)
        for (int w = threadIdx.x; w < rr * rr; w += blockDim.x) {
          const int i = w / rr, j = w % rr;
          double v = 0.0;
          if (i != j && (i < k || j < k)) {
            const double si = sv[(int)ordd[i]], sj = sv[(int)ordd[j]];
            const double den = sj * sj - si * si;
            const double Jij = (j < k) ? J[i * k + j] : 0.0;
            const double Jji = (i < k) ? J[j * k + i] : 0.0;
            if (den != 0.0) v = (Jij - Jji) / den * sj;
          }
          In[w] = v;
        }
        bsync();
        // W[ju][j] = (sum_i U_i[ju] In[i][j] + [j < k] (U-bar_j - sum_i U_i J_ij)[ju] / s_j) / s_j
        for (int w = threadIdx.x; w < m * rr; w += blockDim.x) {
          const int ju = w / rr, j = w % rr;
          const double isj = 1.0 / sv[(int)ordd[j]];
          double acc = 0.0, proj = 0.0;
          for (int i = 0; i < rr; ++i) {
            const double ui = V[(int64_t)(int)ordd[i] * m + ju];
            acc += ui * In[i * rr + j];
            if (j < k) proj += ui * J[i * k + j];
          }
          if (j < k) acc += (Ub[ju * k + j] - proj) * isj;
          W[w] = acc * isj;
        }
        bsync();
        // M-bar = inv0 V_k C-bar + W MT^T  (MT_j = s_j times the right singular vector)
        for (int w = threadIdx.x; w < m * n; w += blockDim.x) {
          const int ju = w / n, c = w % n;
          double acc = 0.0;
          for (int kk = 0; kk < k; ++kk) acc += V[(int64_t)(int)ordd[kk] * m + ju] * Cbar[kk * n + c];
          acc *= inv0;
          for (int j = 0; j < rr; ++j) acc += W[ju * rr + j] * MT[(int64_t)(int)ordd[j] * n + c];
          Mb[w] = acc;
        }
      }
      bsync();
      // T1-bar and F-bar
      for (int w = threadIdx.x; w < n1; w += blockDim.x) {
        int q0 = w;
        const int j = q0 % cJ; q0 /= cJ;
        const int bb = q0 % aR; q0 /= aR;
        const int d = q0 % aD; q0 /= aD;
        const int pp = q0 % 2; q0 /= 2;
        const int l = q0;
        double acc = 0.0;
        for (int r = 0; r < Rr; ++r)
          for (int q = 0; q < 2; ++q)
            for (int u = 0; u < U; ++u)
              acc += Mb[(j * U + u) * n + (bb * Rr + r) * 2 + q] * F[(pp ^ q) * nF + ((l * Rr + r) * aD + d) * U + u];
        T1b[w] = acc;
      }
      for (int w = threadIdx.x; w < 2 * nF; w += blockDim.x) {
        const int c = w / nF;
        int q0 = w % nF;
        const int u = q0 % U; q0 /= U;
        const int d = q0 % aD; q0 /= aD;
        const int r = q0 % Rr; q0 /= Rr;
        const int l = q0;
        double acc = 0.0;
        for (int pp = 0; pp < 2; ++pp) {
          const int q = pp ^ c;
          for (int bb = 0; bb < aR; ++bb)
            for (int j = 0; j < cJ; ++j)
              acc += T1[(((l * 2 + pp) * aD + d) * aR + bb) * cJ + j] * Mb[(j * U + u) * n + (bb * Rr + r) * 2 + q];
        }
        Fb[w] = acc;
      }
      bsync();
      // C-bar of the carry entering this column, A-bar of the input MPS tensor
      double* Cn = Cb[cb ^ 1];
      for (int w = threadIdx.x; w < cJ * aL * cL * 2; w += blockDim.x) {
        int q0 = w;
        const int pp = q0 % 2; q0 /= 2;
        const int l = q0 % cL; q0 /= cL;
        const int aa = q0 % aL; q0 /= aL;
        const int j = q0;
        double acc = 0.0;
        if (l < L)
          for (int d = 0; d < aD; ++d)
            for (int bb = 0; bb < aR; ++bb)
              acc += T1b[(((l * 2 + pp) * aD + d) * aR + bb) * cJ + j] * A[(aa * aD + d) * aR + bb];
        Cn[w] = acc;
      }
      for (int w = threadIdx.x; w < aL * aD * aR; w += blockDim.x) {
        int q0 = w;
        const int bb = q0 % aR; q0 /= aR;
        const int d = q0 % aD; q0 /= aD;
        const int aa = q0;
        double acc = 0.0;
        for (int j = 0; j < cJ; ++j)
          for (int l = 0; l < L && l < cL; ++l)
            for (int pp = 0; pp < 2; ++pp)
              acc += C[((j * aL + aa) * cL + l) * 2 + pp] * T1b[(((l * 2 + pp) * aD + d) * aR + bb) * cJ + j];
        Ain[(int64_t)x * mA + w] = acc;
      }
      // site adjoints: G-bar, R-bar, lambda-bar
      if (s >= 0) {
        const FinalSite& fs = a.finals[s];
        double* gb = gbar + (int64_t)s * a.max_site;
        double rp[2 * kMaxPhys];
        for (int w = 0; w < 2 * kMaxPhys; ++w) rp[w] = 0.0;
        for (int e = threadIdx.x; e < nF; e += blockDim.x) {
          const double wgt = wg[e];
          const int off = offs[e];
          for (int ph = 0; ph < fs.P; ++ph) {
            gb[(int64_t)ph * nF + off] = (fs.R[ph * 2] * Fb[e] + fs.R[ph * 2 + 1] * Fb[nF + e]) * wgt;
            const double gv = g[(int64_t)ph * nF + off] * wgt;
            rp[ph * 2] += Fb[e] * gv;
            rp[ph * 2 + 1] += Fb[nF + e] * gv;
          }
        }
        for (int w = 0; w < fs.P * 2; ++w) {
          const double tot = block_sum(rp[w], red);
          if (threadIdx.x == 0) Rbar[(int64_t)s * 8 + w] = tot;
        }
        // lambda-bar: sqrt(lambda) on each leg; entries of digit d of direction dir are
        // e = h * (dim * st) + d * st + l in the [l][r][d][u] order
        for (int e = threadIdx.x; e < nF; e += blockDim.x) wg[e] = Fb[e] * F[e] + Fb[nF + e] * F[nF + e];
        bsync();
        const int dims4[4] = {L, Rr, aD, U}, st4[4] = {Rr * aD * U, aD * U, U, 1};
        int first[5], n_out = 0;
        for (int dir = 0; dir < 4; ++dir) { first[dir] = n_out; if (fs.dir_pos[dir] >= 0) n_out += dims4[dir]; }
        first[4] = n_out;
        if (n_out > 0) {
          const int parts = (int)blockDim.x / n_out, t = threadIdx.x;
          double acc = 0.0;
          if (t < parts * n_out) {
            const int o = t % n_out, part = t / n_out;
            int dir = 0;
            while (!(fs.dir_pos[dir] >= 0 && o >= first[dir] && o < first[dir] + dims4[dir])) ++dir;
            const int d = o - first[dir], dk = dims4[dir], sk = st4[dir], cnt = nF / dk;
            for (int e = part; e < cnt; e += parts) acc += wg[(e / sk) * dk * sk + d * sk + e % sk];
          }
          red2[t] = acc;
          bsync();
          if (t < n_out) {
            double tot = 0.0;
            for (int part = 0; part < parts; ++part) tot += red2[part * n_out + t];
            int dir = 0;
            while (!(fs.dir_pos[dir] >= 0 && t >= first[dir] && t < first[dir] + dims4[dir])) ++dir;
            const int d = t - first[dir];
            const double l2 = lam[fs.dir_bond[dir] * chi + d];
            // the two sides of a bond are different sites, handled at different (x, y)
            if (l2 > 0.0) lambar[fs.dir_bond[dir] * chi + d] += tot / (2.0 * l2);
          }
        }
      }
      bsync();
      cb ^= 1;
    }
    double* t = Aout; Aout = Ain; Ain = t;
    bsync();
  }
}

// Per-gate scratch of the core adjoint (doubles, L2 = 2 chi; CoreScr_elems in sweep.cuh is its
// size and must follow this carving): see gate_bwd.
struct CoreScr {
  double *C[2], *Uq, *Vq, *Ub, *Vb, *J, *K, *In, *Th, *Tmp, *W1, *W2, *Mx[2], *Xx[2], *Lb, *wrow;
  __device__ CoreScr(double* base, int chi, int64_t max_oi) {
    const int L2 = 2 * chi;
    double* q = base;
    auto take = [&](int64_t n) { double* r = q; q += n; return r; };
    C[0] = take(L2 * chi); C[1] = take(L2 * chi);
    Uq = take(L2 * L2); Vq = take(L2 * L2); Ub = take(L2 * chi); Vb = take(L2 * chi);
    J = take(L2 * chi); K = take(L2 * chi); In = take(L2 * L2); Th = take(L2 * L2); Tmp = take(L2 * L2);
    W1 = take(L2 * L2); W2 = take(L2 * L2);
    Mx[0] = take(L2 * L2); Mx[1] = take(L2 * L2); Xx[0] = take(chi * L2); Xx[1] = take(chi * L2);
    Lb = take(4 * chi); wrow = take(max_oi);
  }
  // total size: CoreScr_elems (sweep.cuh)
};

__device__ __forceinline__ int side_rows(const SideDesc& sd, int& lo0, int& hi0, int& lo1, int& hi1) {
  int np = 0;
  lo0 = hi0 = lo1 = hi1 = 0;
  for (int sg = 0; sg < sd.P; ++sg)
    if (sg < (sg ^ sd.mask)) {
      if (np == 0) { lo0 = sg; hi0 = sg ^ sd.mask; } else { lo1 = sg; hi1 = sg ^ sd.mask; }
      ++np;
    }
  return np;
}

// Adjoint of gate g (see the file comment).  gbar[site] holds the adjoint of the gate's
// output tensors on entry and of its input tensors on exit; lam[bond] goes back to the
// value before the gate; lambar[bond] becomes the adjoint of that value.
__device__ void gate_bwd(const AdjArgs& a, int b, int g, double* scr, double* gbar, double* lambar, double* lam,
                         double* red) {
  const GateDesc& gd = a.gates[g];
  const int D = gd.D, chi = a.chi, bond = gd.bond, L2 = 2 * chi, CC = chi * chi;
  const double* rec = a.rec_core + ((int64_t)(g - a.rec_gate0) * a.B + b) * core_rec_elems(chi);
  const int rk[4] = {(int)rec[0], (int)rec[1], (int)rec[2], (int)rec[3]};
  const int k = (int)rec[4];
  const double s0 = rec[5];
  const double* lam_old = rec + 8;
  const double* Rf = rec + 8 + chi;      // R[blk][li][q] at blk * CC + li * D + q
  const double* Ri = Rf + 4 * CC;        // Rinv[blk][q][li] at blk * CC + q * D + li
  const double* US = Ri + 4 * CC;        // column-major, ld L2
  const double* VV = US + L2 * L2;
  const double* sv = VV + L2 * L2;
  const double* ordd = sv + L2;
  const int rAp = rk[0], rA = rk[0] + rk[1], rBp = rk[2], rB = rk[2] + rk[3];
  const int roff[2][2] = {{0, rAp}, {0, rBp}};
  CoreScr cs(scr + a.o_core, chi, a.max_site);
  double* rsum = scr + a.o_r;
  const double p = gd.p;
  const double cpm = 0.5 * (1.0 - 2.0 * p);
  auto cval = [&](int ka, int kb) { return ka == kb ? 0.5 : cpm; };
  const double* hist = a.hist + (int64_t)b * a.hist_elems;
  // (a) X-bar = G_new-bar / env, environment adjoints of G_new = X / env; (b) C = M'^T X-bar
  double* rq = scr + a.o_xbar + 2 * a.max_site;   // per-(row, column) partial sums (see prepare_reverse)
  for (int X = 0; X < 2; ++X) {
    const SideDesc& sd = gd.side[X];
    const int OI = sd.outer * sd.inner, Dn = gd.Dn;
    const double* Gn = hist + sd.out_off;
    const double* Gnb = gbar + (int64_t)sd.site * a.max_site;
    double* xb = scr + a.o_xbar + (int64_t)X * a.max_site;
    for (int w = threadIdx.x; w < OI * Dn; w += blockDim.x) {
      int dig[kMaxBonds];
      const int oi = w / Dn, j = w % Dn;
      const int o = oi / sd.inner, i = oi % sd.inner;
      const double wt = env_weight(sd, o, i, lam, chi, dig);
      if (j == 0) cs.wrow[oi] = wt;
      const double winv = wt > 0.0 ? 1.0 / wt : 0.0;
      double r = 0.0;
      for (int ph = 0; ph < sd.P; ++ph) {
        const int64_t e = (((int64_t)ph * sd.outer + o) * Dn + j) * sd.inner + i;
        r += Gnb[e] * Gn[e];
        xb[e] = (j < k) ? Gnb[e] * winv : 0.0;
      }
      rq[w] = r;
    }
    bsync();
    for (int oi = threadIdx.x; oi < OI; oi += blockDim.x) {
      double r = 0.0;
      for (int j = 0; j < Dn; ++j) r += rq[oi * Dn + j];
      rsum[oi] = r;
    }
    bsync();
    env_lambar(sd, rsum, lam, lambar, chi, -1.0, red);
    int lo[2], hi[2];
    const int np = side_rows(sd, lo[0], hi[0], lo[1], hi[1]);
    const double* Gi = hist + sd.in_off;
    // C[kap][q][j]: tiles of 32 outputs; warp w takes rows w, w + nw, ...; lanes take outputs
    const int NO = 2 * D * k, nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrows = np * OI;
    for (int o0 = 0; o0 < NO; o0 += 32) {
      const int out = o0 + lane;
      double acc = 0.0;
      if (out < NO) {
        const int kap = out / (D * k), q = (out / k) % D, j = out % k;
        for (int row = warp; row < nrows; row += nw) {
          const int pr = row / OI, oi = row % OI;
          const int o = oi / sd.inner, i = oi % sd.inner;
          const double gl = Gi[(((int64_t)lo[pr] * sd.outer + o) * D + q) * sd.inner + i];
          const double gh = Gi[(((int64_t)hi[pr] * sd.outer + o) * D + q) * sd.inner + i];
          const double xl = xb[(((int64_t)lo[pr] * sd.outer + o) * Dn + j) * sd.inner + i];
          const double xh = xb[(((int64_t)hi[pr] * sd.outer + o) * Dn + j) * sd.inner + i];
          acc += cs.wrow[oi] * (kap == 0 ? (gl + gh) * (xl + xh) : (gl - gh) * (xl - xh));
        }
      }
      red[threadIdx.x] = acc;
      bsync();
      if (warp == 0 && out < NO) {
        double tot = 0.0;
        for (int ww = 0; ww < nw; ++ww) tot += red[ww * 32 + lane];
        const int kap = out / (D * k), q = (out / k) % D, j = out % k;
        cs.C[X][(kap * D + q) * chi + j] = tot * kRs2;   // M'_lo = (Y, Z) / sqrt2, M'_hi = (Y, -Z) / sqrt2
      }
      bsync();
    }
  }
  // (c) adjoint of the core theta = R_A Lambda' R_B^T (rA x rB) from its recorded SVD
  int rr = 0;
  {
    const double smax = sv[(int)ordd[0]];
    const int rmax = rA < rB ? rA : rB;
    while (rr < rmax && sv[(int)ordd[rr]] > 1e-13 * smax) ++rr;
  }
  for (int w = threadIdx.x; w < rA * rr; w += blockDim.x) {
    const int row = w / rr, i = w % rr, ci = (int)ordd[i];
    cs.Uq[row * L2 + i] = US[ci * L2 + row] / sv[ci];
  }
  for (int w = threadIdx.x; w < rB * rr; w += blockDim.x) {
    const int row = w / rr, i = w % rr, ci = (int)ordd[i];
    cs.Vq[row * L2 + i] = VV[ci * L2 + row];
  }
  for (int w = threadIdx.x; w < rA * k; w += blockDim.x) {
    const int row = w / k, j = w % k, kap = row < rAp ? 0 : 1, li = row - roff[0][kap];
    double acc = 0.0;
    for (int q = 0; q < D; ++q) acc += Ri[kap * CC + q * D + li] * cs.C[0][(kap * D + q) * chi + j];
    cs.Ub[row * chi + j] = acc;
  }
  for (int w = threadIdx.x; w < rB * k; w += blockDim.x) {
    const int row = w / k, j = w % k, kap = row < rBp ? 0 : 1, lj = row - roff[1][kap];
    double acc = 0.0;
    for (int q = 0; q < D; ++q) acc += Ri[(2 + kap) * CC + q * D + lj] * cs.C[1][(kap * D + q) * chi + j];
    cs.Vb[row * chi + j] = acc;
  }
  bsync();
  for (int w = threadIdx.x; w < rr * k; w += blockDim.x) {
    const int i = w / k, j = w % k;
    double aj = 0.0, ak = 0.0;
    for (int row = 0; row < rA; ++row) aj += cs.Uq[row * L2 + i] * cs.Ub[row * chi + j];
    for (int row = 0; row < rB; ++row) ak += cs.Vq[row * L2 + i] * cs.Vb[row * chi + j];
    cs.J[i * chi + j] = aj;
    cs.K[i * chi + j] = ak;
  }
  bsync();
  const double* lbn = lambar + (int64_t)bond * chi;   // adjoint of the new lambda = S / s_1
  for (int w = threadIdx.x; w < rr * rr; w += blockDim.x) {
    const int i = w / rr, j = w % rr;
    const double si = sv[(int)ordd[i]], sj = sv[(int)ordd[j]];
    double v = (i == j && j < k) ? lbn[j] / s0 : 0.0;
    if (i != j) {
      const double den = sj * sj - si * si;
      if (den != 0.0) {
        const double Jij = j < k ? cs.J[i * chi + j] : 0.0, Jji = i < k ? cs.J[j * chi + i] : 0.0;
        const double Kij = j < k ? cs.K[i * chi + j] : 0.0, Kji = i < k ? cs.K[j * chi + i] : 0.0;
        v += (Jij - Jji) / den * sj + si * (Kij - Kji) / den;
      }
    }
    cs.In[i * L2 + j] = v;
  }
  bsync();
  for (int w = threadIdx.x; w < rr * rB; w += blockDim.x) {   // Tmp = In Vq^T  (rr x rB)
    const int i = w / rB, c = w % rB;
    double acc = 0.0;
    for (int j = 0; j < rr; ++j) acc += cs.In[i * L2 + j] * cs.Vq[c * L2 + j];
    cs.Tmp[i * L2 + c] = acc;
  }
  bsync();
  for (int w = threadIdx.x; w < rA * rB; w += blockDim.x) {   // theta-bar (rA x rB)
    const int r = w / rB, c = w % rB;
    double acc = 0.0;
    for (int i = 0; i < rr; ++i) acc += cs.Uq[r * L2 + i] * cs.Tmp[i * L2 + c];
    for (int j = 0; j < k; ++j) {
      const double sj = sv[(int)ordd[j]];
      double p1 = cs.Ub[r * chi + j], p2 = cs.Vb[c * chi + j];
      for (int i = 0; i < rr; ++i) {
        p1 -= cs.Uq[r * L2 + i] * cs.J[i * chi + j];
        p2 -= cs.Vq[c * L2 + i] * cs.K[i * chi + j];
      }
      acc += (p1 * cs.Vq[c * L2 + j] + cs.Uq[r * L2 + j] * p2) / sj;
    }
    cs.Th[r * L2 + c] = acc;
  }
  bsync();
  // Lambda'-bar on the diagonal of each kappa block: Lb[ka][kb][q]
  for (int w = threadIdx.x; w < 4 * D; w += blockDim.x) {
    const int ka = w / (2 * D), kb = (w / D) % 2, q = w % D;
    double acc = 0.0;
    for (int li = 0; li < rk[ka]; ++li) {
      const double ra = Rf[ka * CC + li * D + q];
      if (ra == 0.0) continue;
      double t = 0.0;
      for (int lj = 0; lj < rk[2 + kb]; ++lj)
        t += cs.Th[(roff[0][ka] + li) * L2 + roff[1][kb] + lj] * Rf[(2 + kb) * CC + lj * D + q];
      acc += ra * t;
    }
    cs.Lb[(ka * 2 + kb) * chi + q] = acc;
  }
  // W1 = theta-bar - U-bar S^-1 V_k^T (rA x rB); W1B = theta-bar^T - V-bar S^-1 U_k^T (rB x rA)
  for (int w = threadIdx.x; w < rA * rB; w += blockDim.x) {
    const int r = w / rB, c = w % rB;
    double a1 = cs.Th[r * L2 + c], a2 = a1;
    for (int j = 0; j < k; ++j) {
      const double isj = 1.0 / sv[(int)ordd[j]];
      a1 -= cs.Ub[r * chi + j] * cs.Vq[c * L2 + j] * isj;
      a2 -= cs.Vb[c * chi + j] * cs.Uq[r * L2 + j] * isj;
    }
    cs.W1[r * L2 + c] = a1;
    cs.Tmp[c * L2 + r] = a2;   // W1B
  }
  bsync();
  // lambda-bar of the old bond weight and p-bar (one thread: fixed order)
  double* lbo = cs.J;   // free now
  if (threadIdx.x == 0) {
    double pb = 0.0;
    for (int q = 0; q < D; ++q) {
      const double pp = cs.Lb[0 * chi + q], pm = cs.Lb[1 * chi + q], mp = cs.Lb[2 * chi + q], mm = cs.Lb[3 * chi + q];
      lbo[q] = 0.5 * (pp + mm) + cpm * (pm + mp);
      pb -= lam_old[q] * (pm + mp);
    }
    a.pbar[(int64_t)b * a.n_gates + g] = pb;
  }
  // W2 = W1 R_B Lambda' (rA x 2D), W2B = W1B R_A Lambda' (rB x 2D)  (stored in W2 and In)
  for (int w = threadIdx.x; w < (rA + rB) * 2 * D; w += blockDim.x) {
    const bool sideB = w >= rA * 2 * D;
    const int ww = sideB ? w - rA * 2 * D : w;
    const int r = ww / (2 * D), col = ww % (2 * D), kp = col / D, q2 = col % D;
    double acc = 0.0;
    for (int kx = 0; kx < 2; ++kx) {
      const int blk = sideB ? kx : 2 + kx;           // the other side's R blocks
      const int rkx = rk[blk], off = roff[sideB ? 0 : 1][kx];
      double t = 0.0;
      for (int l = 0; l < rkx; ++l)
        t += (sideB ? cs.Tmp[r * L2 + off + l] : cs.W1[r * L2 + off + l]) * Rf[blk * CC + l * D + q2];
      acc += t * cval(kx, kp);
    }
    acc *= lam_old[q2];
    if (sideB) cs.In[r * L2 + col] = acc; else cs.W2[r * L2 + col] = acc;
  }
  bsync();
  // Mx = R^+ W2 (2D x 2D) per side; Xx = S^-1 [V_k or U_k]^T R_other Lambda' (k x 2D)
  for (int w = threadIdx.x; w < 2 * (2 * D) * (2 * D); w += blockDim.x) {
    const int X = w / (4 * D * D), ww = w % (4 * D * D);
    const int row = ww / (2 * D), col = ww % (2 * D), kap = row / D, q = row % D;
    const int blk = X == 0 ? kap : 2 + kap;
    const double* W2x = X == 0 ? cs.W2 : cs.In;
    double acc = 0.0;
    for (int l = 0; l < rk[blk]; ++l) acc += Ri[blk * CC + q * D + l] * W2x[(roff[X][kap] + l) * L2 + col];
    cs.Mx[X][row * L2 + col] = acc;
  }
  for (int w = threadIdx.x; w < 2 * k * 2 * D; w += blockDim.x) {
    const int X = w / (k * 2 * D), ww = w % (k * 2 * D);
    const int j = ww / (2 * D), col = ww % (2 * D), kp = col / D, q2 = col % D;
    const double* Fq = X == 0 ? cs.Vq : cs.Uq;   // the other side's singular vectors
    double acc = 0.0;
    for (int kx = 0; kx < 2; ++kx) {
      const int blk = X == 0 ? 2 + kx : kx;
      const int off = roff[X == 0 ? 1 : 0][kx];
      double t = 0.0;
      for (int l = 0; l < rk[blk]; ++l) t += Fq[(off + l) * L2 + j] * Rf[blk * CC + l * D + q2];
      acc += t * cval(kx, kp);
    }
    cs.Xx[X][j * L2 + col] = acc * lam_old[q2] / sv[(int)ordd[j]];
  }
  bsync();
  // (d) row update: M'-bar = M' Mx + X-bar Xx, back through the kappa basis, the doubling
  // and the environment weights; G_in-bar into gbar[site].  One thread per (row, q): the
  // columns (+, q) and (-, q) of the lo and hi rows.
  for (int X = 0; X < 2; ++X) {
    const SideDesc& sd = gd.side[X];
    const int OI = sd.outer * sd.inner, Dn = gd.Dn;
    int lo[2], hi[2];
    const int np = side_rows(sd, lo[0], hi[0], lo[1], hi[1]);
    const double* Gi = hist + sd.in_off;
    const double* xb = scr + a.o_xbar + (int64_t)X * a.max_site;
    double* gout = gbar + (int64_t)sd.site * a.max_site;
    const double* Mx = cs.Mx[X];
    const double* Xx = cs.Xx[X];
    for (int w = threadIdx.x; w < OI * D; w += blockDim.x) {
      int dig[kMaxBonds];
      const int oi = w / D, q = w % D;
      const int o = oi / sd.inner, i = oi % sd.inner;
      const double wt = env_weight(sd, o, i, lam, chi, dig);
      double r = 0.0;
      for (int pr = 0; pr < np; ++pr) {
        const int64_t bl = ((int64_t)lo[pr] * sd.outer + o) * D * sd.inner + i;
        const int64_t bh = ((int64_t)hi[pr] * sd.outer + o) * D * sd.inner + i;
        double lp = 0.0, hp = 0.0, lm = 0.0, hm = 0.0;   // M'-bar lo/hi at columns (+, q), (-, q)
        for (int c = 0; c < D; ++c) {
          const double gl = Gi[bl + (int64_t)c * sd.inner], gh = Gi[bh + (int64_t)c * sd.inner];
          const double y = wt * (gl + gh) * kRs2, z = wt * (gl - gh) * kRs2;
          const double mpp = Mx[c * L2 + q], mpm = Mx[c * L2 + D + q];
          const double mmp = Mx[(D + c) * L2 + q], mmm = Mx[(D + c) * L2 + D + q];
          lp += y * mpp + z * mmp;
          hp += y * mpp - z * mmp;
          lm += y * mpm + z * mmm;
          hm += y * mpm - z * mmm;
        }
        const int64_t xl0 = ((int64_t)lo[pr] * sd.outer + o) * Dn * sd.inner + i;
        const int64_t xh0 = ((int64_t)hi[pr] * sd.outer + o) * Dn * sd.inner + i;
        for (int j = 0; j < k; ++j) {
          const double xl = xb[xl0 + (int64_t)j * sd.inner], xh = xb[xh0 + (int64_t)j * sd.inner];
          const double xp = Xx[j * L2 + q], xm = Xx[j * L2 + D + q];
          lp += xl * xp;
          hp += xh * xp;
          lm += xl * xm;
          hm += xh * xm;
        }
        const double yb = (lp + hp) * kRs2, zb = (lm - hm) * kRs2;
        const double gbl = yb + zb, gbh = yb - zb;   // adjoints of the weighted lo / hi entries
        const int64_t el = bl + (int64_t)q * sd.inner, eh = bh + (int64_t)q * sd.inner;
        r += gbl * wt * Gi[el] + gbh * wt * Gi[eh];
        gout[el] = gbl * wt;
        gout[eh] = gbh * wt;
      }
      rq[w] = r;
    }
    bsync();
    for (int oi = threadIdx.x; oi < OI; oi += blockDim.x) {
      double r = 0.0;
      for (int q = 0; q < D; ++q) r += rq[oi * D + q];
      rsum[oi] = r;
    }
    bsync();
    env_lambar(sd, rsum, lam, lambar, chi, 1.0, red);
  }
  // the bond's weight and its adjoint go back to before the gate
  for (int q = threadIdx.x; q < chi; q += blockDim.x) {
    lambar[(int64_t)bond * chi + q] = q < D ? lbo[q] : 0.0;
    lam[(int64_t)bond * chi + q] = q < D ? lam_old[q] : 0.0;
  }
  bsync();
}

// Adjoint of the site-local operator of (layer t, site s): psi_out = sc K' psi_in.
__device__ void local_bwd(const AdjArgs& a, int b, int t, int s, double* gbar, double* red) {
  const LocalDesc& ld = a.locals[(int64_t)t * a.S + s];
  const int P = ld.P, rest = ld.rest;
  const double* gin = a.hist + (int64_t)b * a.hist_elems + ld.off;
  double* gb = gbar + (int64_t)s * a.max_site;
  const double sc = a.rec_sc[((int64_t)(t - a.t_begin) * a.B + b) * a.S + s];
  const int m = a.det[(int64_t)(a.wave_first + b) * a.n_det + ld.det] & 1;
  double acc[kMaxPhys * kMaxPhys];
  for (int e = 0; e < P * P; ++e) acc[e] = 0.0;
  for (int r = threadIdx.x; r < rest; r += blockDim.x)
    for (int i = 0; i < P; ++i) {
      const double gv = gb[(int64_t)i * rest + r];
      for (int kk = 0; kk < P; ++kk) acc[i * P + kk] += gv * gin[(int64_t)kk * rest + r];
    }
  double* Kb = a.Kbar + ((int64_t)b * a.T * a.S + (int64_t)t * a.S + s) * 16;
  for (int e = 0; e < P * P; ++e) {
    const double tot = block_sum(acc[e], red);
    const int i = e / P, kk = e % P;   // K'-bar[i][kk] -> K-bar[i ^ m][kk]
    if (threadIdx.x == 0) Kb[(i ^ m) * P + kk] = sc * tot;
  }
  for (int r = threadIdx.x; r < rest; r += blockDim.x) {
    double v[kMaxPhys];
    for (int i = 0; i < P; ++i) v[i] = gb[(int64_t)i * rest + r];
    for (int kk = 0; kk < P; ++kk) {
      double t2 = 0.0;
      for (int i = 0; i < P; ++i) t2 += ld.K[(i ^ m) * P + kk] * v[i];
      gb[(int64_t)kk * rest + r] = sc * t2;
    }
  }
  bsync();
}

}  // namespace

__global__ void __launch_bounds__(256, 4) k_adjoint(AdjArgs a) {
  __shared__ double red[33];
  __shared__ double red2[256];
  const int b = blockIdx.x;
  double* scr = a.scratch + (int64_t)b * a.scr_stride;
  double* gbar = scr + a.o_gbar;
  double* lambar = scr + a.o_lambar;
  double* lam = a.lam + (int64_t)b * a.nbonds * a.chi;
  double* Kb = a.Kbar + (int64_t)b * a.T * a.S * 16;
  double* pb = a.pbar + (int64_t)b * a.n_gates;
  double* Rb = a.Rbar + (int64_t)b * a.S * 8;
  if (a.do_final) {
    for (int w = threadIdx.x; w < a.T * a.S * 16; w += blockDim.x) Kb[w] = 0.0;
    for (int w = threadIdx.x; w < a.n_gates; w += blockDim.x) pb[w] = 0.0;
    for (int w = threadIdx.x; w < a.S * 8; w += blockDim.x) Rb[w] = 0.0;
    for (int w = threadIdx.x; w < a.nbonds * a.chi; w += blockDim.x) lambar[w] = 0.0;
    __syncthreads();
  }
  const double z = a.Z[2 * b] + a.Z[2 * b + 1];
  if (!(z > 0.0) || !(z < INFINITY)) return;   // probability 0: contributes nothing
  if (a.do_final) {
    final_bwd(a, b, scr, gbar, lambar, Rb, red, red2);
    __syncthreads();
  }
  // the layers of this segment, backwards (gbar, lambar and lam carry over between segments)
  for (int t = a.t_end - 1; t >= a.t_begin; --t) {
    for (int rd = a.layer_round[t + 1] - 1; rd >= a.layer_round[t]; --rd)
      for (int g = a.round_first[rd + 1] - 1; g >= a.round_first[rd]; --g) gate_bwd(a, b, g, scr, gbar, lambar, lam, red2);
    for (int s = 0; s < a.S; ++s) local_bwd(a, b, t, s, gbar, red);
  }
}

cudaError_t launch_adjoint(const AdjArgs& a, int threads, cudaStream_t st) {
  if (a.B <= 0) return cudaSuccess;
  k_adjoint<<<a.B, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace td
