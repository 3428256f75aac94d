// Simple-update truncation core of one gate (Sec. 4), one team of threads per (gate, shot).
//
// Input: the four Gram blocks G_{X,kappa} (X = A, B; kappa = +, -) of the two sides'
// matrices in the kappa basis of the doubled bond (see sweep.cu).  A pivoted Cholesky
// factor R of each block (G = R^T R, rank-revealing) is an R factor of that side's QR
// decomposition, so the two-site core of the simple update is
//     theta = [c(ka, kb) R_{A ka} Lambda R_{B kb}^T],  c(+,+) = c(-,-) = 1/2,
//     c(+,-) = c(-,+) = (1 - 2p)/2,
// (for the diagonal gate diag(w(r + s_a + s_b)) of the generator picture kappa is the
// physical bit, the blocks are the lo and hi rows themselves and c(ka, kb) = w(r + ka + kb)),
// a (rA x rB) matrix, rA, rB <= 2D.  Its SVD theta = U S V^T is truncated to k <= chi values
// (cutoff and multiplet rule), the bond weight becomes S/s_1 (ln s_1 to the log-scale) and
// the update transforms T_{X kappa} = R_{X kappa}^+ [U or V]_{kappa rows, :k} / sqrt2 are
// written for k_update.
//
// The Gram blocks arrive in FP64 on both paths (summed in FP64 from the stored tensors).
//
// The SVD of theta is FP64 one-sided Jacobi.  With `precond` (the mixed-precision path) it
// is first solved in FP32 on a scaled copy; the FP32 right factor, re-orthogonalised in
// FP64 by one Newton-Schulz step V <- V (3I - V^T V)/2, preconditions the FP64 Jacobi
// sweeps, which are run to convergence (mixed-precision Jacobi: precondition with a
// low-precision factor, finish in high precision).  The FP32 solve cannot resolve singular
// values below ~1e-7 of the largest, and the simple update is sensitive to the ones it keeps
// down to the cutoff, so the FP64 sweeps are not cut short.
#include <cfloat>
#include <cmath>

#include "sweep.cuh"
#include "team.cuh"

namespace td {

// Team-shared layout of one item (doubles): five regions of regsz(Dm) = 2Dm x (2Dm + 1)
// (a 2Dm x 2Dm matrix with an odd leading dimension) plus small arrays.
struct CoreSmem {
  double* reg[5];
  double* lam;     // [Dm]
  double* sv;      // [2Dm]
  double* aux;     // [4][Dm] reciprocal Cholesky diagonals, then [2Dm] reciprocal singular values
  int* piv;        // [4][Dm]
  int* order;      // [2Dm]
  int* meta;       // [16]
  static __host__ __device__ size_t regsz(int Dm) { return 4 * (size_t)Dm * Dm + 2 * (size_t)Dm + 2; }
  static __host__ __device__ size_t doubles(int Dm) { return 5 * regsz(Dm) + 7 * (size_t)Dm + 8; }
  static __host__ __device__ size_t ints(int Dm) { return 6 * (size_t)Dm + 16; }
  static __host__ __device__ size_t bytes(int Dm) { return doubles(Dm) * 8 + ints(Dm) * 4 + 16; }
  __device__ void carve(unsigned char* base, int Dm) {
    double* d = reinterpret_cast<double*>(base);
    for (int i = 0; i < 5; ++i) reg[i] = d + (size_t)i * regsz(Dm);
    lam = d + 5 * regsz(Dm);
    sv = lam + Dm;
    aux = sv + 2 * Dm + 8;
    int* ip = reinterpret_cast<int*>(aux + 4 * Dm);
    piv = ip;
    order = piv + 4 * Dm;
    meta = order + 2 * Dm;
  }
};

__device__ __forceinline__ Team make_team(int team_threads) {
  Team tm;
  tm.nt = team_threads;
  tm.tid = threadIdx.x % team_threads;
  tm.bar = 1 + threadIdx.x / team_threads;
  return tm;
}

// The four Gram blocks of item (gate, shot) in FP64: the sum, in chunk order, of the
// partial Grams of its row chunks.
__device__ __forceinline__ void load_gram(const Team& tm, const double* gram, int64_t item, int nchunk, int chi,
                                          int D, double* G) {
  const int DD = D * D;
  const double* src = gram + item * nchunk * 4 * chi * chi;
  for (int w = tm.tid; w < 4 * DD; w += tm.nt) {
    const int64_t off = (int64_t)(w / DD) * chi * chi + w % DD;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += src[(int64_t)c * 4 * chi * chi + off];
    G[w] = s;
  }
}

__global__ void k_core2(SweepArgs a, const GateDesc* __restrict__ gates, const double* __restrict__ gram,
                        double* __restrict__ tbuf, int S, int n_items, int team_threads, int Dm, int precond) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Team tm = make_team(team_threads);
  const int team = threadIdx.x / team_threads;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x / team_threads) + team;
  if (item >= n_items) return;
  CoreSmem sm;
  sm.carve(smem_raw + (size_t)team * CoreSmem::bytes(Dm), Dm);
  const int gi = (int)(item / a.B), b = (int)(item % a.B);
  const GateDesc& gd = gates[gi];
  const int D = gd.D, Dn = gd.Dn, chi = a.chi, DD = D * D;
  int* meta = sm.meta;
  double* slot = reinterpret_cast<double*>(sm.sv + 2 * Dm);   // one spare double after sv
  double* RG = sm.reg[0];
  double* RF = sm.reg[1];
  double* RI = sm.reg[2];
  double* TH = sm.reg[3];
  double* VV = sm.reg[4];
  load_gram(tm, gram, item, a.gram_chunks, chi, D, RG);
  double* lamg = a.lam + ((int64_t)b * a.nbonds + gd.bond) * chi;
  for (int w = tm.tid; w < D; w += tm.nt) sm.lam[w] = lamg[w];
  tm.sync();
  // pivot tolerance per block: gram_cutoff times the side's largest diagonal (< 0: empty)
  if (tm.tid < 4) {
    const int side = tm.tid / 2;
    double e = 0.0;
    for (int blk = 2 * side; blk < 2 * side + 2; ++blk)
      for (int j = 0; j < D; ++j) e = fmax(e, RG[blk * DD + j * D + j]);
    sm.sv[tm.tid] = e > 0.0 ? a.gram_cutoff * e : -1.0;
  }
  tm.sync();
  int* rkp = meta + 12;
  team_pchol4(tm, RG, D, DD, sm.sv, RF, sm.piv, sm.aux, Dm, rkp);
  team_pchol_rinv4(tm, RF, D, DD, sm.piv, sm.aux, Dm, rkp, RI);
  int rk[4];
  for (int blk = 0; blk < 4; ++blk) rk[blk] = rkp[blk];
  double* Rm = RF;           // R factor rows (r x D, ld D) per block
  const double* Rinv = RI;   // right inverse (D x r, ld D) per block
  double* FF = RG;           // scratch free during the SVD (the Gram is consumed)
  double* TT = RF;           // scratch free once theta is formed (R is consumed)
  const int rAp = rk[0], rA = rk[0] + rk[1], rBp = rk[2], rB = rk[2] + rk[3];
  double* tout = tbuf + item * 4 * chi * chi;
  // record for the reverse sweep: ranks, old lambda, R factors and right inverses
  double* rec = a.rec_core ? a.rec_core + ((int64_t)(a.gate_base + gi - a.rec_gate0) * a.B + b) * core_rec_elems(chi)
                           : nullptr;
  const int CC = chi * chi, L2 = 2 * chi;
  if (rec) {
    if (tm.tid < 4) rec[tm.tid] = rk[tm.tid];
    if (tm.tid == 4) { rec[4] = 0.0; rec[5] = 0.0; }
    for (int w = tm.tid; w < D; w += tm.nt) rec[8 + w] = sm.lam[w];
    for (int w = tm.tid; w < 4 * DD; w += tm.nt) {
      rec[8 + chi + (w / DD) * CC + w % DD] = RF[w];
      rec[8 + chi + 4 * CC + (w / DD) * CC + w % DD] = RI[w];
    }
  }
  if (rA == 0 || rB == 0) {            // zero state: this shot has probability 0
    for (int w = tm.tid; w < 4 * chi * chi; w += tm.nt) tout[w] = 0.0;
    for (int w = tm.tid; w < Dn; w += tm.nt) lamg[w] = 0.0;
    if (tm.tid == 0) a.logacc[(int64_t)b * a.nslots + S + gd.bond] = -INFINITY;
    return;
  }
  const Override* ov = vshot_ovr(a.vs, a.ovr, a.wave_first, b, kOvrGate, a.gate_base + gi);
  const double p = ov ? ov->val[0] : gd.p;
  // core coefficients c(ka, kb): kappa = +/- for the gate (1-p) I x I + p X x X; for the
  // diagonal gate of the generator picture kappa is the physical bit itself and
  // c(ka, kb) = w(r + ka + kb), w = (1-p, p), with r the shot's bit of the gate's qubit
  double c_eq = 0.5, c_ne = 0.5 * (1.0 - 2.0 * p);
  if (gd.diag) {
    const int r = a.det[(int64_t)vshot_row(a.vs, a.wave_first, b) * a.n_det + gd.rcol] & 1;
    c_eq = r ? p : 1.0 - p;
    c_ne = r ? 1.0 - p : p;
  }
  for (int w = tm.tid; w < rA * D; w += tm.nt) {     // R_A Lambda, in place
    const int i = w / D, q = w % D;
    const int ka = i < rAp ? 0 : 1, li = i - ka * rAp;
    Rm[ka * DD + li * D + q] *= sm.lam[q];
  }
  tm.sync();
  // theta[i][j] = c(ki, kj) sum_q (R_{A ki} Lambda)[li][q] R_{B kj}[lj][q]  (column-major)
  const int ldt = odd_ld(rA), ldv = odd_ld(rB);
  for (int w = tm.tid; w < rA * rB; w += tm.nt) {
    const int j = w / rA, i = w % rA;
    const int ka = i < rAp ? 0 : 1, li = i - ka * rAp;
    const int kb = j < rBp ? 0 : 1, lj = j - kb * rBp;
    const double* ra = Rm + ka * DD + li * D;
    const double* rb = Rm + (2 + kb) * DD + lj * D;
    double s = 0.0;
    for (int q = 0; q < D; ++q) s += ra[q] * rb[q];
    TH[j * ldt + i] = (ka == kb ? c_eq : c_ne) * s;
  }
  tm.sync();
  if (precond)
    svd_precond(tm, TH, ldt, rA, rB, VV, ldv, FF, TT, meta + 8, slot);
  else
    team_svd_onesided<double>(tm, TH, ldt, rA, rB, VV, ldv, meta + 8, 40, true);
  team_col_norms<double>(tm, TH, ldt, rA, rB, sm.sv);
  team_sort_desc<double>(tm, sm.sv, rB, sm.order);
  if (tm.tid == 0) {
    double srt[2 * kMaxChi];
    for (int j = 0; j < rB; ++j) srt[j] = sm.sv[sm.order[j]];
    int k = 0;
    if (srt[0] > 0.0) k = team_keep_count<double>(srt, rB < rA ? rB : rA, Dn, a.svd_cutoff, a.multiplet_rtol);
    meta[0] = k;
    if (a.stats && k > 0) {
      // discarded fraction sum_{j >= k} s_j^2 / sum_j s_j^2; the shot's gates of a round run
      // concurrently: the max on the bit patterns (non-negative doubles order as them)
      double tot = 0.0, disc = 0.0;
      for (int j = 0; j < rB; ++j) {
        const double q = srt[j] * srt[j];
        tot += q;
        if (j >= k) disc += q;
      }
      const double f = tot > 0.0 ? disc / tot : 0.0;
      double* st = a.stats + (int64_t)(a.wave_first + b) * 4;
      atomicMax(reinterpret_cast<unsigned long long*>(st), (unsigned long long)__double_as_longlong(f));
      atomicAdd(st + 1, f);
    }
  }
  tm.sync();
  const int k = meta[0];
  const double s0 = sm.sv[sm.order[0]];
  if (k == 0 || !(s0 > 0.0)) {
    for (int w = tm.tid; w < 4 * chi * chi; w += tm.nt) tout[w] = 0.0;
    for (int w = tm.tid; w < Dn; w += tm.nt) lamg[w] = 0.0;
    if (tm.tid == 0) a.logacc[(int64_t)b * a.nslots + S + gd.bond] = -INFINITY;
    return;
  }
  if (rec) {
    double* rUS = rec + 8 + chi + 8 * CC;
    double* rV = rUS + L2 * L2;
    double* rsv = rV + L2 * L2;
    double* rord = rsv + L2;
    for (int w = tm.tid; w < rA * rB; w += tm.nt) rUS[(w / rA) * L2 + w % rA] = TH[(w / rA) * ldt + w % rA];
    for (int w = tm.tid; w < rB * rB; w += tm.nt) rV[(w / rB) * L2 + w % rB] = VV[(w / rB) * ldv + w % rB];
    for (int w = tm.tid; w < rB; w += tm.nt) { rsv[w] = sm.sv[w]; rord[w] = sm.order[w]; }
    if (tm.tid == 0) { rec[4] = k; rec[5] = s0; }
  }
  for (int j = tm.tid; j < k; j += tm.nt) sm.aux[j] = 1.0 / sm.sv[sm.order[j]];
  tm.sync();
  const double rs2 = gd.diag ? 1.0 : 0.70710678118654752440;   // the kappa basis' 1/sqrt2
  // T_{A kap}[q][j] = sum_{li} R^+_{A kap}[q][li] U[kap rows li][order j] / sqrt2, U = theta_out / s
  for (int w = tm.tid; w < 2 * D * Dn; w += tm.nt) {
    const int kap = w / (D * Dn), q = (w / Dn) % D, j = w % Dn;
    double acc = 0.0;
    if (j < k) {
      const int cj = sm.order[j];
      const int r = rk[kap], off = kap ? rAp : 0;
      const double* ri = Rinv + kap * DD + q * D;
      const double* u = TH + cj * ldt + off;
      for (int li = 0; li < r; ++li) acc += ri[li] * u[li];
      acc *= sm.aux[j];
    }
    tout[(int64_t)kap * chi * chi + q * Dn + j] = acc * rs2;
  }
  for (int w = tm.tid; w < 2 * D * Dn; w += tm.nt) {
    const int kap = w / (D * Dn), q = (w / Dn) % D, j = w % Dn;
    double acc = 0.0;
    if (j < k) {
      const int cj = sm.order[j];
      const int r = rk[2 + kap], off = kap ? rBp : 0;
      const double* ri = Rinv + (2 + kap) * DD + q * D;
      const double* v = VV + cj * ldv + off;
      for (int lj = 0; lj < r; ++lj) acc += ri[lj] * v[lj];
    }
    tout[(int64_t)(2 + kap) * chi * chi + q * Dn + j] = acc * rs2;
  }
  const double is0 = sm.aux[0];
  for (int j = tm.tid; j < Dn; j += tm.nt) lamg[j] = (j < k) ? sm.sv[sm.order[j]] * is0 : 0.0;
  if (tm.tid == 0) a.logacc[(int64_t)b * a.nslots + S + gd.bond] += log(s0);
}

// ---- launch configuration ---------------------------------------------------------------
// Team size by bond dimension: small cores get one warp each (8 per block), larger ones a
// group of warps, so that no block-wide barrier serialises independent gates.  The team is
// split into four segments of at least Dm lanes for the four Cholesky factorisations.
static void core_shape(int Dm, int& team_threads, int& teams) {
  if (Dm <= 8) { team_threads = 32; teams = 8; }
  else if (Dm <= 16) { team_threads = 64; teams = 2; }
  else { team_threads = 128; teams = 1; }
}

size_t core2_smem_bytes(int Dm) {
  int tt, teams;
  core_shape(Dm, tt, teams);
  return (size_t)teams * CoreSmem::bytes(Dm);
}

template <typename R>
cudaError_t launch_core2(const SweepArgs& a, const GateDesc* g, int count, int Dm, const double* gram, double* tbuf,
                         int S, bool precond, cudaStream_t st) {
  int tt, teams;
  core_shape(Dm, tt, teams);
  const int64_t n_items = (int64_t)count * a.B;
  const size_t smem = (size_t)teams * CoreSmem::bytes(Dm);
  cudaError_t e = cudaFuncSetAttribute(k_core2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((n_items + teams - 1) / teams);
  k_core2<<<blocks, tt * teams, smem, st>>>(a, g, gram, tbuf, S, (int)n_items, tt, Dm, precond ? 1 : 0);
  return cudaGetLastError();
}

template cudaError_t launch_core2<double>(const SweepArgs&, const GateDesc*, int, int, const double*, double*, int,
                                          bool, cudaStream_t);
template cudaError_t launch_core2<float>(const SweepArgs&, const GateDesc*, int, int, const double*, double*, int,
                                         bool, cudaStream_t);

}  // namespace td
