// Kernel argument blocks and launchers of the sweep (sweep.cu) and the final contraction
// (final.cu).
#pragma once

#include <cuda_runtime.h>

#include "td_internal.h"

namespace td {

struct SweepArgs {
  void* gamma;              // site tensors, [B][shot_elems] of the storage type
  int64_t shot_elems;
  double* lam;              // [B][nbonds][chi] bond weights
  double* logacc;           // [B][nslots] log-scale accumulators (sites, bonds, final)
  const uint8_t* det;       // [*][n_det] detector bits of the whole call
  int32_t nbonds, chi, nslots, n_det;
  int32_t wave_first;       // first shot of this wave in `det`
  int32_t B;                // shots in this wave
  int32_t gram_chunks;      // partial Grams per (gate, shot) of the current round (row chunks)
  int32_t chunk_rows;       // rows per Gram / update job (0: kChunkRows)
  double gram_cutoff, svd_cutoff, multiplet_rtol;
  // gradient pass (null otherwise): virtual shots [*] and their override table
  const VShot* vs;
  const Override* ovr;
  int32_t layer;            // current layer (local operators)
  int32_t gate_base;        // global index of the round's first gate (core)
  // recording for the reverse sweep (null otherwise)
  double* rec_sc;           // [B][S] scale of this layer's site-local operators
  double* rec_core;         // [gates][B][kCoreRec(chi)] truncation cores (global gate - rec_gate0)
  int32_t rec_gate0;        // first gate of the recorded segment
  int32_t tc;               // Gram pass on the tensor cores (TD_FP32, TD_TC)
  int32_t precond;          // truncation cores: FP32-preconditioned FP64 Jacobi (TD_FP32, TD_TC)
  int* status;              // device status word: a kernel that gives up writes its td_status
  // truncation statistics (null: none): [call shot][4], entries 0, 1 = the largest and the
  // summed discarded fraction of the simple-update truncations (index wave_first + b)
  double* stats;
};

// Per-gate record of the truncation core for the reverse sweep (doubles), Dm = chi:
// meta[8] (rk0..3, k, s0, unused), lam_old[Dm], R[4][Dm*Dm] (rows r x D, ld D, before the
// lambda scaling), Rinv[4][Dm*Dm] (D x r, ld D), U S [(2Dm)(2Dm)] (theta V after the Jacobi
// sweeps, column-major ld 2Dm, unsorted columns), V [(2Dm)(2Dm)] (same), sv[2Dm], order[2Dm].
__host__ __device__ inline int64_t core_rec_elems(int Dm) { return 8 + Dm + 8LL * Dm * Dm + 8LL * Dm * Dm + 4 * Dm + 8; }

// Detector row and override of shot b of a wave (plain decode: row wave_first + b, none).
__device__ __forceinline__ int vshot_row(const VShot* vs, int wave_first, int b) {
  return vs ? vs[wave_first + b].base : wave_first + b;
}
__device__ __forceinline__ const Override* vshot_ovr(const VShot* vs, const Override* ovr, int wave_first, int b,
                                                     int kind, int target) {
  if (!vs) return nullptr;
  const Override* o = ovr + vs[wave_first + b].ovr;
  return (o->kind == kind && o->target == target) ? o : nullptr;
}

struct FinalArgs {
  const void* gamma;
  int64_t shot_elems;
  const double* lam;
  double* logacc;
  const FinalSite* sites;
  const int32_t* grid_site;  // [ny][nx]
  void* scratch;             // [B][scratch_elems] of the accumulation type (global)
  double* Z;                 // [B][2]
  int64_t scratch_elems;
  int64_t off_mps0, off_mps1, mps_stride;   // boundary MPS (global scratch)
  int64_t off_work;          // work region in the global scratch (when not in shared memory)
  int64_t work_elems;        // work region size (elements)
  int64_t w_F, w_W, w_MT, w_C0, w_C1, w_s, w_ord;   // offsets inside the work region
  int64_t w_Q, w_R, w_P, w_T;   // QR copy of M^T, its triangular factor, FP32-preconditioning scratch
  int32_t precond;           // cut SVDs: FP32-preconditioned FP64 Jacobi (mixed path)
  int32_t use_smem;          // work region in dynamic shared memory
  int32_t threads;           // threads per block (one block per shot)
  int32_t nbonds, chi, nslots, slot;
  int32_t nx, ny, chi_mps;
  int32_t B;
  double svd_cutoff, multiplet_rtol;
  const VShot* vs;           // gradient pass: virtual shots and overrides (null otherwise)
  const Override* ovr;
  int32_t wave_first;
  // recording for the reverse sweep (FP64 only; null otherwise): per shot rec_stride
  // doubles, one slot of rec_slot doubles per (row, column); see FinRecSlot
  double* rec;
  int64_t rec_stride, rec_slot;
  double* stats;             // truncation statistics (null: none): entries 2, 3 of [call shot][4] = the
                             // largest and the summed discarded fraction of the zip-up cuts
  int32_t rec_mC, rec_mA, rec_m, rec_n;   // capacities: carry, MPS tensor, cut rows, cut columns
};

// Layout of one (row, column) slot of the final-contraction record: meta[16] = (kind,
// cJ, aL, cL, aD, aR, L, Rr, U, m, n, k, e2; kind 0 cut, 1 last row, 2 last column), the
// carry C [cJ][aL][cL][2], the MPS tensor A [aL][aD][aR], then for a cut: the left singular
// vectors V (m x m, column-major ld m, unsorted), M^T after the Jacobi sweeps (n x m,
// column-major ld n), the column norms sv[m] and the order[m].
struct FinRecSlot {
  int64_t C, A, V, MT, sv, ord, size;
  __host__ __device__ FinRecSlot(int mC, int mA, int m, int n) {
    C = 16; A = C + mC; V = A + mA; MT = V + (int64_t)m * m; sv = MT + (int64_t)n * m; ord = sv + m; size = ord + m;
  }
};

// Reverse sweep (adjoint.cu): one block per shot of the wave, FP64.
struct AdjArgs {
  const double* hist;          // [B][hist_elems] forward site tensors, versioned layout
  int64_t hist_elems;
  double* lam;                 // [B][nbonds][chi] lambda after the sweep (restored backwards)
  const double* Z;             // [B][2] final contraction values
  const double* rec_core;      // [segment gates][B][core_rec_elems(chi)] (gate - rec_gate0)
  const double* rec_sc;        // [segment layers][B][S] scales of the site-local operators (layer - t_begin)
  const double* rec_fin;       // [B][fin_stride] final-contraction record
  int64_t fin_stride, fin_slot;
  int32_t fin_mC, fin_mA, fin_m, fin_n;
  const GateDesc* gates;       // versioned gate descriptors
  const LocalDesc* locals;     // versioned local descriptors [T * S]
  const FinalSite* finals;     // versioned final sites [S]
  const int32_t* grid_site;    // [ny][nx]
  const int32_t* round_first;  // [n_rounds + 1] first gate of every round, in sweep order
  const int32_t* layer_round;  // [T + 1] first round of every layer
  const uint8_t* det;
  int32_t n_det, wave_first;
  double* scratch;             // [B][scr_stride]
  int64_t scr_stride;
  int64_t o_gbar, o_xbar, o_r, o_lambar, o_core, o_fin;   // offsets in a shot's scratch
  int64_t max_site;            // elements per site slot of gbar
  int64_t fo_F, fo_Fb, fo_T1, fo_T1b, fo_M, fo_Mb, fo_C0, fo_C1, fo_A0, fo_A1, fo_Ub, fo_W, fo_J, fo_In, fo_wg,
      fo_off;                  // final-contraction scratch
  int32_t S, T, nbonds, chi, nx, ny, B, n_gates, max_final_D, mps_stride;
  int32_t t_begin, t_end;      // layers walked by this launch (backwards), a segment of the sweep
  int32_t rec_gate0;           // first gate of the segment (rec_core index origin)
  int32_t do_final;            // this launch starts the reverse sweep: adjoint of the final contraction
  double* Kbar;                // [B][T * S][16]
  double* pbar;                // [B][n_gates]
  double* Rbar;                // [B][S][8]
};
cudaError_t launch_adjoint(const AdjArgs& a, int threads, cudaStream_t st);
// Scratch of the per-gate core adjoint (doubles) for bond cap chi and rows up to max_oi.
inline int64_t CoreScr_elems(int chi, int64_t max_oi) {
  const int64_t L2 = 2 * chi;
  return 2 * L2 * chi + 2 * L2 * L2 + 4 * L2 * chi + 5 * L2 * L2 + 2 * L2 * L2 + 2 * chi * L2 + 4 * chi + max_oi;
}

struct FinalizeArgs {
  const double* Z;
  const double* logacc;
  const uint8_t* det;
  double* logp;              // [*][2] or null
  int32_t* decision;         // [*] or null
  double* margin;            // [*] or null
  int32_t nslots, n_det, wave_first, B, offset_all;
  double mix[4];
  const VShot* vs;           // gradient pass (null otherwise)
  int* status;               // device status word (TD_ERR_NUMERIC for a non-finite shot), or null
};

// Optional timing hooks around each kernel launch (kernel class ids of td_kernel_class).
struct Prof {
  virtual void begin(int k) = 0;
  virtual void end(int k) = 0;
  virtual ~Prof() {}
};

template <typename T, typename R>
cudaError_t launch_sweep_init(const SweepArgs& a, const LocalDesc* locals0, int S, cudaStream_t st);
template <typename T, typename R>
cudaError_t launch_local(const SweepArgs& a, const LocalDesc* locals, int S, cudaStream_t st);
template <typename T, typename R>
cudaError_t launch_round(const SweepArgs& a, const GateDesc* gates, const Round& rd, double* gram, double* tbuf, int S,
                         cudaStream_t st, Prof* prof = nullptr);
template <typename T, typename R>
cudaError_t launch_final(const FinalArgs& f, cudaStream_t st);
cudaError_t launch_finalize(const FinalizeArgs& f, cudaStream_t st);
// Gradient pass (grad.cu): log P per shot and d mean log P / d p_j from the virtual shots'
// log p [B * NV][2]; act[j] = the mechanism's position among the forced ones, or -1.
cudaError_t launch_grad_combine(const double* vlogp, int64_t B, int32_t NV, const int32_t* act, int32_t n_mech,
                                double* logP, double* grad, cudaStream_t st);

// Checkpoint copies of the reverse sweep (grad.cu).
cudaError_t launch_copy_sites(const double* src, int64_t src_stride, const int64_t* src_off, double* dst,
                              int64_t dst_stride, const int64_t* dst_off, const int64_t* len, int S, int B,
                              cudaStream_t st);
cudaError_t launch_copy_rows(const double* src, int64_t src_stride, int64_t src_off, double* dst, int64_t dst_stride,
                             int64_t dst_off, int64_t n, int B, cudaStream_t st);

// Truncation core (core.cu): the simple-update core of every gate of a round; Dm = the
// round's largest active bond dimension; gram: FP64 partial Grams.
template <typename R>
cudaError_t launch_core2(const SweepArgs& a, const GateDesc* g, int count, int Dm, const double* gram, double* tbuf,
                         int S, bool precond, cudaStream_t st);
size_t core2_smem_bytes(int Dm);

// Gram and update passes (absorb.cu), one warp per (gate side, shot, chunk of kChunkRows
// rows); Dm = the round's largest bond dimension (before or after the gate).
constexpr int kChunkRows = 2048;      // default
constexpr int kMinChunkRows = 512;    // smallest schedule candidate (sizes the partial-Gram buffer)
int absorb_chunks(int max_rows, int chunk_rows);
template <typename T>
cudaError_t launch_gram2(const SweepArgs& a, const GateDesc* g, int count, int Dm, double* gram, int nchunk,
                         int chunk_rows, cudaStream_t st);
// Tensor-core Gram (absorb.cu; bond dimensions 4..16; T: storage type).
bool gram_tc_supported(int maxD);
template <typename T>
cudaError_t launch_gram_tc(const SweepArgs& a, const GateDesc* g, int count, int maxD, double* gram, int nchunk,
                           int chunk_rows, cudaStream_t st);
template <typename T>
cudaError_t launch_update2(const SweepArgs& a, const GateDesc* g, int count, int Dm, const double* tbuf, int nchunk,
                           int chunk_rows, cudaStream_t st);

// Static scratch of the allocation-free final contraction (final.cu).
constexpr size_t kStaticFinalScratchBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxStaticDevices = 64;
// Device address of the static scratch on the current device (looked up on first use).
cudaError_t static_final_scratch(void** ptr);

}  // namespace td
