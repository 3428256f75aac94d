// C ABI of libtd (include/td.h): network construction, device workspace, and the launch
// sequence of one decoding call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gen.cuh"
#include "sweep.cuh"
#include "td_internal.h"
#include "team.cuh"

namespace {
thread_local std::string g_err;

// Schedule candidates of td_network_tune: k_final block size and rows per Gram / update job.
constexpr int kFinalThreads[] = {256, 512, 1024};
constexpr int kChunkCandidates[] = {512, 1024, 2048, 4096};

td_status fail(td_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

td_status cuda_fail(cudaError_t e, const char* what) {
  return fail(TD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace

struct td_network {
  td::Plan plan;
  int32_t wave = 0;
  size_t elem = 8;            // bytes per storage element of the site tensors
  static constexpr size_t felem = 8;   // bytes per element of the final contraction (FP64 on both paths)
  void* d_gamma = nullptr;
  double* d_lam = nullptr;
  double* d_logacc = nullptr;
  double* d_gram = nullptr;
  double* d_tbuf = nullptr;
  void* d_fscr = nullptr;
  double* d_Z = nullptr;
  int* d_status = nullptr;      // device status word (td_network_check)
  td::GateDesc* d_gates = nullptr;
  td::LocalDesc* d_locals = nullptr;
  td::FinalSite* d_finals = nullptr;
  int32_t* d_grid = nullptr;
  uint8_t* d_det_stage = nullptr;
  double* d_logp_stage = nullptr;
  int32_t nslots = 0;
  td::FinalArgs fin{};
  int64_t fscr_elems = 0;       // final-contraction scratch per shot (largest candidate layout)
  int smem_optin = 0;
  int32_t chunk_rows = td::kChunkRows;   // rows per Gram / update job
  size_t bytes = 0;
  int64_t launches_per_wave = 0;
  std::vector<void*> allocs;
  // copy of the problem (the gradient pass rebuilds the parameter objects at other rates)
  std::vector<int32_t> H_indptr, H_indices, L_indptr, L_indices, det_xyt;
  std::vector<double> rates;
  int32_t n_obs = 0;
  td_options opt{};
  // gradient pass: override table for the current rates, per-mechanism entries (0: none)
  std::vector<double> ovr_rates;
  std::vector<td::Override> ovr_host;
  std::vector<int32_t> ovr_of;           // [n_mech][2] override index at p_j = 0, 1
  td::Override* d_ovr = nullptr;
  size_t d_ovr_cap = 0;
  td::VShot* d_vs = nullptr;
  size_t d_vs_cap = 0;
  double* d_vlogp = nullptr;
  size_t d_vlogp_cap = 0;
  int32_t* d_act = nullptr;
  size_t d_act_cap = 0;
  // reverse sweep: versioned descriptors, round tables, per-wave buffers (grad_wave shots)
  td::GateDesc* d_hgates = nullptr;
  td::LocalDesc* d_hlocals = nullptr;
  td::FinalSite* d_hfinals = nullptr;
  int32_t* d_round_first = nullptr;
  int32_t* d_layer_round = nullptr;
  int64_t *d_seg_in_off = nullptr, *d_seg_out_off = nullptr, *d_seg_len = nullptr, *d_ckpt_off = nullptr;
  double* d_ckpt = nullptr;      // [grad_wave][ckpt_shot_elems] checkpointed segment inputs
  int32_t grad_wave = 0;
  int64_t gfscr_elems = 0;      // per-shot elements of d_gfscr as allocated
  double *d_hist = nullptr, *d_rec_core = nullptr, *d_rec_sc = nullptr, *d_rec_fin = nullptr, *d_adj_scr = nullptr,
         *d_gfscr = nullptr, *d_Kbar = nullptr, *d_pbar = nullptr, *d_Rbar = nullptr, *d_glogp = nullptr;
  td::AdjArgs adj{};
  td::FinalArgs gfin{};
  // generator network: elimination transform, pivot columns, xbar, and per-chunk rows
  unsigned long long* d_gen_trans = nullptr;
  int32_t* d_gen_col = nullptr;
  uint8_t* d_gen_xbar = nullptr;
  uint8_t* d_gen_rows = nullptr;     // [2 gen_chunk][n_qubits]
  int32_t* d_gen_cls = nullptr;      // [gen_chunk]
  double* d_gen_lp = nullptr;        // [2 gen_chunk][2]
  int64_t gen_chunk = 0;             // shots per chunk (two sweep rows each)
  td_dem dem_view(const double* p) const {
    td_dem d{};
    d.n_det = plan.n_det; d.n_mech = plan.n_mech; d.n_obs = n_obs;
    d.H_indptr = H_indptr.data(); d.H_indices = H_indices.data();
    d.L_indptr = L_indptr.data(); d.L_indices = L_indices.data();
    d.p = p;
    return d;
  }
  td_layout layout_view() const {
    td_layout l{};
    l.det_xyt = det_xyt.data();
    return l;
  }
  // growable device buffer (freed with the network)
  template <typename P>
  bool reserve(P*& ptr, size_t& cap, size_t n) {
    if (n <= cap && ptr) return true;
    if (ptr) {
      cudaFree(ptr);
      allocs.erase(std::remove(allocs.begin(), allocs.end(), (void*)ptr), allocs.end());
      ptr = nullptr;
      cap = 0;
    }
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(P)) != cudaSuccess) { cudaGetLastError(); return false; }
    allocs.push_back(q);
    ptr = reinterpret_cast<P*>(q);
    cap = n;
    return true;
  }
  // kernel timing (td_network_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;

  ~td_network() {
    for (void* p : allocs) cudaFree(p);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (auto& u : ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
  }
  cudaEvent_t take_event() {
    if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // Brackets one launch of kernel class k with events when profiling.
  struct Mark {
    td_network* n; int k; cudaStream_t s; cudaEvent_t a = nullptr;
    Mark(td_network* net, int cls, cudaStream_t st) : n(net), k(cls), s(st) {
      if (n->profiling) { a = n->take_event(); cudaEventRecord(a, s); }
    }
    ~Mark() {
      if (a) { cudaEvent_t b = n->take_event(); cudaEventRecord(b, s); n->ev_used.push_back({k, {a, b}}); }
    }
  };
  template <typename P>
  bool alloc(P*& ptr, size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(p);
    bytes += n;
    ptr = reinterpret_cast<P*>(p);
    return true;
  }
};

// Final-contraction layout (work region offsets, shared or global memory) for a block of
// `threads` threads (the Jacobi lane groups and leading dimensions depend on it).
static void final_layout(td_network* net, int threads, bool allow_smem = true) {
  const td::Plan& P = net->plan;
  const int cm = P.chi_mps, Dm = P.max_final_D;
  const int64_t cmx = std::max(cm, 2);
  const int64_t mps_stride = ((int64_t)cm * Dm * cmx + 3) / 4 * 4;
  const int64_t mF = 2LL * Dm * Dm * Dm * Dm;
  net->fin.threads = threads;
  int64_t mMT = 0, mV = 0;   // M^T (n x m) and V (m x m) with the bank-spreading leading dimensions
  {
    const int n_max = (int)(cmx * Dm * 2), m_max = cm * Dm;
    for (int m = 1; m <= m_max; ++m) {
      const int g = td::team_svd_group(threads, n_max, m);
      mMT = std::max<int64_t>(mMT, (int64_t)m * td::bank_ld32(n_max, g));
      mV = std::max<int64_t>(mV, (int64_t)m * td::bank_ld32(m, g));
    }
  }
  // QR-reduced cuts (n >= m): the copy of M^T (n x m, ld n), the m x m factor R and V with the
  // leading dimensions of an m x m Jacobi, and the FP32-preconditioning scratch
  int64_t mR = 0;
  {
    const int m_max = cm * Dm;
    for (int m = 1; m <= m_max; ++m) {
      const int g = td::team_svd_group(threads, m, m);
      mR = std::max<int64_t>(mR, (int64_t)m * td::bank_ld32(m, g));
    }
  }
  int64_t mQ = (int64_t)cmx * Dm * 2 * cm * Dm;
  {
    // wide cuts (n < m): M (m x n) with the leading dimension of an n-column Jacobi (in the
    // QR copy's region) and its n x n rotation (in V's region)
    const int m_max = cm * Dm;
    for (int m = 2; m <= m_max; ++m)
      for (int n = 1; n < m; ++n) {
        const int g = td::team_svd_group(threads, m, n);
        mQ = std::max<int64_t>(mQ, (int64_t)n * td::bank_ld32(m, g));
        mV = std::max<int64_t>(mV, (int64_t)n * td::bank_ld32(n, g));
      }
  }
  const int64_t mP = (int64_t)(cm * Dm + 1) * cm * Dm, mT = (int64_t)cm * Dm * cm * Dm;
  const int64_t mW = std::max<int64_t>({(int64_t)cm * Dm * 2 * Dm * cmx, mV, mR});
  const int64_t mC = (int64_t)cm * cmx * Dm * 2;
  const int64_t mS = 2LL * cm * Dm;
  const int64_t mOrd = ((int64_t)cm * Dm * 4 + net->felem - 1) / net->felem;
  int64_t wacc = 0;
  auto wtake = [&](int64_t n) { int64_t r = wacc; wacc += (n + 3) / 4 * 4; return r; };
  net->fin.w_F = wtake(mF);
  net->fin.w_W = wtake(mW);
  net->fin.w_MT = wtake(mMT);
  net->fin.w_C0 = wtake(mC);
  net->fin.w_C1 = wtake(mC);
  net->fin.w_s = wtake(mS);
  net->fin.w_ord = wtake(mOrd);
  // the QR copy is dead once R is extracted, before the preconditioning scratch is used
  net->fin.w_Q = wtake(std::max<int64_t>(mQ, (mP + 3) / 4 * 4 + mT));
  net->fin.w_P = net->fin.w_Q;
  net->fin.w_T = net->fin.w_Q + (mP + 3) / 4 * 4;
  net->fin.w_R = wtake(mR);
  net->fin.work_elems = wacc;
  net->fin.precond = (P.precision == TD_FP64) ? 0 : 1;
  const size_t static_smem = 8 * 1024;   // k_final's own shared arrays
  net->fin.use_smem = (allow_smem && (size_t)wacc * net->felem + static_smem <= (size_t)net->smem_optin) ? 1 : 0;
  int64_t acc = 0;
  auto take = [&](int64_t n) { int64_t r = acc; acc += (n + 3) / 4 * 4; return r; };
  net->fin.off_mps0 = take(mps_stride * P.nx);
  net->fin.off_mps1 = take(mps_stride * P.nx);
  net->fin.mps_stride = mps_stride;
  net->fin.off_work = net->fin.use_smem ? 0 : take(wacc);
  net->fin.scratch_elems = acc;
}

extern "C" {

void td_default_options(td_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->chi = 8;
  opt->chi_mps = 16;
  opt->precision = TD_FP64;
  opt->ckpt_stride = 0;
  opt->svd_cutoff = 1e-12;
  opt->multiplet_rtol = 1e-8;
  opt->gram_cutoff = -1.0;   // per precision
  opt->mem_budget = size_t(16) << 30;
  opt->max_wave = 0;
}

const char* td_last_error(void) { return g_err.c_str(); }

static td_status finish_build(td_network* net, const td_options& o, td_network** out);

td_status td_build_network(const td_dem* dem, const td_layout* layout, const td_options* opt, td_network** out) {
  g_err.clear();
  if (!dem || !layout || !out) return fail(TD_ERR_INVALID, "null argument");
  *out = nullptr;
  td_options o;
  if (opt) o = *opt; else td_default_options(&o);
  td_network* net = new (std::nothrow) td_network();
  if (!net) return fail(TD_ERR_OOM, "host allocation failed");
  std::string err;
  td_status st = td::build_plan(*dem, *layout, o, net->plan, err);
  if (st != TD_OK) { delete net; return fail(st, err); }
  net->H_indptr.assign(dem->H_indptr, dem->H_indptr + dem->n_det + 1);
  net->H_indices.assign(dem->H_indices, dem->H_indices + dem->H_indptr[dem->n_det]);
  net->L_indptr.assign(dem->L_indptr, dem->L_indptr + dem->n_obs + 1);
  net->L_indices.assign(dem->L_indices, dem->L_indices + dem->L_indptr[dem->n_obs]);
  net->det_xyt.assign(layout->det_xyt, layout->det_xyt + 3 * (size_t)dem->n_det);
  net->rates.assign(dem->p, dem->p + dem->n_mech);
  net->n_obs = dem->n_obs;
  return finish_build(net, o, out);
}

td_status td_build_gen_network(const td_gen* gen, const td_options* opt, td_network** out) {
  g_err.clear();
  if (!gen || !out) return fail(TD_ERR_INVALID, "null argument");
  *out = nullptr;
  td_options o;
  if (opt) o = *opt; else td_default_options(&o);
  td_network* net = new (std::nothrow) td_network();
  if (!net) return fail(TD_ERR_OOM, "host allocation failed");
  std::string err;
  td_status st = td::build_gen_plan(*gen, o, net->plan, err);
  if (st != TD_OK) { delete net; return fail(st, err); }
  if (net->plan.check_words > 3000) { delete net; return fail(TD_ERR_UNSUPPORTED, "more than 192000 checks"); }
  net->n_obs = 1;
  net->rates.assign(gen->p, gen->p + gen->n_qubits);
  return finish_build(net, o, out);
}

// Device workspace of a planned network (both kinds); deletes net on failure.
static td_status finish_build(td_network* net, const td_options& o, td_network** out) {
  td::Plan& P = net->plan;
  if (P.nx > td::kMaxGridX) { delete net; return fail(TD_ERR_UNSUPPORTED, "grid wider than 64 sites"); }
  net->opt = o;
  const int chi = P.chi, cm = P.chi_mps, Dm = P.max_final_D;
  if ((int64_t)cm * Dm > td::kMaxFinalBond) {
    delete net;
    return fail(TD_ERR_UNSUPPORTED, "chi_mps * final bond dimension must be <= 1024");
  }
  net->elem = (o.precision == TD_FP32) ? 4 : 8;
  net->nslots = P.S + P.n_bonds + 1;

  // final-contraction scratch per shot (elements of the accumulation type): the boundary
  // MPS (two buffers) in global memory, and the work region of one block -- in shared
  // memory when it fits, otherwise after the MPS in global memory.  Block size of k_final:
  // 512 threads once the widest cut has >= 128 columns (more lanes per column pair in the
  // Jacobi steps: rotated d=9, chi=16, chi_mps=8 runs 1.9x faster), 256 below (no gain at 64
  // columns); td_network_tune may pick another of kFinalThreads.  The scratch is sized for
  // the largest layout of all candidates.
  int dev = 0;
  net->smem_optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&net->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    net->smem_optin = 0;
  }
  int64_t acc = 0;
  for (int th : kFinalThreads)
    for (int sm = 0; sm < 2; ++sm) {
      final_layout(net, th, sm == 1);
      acc = std::max<int64_t>(acc, net->fin.scratch_elems);
    }
  final_layout(net, (int64_t)cm * Dm >= 128 ? 512 : 256);
  net->fscr_elems = acc;

  int max_chunks = 1;
  for (const td::LayerPlan& L : P.layers)
    for (const td::Round& rd : L.rounds) max_chunks = std::max(max_chunks, td::absorb_chunks(rd.max_rows, td::kMinChunkRows));
  const size_t per_shot = P.shot_elems * net->elem + (size_t)P.n_bonds * chi * 8 + (size_t)net->nslots * 8 +
                          (size_t)P.max_round_gates * 4 * chi * chi * (8 * max_chunks + 8) +
                          (size_t)net->fscr_elems * net->felem + 16 + (size_t)P.n_det + 16;
  const size_t budget = o.mem_budget ? o.mem_budget : (size_t(16) << 30);
  int64_t wave = (int64_t)(budget / std::max<size_t>(per_shot, 1));
  if (o.max_wave > 0) wave = std::min<int64_t>(wave, o.max_wave);
  wave = std::min<int64_t>(wave, 65535);
  if (wave < 1) { delete net; return fail(TD_ERR_OOM, "mem_budget too small for one shot"); }
  net->wave = (int32_t)wave;

  bool ok = net->alloc(net->d_gamma, (size_t)wave * P.shot_elems * net->elem) &&
            net->alloc(net->d_lam, (size_t)wave * P.n_bonds * chi * 8) &&
            net->alloc(net->d_logacc, (size_t)wave * net->nslots * 8) &&
            net->alloc(net->d_gram, (size_t)std::max(P.max_round_gates, 1) * wave * 4 * chi * chi * 8 * max_chunks) &&
            net->alloc(net->d_tbuf, (size_t)std::max(P.max_round_gates, 1) * wave * 4 * chi * chi * 8) &&
            net->alloc(net->d_fscr, (size_t)wave * net->fscr_elems * net->felem) &&
            net->alloc(net->d_Z, (size_t)wave * 2 * 8) &&
            net->alloc(net->d_gates, sizeof(td::GateDesc) * P.gates.size()) &&
            net->alloc(net->d_locals, sizeof(td::LocalDesc) * P.locals.size()) &&
            net->alloc(net->d_finals, sizeof(td::FinalSite) * P.finals.size()) &&
            net->alloc(net->d_grid, sizeof(int32_t) * P.grid_site.size()) &&
            net->alloc(net->d_det_stage, (size_t)wave * P.n_det) &&
            net->alloc(net->d_logp_stage, (size_t)wave * 2 * 8) &&
            net->alloc(net->d_status, sizeof(int));
  if (ok && P.gen) {
    net->gen_chunk = std::max<int64_t>(1, wave / 2);
    ok = net->alloc(net->d_gen_trans, sizeof(unsigned long long) * P.gen_rows.size()) &&
         net->alloc(net->d_gen_col, sizeof(int32_t) * std::max<size_t>(P.gen_col.size(), 1)) &&
         net->alloc(net->d_gen_xbar, P.gen_xbar.size()) &&
         net->alloc(net->d_gen_rows, (size_t)2 * net->gen_chunk * P.n_qubits) &&
         net->alloc(net->d_gen_cls, sizeof(int32_t) * net->gen_chunk) &&
         net->alloc(net->d_gen_lp, sizeof(double) * 4 * net->gen_chunk);
  }
  if (!ok) { delete net; return fail(TD_ERR_OOM, "device allocation failed"); }
  cudaError_t e;
  if ((!P.gates.empty() && (e = cudaMemcpy(net->d_gates, P.gates.data(), sizeof(td::GateDesc) * P.gates.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemcpy(net->d_locals, P.locals.data(), sizeof(td::LocalDesc) * P.locals.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(net->d_finals, P.finals.data(), sizeof(td::FinalSite) * P.finals.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(net->d_grid, P.grid_site.data(), sizeof(int32_t) * P.grid_site.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    delete net;
    return cuda_fail(e, "descriptor upload");
  }
  if (P.gen &&
      ((e = cudaMemcpy(net->d_gen_trans, P.gen_rows.data(), sizeof(unsigned long long) * P.gen_rows.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
       (!P.gen_col.empty() && (e = cudaMemcpy(net->d_gen_col, P.gen_col.data(), sizeof(int32_t) * P.gen_col.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
       (e = cudaMemcpy(net->d_gen_xbar, P.gen_xbar.data(), P.gen_xbar.size(), cudaMemcpyHostToDevice)) != cudaSuccess)) {
    delete net;
    return cuda_fail(e, "generator tables upload");
  }
  if ((e = cudaMemset(net->d_status, 0, sizeof(int))) != cudaSuccess) { delete net; return cuda_fail(e, "status init"); }
  // pageable uploads may still be in flight when cudaMemcpy returns
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) { delete net; return cuda_fail(e, "descriptor upload"); }
  int64_t launches = 1 + 2 + (P.gen ? 2 : 0);   // init, final, finalize (+ rows, combine)
  const int per_round = 3;   // Gram, core, update
  for (const td::LayerPlan& L : P.layers) launches += 1 + per_round * (int64_t)L.rounds.size();
  net->launches_per_wave = launches;
  *out = net;
  return TD_OK;
}

struct NetProf : td::Prof {
  td_network* n; cudaStream_t s; cudaEvent_t a = nullptr;
  NetProf(td_network* net, cudaStream_t st) : n(net), s(st) {}
  void begin(int) override { if (n->profiling) { a = n->take_event(); cudaEventRecord(a, s); } }
  void end(int k) override {
    if (a) { cudaEvent_t b = n->take_event(); cudaEventRecord(b, s); n->ev_used.push_back({k, {a, b}}); a = nullptr; }
  }
};

static td_status run(td_network* net, const uint8_t* det, int64_t B, double* logp, int32_t* decision, double* margin,
                     cudaStream_t st, void* final_scratch = nullptr, const td::VShot* vs = nullptr,
                     const td::Override* ovr = nullptr, double* stats = nullptr) {
  td::Plan& P = net->plan;
  if (stats && B > 0) {
    const cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(double) * 4 * (size_t)B, st);
    if (e != cudaSuccess) return cuda_fail(e, "statistics reset");
  }
  NetProf prof(net, st);
  for (int64_t w0 = 0; w0 < B; w0 += net->wave) {
    const int32_t Bw = (int32_t)std::min<int64_t>(net->wave, B - w0);
    td::SweepArgs a{};
    a.gamma = net->d_gamma;
    a.shot_elems = P.shot_elems;
    a.lam = net->d_lam;
    a.logacc = net->d_logacc;
    a.det = det;
    a.nbonds = P.n_bonds;
    a.chi = P.chi;
    a.nslots = net->nslots;
    a.n_det = P.n_det;
    a.wave_first = (int32_t)w0;
    a.B = Bw;
    a.gram_cutoff = P.gram_cutoff;
    a.svd_cutoff = P.svd_cutoff;
    a.multiplet_rtol = P.multiplet_rtol;
    a.vs = vs;
    a.ovr = ovr;
    a.chunk_rows = net->chunk_rows;
    a.tc = P.precision == TD_FP64 ? 0 : 1;
    a.precond = P.precision == TD_FP64 ? 0 : 1;
    a.status = net->d_status;
    a.stats = stats;
    const bool f64 = P.precision != TD_FP32;   // storage type
    cudaError_t e;
    {
      td_network::Mark mk(net, TD_K_INIT, st);
      e = f64 ? td::launch_sweep_init<double, double>(a, net->d_locals, P.S, st)
              : td::launch_sweep_init<float, float>(a, net->d_locals, P.S, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "init launch");
    for (int32_t t = 0; t < P.T; ++t) {
      const td::LayerPlan& L = P.layers[t];
      a.layer = t;
      {
        td_network::Mark mk(net, TD_K_LOCAL, st);
        e = f64 ? td::launch_local<double, double>(a, net->d_locals + L.local_first, P.S, st)
                : td::launch_local<float, float>(a, net->d_locals + L.local_first, P.S, st);
      }
      if (e != cudaSuccess) return cuda_fail(e, "local launch");
      for (const td::Round& rd : L.rounds) {
        e = f64 ? td::launch_round<double, double>(a, net->d_gates, rd, net->d_gram, net->d_tbuf, P.S, st, &prof)
                : td::launch_round<float, float>(a, net->d_gates, rd, net->d_gram, net->d_tbuf, P.S, st, &prof);
        if (e != cudaSuccess) return cuda_fail(e, "gate round launch");
      }
    }
    td::FinalArgs f = net->fin;
    f.gamma = net->d_gamma;
    f.shot_elems = P.shot_elems;
    f.lam = net->d_lam;
    f.logacc = net->d_logacc;
    f.sites = net->d_finals;
    f.grid_site = net->d_grid;
    f.scratch = final_scratch ? final_scratch : net->d_fscr;
    f.Z = net->d_Z;
    f.nbonds = P.n_bonds;
    f.chi = P.chi;
    f.nslots = net->nslots;
    f.slot = P.S + P.n_bonds;
    f.nx = P.nx;
    f.ny = P.ny;
    f.chi_mps = P.chi_mps;
    f.B = Bw;
    f.svd_cutoff = P.svd_cutoff;
    f.multiplet_rtol = P.multiplet_rtol;
    f.vs = vs;
    f.ovr = ovr;
    f.wave_first = (int32_t)w0;
    f.stats = stats;
    {
      td_network::Mark mk(net, TD_K_FINAL, st);
      e = f64 ? td::launch_final<double, double>(f, st) : td::launch_final<float, double>(f, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "final launch");
    td::FinalizeArgs z{};
    z.Z = net->d_Z;
    z.logacc = net->d_logacc;
    z.det = det;
    z.logp = logp;
    z.decision = decision;
    z.margin = margin;
    z.nslots = net->nslots;
    z.n_det = P.n_det;
    z.wave_first = (int32_t)w0;
    z.B = Bw;
    z.offset_all = P.offset_all;
    for (int i = 0; i < 4; ++i) z.mix[i] = P.glob_mix[i];
    z.vs = vs;
    z.status = net->d_status;
    {
      td_network::Mark mk(net, TD_K_FINALIZE, st);
      e = td::launch_finalize(z, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "finalize launch");
  }
  return TD_OK;
}

static td_status check_call(td_network* net, const void* det, int64_t B) {
  if (!net) return fail(TD_ERR_INVALID, "null network");
  if (net->plan.gen) return fail(TD_ERR_INVALID, "generator network: decode with td_gen_coset_logprob / td_gen_decode");
  if (B < 0) return fail(TD_ERR_INVALID, "B must be >= 0");
  if (B > 0 && !det) return fail(TD_ERR_INVALID, "null detector buffer");
  if (B > (int64_t)1 << 31) return fail(TD_ERR_INVALID, "B too large");
  return TD_OK;
}

td_status td_coset_logprob(td_network* net, const uint8_t* det_dev, int64_t B, double* logp_dev, void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_dev, B);
  if (s != TD_OK) return s;
  if (B > 0 && !logp_dev) return fail(TD_ERR_INVALID, "null output buffer");
  return run(net, det_dev, B, logp_dev, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

td_status td_coset_logprob_stats(td_network* net, const uint8_t* det_dev, int64_t B, double* logp_dev,
                                 double* stats_dev, void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_dev, B);
  if (s != TD_OK) return s;
  if (B > 0 && (!logp_dev || !stats_dev)) return fail(TD_ERR_INVALID, "null output buffer");
  return run(net, det_dev, B, logp_dev, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream), nullptr, nullptr,
             nullptr, stats_dev);
}

td_status td_decode(td_network* net, const uint8_t* det_dev, int64_t B, int32_t* decision_dev, double* margin_dev,
                    void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_dev, B);
  if (s != TD_OK) return s;
  if (B > 0 && !decision_dev) return fail(TD_ERR_INVALID, "null decision buffer");
  return run(net, det_dev, B, nullptr, decision_dev, margin_dev, reinterpret_cast<cudaStream_t>(stream));
}

static td_status run_gen(td_network* net, const uint8_t* syn, int64_t B, double* logp, int32_t* decision,
                         double* margin, cudaStream_t st) {
  td::Plan& P = net->plan;
  for (int64_t c0 = 0; c0 < B; c0 += net->gen_chunk) {
    const int64_t Bc = std::min<int64_t>(net->gen_chunk, B - c0);
    td::GenRowsArgs g{};
    g.syn = syn + c0 * P.n_checks;
    g.B = Bc;
    g.n_checks = P.n_checks;
    g.words = P.check_words;
    g.trans = net->d_gen_trans;
    g.rank = P.gen_rank;
    g.col = net->d_gen_col;
    g.xbar = net->d_gen_xbar;
    g.n_cols = P.n_qubits;
    g.rows = net->d_gen_rows;
    g.cls = net->d_gen_cls;
    cudaError_t e;
    {
      td_network::Mark mk(net, TD_K_INIT, st);
      e = td::launch_gen_rows(g, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "representative launch");
    td_status s = run(net, net->d_gen_rows, 2 * Bc, net->d_gen_lp, nullptr, nullptr, st);
    if (s != TD_OK) return s;
    td::GenCombineArgs z{};
    z.row_logp = net->d_gen_lp;
    z.cls = net->d_gen_cls;
    z.B = Bc;
    z.log_offset = P.gen_log_offset;
    z.logp = logp ? logp + 2 * c0 : nullptr;
    z.decision = decision ? decision + c0 : nullptr;
    z.margin = margin ? margin + c0 : nullptr;
    {
      td_network::Mark mk(net, TD_K_FINALIZE, st);
      e = td::launch_gen_combine(z, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "class combine launch");
  }
  return TD_OK;
}

static td_status check_gen_call(td_network* net, const void* syn, int64_t B) {
  if (!net) return fail(TD_ERR_INVALID, "null network");
  if (!net->plan.gen) return fail(TD_ERR_INVALID, "detector network: decode with td_coset_logprob / td_decode");
  if (B < 0) return fail(TD_ERR_INVALID, "B must be >= 0");
  if (B > 0 && !syn) return fail(TD_ERR_INVALID, "null syndrome buffer");
  if (B > (int64_t)1 << 30) return fail(TD_ERR_INVALID, "B too large");
  return TD_OK;
}

td_status td_gen_rows_host(const td_gen* gen, const uint8_t* syn_host, int64_t B, uint8_t* rows_host,
                           int32_t* cls_host, int32_t* col_host) {
  g_err.clear();
  if (!gen || B < 0 || (B > 0 && (!syn_host || !rows_host || !cls_host))) return fail(TD_ERR_INVALID, "null argument");
  td_options o;
  td_default_options(&o);
  td::Plan P;
  std::string err;
  td_status st = td::build_gen_plan(*gen, o, P, err);
  if (st != TD_OK) return fail(st, err);
  const int nq = P.n_qubits, nc = P.n_checks, words = P.check_words;
  std::vector<uint64_t> mw(words);
  for (int64_t b = 0; b < B; ++b) {
    std::fill(mw.begin(), mw.end(), 0ull);
    for (int c = 0; c < nc; ++c)
      if (syn_host[b * nc + c] & 1) mw[c / 64] |= 1ull << (c % 64);
    auto dot = [&](int i) {
      int par = 0;
      for (int w = 0; w < words; ++w) par ^= __builtin_popcountll(P.gen_rows[(size_t)i * words + w] & mw[w]);
      return par & 1;
    };
    uint8_t* r0 = rows_host + 2 * b * nq;
    uint8_t* r1 = r0 + nq;
    std::fill(r0, r0 + nq, (uint8_t)0);
    for (int i = 0; i < P.gen_rank; ++i)
      if (dot(i)) r0[P.gen_col[i]] = 1;
    int bad = 0;
    for (int i = P.gen_rank; i < nc; ++i) bad |= dot(i);
    for (int j = 0; j < nq; ++j) r1[j] = r0[j] ^ P.gen_xbar[j];
    cls_host[b] = bad ? -1 : dot(nc);
  }
  if (col_host) std::copy(P.gen_qcol.begin(), P.gen_qcol.end(), col_host);
  return TD_OK;
}

td_status td_gen_coset_logprob(td_network* net, const uint8_t* syn_dev, int64_t B, double* logp_dev, void* stream) {
  g_err.clear();
  td_status s = check_gen_call(net, syn_dev, B);
  if (s != TD_OK) return s;
  if (B > 0 && !logp_dev) return fail(TD_ERR_INVALID, "null output buffer");
  return run_gen(net, syn_dev, B, logp_dev, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

td_status td_gen_decode(td_network* net, const uint8_t* syn_dev, int64_t B, int32_t* decision_dev, double* margin_dev,
                        void* stream) {
  g_err.clear();
  td_status s = check_gen_call(net, syn_dev, B);
  if (s != TD_OK) return s;
  if (B > 0 && !decision_dev) return fail(TD_ERR_INVALID, "null decision buffer");
  return run_gen(net, syn_dev, B, nullptr, decision_dev, margin_dev, reinterpret_cast<cudaStream_t>(stream));
}

td_status td_coset_logprob_host(td_network* net, const uint8_t* det_host, int64_t B, double* logp_host, void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_host, B);
  if (s != TD_OK) return s;
  if (B > 0 && !logp_host) return fail(TD_ERR_INVALID, "null output buffer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int32_t n_det = net->plan.n_det;
  for (int64_t w0 = 0; w0 < B; w0 += net->wave) {
    const int64_t Bw = std::min<int64_t>(net->wave, B - w0);
    cudaError_t e = cudaMemcpyAsync(net->d_det_stage, det_host + w0 * n_det, (size_t)Bw * n_det,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "detector copy");
    s = run(net, net->d_det_stage, Bw, net->d_logp_stage, nullptr, nullptr, st);
    if (s != TD_OK) return s;
    e = cudaMemcpyAsync(logp_host + w0 * 2, net->d_logp_stage, (size_t)Bw * 2 * sizeof(double),
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
  }
  return td_network_check(net, stream);
}

td_status td_network_check(td_network* net, void* stream) {
  if (!net) return fail(TD_ERR_INVALID, "null network");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  int code = 0;
  if ((e = cudaMemcpy(&code, net->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "status read");
  if (code == TD_OK) return TD_OK;
  if ((e = cudaMemset(net->d_status, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "status reset");
  return fail((td_status)code,
              code == TD_ERR_TIMEOUT ? "a tensor-core kernel gave up waiting for its MMAs; the results of the calls "
                                       "since the last check are not valid"
              : code == TD_ERR_NUMERIC ? "a shot met a non-finite intermediate; its log-probabilities are NaN"
                                       : "a kernel recorded an error status");
}

td_status td_coset_logprob_static(td_network* net, const uint8_t* det_dev, int64_t B, double* logp_dev,
                                  void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_dev, B);
  if (s != TD_OK) return s;
  if (B > 0 && !logp_dev) return fail(TD_ERR_INVALID, "null output buffer");
  const size_t per_shot = (size_t)net->fin.scratch_elems * net->felem;
  const int64_t cap = (int64_t)std::min<size_t>(td::kStaticFinalScratchBytes / std::max<size_t>(per_shot, 1),
                                                (size_t)net->wave);
  if (B > cap)
    return fail(TD_ERR_INVALID, "B = " + std::to_string(B) + " exceeds the static scratch capacity of this network: " +
                                    std::to_string(cap) + " shots (" + std::to_string(per_shot) +
                                    " bytes of final-contraction scratch per shot in a " +
                                    std::to_string(td::kStaticFinalScratchBytes >> 20) + " MiB array)");
  if (B == 0) return TD_OK;
  void* scr = nullptr;
  cudaError_t e = td::static_final_scratch(&scr);
  if (e != cudaSuccess) return cuda_fail(e, "static scratch lookup");
  // kernel timing (td_network_profile) creates CUDA events on demand: this call records
  // none, so that it stays free of every allocation
  const bool prof = net->profiling;
  net->profiling = false;
  s = run(net, det_dev, B, logp_dev, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream), scr);
  net->profiling = prof;
  return s;
}

// ---- gradient pass ----------------------------------------------------------------------
// The parameter objects of a plan that depend on the rates: site-local K, gate p, readout R.
static int differing_object(const td::Plan& A, const td::Plan& B, td::Override& o) {
  int found = 0;
  for (size_t i = 0; i < A.locals.size(); ++i)
    if (std::memcmp(A.locals[i].K, B.locals[i].K, sizeof(A.locals[i].K)) != 0) {
      o.kind = td::kOvrLocal;
      o.target = (int32_t)i;   // layer * S + site (locals are emitted layer by layer)
      std::memset(o.val, 0, sizeof(o.val));
      std::memcpy(o.val, B.locals[i].K, sizeof(B.locals[i].K));
      ++found;
    }
  for (size_t i = 0; i < A.gates.size(); ++i)
    if (A.gates[i].p != B.gates[i].p) {
      o.kind = td::kOvrGate;
      o.target = (int32_t)i;
      std::memset(o.val, 0, sizeof(o.val));
      o.val[0] = B.gates[i].p;
      ++found;
    }
  for (size_t i = 0; i < A.finals.size(); ++i)
    if (std::memcmp(A.finals[i].R, B.finals[i].R, sizeof(A.finals[i].R)) != 0) {
      o.kind = td::kOvrRead;
      o.target = (int32_t)i;
      std::memset(o.val, 0, sizeof(o.val));
      std::memcpy(o.val, B.finals[i].R, sizeof(B.finals[i].R));
      ++found;
    }
  return found;
}

static bool same_structure(const td::Plan& A, const td::Plan& B) {
  return A.locals.size() == B.locals.size() && A.gates.size() == B.gates.size() &&
         A.finals.size() == B.finals.size() && A.shot_elems == B.shot_elems && A.n_bonds == B.n_bonds;
}

// Sets the network's rates to `rates` (parameter objects rebuilt and uploaded) and builds
// the override table of every mechanism forced to 0 and to 1.
static td_status prepare_overrides(td_network* net, const std::vector<double>& rates, cudaStream_t st) {
  if (!net->ovr_rates.empty() && net->ovr_rates == rates) return TD_OK;
  std::string err;
  td::Plan& P = net->plan;
  const td_layout lay = net->layout_view();
  if (rates != net->rates) {
    td::Plan Q;
    const td_dem d = net->dem_view(rates.data());
    td_status s = td::build_plan(d, lay, net->opt, Q, err);
    if (s != TD_OK) return fail(s, "rates: " + err);
    if (!same_structure(P, Q)) return fail(TD_ERR_INVALID, "rates change the network's structure");
    for (size_t i = 0; i < P.locals.size(); ++i) std::memcpy(P.locals[i].K, Q.locals[i].K, sizeof(P.locals[i].K));
    for (size_t i = 0; i < P.gates.size(); ++i) P.gates[i].p = Q.gates[i].p;
    for (size_t i = 0; i < P.finals.size(); ++i) std::memcpy(P.finals[i].R, Q.finals[i].R, sizeof(P.finals[i].R));
    std::memcpy(P.glob_mix, Q.glob_mix, sizeof(P.glob_mix));
    cudaError_t e;
    if ((!P.gates.empty() && (e = cudaMemcpyAsync(net->d_gates, P.gates.data(), sizeof(td::GateDesc) * P.gates.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(net->d_locals, P.locals.data(), sizeof(td::LocalDesc) * P.locals.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(net->d_finals, P.finals.data(), sizeof(td::FinalSite) * P.finals.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail(e, "descriptor upload");
    net->rates = rates;
  }
  const int32_t n_mech = P.n_mech;
  net->ovr_host.assign(1, td::Override{});
  net->ovr_host[0].kind = td::kOvrNone;
  net->ovr_of.assign(2 * (size_t)n_mech, 0);
  std::vector<double> r = rates;
  for (int32_t j = 0; j < n_mech; ++j) {
    for (int x = 0; x < 2; ++x) {
      r[j] = (double)x;
      td::Plan Q;
      const td_dem d = net->dem_view(r.data());
      td_status s = td::build_plan(d, lay, net->opt, Q, err);
      if (s != TD_OK) return fail(s, "forced rate: " + err);
      if (!same_structure(P, Q)) return fail(TD_ERR_INVALID, "forcing a rate changes the network's structure");
      td::Override o{};
      const int nd = differing_object(P, Q, o);
      if (nd > 1) return fail(TD_ERR_INVALID, "a mechanism rate enters more than one parameter object");
      if (nd == 1) {
        net->ovr_of[2 * (size_t)j + x] = (int32_t)net->ovr_host.size();
        net->ovr_host.push_back(o);
      }
    }
    r[j] = rates[j];
  }
  if (!net->reserve(net->d_ovr, net->d_ovr_cap, net->ovr_host.size())) return fail(TD_ERR_OOM, "override table");
  cudaError_t e = cudaMemcpyAsync(net->d_ovr, net->ovr_host.data(), sizeof(td::Override) * net->ovr_host.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "override upload");
  net->ovr_rates = rates;
  return TD_OK;
}

td_status td_grad_logprob_forced(td_network* net, const uint8_t* det_dev, int64_t B, const double* p_dev,
                                 double* logP_dev, double* grad_dev, void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_dev, B);
  if (s != TD_OK) return s;
  if (!grad_dev || (B > 0 && !logP_dev)) return fail(TD_ERR_INVALID, "null output buffer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int32_t n_mech = net->plan.n_mech;
  std::vector<double> rates = net->rates;
  cudaError_t e;
  if (p_dev) {
    e = cudaMemcpyAsync(rates.data(), p_dev, sizeof(double) * n_mech, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "rate copy");
    for (int32_t j = 0; j < n_mech; ++j)
      if (!(rates[j] >= 0.0 && rates[j] <= 1.0)) return fail(TD_ERR_INVALID, "rate outside [0, 1]");
  }
  // the override table is built on the host; no kernel of an earlier call may still read it
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  s = prepare_overrides(net, rates, st);
  if (s != TD_OK) return s;
  // forced mechanisms, in order; virtual shots b * NV + (0 | 1 + 2a + x)
  std::vector<int32_t> act(n_mech, -1);
  std::vector<int32_t> forced;
  for (int32_t j = 0; j < n_mech; ++j)
    if (net->ovr_of[2 * (size_t)j] || net->ovr_of[2 * (size_t)j + 1]) {
      act[j] = (int32_t)forced.size();
      forced.push_back(j);
    }
  const int32_t NV = 1 + 2 * (int32_t)forced.size();
  const int64_t Bv = B * NV;
  if (Bv > ((int64_t)1 << 31) - 1) return fail(TD_ERR_INVALID, "B * (1 + 2 * forced mechanisms) exceeds 2^31 - 1");
  if (!net->reserve(net->d_act, net->d_act_cap, (size_t)n_mech) ||
      !net->reserve(net->d_vs, net->d_vs_cap, (size_t)Bv) ||
      !net->reserve(net->d_vlogp, net->d_vlogp_cap, (size_t)Bv * 2))
    return fail(TD_ERR_OOM, "gradient pass buffers");
  std::vector<td::VShot> vs((size_t)Bv);
  for (int64_t b = 0; b < B; ++b) {
    td::VShot* v = &vs[(size_t)(b * NV)];
    v[0].base = (int32_t)b;
    v[0].ovr = 0;
    for (size_t a = 0; a < forced.size(); ++a)
      for (int x = 0; x < 2; ++x) {
        v[1 + 2 * a + x].base = (int32_t)b;
        v[1 + 2 * a + x].ovr = net->ovr_of[2 * (size_t)forced[a] + x];
      }
  }
  // pageable sources: each asynchronous copy has staged its source when it returns
  if (n_mech > 0 && (e = cudaMemcpyAsync(net->d_act, act.data(), sizeof(int32_t) * n_mech, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "gradient map upload");
  if (Bv > 0 && (e = cudaMemcpyAsync(net->d_vs, vs.data(), sizeof(td::VShot) * (size_t)Bv, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "virtual shot upload");
  if (Bv > 0) {
    s = run(net, det_dev, Bv, net->d_vlogp, nullptr, nullptr, st, nullptr, net->d_vs, net->d_ovr);
    if (s != TD_OK) return s;
  }
  e = td::launch_grad_combine(net->d_vlogp, B, NV, net->d_act, n_mech, logP_dev, grad_dev, st);
  if (e != cudaSuccess) return cuda_fail(e, "gradient combine launch");
  return TD_OK;
}

// ---- reverse sweep ----------------------------------------------------------------------
// Buffers and layouts of the reverse sweep for waves of up to net->grad_wave shots.
static td_status prepare_reverse(td_network* net, int64_t B) {
  td::Plan& P = net->plan;
  const int chi = P.chi, cm = P.chi_mps, Dm = P.max_final_D, cmx = std::max(cm, 2);
  const int64_t max_site = (P.max_site_elems + 3) / 4 * 4;
  const int64_t mA = net->fin.mps_stride;
  const int64_t mC = (int64_t)cm * cmx * Dm * 2;
  const int m_max = cm * Dm, n_max = cmx * Dm * 2;
  const td::FinRecSlot ly((int)mC, (int)mA, m_max, n_max);
  const int64_t fin_slot = (ly.size + 3) / 4 * 4;
  const int64_t fin_stride = fin_slot * P.nx * P.ny;
  const int64_t core_rec = td::core_rec_elems(chi);
  // adjoint scratch per shot
  int64_t acc = 0;
  auto take = [&](int64_t n) { int64_t r = acc; acc += (n + 3) / 4 * 4; return r; };
  td::AdjArgs& A = net->adj;
  A = td::AdjArgs{};
  A.max_site = max_site;
  A.o_gbar = take(max_site * P.S);
  A.o_xbar = take(3 * max_site);   // two sides' X-bar, then per-(row, column) partial sums
  A.o_r = take(max_site);
  A.o_lambar = take((int64_t)P.n_bonds * chi);
  A.o_core = take(td::CoreScr_elems(chi, max_site));
  const int64_t mF = 2LL * Dm * Dm * Dm * Dm, mT1 = (int64_t)Dm * 2 * Dm * cmx * cm, mMN = (int64_t)m_max * n_max;
  A.fo_F = take(mF); A.fo_Fb = take(mF);
  A.fo_T1 = take(mT1); A.fo_T1b = take(mT1);
  A.fo_M = take(mMN); A.fo_Mb = take(mMN);
  A.fo_C0 = take(mMN); A.fo_C1 = take(mMN);
  A.fo_A0 = take(mA * P.nx); A.fo_A1 = take(mA * P.nx);
  A.fo_Ub = take((int64_t)m_max * cm); A.fo_W = take((int64_t)m_max * m_max); A.fo_J = take((int64_t)m_max * cm);
  A.fo_In = take((int64_t)m_max * m_max); A.fo_wg = take(mF / 2); A.fo_off = take(mF / 4 + 1);
  A.scr_stride = acc;
  // FP64 final contraction of the recorded forward: work region in global scratch
  td::FinalArgs& G = net->gfin;
  G = net->fin;
  G.use_smem = 0;
  G.precond = 0;
  G.off_work = (net->fin.off_mps1 + mA * P.nx + 3) / 4 * 4;
  G.scratch_elems = G.off_work + net->fin.work_elems;
  G.rec_stride = fin_stride; G.rec_slot = fin_slot;
  G.rec_mC = (int32_t)mC; G.rec_mA = (int32_t)mA; G.rec_m = m_max; G.rec_n = n_max;
  const int64_t n_gates = (int64_t)P.gates.size();
  const int32_t nseg = (int32_t)P.seg_first_layer.size() - 1;
  int64_t seg_gates = 1;
  for (int32_t j = 0; j < nseg; ++j) seg_gates = std::max<int64_t>(seg_gates, P.seg_first_gate[j + 1] - P.seg_first_gate[j]);
  const int64_t seg_layers = P.ckpt_stride;
  const size_t per_shot = 8 * (size_t)(P.hist_shot_elems + P.ckpt_shot_elems + seg_gates * core_rec + seg_layers * P.S +
                                       fin_stride + A.scr_stride + G.scratch_elems + (int64_t)P.T * P.S * 16 + n_gates +
                                       P.S * 8 + 2);
  const size_t budget = net->opt.mem_budget ? net->opt.mem_budget : (size_t(16) << 30);
  int64_t gw = std::min<int64_t>({(int64_t)net->wave, std::max<int64_t>(B, 1),
                                   std::max<int64_t>(1, (int64_t)(budget / std::max<size_t>(per_shot, 1)))});
  // smaller calls reuse the buffers, unless the final contraction's layout (set by the
  // launch schedule) needs more scratch than was allocated
  if (net->d_hist && gw <= net->grad_wave && G.scratch_elems <= net->gfscr_elems) return TD_OK;
  gw = std::max<int64_t>(gw, net->grad_wave);
  for (double** pp : {&net->d_hist, &net->d_rec_core, &net->d_rec_sc, &net->d_rec_fin, &net->d_adj_scr, &net->d_gfscr,
                      &net->d_Kbar, &net->d_pbar, &net->d_Rbar, &net->d_glogp, &net->d_ckpt})
    if (*pp) {
      cudaFree(*pp);
      net->allocs.erase(std::remove(net->allocs.begin(), net->allocs.end(), (void*)*pp), net->allocs.end());
      *pp = nullptr;
    }
  net->grad_wave = 0;
  auto res = [&](double*& ptr, int64_t n) { size_t c = 0; return net->reserve(ptr, c, (size_t)n); };
  if (!res(net->d_hist, gw * P.hist_shot_elems) || !res(net->d_rec_core, seg_gates * gw * core_rec) ||
      !res(net->d_ckpt, std::max<int64_t>(gw * P.ckpt_shot_elems, 1)) ||
      !res(net->d_rec_sc, seg_layers * gw * P.S) || !res(net->d_rec_fin, gw * fin_stride) ||
      !res(net->d_adj_scr, gw * A.scr_stride) || !res(net->d_gfscr, gw * G.scratch_elems) ||
      !res(net->d_Kbar, gw * P.T * P.S * 16) || !res(net->d_pbar, gw * std::max<int64_t>(n_gates, 1)) ||
      !res(net->d_Rbar, gw * P.S * 8) || !res(net->d_glogp, gw * 2))
    return fail(TD_ERR_OOM, "reverse-sweep buffers");
  if (!net->d_hgates) {
    std::vector<int32_t> rf, lr;
    int32_t nr = 0;
    for (const td::LayerPlan& L : P.layers) {
      lr.push_back(nr);
      for (const td::Round& R : L.rounds) { rf.push_back(R.first); ++nr; }
    }
    lr.push_back(nr);
    rf.push_back((int32_t)P.gates.size());
    size_t c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0, c6 = 0, c7 = 0, c8 = 0, c9 = 0;
    const size_t nst = P.seg_in_off.size();
    if (!net->reserve(net->d_hgates, c1, std::max<size_t>(P.hist_gates.size(), 1)) ||
        !net->reserve(net->d_hlocals, c2, P.hist_locals.size()) || !net->reserve(net->d_hfinals, c3, P.hist_finals.size()) ||
        !net->reserve(net->d_round_first, c4, rf.size()) || !net->reserve(net->d_layer_round, c5, lr.size()) ||
        !net->reserve(net->d_seg_in_off, c6, nst) || !net->reserve(net->d_seg_out_off, c7, nst) ||
        !net->reserve(net->d_seg_len, c8, nst) || !net->reserve(net->d_ckpt_off, c9, nst))
      return fail(TD_ERR_OOM, "reverse-sweep descriptors");
    cudaError_t e;
    if ((e = cudaMemcpy(net->d_seg_in_off, P.seg_in_off.data(), 8 * nst, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(net->d_seg_out_off, P.seg_out_off.data(), 8 * nst, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(net->d_seg_len, P.seg_in_elems.data(), 8 * nst, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(net->d_ckpt_off, P.ckpt_off.data(), 8 * nst, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "reverse-sweep segment tables");
    if ((!P.hist_gates.empty() && (e = cudaMemcpy(net->d_hgates, P.hist_gates.data(), sizeof(td::GateDesc) * P.hist_gates.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(net->d_hlocals, P.hist_locals.data(), sizeof(td::LocalDesc) * P.hist_locals.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(net->d_hfinals, P.hist_finals.data(), sizeof(td::FinalSite) * P.hist_finals.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(net->d_round_first, rf.data(), sizeof(int32_t) * rf.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(net->d_layer_round, lr.data(), sizeof(int32_t) * lr.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess)
      return cuda_fail(e, "reverse-sweep descriptor upload");
  }
  net->grad_wave = (int32_t)gw;
  net->gfscr_elems = G.scratch_elems;
  return TD_OK;
}

// The versioned descriptors carry the rates of the build; after a change of rates they are
// refreshed from the plan (same structure, new K, p and R).
static td_status refresh_hist_params(td_network* net, cudaStream_t st) {
  td::Plan& P = net->plan;
  for (size_t i = 0; i < P.hist_locals.size(); ++i) std::memcpy(P.hist_locals[i].K, P.locals[i].K, sizeof(P.locals[i].K));
  for (size_t i = 0; i < P.hist_gates.size(); ++i) P.hist_gates[i].p = P.gates[i].p;
  for (size_t i = 0; i < P.hist_finals.size(); ++i) std::memcpy(P.hist_finals[i].R, P.finals[i].R, sizeof(P.finals[i].R));
  cudaError_t e;
  if ((!P.hist_gates.empty() && (e = cudaMemcpyAsync(net->d_hgates, P.hist_gates.data(), sizeof(td::GateDesc) * P.hist_gates.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) ||
      (e = cudaMemcpyAsync(net->d_hlocals, P.hist_locals.data(), sizeof(td::LocalDesc) * P.hist_locals.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(net->d_hfinals, P.hist_finals.data(), sizeof(td::FinalSite) * P.hist_finals.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "reverse-sweep descriptor upload");
  return TD_OK;
}

td_status td_grad_logprob(td_network* net, const uint8_t* det_dev, int64_t B, const double* p_dev, double* logP_dev,
                          double* grad_dev, void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_dev, B);
  if (s != TD_OK) return s;
  if (!grad_dev || (B > 0 && !logP_dev)) return fail(TD_ERR_INVALID, "null output buffer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  td::Plan& P = net->plan;
  const int32_t n_mech = P.n_mech, S = P.S, T = P.T, chi = P.chi;
  const int64_t n_gates = (int64_t)P.gates.size();
  std::vector<double> rates = net->rates;
  cudaError_t e;
  if (p_dev) {
    e = cudaMemcpyAsync(rates.data(), p_dev, sizeof(double) * n_mech, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "rate copy");
    for (int32_t j = 0; j < n_mech; ++j)
      if (!(rates[j] >= 0.0 && rates[j] <= 1.0)) return fail(TD_ERR_INVALID, "rate outside [0, 1]");
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  s = prepare_overrides(net, rates, st);   // objects at the rates and at every forced rate
  if (s != TD_OK) return s;
  s = prepare_reverse(net, B);
  if (s != TD_OK) return s;
  s = refresh_hist_params(net, st);
  if (s != TD_OK) return s;
  std::vector<double> Ksum((size_t)T * S * 16, 0.0), psum((size_t)n_gates, 0.0), Rsum((size_t)S * 8, 0.0);
  std::vector<double> hK, hp, hR;
  const int64_t gw = net->grad_wave;
  const int32_t nseg = (int32_t)P.seg_first_layer.size() - 1;
  for (int64_t w0 = 0; w0 < B; w0 += gw) {
    const int32_t Bw = (int32_t)std::min<int64_t>(gw, B - w0);
    td::SweepArgs a{};
    a.gamma = net->d_hist;
    a.shot_elems = P.hist_shot_elems;
    a.lam = net->d_lam;
    a.logacc = net->d_logacc;
    a.det = det_dev;
    a.nbonds = P.n_bonds; a.chi = chi; a.nslots = net->nslots; a.n_det = P.n_det;
    a.wave_first = (int32_t)w0;
    a.B = Bw;
    a.gram_cutoff = P.gram_cutoff; a.svd_cutoff = P.svd_cutoff; a.multiplet_rtol = P.multiplet_rtol;
    a.rec_core = net->d_rec_core;
    a.chunk_rows = net->chunk_rows;
    a.status = net->d_status;
    const int64_t lam_elems = (int64_t)P.n_bonds * chi, lam_stride = lam_elems;
    // forward sweep of segment j in the versioned layout, recording its cores and scales;
    // a segment j >= 1 starts from its checkpoint (tensors and bond weights), segment 0
    // from the product state
    auto forward_segment = [&](int32_t j) -> td_status {
      cudaError_t e2;
      if (j == 0) {
        if ((e2 = td::launch_sweep_init<double, double>(a, net->d_hlocals, S, st)) != cudaSuccess)
          return cuda_fail(e2, "init launch");
      } else {
        if ((e2 = td::launch_copy_sites(net->d_ckpt, P.ckpt_shot_elems, net->d_ckpt_off + (size_t)j * S, net->d_hist,
                                        P.hist_shot_elems, net->d_seg_in_off + (size_t)j * S,
                                        net->d_seg_len + (size_t)j * S, S, Bw, st)) != cudaSuccess ||
            (e2 = td::launch_copy_rows(net->d_ckpt, P.ckpt_shot_elems, P.ckpt_lam_off[j], net->d_lam, lam_stride, 0,
                                       lam_elems, Bw, st)) != cudaSuccess)
          return cuda_fail(e2, "checkpoint restore");
      }
      const int32_t t0 = P.seg_first_layer[j], t1 = P.seg_first_layer[j + 1];
      a.rec_gate0 = P.seg_first_gate[j];
      for (int32_t t = t0; t < t1; ++t) {
        a.layer = t;
        a.rec_sc = net->d_rec_sc + (int64_t)(t - t0) * Bw * S;
        if ((e2 = td::launch_local<double, double>(a, net->d_hlocals + (int64_t)t * S, S, st)) != cudaSuccess)
          return cuda_fail(e2, "local launch");
        for (const td::Round& rd : P.layers[t].rounds)
          if ((e2 = td::launch_round<double, double>(a, net->d_hgates, rd, net->d_gram, net->d_tbuf, S, st)) != cudaSuccess)
            return cuda_fail(e2, "gate round launch");
      }
      return TD_OK;
    };
    cudaError_t e;
    for (int32_t j = 0; j < nseg; ++j) {
      if (j > 0) {
        // checkpoint: the previous segment's output tensors and the bond weights
        if ((e = td::launch_copy_sites(net->d_hist, P.hist_shot_elems, net->d_seg_out_off + (size_t)(j - 1) * S,
                                       net->d_ckpt, P.ckpt_shot_elems, net->d_ckpt_off + (size_t)j * S,
                                       net->d_seg_len + (size_t)j * S, S, Bw, st)) != cudaSuccess ||
            (e = td::launch_copy_rows(net->d_lam, lam_stride, 0, net->d_ckpt, P.ckpt_shot_elems, P.ckpt_lam_off[j],
                                      lam_elems, Bw, st)) != cudaSuccess)
          return cuda_fail(e, "checkpoint save");
      }
      s = forward_segment(j);
      if (s != TD_OK) return s;
    }
    td::FinalArgs f = net->gfin;
    f.gamma = net->d_hist; f.shot_elems = P.hist_shot_elems; f.lam = net->d_lam; f.logacc = net->d_logacc;
    f.sites = net->d_hfinals; f.grid_site = net->d_grid; f.scratch = net->d_gfscr; f.Z = net->d_Z;
    f.nbonds = P.n_bonds; f.chi = chi; f.nslots = net->nslots; f.slot = S + P.n_bonds;
    f.nx = P.nx; f.ny = P.ny; f.chi_mps = P.chi_mps; f.B = Bw;
    f.svd_cutoff = P.svd_cutoff; f.multiplet_rtol = P.multiplet_rtol;
    f.rec = net->d_rec_fin;
    if ((e = td::launch_final<double, double>(f, st)) != cudaSuccess) return cuda_fail(e, "final launch");
    td::FinalizeArgs z{};
    z.Z = net->d_Z; z.logacc = net->d_logacc; z.det = det_dev + w0 * P.n_det; z.logp = net->d_glogp;
    z.nslots = net->nslots; z.n_det = P.n_det; z.wave_first = 0; z.B = Bw; z.offset_all = P.offset_all;
    for (int i = 0; i < 4; ++i) z.mix[i] = P.glob_mix[i];
    if ((e = td::launch_finalize(z, st)) != cudaSuccess) return cuda_fail(e, "finalize launch");
    if ((e = td::launch_grad_combine(net->d_glogp, Bw, 1, nullptr, 0, logP_dev + w0, nullptr, st)) != cudaSuccess)
      return cuda_fail(e, "log P launch");
    td::AdjArgs A = net->adj;
    A.hist = net->d_hist; A.hist_elems = P.hist_shot_elems; A.lam = net->d_lam; A.Z = net->d_Z;
    A.rec_core = net->d_rec_core; A.rec_sc = net->d_rec_sc; A.rec_fin = net->d_rec_fin;
    A.fin_stride = f.rec_stride; A.fin_slot = f.rec_slot;
    A.fin_mC = f.rec_mC; A.fin_mA = f.rec_mA; A.fin_m = f.rec_m; A.fin_n = f.rec_n;
    A.gates = net->d_hgates; A.locals = net->d_hlocals; A.finals = net->d_hfinals; A.grid_site = net->d_grid;
    A.round_first = net->d_round_first; A.layer_round = net->d_layer_round;
    A.det = det_dev; A.n_det = P.n_det; A.wave_first = (int32_t)w0;
    A.scratch = net->d_adj_scr;
    A.S = S; A.T = T; A.nbonds = P.n_bonds; A.chi = chi; A.nx = P.nx; A.ny = P.ny; A.B = Bw;
    A.n_gates = (int32_t)n_gates; A.max_final_D = P.max_final_D; A.mps_stride = (int32_t)net->fin.mps_stride;
    A.Kbar = net->d_Kbar; A.pbar = net->d_pbar; A.Rbar = net->d_Rbar;
    // reverse sweep, one segment at a time from the last: the last segment's record is in
    // place; every earlier one is recomputed from its checkpoint first
    for (int32_t j = nseg - 1; j >= 0; --j) {
      if (j < nseg - 1) {
        s = forward_segment(j);
        if (s != TD_OK) return s;
      }
      A.t_begin = P.seg_first_layer[j];
      A.t_end = P.seg_first_layer[j + 1];
      A.rec_gate0 = P.seg_first_gate[j];
      A.do_final = (j == nseg - 1) ? 1 : 0;
      if ((e = td::launch_adjoint(A, 256, st)) != cudaSuccess) return cuda_fail(e, "adjoint launch");
    }
    hK.resize((size_t)Bw * T * S * 16); hp.resize((size_t)Bw * n_gates); hR.resize((size_t)Bw * S * 8);
    if ((e = cudaMemcpyAsync(hK.data(), net->d_Kbar, sizeof(double) * hK.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (n_gates > 0 && (e = cudaMemcpyAsync(hp.data(), net->d_pbar, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(hR.data(), net->d_Rbar, sizeof(double) * hR.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail(e, "adjoint copy");
    for (int32_t b = 0; b < Bw; ++b) {
      for (size_t i = 0; i < Ksum.size(); ++i) Ksum[i] += hK[(size_t)b * Ksum.size() + i];
      for (size_t i = 0; i < psum.size(); ++i) psum[i] += hp[(size_t)b * psum.size() + i];
      for (size_t i = 0; i < Rsum.size(); ++i) Rsum[i] += hR[(size_t)b * Rsum.size() + i];
    }
  }
  // rates: d mean log P / d p_j = sum over objects of object-bar . (object(p_j=1) - object(p_j=0)) / B
  std::vector<double> grad(n_mech, 0.0);
  for (int32_t j = 0; j < n_mech && B > 0; ++j) {
    const int32_t o0 = net->ovr_of[2 * (size_t)j], o1 = net->ovr_of[2 * (size_t)j + 1];
    if (!o0 && !o1) continue;
    const td::Override& ref = net->ovr_host[o1 ? o1 : o0];
    double acc = 0.0;
    if (ref.kind == td::kOvrLocal) {
      const double* base = P.locals[ref.target].K;
      const double* v1 = o1 ? net->ovr_host[o1].val : base;
      const double* v0 = o0 ? net->ovr_host[o0].val : base;
      for (int e2 = 0; e2 < 16; ++e2) acc += Ksum[(size_t)ref.target * 16 + e2] * (v1[e2] - v0[e2]);
    } else if (ref.kind == td::kOvrGate) {
      const double base = P.gates[ref.target].p;
      const double v1 = o1 ? net->ovr_host[o1].val[0] : base, v0 = o0 ? net->ovr_host[o0].val[0] : base;
      acc = psum[ref.target] * (v1 - v0);
    } else if (ref.kind == td::kOvrRead) {
      const double* base = P.finals[ref.target].R;
      const double* v1 = o1 ? net->ovr_host[o1].val : base;
      const double* v0 = o0 ? net->ovr_host[o0].val : base;
      for (int e2 = 0; e2 < 8; ++e2) acc += Rsum[(size_t)ref.target * 8 + e2] * (v1[e2] - v0[e2]);
    }
    grad[j] = acc / (double)B;
  }
  if (n_mech > 0) {
    e = cudaMemcpyAsync(grad_dev, grad.data(), sizeof(double) * n_mech, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "gradient copy");
  }
  return TD_OK;
}

// ---- schedule -------------------------------------------------------------------------------
td_status td_network_set_schedule(td_network* net, int32_t final_threads, int32_t final_smem, int32_t chunk_rows) {
  g_err.clear();
  if (!net) return fail(TD_ERR_INVALID, "null network");
  bool ok_t = false, ok_c = false;
  for (int th : kFinalThreads) ok_t |= (th == final_threads);
  for (int c : kChunkCandidates) ok_c |= (c == chunk_rows);
  if (!ok_t) return fail(TD_ERR_INVALID, "final_threads must be 256, 512 or 1024");
  if (!ok_c) return fail(TD_ERR_INVALID, "chunk_rows must be 512, 1024, 2048 or 4096");
  final_layout(net, final_threads, final_smem != 0);
  net->chunk_rows = chunk_rows;
  return TD_OK;
}

td_status td_network_tune(td_network* net, const uint8_t* det_dev, int64_t B, int32_t* final_threads,
                          int32_t* final_smem, int32_t* chunk_rows, double* ms_best, void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_dev, B);
  if (s != TD_OK) return s;
  if (B < 1) return fail(TD_ERR_INVALID, "tuning needs at least one shot");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t Bs = std::min<int64_t>(B, net->wave);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "event create");
  }
  auto time_one = [&](float& ms) -> td_status {
    td_status r = run(net, det_dev, Bs, net->d_logp_stage, nullptr, nullptr, st);   // warm-up
    if (r != TD_OK) return r;
    cudaEventRecord(e0, st);
    r = run(net, det_dev, Bs, net->d_logp_stage, nullptr, nullptr, st);
    if (r != TD_OK) return r;
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    return e == cudaSuccess ? TD_OK : cuda_fail(e, "tuning timing");
  };
  // coordinate descent: the final contraction's block size and work-region placement at the
  // current chunk size, then the chunk size at the best of those
  int best_t = net->fin.threads, best_sm = 1, best_c = net->chunk_rows;
  final_layout(net, best_t, true);
  float best = 0.0f;
  s = time_one(best);
  for (int th : kFinalThreads)
    for (int sm = 1; sm >= 0; --sm) {
      if (s != TD_OK) break;
      if (th == best_t && sm == 1) continue;
      final_layout(net, th, sm == 1);
      float ms = 0.0f;
      s = time_one(ms);
      if (s == TD_OK && ms < best) { best = ms; best_t = th; best_sm = sm; }
    }
  final_layout(net, best_t, best_sm == 1);
  for (int c : kChunkCandidates) {
    if (s != TD_OK) break;
    if (c == best_c) continue;
    net->chunk_rows = c;
    float ms = 0.0f;
    s = time_one(ms);
    if (s == TD_OK && ms < best) { best = ms; best_c = c; }
  }
  net->chunk_rows = best_c;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != TD_OK) return s;
  if (final_threads) *final_threads = best_t;
  if (final_smem) *final_smem = net->fin.use_smem;
  if (chunk_rows) *chunk_rows = best_c;
  if (ms_best) *ms_best = best;
  return TD_OK;
}

td_status td_debug_sweep(td_network* net, const uint8_t* det_dev, int64_t B, int32_t n_gates, double* lam_dev,
                         double* logacc_dev, int32_t* applied, void* stream) {
  g_err.clear();
  td_status s = check_call(net, det_dev, B);
  if (s != TD_OK) return s;
  if (!lam_dev || !applied) return fail(TD_ERR_INVALID, "null output");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  td::Plan& P = net->plan;
  const int32_t Bw = (int32_t)std::min<int64_t>(net->wave, B);
  td::SweepArgs a{};
  a.gamma = net->d_gamma; a.shot_elems = P.shot_elems; a.lam = net->d_lam; a.logacc = net->d_logacc;
  a.det = det_dev; a.nbonds = P.n_bonds; a.chi = P.chi; a.nslots = net->nslots; a.n_det = P.n_det;
  a.wave_first = 0; a.B = Bw;
  a.gram_cutoff = P.gram_cutoff; a.svd_cutoff = P.svd_cutoff; a.multiplet_rtol = P.multiplet_rtol;
  a.tc = P.precision == TD_FP64 ? 0 : 1;
  a.precond = P.precision == TD_FP64 ? 0 : 1;
  a.status = net->d_status;
  const bool f64 = P.precision != TD_FP32;   // storage type
  cudaError_t e = f64 ? td::launch_sweep_init<double, double>(a, net->d_locals, P.S, st)
                      : td::launch_sweep_init<float, float>(a, net->d_locals, P.S, st);
  if (e != cudaSuccess) return cuda_fail(e, "init launch");
  int32_t done = 0;
  for (int32_t t = 0; t < P.T && done < n_gates; ++t) {
    const td::LayerPlan& L = P.layers[t];
    e = f64 ? td::launch_local<double, double>(a, net->d_locals + L.local_first, P.S, st)
            : td::launch_local<float, float>(a, net->d_locals + L.local_first, P.S, st);
    if (e != cudaSuccess) return cuda_fail(e, "local launch");
    for (const td::Round& rd : L.rounds) {
      if (done >= n_gates) break;
      e = f64 ? td::launch_round<double, double>(a, net->d_gates, rd, net->d_gram, net->d_tbuf, P.S, st)
              : td::launch_round<float, float>(a, net->d_gates, rd, net->d_gram, net->d_tbuf, P.S, st);
      if (e != cudaSuccess) return cuda_fail(e, "gate round launch");
      done += rd.count;
    }
  }
  e = cudaMemcpyAsync(lam_dev, net->d_lam, sizeof(double) * Bw * P.n_bonds * P.chi, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && logacc_dev)
    e = cudaMemcpyAsync(logacc_dev, net->d_logacc, sizeof(double) * Bw * net->nslots, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "debug copy");
  *applied = done;
  return TD_OK;
}

td_status td_network_get_info(const td_network* net, td_network_info* info) {
  if (!net || !info) return fail(TD_ERR_INVALID, "null argument");
  const td::Plan& P = net->plan;
  info->n_sites = P.S;
  info->n_layers = P.T;
  info->n_bonds = P.n_bonds;
  info->n_gates = (int32_t)P.gates.size();
  info->n_counter_sites = P.n_counter_sites;
  info->nx = P.nx;
  info->ny = P.ny;
  info->wave = net->wave;
  info->chi = P.chi;
  info->chi_mps = P.chi_mps;
  info->precision = P.precision;
  info->offset_all = P.offset_all;
  info->generator = P.gen;
  info->workspace_bytes = net->bytes;
  info->launches_per_wave = net->launches_per_wave;
  return TD_OK;
}

td_status td_network_get_work(const td_network* net, double* bytes, double* flops, double* fp64_flops) {
  g_err.clear();
  if (!net || !bytes || !flops || !fp64_flops) return fail(TD_ERR_INVALID, "null argument");
  const td::Plan& P = net->plan;
  const double el = (double)net->elem;
  const bool f64 = P.precision == TD_FP64;   // the update in FP64 arithmetic on FP64 storage only counts as FP64 work
  for (int k = 0; k < TD_K_COUNT; ++k) { bytes[k] = 0; flops[k] = 0; fp64_flops[k] = 0; }
  auto eig = [](double n) { return 9.0 * n * n * n; };
  auto svd = [](double m, double n) {
    if (m < n) std::swap(m, n);
    return 4.0 * m * m * n + 8.0 * m * n * n + 9.0 * n * n * n;
  };
  // singular values and left singular vectors of an m x n matrix (a zip-up cut keeps left
  // vectors only): R-SVD counts, Sigma and U1 (6 m n^2 + 11 n^3) for m >= n, Sigma and the
  // square left factor through a QR of the transpose (2 n m^2 + 11 m^3) for m < n
  auto svd_left = [](double m, double n) {
    return m >= n ? 6.0 * m * n * n + 11.0 * n * n * n : 2.0 * n * m * m + 11.0 * m * m * m;
  };
  bytes[TD_K_INIT] = 0;
  for (const td::LocalDesc& d : P.locals) {
    bytes[TD_K_LOCAL] += 2.0 * d.P * d.rest * el;
    flops[TD_K_LOCAL] += 2.0 * d.P * d.P * d.rest;
  }
  for (const td::GateDesc& g : P.gates) {
    const double D = g.D, Dn = g.Dn;
    for (int sd_i = 0; sd_i < 2; ++sd_i) {
      const td::SideDesc& sd = g.side[sd_i];
      const double OI = (double)sd.outer * sd.inner;
      const double rows = sd.P / 2 * OI;
      const double in = sd.P * OI * D * el, out = sd.P * OI * Dn * el;
      bytes[TD_K_GRAM] += in;
      flops[TD_K_GRAM] += 2.0 * rows * 2.0 * D * D;               // G+ and G-, FP64 accumulation
      fp64_flops[TD_K_GRAM] += 2.0 * rows * 2.0 * D * D;
      bytes[TD_K_UPDATE] += in + out;
      flops[TD_K_UPDATE] += 2.0 * rows * 2.0 * D * Dn;            // Y T+ and Z T-
      if (f64) fp64_flops[TD_K_UPDATE] += 2.0 * rows * 2.0 * D * Dn;
    }
    // four pivoted Cholesky factors and triangular inverses, theta, SVD, transforms
    const double core = 8.0 * D * D * D / 3.0 + 8.0 * D * D * D + svd(2 * D, 2 * D) + 2.0 * 4.0 * D * Dn * 2 * D;
    flops[TD_K_CORE] += core;
    fp64_flops[TD_K_CORE] += core;
    bytes[TD_K_CORE] += 4.0 * D * D * 8 + 4.0 * D * Dn * 8;
  }
  // final contraction: zip-up with static dims, kept bond min(chi_mps, m, n) at every cut
  std::vector<double> mL(P.nx, 1), mDn(P.nx, 1), mR(P.nx, 1);
  mR[P.nx - 1] = 2;
  for (int y = 0; y < P.ny; ++y) {
    double cJ = 1;
    std::vector<double> nL(P.nx), nD(P.nx), nR(P.nx);
    for (int x = 0; x < P.nx; ++x) {
      const int s = P.grid_site[(size_t)y * P.nx + x];
      double L = 1, R = 1, Dd = 1, U = 1;
      if (s >= 0) {
        const td::FinalSite& f = P.finals[s];
        L = f.dir_dim[0]; R = f.dir_dim[1]; Dd = f.dir_dim[2]; U = f.dir_dim[3];
        double rest = L * R * Dd * U;
        bytes[TD_K_FINAL] += f.P * rest * el;
      }
      const double aL = mL[x], aD = mDn[x], aR = mR[x];
      // the site's class-1 half is zero when its readout flips no class: one parity term
      double cls1 = 0;
      if (s >= 0)
        for (int ph = 0; ph < P.finals[s].P; ++ph) cls1 = cls1 || P.finals[s].R[ph * 2 + 1] != 0.0;
      flops[TD_K_FINAL] += 2.0 * cJ * L * 2 * aD * aR * aL + 2.0 * cJ * U * aR * R * 2 * (L * (cls1 ? 2 : 1) * aD);
      const double m = cJ * U, n = aR * R * 2;
      if (x < P.nx - 1 && y < P.ny - 1) {
        flops[TD_K_FINAL] += svd_left(m, n);
        const double k = std::min<double>(P.chi_mps, std::min(m, n));
        nL[x] = cJ; nD[x] = U; nR[x] = k;
        cJ = k;
      } else if (x < P.nx - 1) {
        nL[x] = cJ; nD[x] = U; nR[x] = m;
        cJ = m;
      } else {
        nL[x] = cJ; nD[x] = U; nR[x] = 2;
      }
    }
    mL = nL; mDn = nD; mR = nR;
  }
  fp64_flops[TD_K_FINAL] = flops[TD_K_FINAL];   // FP64 on both paths
  bytes[TD_K_FINALIZE] = (double)net->nslots * 8 + P.n_det + 16;
  return TD_OK;
}

td_status td_network_profile(td_network* net, int32_t enable, double* ms, int64_t* launches) {
  g_err.clear();
  if (!net) return fail(TD_ERR_INVALID, "null network");
  if (ms && launches) {
    for (int k = 0; k < TD_K_COUNT; ++k) { ms[k] = 0; launches[k] = 0; }
    for (auto& u : net->ev_used) {
      cudaError_t e = cudaEventSynchronize(u.second.second);
      if (e != cudaSuccess) return cuda_fail(e, "profile event");
      float t = 0;
      e = cudaEventElapsedTime(&t, u.second.first, u.second.second);
      if (e != cudaSuccess) return cuda_fail(e, "profile elapsed");
      ms[u.first] += t;
      launches[u.first] += 1;
    }
  }
  for (auto& u : net->ev_used) { net->ev_pool.push_back(u.second.first); net->ev_pool.push_back(u.second.second); }
  net->ev_used.clear();
  net->profiling = enable != 0;
  return TD_OK;
}

void td_free_network(td_network* net) { delete net; }

}  // extern "C"
