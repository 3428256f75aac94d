// Host planner: DEM + layout -> layered detector network and its gate schedule.
//
// Follows Sec. 2.4 (DEM triple, merging of mechanisms with identical detectors and class
// effect), Sec. 3.4 (a DEM's detector network: mechanisms are weighted equality nodes,
// detectors parity nodes) and the layered form of Sec. 4 / Sec. 5.1 (natural split: a
// mechanism between two checks of one layer is a two-site gate; mechanisms between layers
// are contracted between layers).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <tuple>

#include "td_internal.h"

namespace td {
namespace {

struct Mech {
  std::vector<int32_t> dets;
  int32_t l = 0;
  double p = 0;
  // classification
  int kind = 0;      // 0 global, 1 single, 2 pair, 3 vertical
  int32_t a = -1, b = -1, t = -1;
};

enum { kGlobal = 0, kSingle = 1, kPair = 2, kVert = 3 };

// W[tau][dc]: probability that the XOR of a group's mechanism bits is tau and their class
// flips XOR to dc.
void parity_weights(const std::vector<const Mech*>& group, double W[2][2]) {
  W[0][0] = 1; W[0][1] = 0; W[1][0] = 0; W[1][1] = 0;
  for (const Mech* m : group) {
    double N[2][2] = {{0, 0}, {0, 0}};
    for (int tau = 0; tau < 2; ++tau)
      for (int dc = 0; dc < 2; ++dc) {
        N[tau][dc] += (1 - m->p) * W[tau][dc];
        N[tau ^ 1][dc ^ m->l] += m->p * W[tau][dc];
      }
    std::memcpy(W, N, sizeof(N));
  }
}

void matmul(int P, const double* A, const double* B, double* C) {  // C = A B
  double tmp[kMaxPhys * kMaxPhys];
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      double s = 0;
      for (int k = 0; k < P; ++k) s += A[i * P + k] * B[k * P + j];
      tmp[i * P + j] = s;
    }
  std::memcpy(C, tmp, sizeof(double) * P * P);
}

void eye(int P, double* A) {
  for (int i = 0; i < P * P; ++i) A[i] = 0;
  for (int i = 0; i < P; ++i) A[i * P + i] = 1;
}

// A gate of the layered network: sites a < b of one layer, its colour and position for the
// order inside the layer (colour, y, x of site a, idx), rate, class flip, and for a diagonal
// gate diag(w(r + s_a + s_b)) of the generator picture the detector-row column of r.
struct GateSpec {
  int colour, y, x;
  int32_t idx;
  int32_t a, b;
  double p;
  int32_t l;
  int32_t diag, rcol;
};

// First-stage result of the planner: everything emit_plan needs besides the sites.
struct NetSpec {
  std::vector<int32_t> det_at;                   // [T * S] detector-row column of (site, layer)
  std::vector<double> K;                         // [T * S][16] site-local matrices
  std::vector<std::vector<GateSpec>> layer_gates;   // [T]
  std::vector<double> R;                         // [S][8] readout of the last layer
};

}  // namespace

// Second stage of the planner, shared by detector and generator networks: bonds, the gate
// rounds and the static bond schedule, buffer offsets, descriptors, the final readout and the
// versioned layout of the reverse sweep.  plan's sites, grid and physical dimensions are set.
static td_status emit_plan(NetSpec& ns, const td_options& opt, Plan& plan, std::string& err) {
  const int32_t S = plan.S, T = plan.T;
  (void)err;
  // ---- bonds -------------------------------------------------------------------------------
  std::map<std::pair<int32_t, int32_t>, int32_t> bond_of;
  for (const auto& lg : ns.layer_gates)
    for (const GateSpec& gs : lg) bond_of[{gs.a, gs.b}] = 0;
  for (auto& kv : bond_of) { kv.second = (int32_t)plan.bond_sites.size(); plan.bond_sites.push_back(kv.first); }
  plan.n_bonds = (int32_t)plan.bond_sites.size();
  std::vector<std::vector<int32_t>> site_bonds(S), site_dirs(S);
  for (int32_t s = 0; s < S; ++s) {
    const int32_t x = plan.site_x[s], y = plan.site_y[s];
    const int32_t nbx[4] = {x - 1, x + 1, x, x}, nby[4] = {y, y, y - 1, y + 1};
    for (int dir = 0; dir < 4; ++dir) {
      if (nbx[dir] < 0 || nby[dir] < 0 || nbx[dir] >= plan.nx || nby[dir] >= plan.ny) continue;
      int32_t o = plan.grid_site[(size_t)nby[dir] * plan.nx + nbx[dir]];
      if (o < 0) continue;
      auto it = bond_of.find({std::min(s, o), std::max(s, o)});
      if (it == bond_of.end()) continue;
      site_bonds[s].push_back(it->second);
      site_dirs[s].push_back(dir);
    }
  }

  // Static schedule: bond dims double per gate up to chi.  Pass 1 finds every site
  // tensor's largest size, pass 2 assigns buffer offsets and emits descriptors.
  std::vector<std::vector<std::vector<GateSpec>>> rounds_of(T);
  for (int32_t t = 0; t < T; ++t) {
    auto& g = ns.layer_gates[t];
    std::sort(g.begin(), g.end(), [](const GateSpec& a, const GateSpec& b) {
      return std::tie(a.colour, a.y, a.x, a.idx) < std::tie(b.colour, b.y, b.x, b.idx);
    });
    for (int colour = 0; colour < 4; ++colour) {
      std::vector<std::vector<GateSpec>> rr;
      std::map<int32_t, int> count;
      for (const GateSpec& gs : g) {
        if (gs.colour != colour) continue;
        int32_t b = bond_of[{gs.a, gs.b}];
        int r = count[b]++;
        if ((int)rr.size() <= r) rr.resize(r + 1);
        rr[r].push_back(gs);
      }
      for (auto& r : rr) rounds_of[t].push_back(r);
    }
  }
  auto site_size = [&](int32_t s, const std::vector<int32_t>& dims) {
    int64_t n = plan.P[s];
    for (int32_t b : site_bonds[s]) n *= dims[b];
    return n;
  };
  std::vector<int64_t> maxsize(S);
  {
    std::vector<int32_t> dims(plan.n_bonds, 1);
    for (int32_t s = 0; s < S; ++s) maxsize[s] = site_size(s, dims);
    for (int32_t t = 0; t < T; ++t)
      for (auto& r : rounds_of[t])
        for (const GateSpec& gs : r) {
          int32_t b = bond_of[{gs.a, gs.b}];
          dims[b] = std::min(plan.chi, 2 * dims[b]);
          maxsize[gs.a] = std::max(maxsize[gs.a], site_size(gs.a, dims));
          maxsize[gs.b] = std::max(maxsize[gs.b], site_size(gs.b, dims));
        }
  }
  std::vector<int64_t> base(S);
  int64_t acc = 0;
  for (int32_t s = 0; s < S; ++s) { base[s] = acc; acc += 2 * ((maxsize[s] + 3) / 4 * 4); }
  plan.shot_elems = acc;
  auto buf_off = [&](int32_t s, int k) { return base[s] + k * ((maxsize[s] + 3) / 4 * 4); };

  std::vector<int32_t> dims(plan.n_bonds, 1), cur(S, 0);
  plan.layers.resize(T);
  for (int32_t t = 0; t < T; ++t) {
    LayerPlan& L = plan.layers[t];
    L.local_first = (int32_t)plan.locals.size();
    for (int32_t s = 0; s < S; ++s) {
      LocalDesc ld{};
      ld.P = plan.P[s];
      ld.det = ns.det_at[(size_t)t * S + s];
      ld.rest = (int32_t)(site_size(s, dims) / plan.P[s]);
      ld.off = buf_off(s, cur[s]);
      ld.out_off = ld.off;
      for (int i = 0; i < 16; ++i) ld.K[i] = ns.K[((size_t)t * S + s) * 16 + i];
      plan.locals.push_back(ld);
    }
    for (auto& r : rounds_of[t]) {
      Round R{};
      R.first = (int32_t)plan.gates.size();
      R.count = (int32_t)r.size();
      for (const GateSpec& gs : r) {
        GateDesc g{};
        g.bond = bond_of[{gs.a, gs.b}];
        g.D = dims[g.bond];
        g.Dn = std::min(plan.chi, 2 * g.D);
        g.p = gs.p;
        g.diag = gs.diag;
        g.rcol = gs.rcol;
        const int32_t ends[2] = {gs.a, gs.b};
        for (int side = 0; side < 2; ++side) {
          SideDesc& sd = g.side[side];
          const int32_t s = ends[side];
          sd.site = s;
          sd.P = plan.P[s];
          sd.mask = 1 | ((side == 0 && gs.l) ? 2 : 0);
          sd.nb = (int32_t)site_bonds[s].size();
          sd.pos = -1;
          sd.outer = 1; sd.inner = 1;
          for (int k = 0; k < kMaxBonds; ++k) { sd.dims[k] = 1; sd.bond[k] = -1; }
          for (int k = 0; k < sd.nb; ++k) {
            sd.bond[k] = site_bonds[s][k];
            sd.dims[k] = dims[site_bonds[s][k]];
            if (site_bonds[s][k] == g.bond) sd.pos = k;
          }
          for (int k = 0; k < sd.nb; ++k) {
            if (k < sd.pos) sd.outer *= sd.dims[k];
            if (k > sd.pos) sd.inner *= sd.dims[k];
          }
          sd.in_off = buf_off(s, cur[s]);
          sd.out_off = buf_off(s, cur[s] ^ 1);
          R.max_rows = std::max(R.max_rows, sd.P / 2 * sd.outer * sd.inner);
        }
        R.maxD = std::max(R.maxD, g.D);
        R.maxDn = std::max(R.maxDn, g.Dn);
        dims[g.bond] = g.Dn;
        cur[gs.a] ^= 1;
        cur[gs.b] ^= 1;
        plan.gates.push_back(g);
      }
      plan.max_round_gates = std::max(plan.max_round_gates, R.count);
      L.rounds.push_back(R);
    }
  }
  // readout of the last layer
  for (int32_t s = 0; s < S; ++s) {
    FinalSite f{};
    f.P = plan.P[s];
    f.nb = (int32_t)site_bonds[s].size();
    for (int d = 0; d < 4; ++d) { f.dir_dim[d] = 1; f.dir_pos[d] = -1; f.dir_bond[d] = -1; }
    for (int k = 0; k < f.nb; ++k) {
      int d = site_dirs[s][k];
      f.dir_pos[d] = k;
      f.dir_bond[d] = site_bonds[s][k];
      f.dir_dim[d] = dims[site_bonds[s][k]];
    }
    f.off = buf_off(s, cur[s]);
    for (int i = 0; i < 8; ++i) f.R[i] = ns.R[(size_t)s * 8 + i];
    plan.finals.push_back(f);
  }
  plan.final_dims = dims;
  for (int32_t d : dims) plan.max_final_D = std::max(plan.max_final_D, d);

  // versioned layout of the reverse sweep, one segment of ckpt_stride layers at a time: every
  // site-local operator and gate output gets a new slot, the slots of a segment start at 0
  // with the segment's input versions; the tensors at the start of every segment but the first
  // are kept in a checkpoint area (with the bond weights), the segment is recomputed from it
  {
    const int32_t k = opt.ckpt_stride >= 1 ? std::min(opt.ckpt_stride, T) : T;
    plan.ckpt_stride = k;
    plan.seg_first_layer.clear();
    plan.seg_first_gate.clear();
    for (int32_t t = 0; t < T; t += k) plan.seg_first_layer.push_back(t);
    const int32_t nseg = (int32_t)plan.seg_first_layer.size();
    plan.seg_first_layer.push_back(T);
    plan.seg_in_off.assign((size_t)nseg * S, 0);
    plan.seg_out_off.assign((size_t)nseg * S, 0);
    plan.seg_in_elems.assign((size_t)nseg * S, 0);
    plan.ckpt_off.assign((size_t)nseg * S, 0);
    plan.ckpt_lam_off.assign(nseg, 0);
    plan.hist_locals.clear();
    plan.hist_gates.clear();
    std::vector<int32_t> hd(plan.n_bonds, 1);
    std::vector<int64_t> ver(S);
    int64_t hmax = 0, cacc = 0;
    size_t gi = 0;
    for (int32_t j = 0; j < nseg; ++j) {
      int64_t hacc = 0;
      auto slot = [&](int64_t n) { int64_t r = hacc; hacc += (n + 3) / 4 * 4; return r; };
      plan.seg_first_gate.push_back((int32_t)gi);
      for (int32_t s2 = 0; s2 < S; ++s2) {
        const int64_t n = site_size(s2, hd);
        ver[s2] = slot(n);
        plan.seg_in_off[(size_t)j * S + s2] = ver[s2];
        plan.seg_in_elems[(size_t)j * S + s2] = n;
        if (j > 0) {
          plan.ckpt_off[(size_t)j * S + s2] = cacc;
          cacc += (n + 3) / 4 * 4;
        }
      }
      if (j > 0) {
        plan.ckpt_lam_off[j] = cacc;
        cacc += (int64_t)plan.n_bonds * plan.chi;
      }
      for (int32_t t = plan.seg_first_layer[j]; t < plan.seg_first_layer[j + 1]; ++t) {
        for (int32_t s2 = 0; s2 < S; ++s2) {
          LocalDesc ld = plan.locals[(size_t)t * S + s2];
          ld.off = ver[s2];
          ld.out_off = slot(site_size(s2, hd));
          ver[s2] = ld.out_off;
          plan.hist_locals.push_back(ld);
        }
        for (const Round& R : plan.layers[t].rounds)
          for (int32_t q = 0; q < R.count; ++q, ++gi) {
            GateDesc g = plan.gates[gi];
            const int32_t ends[2] = {g.side[0].site, g.side[1].site};
            hd[g.bond] = g.Dn;
            for (int side = 0; side < 2; ++side) {
              SideDesc& sd = g.side[side];
              sd.in_off = ver[ends[side]];
              sd.out_off = slot(site_size(ends[side], hd));
              ver[ends[side]] = sd.out_off;
            }
            plan.hist_gates.push_back(g);
          }
      }
      for (int32_t s2 = 0; s2 < S; ++s2) plan.seg_out_off[(size_t)j * S + s2] = ver[s2];
      hmax = std::max(hmax, hacc);
    }
    plan.seg_first_gate.push_back((int32_t)gi);
    plan.hist_finals = plan.finals;
    for (int32_t s2 = 0; s2 < S; ++s2) plan.hist_finals[s2].off = ver[s2];
    plan.hist_shot_elems = hmax;
    plan.ckpt_shot_elems = cacc;
    plan.max_site_elems = 1;
    for (int32_t s2 = 0; s2 < S; ++s2) plan.max_site_elems = std::max(plan.max_site_elems, maxsize[s2]);
  }
  return TD_OK;
}

td_status build_plan(const td_dem& dem, const td_layout& layout, const td_options& opt, Plan& plan,
                     std::string& err) {
  // ---- validation ------------------------------------------------------------------
  if (dem.n_det < 1 || dem.n_mech < 0 || dem.n_obs < 0) { err = "n_det must be >= 1, n_mech and n_obs >= 0"; return TD_ERR_INVALID; }
  if (dem.n_obs != 1) { err = "this build supports exactly one logical observable (n_obs = 1)"; return TD_ERR_UNSUPPORTED; }
  if (!dem.H_indptr || !dem.L_indptr || !dem.p || !layout.det_xyt ||
      (!dem.H_indices && dem.H_indptr[dem.n_det] > 0) || (!dem.L_indices && dem.L_indptr[dem.n_obs] > 0)) {
    err = "null DEM or layout array"; return TD_ERR_INVALID;
  }
  if (opt.chi < 1 || opt.chi > kMaxChi) { err = "chi must be in [1, 32]"; return opt.chi < 1 ? TD_ERR_INVALID : TD_ERR_UNSUPPORTED; }
  if (opt.chi_mps < 1) { err = "chi_mps must be >= 1"; return TD_ERR_INVALID; }
  if (opt.precision < TD_FP64 || opt.precision > TD_TC) { err = "unknown precision"; return TD_ERR_INVALID; }
  if (!(opt.svd_cutoff >= 0 && opt.svd_cutoff < 1) || !(opt.multiplet_rtol >= 0 && opt.multiplet_rtol < 1) ||
      !(opt.gram_cutoff < 1)) { err = "cutoffs must be in [0, 1)"; return TD_ERR_INVALID; }
  const int32_t n_det = dem.n_det, n_mech = dem.n_mech;
  std::vector<std::vector<int32_t>> mdets(n_mech);
  std::vector<int32_t> mobs(n_mech, 0);
  if (dem.H_indptr[0] != 0) { err = "H_indptr[0] must be 0"; return TD_ERR_INVALID; }
  for (int32_t i = 0; i < n_det; ++i) {
    if (dem.H_indptr[i + 1] < dem.H_indptr[i]) { err = "H_indptr not monotone"; return TD_ERR_INVALID; }
    for (int32_t k = dem.H_indptr[i]; k < dem.H_indptr[i + 1]; ++k) {
      int32_t j = dem.H_indices[k];
      if (j < 0 || j >= n_mech) { err = "H index out of range"; return TD_ERR_INVALID; }
      if (std::find(mdets[j].begin(), mdets[j].end(), i) != mdets[j].end()) { err = "duplicate entry in H"; return TD_ERR_INVALID; }
      mdets[j].push_back(i);
    }
  }
  if (dem.L_indptr[0] != 0 || dem.L_indptr[1] < 0) { err = "bad L_indptr"; return TD_ERR_INVALID; }
  for (int32_t k = dem.L_indptr[0]; k < dem.L_indptr[1]; ++k) {
    int32_t j = dem.L_indices[k];
    if (j < 0 || j >= n_mech) { err = "L index out of range"; return TD_ERR_INVALID; }
    if (mobs[j]) { err = "duplicate entry in l"; return TD_ERR_INVALID; }
    mobs[j] = 1;
  }
  for (int32_t j = 0; j < n_mech; ++j)
    if (!(dem.p[j] >= 0.0 && dem.p[j] <= 1.0)) { err = "mechanism probability outside [0, 1]"; return TD_ERR_INVALID; }
  for (int32_t i = 0; i < 3 * n_det; ++i)
    if (layout.det_xyt[i] < 0 || layout.det_xyt[i] > (1 << 14)) { err = "detector coordinate outside [0, 16384]"; return TD_ERR_INVALID; }

  // ---- sites and layers ----------------------------------------------------------------
  plan = Plan();
  plan.n_det = n_det; plan.n_mech = n_mech; plan.n_obs = dem.n_obs;
  plan.chi = opt.chi; plan.chi_mps = opt.chi_mps; plan.precision = opt.precision;
  plan.svd_cutoff = opt.svd_cutoff; plan.multiplet_rtol = opt.multiplet_rtol;
  // Gram directions below this fraction of the side's largest diagonal are rounding noise
  // of the FP64 sums (both storage types accumulate the Gram in FP64).
  plan.gram_cutoff = opt.gram_cutoff >= 0 ? opt.gram_cutoff : 1e-15;
  std::set<std::pair<int32_t, int32_t>> yx;
  int32_t T = 0;
  for (int32_t i = 0; i < n_det; ++i) {
    yx.insert({layout.det_xyt[3 * i + 1], layout.det_xyt[3 * i]});
    T = std::max(T, layout.det_xyt[3 * i + 2] + 1);
    plan.nx = std::max(plan.nx, layout.det_xyt[3 * i] + 1);
    plan.ny = std::max(plan.ny, layout.det_xyt[3 * i + 1] + 1);
  }
  const int32_t S = (int32_t)yx.size();
  plan.S = S; plan.T = T;
  plan.grid_site.assign((size_t)plan.nx * plan.ny, -1);
  for (auto& q : yx) {
    int32_t s = (int32_t)plan.site_x.size();
    plan.site_x.push_back(q.second); plan.site_y.push_back(q.first);
    plan.grid_site[(size_t)q.first * plan.nx + q.second] = s;
  }
  std::vector<int32_t> det_site(n_det), det_layer(n_det), det_at((size_t)S * T, -1);
  for (int32_t i = 0; i < n_det; ++i) {
    int32_t s = plan.grid_site[(size_t)layout.det_xyt[3 * i + 1] * plan.nx + layout.det_xyt[3 * i]];
    int32_t t = layout.det_xyt[3 * i + 2];
    det_site[i] = s; det_layer[i] = t;
    if (det_at[(size_t)t * S + s] != -1) { err = "two detectors at one (site, layer)"; return TD_ERR_UNSUPPORTED; }
    det_at[(size_t)t * S + s] = i;
  }
  if ((int64_t)S * T != n_det) { err = "every site needs exactly one detector in every layer"; return TD_ERR_UNSUPPORTED; }

  // ---- merge identical mechanisms (Sec. 2.4) --------------------------------------------
  std::map<std::pair<std::vector<int32_t>, int32_t>, int32_t> seen;
  std::vector<Mech> mechs;
  for (int32_t j = 0; j < n_mech; ++j) {
    std::vector<int32_t> d = mdets[j];
    std::sort(d.begin(), d.end());
    auto key = std::make_pair(d, mobs[j]);
    auto it = seen.find(key);
    if (it != seen.end()) {
      Mech& m = mechs[it->second];
      m.p = m.p + dem.p[j] - 2 * m.p * dem.p[j];
    } else {
      seen[key] = (int32_t)mechs.size();
      Mech m; m.dets = d; m.l = mobs[j]; m.p = dem.p[j];
      mechs.push_back(m);
    }
  }

  // ---- classify ----------------------------------------------------------------------------
  for (Mech& m : mechs) {
    if (m.dets.empty()) { m.kind = kGlobal; continue; }
    if (m.dets.size() == 1) { m.kind = kSingle; m.a = det_site[m.dets[0]]; m.t = det_layer[m.dets[0]]; continue; }
    if (m.dets.size() > 2) { err = "mechanism flips more than two detectors"; return TD_ERR_NONLOCAL; }
    int32_t s0 = det_site[m.dets[0]], s1 = det_site[m.dets[1]];
    int32_t t0 = det_layer[m.dets[0]], t1 = det_layer[m.dets[1]];
    if (t0 == t1) {
      int32_t dx = std::abs(plan.site_x[s0] - plan.site_x[s1]), dy = std::abs(plan.site_y[s0] - plan.site_y[s1]);
      if (dx + dy != 1) { err = "two-detector mechanism between non-adjacent sites of one layer"; return TD_ERR_NONLOCAL; }
      m.kind = kPair; m.a = std::min(s0, s1); m.b = std::max(s0, s1); m.t = t0;
    } else if (s0 == s1 && std::abs(t0 - t1) == 1) {
      m.kind = kVert; m.a = s0; m.t = std::min(t0, t1);
    } else {
      err = "two-detector mechanism that is neither in-layer nor vertical"; return TD_ERR_NONLOCAL;
    }
  }

  // ---- class tracking: observable representative with fewer counter sites ----------------
  auto counters_of = [&](bool deformed) {
    std::set<int32_t> cs;
    for (const Mech& m : mechs) {
      int32_t l = m.l ^ ((deformed && m.kind == kSingle) ? 1 : 0);
      if (!l) continue;
      if (m.kind == kPair) cs.insert(m.a);
      else if (m.kind == kSingle && m.t != T - 1) cs.insert(m.a);
      else if (m.kind == kVert) cs.insert(m.a);
    }
    return cs;
  };
  std::set<int32_t> c0 = counters_of(false), c1 = counters_of(true);
  bool deformed = c1.size() < c0.size();
  std::set<int32_t>& cs = deformed ? c1 : c0;
  plan.offset_all = deformed ? 1 : 0;
  if (deformed)
    for (Mech& m : mechs)
      if (m.kind == kSingle) m.l ^= 1;
  plan.P.assign(S, 2);
  for (int32_t s : cs) plan.P[s] = 4;
  plan.n_counter_sites = (int32_t)cs.size();
  for (const Mech& m : mechs)
    if (m.kind == kGlobal && m.l) {
      double G[4] = {1 - m.p, m.p, m.p, 1 - m.p}, R[4];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) R[i * 2 + j] = G[i * 2] * plan.glob_mix[j] + G[i * 2 + 1] * plan.glob_mix[2 + j];
      std::memcpy(plan.glob_mix, R, sizeof(R));
    }

  // ---- network spec: per-layer local operators, gates, readout --------------------------
  NetSpec ns;
  ns.det_at = det_at;
  ns.K.assign((size_t)T * S * 16, 0.0);
  ns.layer_gates.resize(T);
  ns.R.assign((size_t)S * 8, 0.0);
  std::vector<std::vector<const Mech*>> vert((size_t)T * S), read(S);
  std::vector<double> pre((size_t)T * S * 16);
  for (int32_t t = 0; t < T; ++t)
    for (int32_t s = 0; s < S; ++s) eye(plan.P[s], &pre[((size_t)t * S + s) * 16]);
  for (int32_t idx = 0; idx < (int32_t)mechs.size(); ++idx) {
    const Mech& m = mechs[idx];
    if (m.kind == kSingle) {
      if (m.t == T - 1) { read[m.a].push_back(&m); continue; }
      const int P = plan.P[m.a];
      const int mask = 1 | (m.l ? 2 : 0);
      double G[16];
      for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) G[i * P + j] = (i == j ? 1 - m.p : 0) + (i == (j ^ mask) ? m.p : 0);
      double* A = &pre[((size_t)m.t * S + m.a) * 16];
      matmul(P, G, A, A);
    } else if (m.kind == kVert) {
      vert[(size_t)m.t * S + m.a].push_back(&m);
    } else if (m.kind == kPair) {
      const int32_t xa = plan.site_x[m.a], ya = plan.site_y[m.a], xb = plan.site_x[m.b], yb = plan.site_y[m.b];
      int colour = (ya == yb) ? (std::min(xa, xb) % 2) : 2 + (std::min(ya, yb) % 2);
      GateSpec gs{};
      gs.colour = colour; gs.y = ya; gs.x = xa; gs.idx = idx;
      gs.a = m.a; gs.b = m.b; gs.p = m.p; gs.l = m.l; gs.diag = 0; gs.rcol = -1;
      ns.layer_gates[m.t].push_back(gs);
    }
  }
  auto post_matrix = [&](int32_t t, int32_t s, double* M) -> bool {   // vertical weights above layer t
    const int P = plan.P[s];
    double W[2][2];
    parity_weights(vert[(size_t)t * S + s], W);
    for (int i = 0; i < P * P; ++i) M[i] = 0;
    for (int ph = 0; ph < P; ++ph) {
      int tau = ph & 1, cl = ph >> 1;
      for (int dc = 0; dc < 2; ++dc) {
        if (W[tau][dc] == 0) continue;
        if (P == 2 && dc) return false;
        M[(tau | ((cl ^ dc) << 1)) * P + ph] += W[tau][dc];
      }
    }
    return true;
  };
  for (int32_t t = 0; t < T; ++t)
    for (int32_t s = 0; s < S; ++s) {
      double* K = &ns.K[((size_t)t * S + s) * 16];
      std::memcpy(K, &pre[((size_t)t * S + s) * 16], sizeof(double) * 16);
      if (t > 0) {
        double post[16];
        if (!post_matrix(t - 1, s, post)) { err = "class-flipping vertical mechanism without counter"; return TD_ERR_INVALID; }
        matmul(plan.P[s], K, post, K);
      }
      for (int i = plan.P[s] * plan.P[s]; i < 16; ++i) K[i] = 0.0;
    }
  for (int32_t s = 0; s < S; ++s) {
    double W[2][2];
    parity_weights(read[s], W);
    for (int ph = 0; ph < plan.P[s]; ++ph) {
      int tau = ph & 1, cl = ph >> 1;
      for (int c = 0; c < 2; ++c) ns.R[(size_t)s * 8 + ph * 2 + c] = W[tau][c ^ cl];
    }
  }
  return emit_plan(ns, opt, plan, err);
}

}  // namespace td

// ---- generator networks (Sec. 3.2) ------------------------------------------------------------
namespace td {
namespace {

// Dense GF(2) matrix with rows of 64-bit words.
struct Bits {
  int32_t rows = 0, cols = 0, words = 0;
  std::vector<uint64_t> w;
  Bits(int32_t r, int32_t c) : rows(r), cols(c), words((c + 63) / 64), w((size_t)r * ((c + 63) / 64), 0ull) {}
  uint64_t* row(int32_t i) { return &w[(size_t)i * words]; }
  bool get(int32_t i, int32_t j) const { return (w[(size_t)i * words + j / 64] >> (j % 64)) & 1ull; }
  void flip(int32_t i, int32_t j) { w[(size_t)i * words + j / 64] ^= 1ull << (j % 64); }
};

// Reduced row echelon form in place, pivots taken column by column in order among the first
// `ncols` columns; returns the pivot columns (row i has its leading one at pivots[i]).
std::vector<int32_t> rref(Bits& A, int32_t ncols) {
  std::vector<int32_t> piv;
  int32_t r = 0;
  for (int32_t c = 0; c < ncols && r < A.rows; ++c) {
    int32_t k = -1;
    for (int32_t i = r; i < A.rows; ++i)
      if (A.get(i, c)) { k = i; break; }
    if (k < 0) continue;
    if (k != r)
      for (int32_t q = 0; q < A.words; ++q) std::swap(A.row(k)[q], A.row(r)[q]);
    const uint64_t* pr = A.row(r);
    for (int32_t i = 0; i < A.rows; ++i)
      if (i != r && A.get(i, c)) {
        uint64_t* ri = A.row(i);
        for (int32_t q = c / 64; q < A.words; ++q) ri[q] ^= pr[q];
      }
    piv.push_back(c);
    ++r;
  }
  return piv;
}

}  // namespace

td_status build_gen_plan(const td_gen& g, const td_options& opt, Plan& plan, std::string& err) {
  // ---- validation ------------------------------------------------------------------------
  if (g.n_gen < 1 || g.n_qubits < 1 || g.n_checks < 0) { err = "n_gen and n_qubits must be >= 1, n_checks >= 0"; return TD_ERR_INVALID; }
  if (!g.qubit_gens || !g.p || !g.gen_xyt || !g.check_indptr || (!g.check_indices && g.check_indptr[g.n_checks] > 0) ||
      (g.n_xbar > 0 && !g.xbar) || (g.n_zbar > 0 && !g.zbar)) { err = "null array in td_gen"; return TD_ERR_INVALID; }
  if (opt.chi < 1 || opt.chi > kMaxChi) { err = "chi must be in [1, 32]"; return opt.chi < 1 ? TD_ERR_INVALID : TD_ERR_UNSUPPORTED; }
  if (opt.chi_mps < 1) { err = "chi_mps must be >= 1"; return TD_ERR_INVALID; }
  if (opt.precision < TD_FP64 || opt.precision > TD_TC) { err = "unknown precision"; return TD_ERR_INVALID; }
  if (!(opt.svd_cutoff >= 0 && opt.svd_cutoff < 1) || !(opt.multiplet_rtol >= 0 && opt.multiplet_rtol < 1) ||
      !(opt.gram_cutoff < 1)) { err = "cutoffs must be in [0, 1)"; return TD_ERR_INVALID; }
  const int32_t NG = g.n_gen, NQ = g.n_qubits, NC = g.n_checks;
  for (int32_t j = 0; j < NQ; ++j) {
    const int32_t a = g.qubit_gens[2 * j], b = g.qubit_gens[2 * j + 1];
    if (a < 0 || a >= NG || b < -1 || b >= NG || a == b) { err = "qubit_gens entry out of range"; return TD_ERR_INVALID; }
    if (!(g.p[j] >= 0.0 && g.p[j] <= 1.0)) { err = "flip rate outside [0, 1]"; return TD_ERR_INVALID; }
  }
  for (int32_t i = 0; i < 3 * NG; ++i)
    if (g.gen_xyt[i] < 0 || g.gen_xyt[i] > (1 << 14)) { err = "generator coordinate outside [0, 16384]"; return TD_ERR_INVALID; }
  if (g.check_indptr[0] != 0) { err = "check_indptr[0] must be 0"; return TD_ERR_INVALID; }
  Bits H(std::max(NC, 1), NQ);
  for (int32_t i = 0; i < NC; ++i) {
    if (g.check_indptr[i + 1] < g.check_indptr[i]) { err = "check_indptr not monotone"; return TD_ERR_INVALID; }
    for (int32_t k = g.check_indptr[i]; k < g.check_indptr[i + 1]; ++k) {
      const int32_t j = g.check_indices[k];
      if (j < 0 || j >= NQ) { err = "check index out of range"; return TD_ERR_INVALID; }
      if (H.get(i, j)) { err = "duplicate entry in a check"; return TD_ERR_INVALID; }
      H.flip(i, j);
    }
  }
  auto qubit_set = [&](int32_t n, const int32_t* q, std::vector<uint8_t>& v) {
    v.assign(NQ, 0);
    for (int32_t k = 0; k < n; ++k) {
      if (q[k] < 0 || q[k] >= NQ || v[q[k]]) return false;
      v[q[k]] = 1;
    }
    return true;
  };
  std::vector<uint8_t> xb, zb;
  if (!qubit_set(g.n_xbar, g.xbar, xb) || !qubit_set(g.n_zbar, g.zbar, zb)) { err = "xbar / zbar: index out of range or repeated"; return TD_ERR_INVALID; }
  // commutation: every check with every generator and with xbar; zbar with every generator
  {
    std::vector<std::vector<int32_t>> gq(NG);
    for (int32_t j = 0; j < NQ; ++j) {
      gq[g.qubit_gens[2 * j]].push_back(j);
      if (g.qubit_gens[2 * j + 1] >= 0) gq[g.qubit_gens[2 * j + 1]].push_back(j);
    }
    for (int32_t i = 0; i < NC; ++i) {
      for (int32_t v = 0; v < NG; ++v) {
        int par = 0;
        for (int32_t j : gq[v]) par ^= H.get(i, j) ? 1 : 0;
        if (par) { err = "a generator anticommutes with a check (H g != 0)"; return TD_ERR_INVALID; }
      }
      int par = 0;
      for (int32_t j = 0; j < NQ; ++j) par ^= (xb[j] && H.get(i, j)) ? 1 : 0;
      if (par) { err = "xbar has a nonzero syndrome"; return TD_ERR_INVALID; }
    }
    for (int32_t v = 0; v < NG; ++v) {
      int par = 0;
      for (int32_t j : gq[v]) par ^= zb[j];
      if (par) { err = "zbar anticommutes with a generator"; return TD_ERR_INVALID; }
    }
    int par = 0;
    for (int32_t j = 0; j < NQ; ++j) par ^= xb[j] & zb[j];
    if (!par) { err = "xbar and zbar must overlap on an odd number of qubits"; return TD_ERR_INVALID; }
    // rank of the generators (the sum over s counts every coset element 2^(n_gen - rank) times)
    Bits G(NG, NQ);
    for (int32_t v = 0; v < NG; ++v)
      for (int32_t j : gq[v]) G.flip(v, j);
    const int32_t rk = (int32_t)rref(G, NQ).size();
    plan = Plan();
    plan.gen_log_offset = -(double)(NG - rk) * std::log(2.0);
  }

  // ---- sites and layers ----------------------------------------------------------------
  plan.gen = 1;
  plan.n_checks = NC; plan.n_qubits = NQ; plan.n_gen = NG;
  plan.n_det = NQ; plan.n_mech = NQ; plan.n_obs = 1;
  plan.chi = opt.chi; plan.chi_mps = opt.chi_mps; plan.precision = opt.precision;
  plan.svd_cutoff = opt.svd_cutoff; plan.multiplet_rtol = opt.multiplet_rtol;
  plan.gram_cutoff = opt.gram_cutoff >= 0 ? opt.gram_cutoff : 1e-15;
  std::set<std::pair<int32_t, int32_t>> yx;
  int32_t TG = 0;
  for (int32_t v = 0; v < NG; ++v) {
    yx.insert({g.gen_xyt[3 * v + 1], g.gen_xyt[3 * v]});
    TG = std::max(TG, g.gen_xyt[3 * v + 2] + 1);
    plan.nx = std::max(plan.nx, g.gen_xyt[3 * v] + 1);
    plan.ny = std::max(plan.ny, g.gen_xyt[3 * v + 1] + 1);
  }
  const int32_t S = (int32_t)yx.size(), T = TG + 1;   // the generator layers, then the readout layer
  plan.S = S; plan.T = T;
  plan.grid_site.assign((size_t)plan.nx * plan.ny, -1);
  for (auto& q : yx) {
    int32_t s = (int32_t)plan.site_x.size();
    plan.site_x.push_back(q.second); plan.site_y.push_back(q.first);
    plan.grid_site[(size_t)q.first * plan.nx + q.second] = s;
  }
  std::vector<int32_t> gsite(NG), glayer(NG), gen_at((size_t)S * TG, -1);
  for (int32_t v = 0; v < NG; ++v) {
    const int32_t s = plan.grid_site[(size_t)g.gen_xyt[3 * v + 1] * plan.nx + g.gen_xyt[3 * v]], t = g.gen_xyt[3 * v + 2];
    gsite[v] = s; glayer[v] = t;
    if (gen_at[(size_t)t * S + s] != -1) { err = "two generators at one (site, layer)"; return TD_ERR_UNSUPPORTED; }
    gen_at[(size_t)t * S + s] = v;
  }
  if ((int64_t)S * TG != NG) { err = "every site needs exactly one generator in every layer"; return TD_ERR_UNSUPPORTED; }
  plan.P.assign(S, 2);

  // ---- classify the qubits: the edge entering (site, layer t) from below (t = 0: dangling;
  //      t = TG: the dangling edge above the last layer) or an in-layer edge -------------------
  std::vector<int32_t> below((size_t)S * T, -1), col(NQ, -1);
  NetSpec ns;
  ns.layer_gates.resize(T);
  std::vector<int32_t> inlayer;
  for (int32_t j = 0; j < NQ; ++j) {
    const int32_t a = g.qubit_gens[2 * j], b = g.qubit_gens[2 * j + 1];
    int32_t slot = -1;
    if (b < 0) {
      const int32_t s = gsite[a], t = glayer[a];
      if (t == 0 && below[s] < 0) slot = s;
      else if (t == TG - 1 && below[(size_t)TG * S + s] < 0) slot = TG * S + s;
      else { err = "dangling edge inside the lattice"; return TD_ERR_UNSUPPORTED; }
    } else if (glayer[a] == glayer[b]) {
      const int32_t sa = gsite[a], sb = gsite[b];
      const int32_t dx = std::abs(plan.site_x[sa] - plan.site_x[sb]), dy = std::abs(plan.site_y[sa] - plan.site_y[sb]);
      if (dx + dy != 1) { err = "in-layer edge between generators that are not grid neighbours"; return TD_ERR_NONLOCAL; }
      inlayer.push_back(j);
      continue;
    } else if (gsite[a] == gsite[b] && std::abs(glayer[a] - glayer[b]) == 1) {
      slot = std::max(glayer[a], glayer[b]) * S + gsite[a];
      if (below[slot] >= 0) { err = "two vertical edges into one generator"; return TD_ERR_UNSUPPORTED; }
    } else {
      err = "edge that is neither in-layer nor vertical"; return TD_ERR_NONLOCAL;
    }
    below[slot] = j;
    col[j] = slot;
  }
  for (int32_t k = 0; k < S * T; ++k)
    if (below[k] < 0) { err = "every generator needs one edge below, and the last layer one above"; return TD_ERR_UNSUPPORTED; }
  for (size_t k = 0; k < inlayer.size(); ++k) col[inlayer[k]] = S * T + (int32_t)k;

  // ---- network spec --------------------------------------------------------------------------
  ns.det_at.resize((size_t)T * S);
  ns.K.assign((size_t)T * S * 16, 0.0);
  ns.R.assign((size_t)S * 8, 0.0);
  for (int32_t t = 0; t < T; ++t)
    for (int32_t s = 0; s < S; ++s) {
      const int32_t k = t * S + s;
      ns.det_at[k] = k;   // the row's bit r flips the physical leg: X^r
      double* K = &ns.K[(size_t)k * 16];
      if (t < TG) {       // transfer w(s_old + s_new) of the edge below (the old bit is 0 at t = 0)
        const double p = g.p[below[k]];
        K[0] = 1 - p; K[1] = p; K[2] = p; K[3] = 1 - p;
      } else {            // readout layer: the weight of the dangling edge above, then the sum
        K[0] = 1; K[3] = 1;
        const double p = g.p[below[k]];
        ns.R[(size_t)s * 8 + 0] = 1 - p;
        ns.R[(size_t)s * 8 + 2] = p;
      }
    }
  for (int32_t j : inlayer) {
    const int32_t a = g.qubit_gens[2 * j], b = g.qubit_gens[2 * j + 1];
    const int32_t sa = std::min(gsite[a], gsite[b]), sb = std::max(gsite[a], gsite[b]);
    const int32_t xa = plan.site_x[sa], ya = plan.site_y[sa], xb2 = plan.site_x[sb], yb = plan.site_y[sb];
    GateSpec gs{};
    gs.colour = (ya == yb) ? (std::min(xa, xb2) % 2) : 2 + (std::min(ya, yb) % 2);
    gs.y = ya; gs.x = xa; gs.idx = j;
    gs.a = sa; gs.b = sb; gs.p = g.p[j]; gs.l = 0; gs.diag = 1; gs.rcol = col[j];
    ns.layer_gates[glayer[a]].push_back(gs);
  }

  // ---- representative map: elimination of [H | I] ----------------------------------------------
  {
    Bits A(std::max(NC, 1), NQ + std::max(NC, 1));
    for (int32_t i = 0; i < NC; ++i) {
      for (int32_t q = 0; q < H.words; ++q) {
        const uint64_t v = H.row(i)[q];
        for (int bit = 0; bit < 64; ++bit)
          if ((v >> bit) & 1ull) A.flip(i, q * 64 + bit);
      }
      A.flip(i, NQ + i);
    }
    const std::vector<int32_t> piv = NC > 0 ? rref(A, NQ) : std::vector<int32_t>();
    plan.gen_rank = (int32_t)piv.size();
    plan.check_words = std::max(1, (NC + 63) / 64);
    plan.gen_rows.assign((size_t)(NC + 1) * plan.check_words, 0ull);
    for (int32_t i = 0; i < NC; ++i)
      for (int32_t c = 0; c < NC; ++c)
        if (A.get(i, NQ + c)) plan.gen_rows[(size_t)i * plan.check_words + c / 64] ^= 1ull << (c % 64);
    uint64_t* cls = &plan.gen_rows[(size_t)NC * plan.check_words];
    for (int32_t i = 0; i < plan.gen_rank; ++i) {
      plan.gen_col.push_back(col[piv[i]]);
      if (zb[piv[i]])
        for (int32_t q = 0; q < plan.check_words; ++q) cls[q] ^= plan.gen_rows[(size_t)i * plan.check_words + q];
    }
    plan.gen_xbar.assign(NQ, 0);
    for (int32_t j = 0; j < NQ; ++j) plan.gen_xbar[col[j]] = xb[j];
    plan.gen_qcol = col;
  }
  return emit_plan(ns, opt, plan, err);
}

}  // namespace td
