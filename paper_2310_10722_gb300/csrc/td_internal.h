// Internal data structures shared by the host planner and the CUDA kernels.
//
// The network plan is the layered detector network of Sec. 3.4 / Sec. 4 for a graph-like
// DEM: sites are the (x, y) positions of one layer, the boundary state is a PEPS with one
// physical leg per site (the bit of the vertical mechanism entering the layer, plus a class
// counter bit on counter sites), and each layer is absorbed as site-local matrices and
// two-site gates (1-p) I x I + p X x X on grid bonds, each followed by a simple-update
// truncation of its bond to chi.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/td.h"

namespace td {

constexpr int kMaxChi = 32;      // simple-update bond cap supported by the kernels
constexpr int kMaxBonds = 4;     // grid sites have at most 4 bonds
constexpr int kMaxPhys = 4;      // physical leg: vertical bit x class counter bit
constexpr int kMaxGridX = 64;    // grid width (sites per row) of the final contraction
constexpr int kMaxFinalBond = 1024;   // chi_mps x largest final bond dimension

// One endpoint of a gate: the site tensor is stored as [phys][d_0]...[d_{nb-1}] (row
// major, bonds ordered left, right, down, up) and viewed as [phys][outer][D][inner]
// around the active bond at position `pos`.
struct SideDesc {
  int32_t site;
  int32_t P;            // physical dimension (2 or 4)
  int32_t mask;         // physical index flip of the gate's X on this side (1 or 3)
  int32_t nb;           // bonds of the site
  int32_t pos;          // position of the active bond
  int32_t dims[kMaxBonds];   // current bond dimensions (before the gate)
  int32_t bond[kMaxBonds];   // global bond ids (lambda lookup)
  int32_t outer, inner; // product of dims before / after `pos`
  int64_t in_off;       // element offset of the current tensor in a shot block
  int64_t out_off;      // element offset of the updated tensor in a shot block
};

struct GateDesc {
  SideDesc side[2];
  int32_t bond;
  int32_t D, Dn;        // active bond dimension before / after
  double p;             // mechanism probability
  // 0: the gate (1-p) I x I + p X x X of the detector picture; 1: the diagonal gate
  // diag(w(r + s_a + s_b)), w = (1-p, p), of the generator picture (Sec. 3.2) with the bit r
  // read from column rcol of the shot's detector row
  int32_t diag, rcol;
};

// Site-local operator applied at the start of a layer: psi <- X^{m} K psi on the
// physical leg (K = this layer's single-detector mechanisms times the previous layer's
// vertical weights), then rescaled by its largest magnitude.
struct LocalDesc {
  int32_t P;
  int32_t det;          // detector index of (site, layer): its bit flips phys bit 0
  int32_t rest;         // product of the site's current bond dims
  int32_t pad;
  int64_t off;          // element offset of the current tensor in a shot block
  int64_t out_off;      // where the result goes (== off: in place)
  double K[kMaxPhys * kMaxPhys];
};

// Final readout of one site for the 2D contraction: F[c][l][r][d][u] =
// sum_phys R[phys][c] Gamma[phys][bonds] * prod sqrt(lambda).
struct FinalSite {
  int32_t P;
  int32_t nb;
  int32_t dir_dim[4];   // dimension per direction (left, right, down, up); 1 if absent
  int32_t dir_pos[4];   // position of that direction's bond in the site tensor, -1 if absent
  int32_t dir_bond[4];  // global bond id per direction, -1 if absent
  int64_t off;          // element offset of the final tensor in a shot block
  double R[kMaxPhys * 2];
};

// Parameter override of the gradient pass.  The network is affine in every mechanism rate,
// and the rate of one mechanism enters exactly one parameter object: a site-local matrix K
// (single-detector mechanisms of layers < T-1, vertical mechanisms), a gate's p (two-
// detector mechanisms of one layer) or a site's readout R (single-detector mechanisms of
// the last layer).  A virtual shot decodes the detector bits of shot `base` with at most
// one object replaced by its value at p_j = 0 or 1.
enum { kOvrNone = 0, kOvrLocal = 1, kOvrGate = 2, kOvrRead = 3 };
struct Override {
  int32_t kind;
  int32_t target;       // local: layer * S + site; gate: global gate index; readout: site
  double val[kMaxPhys * kMaxPhys];   // K (P x P), p (val[0]) or R (P x 2), row major
};
struct VShot {
  int32_t base;         // row of the detector buffer
  int32_t ovr;          // index into the override table (entry 0: no override)
};

struct Round {             // gates on disjoint bonds, run as one batch
  int32_t first, count;    // range in the gate descriptor array
  int32_t maxD, maxDn;
  int32_t max_rows;        // max over sides of (P/2) * outer * inner
};

struct LayerPlan {
  int32_t local_first;     // S local descriptors
  std::vector<Round> rounds;
};

struct Plan {
  int32_t n_det = 0, n_mech = 0, n_obs = 0;
  int32_t nx = 0, ny = 0, T = 0, S = 0;
  int32_t chi = 8, chi_mps = 16, precision = TD_FP64;
  double svd_cutoff = 1e-12, multiplet_rtol = 1e-8, gram_cutoff = 1e-13;
  std::vector<int32_t> site_x, site_y;
  std::vector<int32_t> grid_site;        // [ny*nx] -> site or -1
  std::vector<int32_t> P;                // per site
  int32_t n_counter_sites = 0;
  int32_t offset_all = 0;                // class offset = parity of all detector bits
  double glob_mix[4] = {1, 0, 0, 1};     // class mixing by mechanisms with no detectors
  std::vector<std::pair<int32_t, int32_t>> bond_sites;
  int32_t n_bonds = 0;
  std::vector<GateDesc> gates;
  std::vector<LocalDesc> locals;
  std::vector<LayerPlan> layers;
  std::vector<FinalSite> finals;
  std::vector<int32_t> final_dims;       // per bond, dimension after the sweep
  int64_t shot_elems = 0;                // PEPS elements per shot (both buffers of all sites)
  int32_t max_round_gates = 0;
  int32_t max_final_D = 1;               // largest bond after the sweep
  // Versioned layout of the reverse sweep: the same schedule with every site-local
  // operator and every gate writing a new copy of its site tensors, so that every
  // intermediate tensor of one segment of ckpt_stride layers is kept (hist_shot_elems per
  // shot: the largest segment).  Offsets are relative to the segment, whose first slots hold
  // its input versions; the input tensors of segments 1.. are checkpointed (ckpt_off, with
  // the bond weights at ckpt_lam_off; ckpt_shot_elems per shot) and the segment recomputed.
  std::vector<LocalDesc> hist_locals;    // off = input version, out_off = output version
  std::vector<GateDesc> hist_gates;      // in_off / out_off = versions
  std::vector<FinalSite> hist_finals;    // off = last version (in the last segment)
  int64_t hist_shot_elems = 0;
  int32_t ckpt_stride = 1;
  std::vector<int32_t> seg_first_layer;  // [nseg + 1]
  std::vector<int32_t> seg_first_gate;   // [nseg + 1]
  std::vector<int64_t> seg_in_off;       // [nseg][S] input versions of the segment
  std::vector<int64_t> seg_out_off;      // [nseg][S] output versions of the segment
  std::vector<int64_t> seg_in_elems;     // [nseg][S] sizes of the input versions
  std::vector<int64_t> ckpt_off;         // [nseg][S] checkpointed input tensors (segments >= 1)
  std::vector<int64_t> ckpt_lam_off;     // [nseg] checkpointed bond weights (segments >= 1)
  int64_t ckpt_shot_elems = 0;
  int64_t max_site_elems = 0;            // largest site tensor of the sweep (elements)
  // Generator network (Sec. 3.2, built by build_gen_plan): a row of the sweep's detector
  // buffer is a representative error r in column order (the edge entering each (site, layer)
  // from below at t * S + site, then the in-layer edges); n_det = n_qubits is the row length.
  // The representative of a syndrome m is linear in m: bit i < gen_rank of the elimination
  // transform gives r at column gen_col[i] (r is zero elsewhere), the bits rank <= i <
  // n_checks vanish exactly when m is a syndrome, the last row gives the class of r.
  int32_t gen = 0;
  int32_t n_checks = 0, n_qubits = 0, n_gen = 0, gen_rank = 0, check_words = 0;
  std::vector<uint64_t> gen_rows;        // [n_checks + 1][check_words]
  std::vector<int32_t> gen_col;          // [gen_rank]
  std::vector<uint8_t> gen_xbar;         // [n_qubits] xbar in column order
  std::vector<int32_t> gen_qcol;         // [n_qubits] column of every qubit
  double gen_log_offset = 0.0;           // -(n_gen - rank of the generators) ln 2
};

// Build the plan from the ABI structures.  Returns TD_OK or an error with `err` set.
td_status build_plan(const td_dem& dem, const td_layout& layout, const td_options& opt, Plan& plan,
                     std::string& err);
// Build the generator network of a CSS sector (td_gen, Sec. 3.2).
td_status build_gen_plan(const td_gen& gen, const td_options& opt, Plan& plan, std::string& err);

}  // namespace td
