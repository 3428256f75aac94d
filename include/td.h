/*
 * td.h -- tensor-network coset decoding of 3D codes on one GB300 (sm_103a).
 *
 * C ABI of libtd.so.  The problem statement is the detector error model (DEM) of Sec. 2.4
 * of "Tensor Network Decoding Beyond 2D" (Piveteau, Chubb, Renes; arXiv 2310.10722):
 * n mechanisms, each occurring independently with probability p_j and flipping the
 * detectors of column j of H and the logical observables of column j of l.  For an
 * observed detector outcome m the library returns, for every class L,
 *
 *     log p_{m,L},   p_{m,L} = sum_{x : Hx = m, l.x = L} prod_j p_j^{x_j} (1-p_j)^{1-x_j}
 *
 * (Sec. 2.4), evaluated approximately by the contraction of Sec. 4: the detector network
 * (Sec. 3.1, 3.4) is swept layer by layer with a PEPS boundary whose bonds are truncated
 * to chi by simple update after every gate, and the final 2D network is contracted by an
 * MPS of bond chi_mps.  With chi and chi_mps at least the untruncated bond dimensions the
 * result is exact.  The decision is argmax_L p_{m,L} (Sec. 2.4, L*(m)).
 *
 * Conventions common to every call
 *   - Host pointers: DEM and layout arrays (read during td_build_network only; the
 *     library keeps its own copy).  Device pointers: per-shot inputs and outputs of the
 *     decoding calls; they must be CUDA device memory of the current device.
 *   - Ownership: the caller owns every buffer it passes.  The library owns the opaque
 *     td_network and its device workspace (allocated by td_build_network, freed by
 *     td_free_network).
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Decoding calls
 *     enqueue their work on it and return without synchronising, except the *_host
 *     variants, which synchronise on it before returning.  A network is not thread safe:
 *     use one network per concurrent stream.
 *   - Errors: every call returns a td_status; td_last_error() describes the last failure
 *     of the calling thread.  Argument errors are detected on the host before any work is
 *     enqueued.  No call aborts the process or throws across the ABI.
 */
#ifndef TD_H_
#define TD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TD_OK = 0,
  TD_ERR_INVALID = 1,      /* bad argument: shapes, bits not in {0,1}, p outside [0,1] */
  TD_ERR_NONLOCAL = 2,     /* a mechanism is not single-site, grid-bond or vertical */
  TD_ERR_OOM = 3,          /* device or host allocation failed */
  TD_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  TD_ERR_TIMEOUT = 5,      /* a bounded device wait gave up (reported by td_network_check) */
  TD_ERR_NUMERIC = 6,      /* a shot met a non-finite intermediate: its logp is NaN, the batch
                              completes (reported by td_network_check) */
  TD_ERR_UNSUPPORTED = 7   /* valid input outside what this build implements */
} td_status;

typedef enum {
  TD_FP64 = 0,   /* the plain FP64 GPU path: FP64 storage and arithmetic on the CUDA cores
                    everywhere, every SVD an FP64 one-sided Jacobi */
  TD_FP32 = 1,   /* mixed precision with FP32 storage of the site tensors: the Gram pass on
                    the tcgen05 tensor cores (below), the update and site operators in FP64
                    arithmetic, every SVD (truncation cores, zip-up cuts) FP32-preconditioned
                    and finished by FP64 Jacobi sweeps, the final contraction and log-sum in
                    FP64 */
  TD_TC = 2      /* mixed precision with FP64 storage (the headline mixed path): as TD_FP32,
                    with the site tensors kept in FP64 */
  /* The tensor-core Gram (bond dimensions 4..16; others use the FP64 CUDA-core Gram): each
   * value of the Gram's operands is cut into eight exact integer BF16 slices below a
   * per-column power-of-two bound (7 bits each from FP64 storage, 56 bits; 6 bits of an
   * exact FP32 pair from FP32 storage, 48 bits), slice products are summed exactly in FP32
   * (TMEM) over at most 1024 rows and combined in FP64. */
} td_precision;

/* DEM triple (H, p, l) of Sec. 2.4, host memory, CSR by rows. */
typedef struct {
  int32_t n_det;             /* detectors (rows of H) */
  int32_t n_mech;            /* error mechanisms (columns of H) */
  int32_t n_obs;             /* logical observables (rows of l); this build supports 1 */
  const int32_t* H_indptr;   /* [n_det + 1] */
  const int32_t* H_indices;  /* [H_indptr[n_det]] mechanism indices of each detector */
  const int32_t* L_indptr;   /* [n_obs + 1] */
  const int32_t* L_indices;  /* [L_indptr[n_obs]] mechanism indices of each observable */
  const double* p;           /* [n_mech], each in [0, 1] */
} td_dem;

/* Space-time layout: integer coordinates (x, y, t) of every detector, host memory,
 * [n_det][3] row-major.  t is the layer (sweep direction, Sec. 4), (x, y) the site of a
 * 2D grid.  Every occupied (x, y) must hold exactly one detector in every layer. */
typedef struct {
  const int32_t* det_xyt;
} td_layout;

typedef struct {
  int32_t chi;             /* simple-update bond cap (Sec. 4; chi_SU of Sec. 5) */
  int32_t chi_mps;         /* final boundary-MPS bond cap (chi_MPS of Sec. 5) */
  int32_t precision;       /* td_precision */
  int32_t ckpt_stride;     /* td_grad_logprob: layers per checkpoint segment of the reverse sweep
                              (<= 0 or >= the layer count: one segment, every intermediate tensor
                              kept).  With k < T, only one segment's intermediate tensors are kept
                              and the tensors at every segment start are checkpointed; each
                              segment but the last is swept forward again from its checkpoint
                              before its reverse sweep.  The gradient is identical either way. */
  double svd_cutoff;       /* keep singular values s_i > svd_cutoff * s_1 */
  double multiplet_rtol;   /* a cut inside s_k - s_{k+1} <= rtol * s_1 drops the multiplet */
  double gram_cutoff;      /* drop Gram eigen-directions below gram_cutoff * max eigenvalue;
                              negative: 1e-15 */
  size_t mem_budget;       /* device workspace cap in bytes (0: 16 GiB) */
  int32_t max_wave;        /* shots processed per wave (0: as many as mem_budget allows) */
} td_options;

typedef struct td_network td_network;

typedef struct {
  int32_t n_sites, n_layers, n_bonds, n_gates, n_counter_sites;
  int32_t nx, ny;
  int32_t wave;              /* shots per wave */
  int32_t chi, chi_mps, precision;
  int32_t offset_all;        /* 1 if the observable was replaced by l + sum of rows of H */
  int32_t generator;         /* 1 for a generator network (td_build_gen_network) */
  size_t workspace_bytes;    /* device bytes held by the network */
  int64_t launches_per_wave; /* kernel launches enqueued per wave */
} td_network_info;

/* Fill `opt` with defaults: chi 8, chi_mps 16, TD_FP64, svd_cutoff 1e-12,
 * multiplet_rtol 1e-8, gram_cutoff -1 (per precision), mem_budget 16 GiB. */
void td_default_options(td_options* opt);

/* Build the layered network of the DEM (Sec. 3.4 detector network in the layered form of
 * Sec. 4; Sec. 2.4 merging of mechanisms with identical detectors and class effect) and
 * allocate its device workspace.  Errors: TD_ERR_INVALID (shapes, ranges),
 * TD_ERR_NONLOCAL (a two-detector mechanism whose detectors are neither grid neighbours
 * in one layer nor one site in consecutive layers, or a mechanism with > 2 detectors),
 * TD_ERR_UNSUPPORTED (n_obs != 1, chi > 32, missing detector at some (site, layer)),
 * TD_ERR_OOM, TD_ERR_CUDA.  On success *out owns the network. */
td_status td_build_network(const td_dem* dem, const td_layout* layout, const td_options* opt,
                           td_network** out);

/* Coset log-probabilities (Sec. 2.4 p_{m,L}; Sec. 4 contraction).
 * det_dev: device uint8 [B][n_det], each 0 or 1 (detector outcomes m).
 * logp_dev: device double [B][2^n_obs]; logp_dev[b][L] = log p_{m_b, L} (-inf if zero).
 * B >= 0 (B = 0 is a no-op).  Asynchronous on `stream`. */
td_status td_coset_logprob(td_network* net, const uint8_t* det_dev, int64_t B, double* logp_dev,
                           void* stream);

/* td_coset_logprob with truncation statistics per shot (a property of this library; the
 * paper reports none): stats_dev, device double [B][4], receives for shot b
 *   [b][0], [b][1]: the largest and the sum over the simple-update truncations (Sec. 4) of
 *                   the discarded fraction sum_{i >= k} s_i^2 / sum_i s_i^2 of the bond's
 *                   singular values s (the squared Frobenius error of that truncation relative
 *                   to the squared norm of the two-site tensor under the bond's environment);
 *   [b][2], [b][3]: the same over the cuts of the final boundary-MPS contraction.
 * Zero where nothing was truncated (values below svd_cutoff * s_1 dropped count, ~1e-24).
 * Overwrites stats_dev[0 .. B); logp_dev as td_coset_logprob.  Asynchronous on `stream`. */
td_status td_coset_logprob_stats(td_network* net, const uint8_t* det_dev, int64_t B, double* logp_dev,
                                 double* stats_dev, void* stream);

/* Decisions L*(m) = argmax_L p_{m,L} (Sec. 2.4; ties -> lowest L) and margins
 * log p_{m,L*} - max_{L != L*} log p_{m,L}.  decision_dev: device int32 [B];
 * margin_dev: device double [B] or NULL.  Asynchronous on `stream`. */
td_status td_decode(td_network* net, const uint8_t* det_dev, int64_t B, int32_t* decision_dev,
                    double* margin_dev, void* stream);

/* td_coset_logprob with host buffers: det_host uint8 [B][n_det] and logp_host double
 * [B][2^n_obs] in host memory (pinned memory gives asynchronous copies).  Copies in, runs
 * and copies out on `stream` in waves; synchronises before returning. */
td_status td_coset_logprob_host(td_network* net, const uint8_t* det_host, int64_t B,
                                double* logp_host, void* stream);

/* td_coset_logprob for callers that cannot call cudaMalloc or cudaFree around a decode --
 * for example code that runs where device memory is fixed up front and no allocator may be
 * called.  This call allocates nothing: the scratch of the final 2D contraction is a
 * file-scope static device array of 64 MiB instead of the network's workspace (the paper
 * has no counterpart; it is a property of this library).  Arguments and results are those
 * of td_coset_logprob.  B may not exceed min(wave, 64 MiB / final-contraction scratch per
 * shot); a larger B returns TD_ERR_INVALID with the capacity in td_last_error().
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current: make that first call before any stream capture.  Every call
 * on a device shares the one array and leaves its contents behind (nothing in it needs to
 * start at zero): calls whose work overlaps on the GPU -- on different streams, or from
 * different threads -- race on it and must be serialised by the caller.  Every GPU that
 * loads the library holds the array until the process exits.  The looked-up address is
 * kept for the life of the process: after cudaDeviceReset on a device it is stale, so do
 * not use this call on that device again in the same process.  Kernel timing
 * (td_network_profile) records none of this call's launches (it would create events). */
td_status td_coset_logprob_static(td_network* net, const uint8_t* det_dev, int64_t B, double* logp_dev,
                                  void* stream);

/* Gradient of the mean total log-probability (1/B) sum_b log P(m_b), P(m) = sum_L p_{m,L}
 * (Sec. 2.4), with respect to every mechanism rate, by a reverse sweep (the paper has no
 * gradient).  The value differentiated is the decoder's own log P: the Sec. 4 sweep at the
 * network's chi and chi_mps, truncations included, so the gradient is consistent with the
 * values (central differences of td_coset_logprob agree while no truncation decision
 * changes; without truncation it is the exact gradient).
 *
 * The call runs the forward sweep once more in FP64 (whatever the network's precision)
 * with the intermediate site tensors of one segment of ckpt_stride layers kept (the inputs of
 * every segment checkpointed, earlier segments recomputed from them) and every truncation
 * core and zip-up cut recorded, then walks it backwards, one block of threads per shot: the adjoint of each
 * truncated SVD (the thin SVD over the nonzero singular values), of the kappa-basis
 * doubling of each gate, of the environment weights and of the site-local operators.  Its
 * result is the adjoint of every parameter object (site-local matrix, gate rate, readout),
 * summed over shots and mapped to the rates on the host through the objects' exact
 * dependence on each rate (each object is affine in each rate).  Mechanisms without
 * detectors only mix the classes and get 0; a shot whose P comes out 0 contributes nothing
 * (the mean still divides by B).
 *
 * det_dev: device uint8 [B][n_det]; p_dev: device double [n_mech] rates in [0, 1], or
 * NULL for the network's current rates.  A p_dev different from the current rates must
 * keep the network's structure (TD_ERR_INVALID otherwise) and becomes the network's rates
 * for this and later calls.  logP_dev: device double [B] (log P of each shot at the rates,
 * from the FP64 sweep); grad_dev: device double [n_mech].
 * Memory: beside the decoding workspace, the recording of up to min(wave, B, mem_budget /
 * per-shot record) shots -- one segment's intermediate tensors and cores, the checkpoints,
 * the final contraction's record -- allocated by the first call and grown by a later call
 * with a larger B; a B above mem_budget / per-shot record runs in several waves.  The
 * call synchronises `stream` (the objects' dependence on the rates is built on the host,
 * and the per-shot adjoints are summed there) and returns when the results are written.
 * Errors: TD_ERR_INVALID (null buffers, rates outside [0, 1]), TD_ERR_OOM, TD_ERR_CUDA. */
td_status td_grad_logprob(td_network* net, const uint8_t* det_dev, int64_t B, const double* p_dev,
                          double* logP_dev, double* grad_dev, void* stream);

/* The same gradient by the affine identity d log P / d p_j = (P_{x_j=1} - P_{x_j=0}) / P, with
 * P_{x_j=x} the network with p_j set to x and each of the three values from the decoder
 * (at the network's chi, chi_mps and precision): B * (1 + 2 n_forced) decodes, batched as
 * virtual shots that each replace one parameter object.  Without truncation it equals
 * td_grad_logprob (both are exact); with truncation it differs from it by the truncation
 * error of the forced networks.  Arguments, rates and errors as td_grad_logprob
 * (TD_ERR_INVALID also when B * (1 + 2 n_forced) >= 2^31); the decodes are queued on
 * `stream` and the call returns without waiting for them. */
td_status td_grad_logprob_forced(td_network* net, const uint8_t* det_dev, int64_t B, const double* p_dev,
                                 double* logP_dev, double* grad_dev, void* stream);

/* ---- Generator networks (Sec. 3.2; the loop sector of Sec. 5.2) ------------------------
 *
 * A CSS sector decoded in the generator picture: qubit j flips independently with rate p_j,
 * n_checks checks (the rows of H) observe the flips, and n_gen stabilizer generators of the
 * other type span the errors equivalent to none -- generator v flips the qubits that name it.
 * For a syndrome m, the class-L coset probability is
 *     p_{m,L} = sum over x with H x = m and (x . zbar) = L of prod_j p_j^{x_j} (1-p_j)^{1-x_j}
 * (Sec. 2.4 with the observable zbar), computed as the coset sum of Sec. 3.2: with r a
 * representative of m, p(coset of r) = sum over s in {0,1}^{n_gen} of
 * prod_j w_j(r_j + sum_{v flipping j} s_v), w_j = (1 - p_j, p_j), divided by 2^(n_gen - rank)
 * when the generators are dependent; the classes are the cosets of r and r + xbar.  The
 * network has one weight per qubit between the generators it touches and is contracted as
 * in Sec. 4: a PEPS over the generators of one layer (physical leg = the generator's bit),
 * swept along t; in-layer qubits are the diagonal two-site gates diag(w(r + s_a + s_b)),
 * each followed by the simple-update truncation to chi; the final 2D network by the boundary
 * MPS (chi_mps).  Nonnegative throughout: the class is carried by the representative.
 *
 * Representative: r is the error supported on the greedy column basis of H (columns in qubit
 * order, a column kept when it is independent of those kept before it) with H r = m; it is
 * unique and computed on the device from a GF(2) elimination done at build time.  A truncated
 * contraction depends on the representative; this rule fixes it.
 *
 * Geometry: gen_xyt places every generator at (x, y, t); every occupied (x, y) holds one
 * generator in every layer t = 0 .. T-1.  A qubit names one or two generators: two in one
 * layer at grid neighbours (an in-layer edge), two at one (x, y) in consecutive layers (a
 * vertical edge), or one (a dangling edge).  Every generator of layer t > 0 has exactly one
 * vertical edge from layer t-1; every generator of layer 0 one dangling edge below and every
 * generator of layer T-1 one dangling edge above (in qubit order, a layer-0 generator's first
 * dangling edge is the one below).  Other geometries are TD_ERR_UNSUPPORTED. */
typedef struct {
  int32_t n_gen;               /* stabilizer generators of the other type (vertices) */
  int32_t n_qubits;            /* qubits (edges) */
  int32_t n_checks;            /* checks (rows of H; the syndrome's length) */
  const int32_t* qubit_gens;   /* [n_qubits][2] generators flipping each qubit; [j][1] = -1 for a
                                  dangling edge */
  const double* p;             /* [n_qubits] flip rates, each in [0, 1] */
  const int32_t* gen_xyt;      /* [n_gen][3] (x, y, t) of every generator */
  const int32_t* check_indptr; /* [n_checks + 1] CSR of H by rows */
  const int32_t* check_indices;/* qubit indices of each check */
  int32_t n_xbar;              /* xbar: a logical of the flipped type (H xbar = 0, not a sum of */
  const int32_t* xbar;         /*   generators): qubit indices */
  int32_t n_zbar;              /* zbar: its conjugate logical (even overlap with every generator, */
  const int32_t* zbar;         /*   odd with xbar): qubit indices; the class of x is x . zbar */
} td_gen;

/* Build the generator network of `gen` (host arrays, copied) and allocate its workspace.
 * The decoding calls of a generator network are td_gen_coset_logprob and td_gen_decode;
 * the detector-network calls (td_coset_logprob and its variants, the gradients, the tuner and
 * td_debug_sweep) return TD_ERR_INVALID on it.  Errors: TD_ERR_INVALID (shapes, ranges, p
 * outside [0, 1], a generator that anticommutes with a check -- H g_v != 0 --, xbar with a
 * syndrome, zbar that anticommutes with a generator or commutes with xbar),
 * TD_ERR_UNSUPPORTED (the geometry rules above, chi > 32), TD_ERR_OOM, TD_ERR_CUDA. */
td_status td_build_gen_network(const td_gen* gen, const td_options* opt, td_network** out);

/* Coset log-probabilities of a generator network.  syn_dev: device uint8 [B][n_checks], each
 * 0 or 1.  logp_dev: device double [B][2]; logp_dev[b][L] = log p_{m_b, L}; both -inf when
 * m_b is not a syndrome (no error has it).  Each shot is two sweeps (r and r + xbar), run as
 * two rows of the network's waves.  B >= 0.  Asynchronous on `stream`. */
td_status td_gen_coset_logprob(td_network* net, const uint8_t* syn_dev, int64_t B, double* logp_dev, void* stream);

/* Decisions argmax_L p_{m,L} (ties -> 0) and margins of a generator network (as td_decode).
 * decision_dev: device int32 [B]; margin_dev: device double [B] or NULL. */
td_status td_gen_decode(td_network* net, const uint8_t* syn_dev, int64_t B, int32_t* decision_dev,
                        double* margin_dev, void* stream);

/* Diagnostic, no device involved (a property of this library): plan the generator network of
 * `gen` on the host and evaluate, for each syndrome of syn_host (uint8 [B][n_checks]), the rows
 * the decoding calls sweep -- rows_host (uint8 [2B][n_qubits]): row 2b = the representative r
 * of syndrome b in the network's column order, row 2b + 1 = r + xbar -- and cls_host (int32 [B]):
 * the class r . zbar, or -1 when syndrome b is not a syndrome.  col_host (int32 [n_qubits], or
 * NULL) receives the column of every qubit: column t * S + s for the edge entering generator
 * (site s, layer t) from below (layer T: the dangling edge above the last layer; sites in
 * (y, x) order), then the in-layer edges in qubit order.  Errors as td_build_gen_network. */
td_status td_gen_rows_host(const td_gen* gen, const uint8_t* syn_host, int64_t B, uint8_t* rows_host,
                           int32_t* cls_host, int32_t* col_host);

/* Launch schedule of the network (a property of this library; the paper has none): the
 * block size of the final contraction's kernel (256, 512 or 1024 threads; the Jacobi lane
 * groups and the work region's layout follow it), whether that kernel's work region may sit
 * in shared memory (final_smem != 0: when it fits; 0: global memory, cached in L1, which
 * leaves room for more blocks per SM), and the rows per job of the Gram and update passes
 * (512, 1024, 2048 or 4096).  Results do not depend on the schedule beyond rounding (the
 * Gram's partial sums and the Jacobi rotations are grouped differently).
 * td_network_set_schedule sets it; TD_ERR_INVALID for other values. */
td_status td_network_set_schedule(td_network* net, int32_t final_threads, int32_t final_smem, int32_t chunk_rows);

/* Autotuner: times decodes of the first min(B, wave) shots of det_dev (device uint8
 * [B][n_det]) under the schedule candidates -- the final contraction's block size and work-
 * region placement at the current chunk size, then the chunk size at the best of those (two
 * decodes per candidate, the second timed with CUDA events on `stream`) -- and keeps the
 * fastest.  Writes the chosen values (final_smem: 1 if the work region is in shared memory)
 * and the best time (ms); each pointer may be NULL.  Synchronous.  Errors as
 * td_coset_logprob; TD_ERR_INVALID for B < 1. */
td_status td_network_tune(td_network* net, const uint8_t* det_dev, int64_t B, int32_t* final_threads,
                          int32_t* final_smem, int32_t* chunk_rows, double* ms_best, void* stream);

td_status td_network_get_info(const td_network* net, td_network_info* info);

/* Device status of the network's kernels (a property of this library): synchronises
 * `stream`, then returns and clears the status that a kernel recorded since the last check
 * -- TD_ERR_TIMEOUT when a tensor-core kernel's bounded wait for its MMAs gave up (its
 * results of that call are not valid), TD_ERR_NUMERIC when a shot met a non-finite
 * intermediate (that shot's log-probabilities are NaN, the others are valid) -- or TD_OK.
 * td_coset_logprob_host checks it too. */
td_status td_network_check(td_network* net, void* stream);

/* Diagnostic: run the sweep of Sec. 4 on the first min(B, wave) shots up to the end of the
 * gate round that contains gate n_gates-1 (site-local operators of a layer run before its
 * first round), then copy the bond weights and the log-scale accumulators.
 * lam_dev: device double [B][n_bonds][chi] (lambda of each bond, zero padded; bonds in
 * the order of their (site a, site b) pairs, sites ordered by (y, x));
 * logacc_dev: device double [B][n_sites + n_bonds + 1] or NULL.  Returns the number of
 * gates applied in *applied.  Asynchronous on `stream`. */
td_status td_debug_sweep(td_network* net, const uint8_t* det_dev, int64_t B, int32_t n_gates, double* lam_dev,
                         double* logacc_dev, int32_t* applied, void* stream);

/* Kernel classes timed by td_network_profile. */
typedef enum {
  TD_K_INIT = 0, TD_K_LOCAL = 1, TD_K_GRAM = 2, TD_K_PRE = 3, TD_K_CORE = 4, TD_K_UPDATE = 5,
  TD_K_FINAL = 6, TD_K_FINALIZE = 7, TD_K_COUNT = 8
} td_kernel_class;

/* Kernel timing with CUDA events recorded on the call's stream around every launch.
 * enable = 1 starts recording (and clears earlier records), 0 stops.  With ms and
 * launches non-NULL (arrays of TD_K_COUNT), synchronises the recorded events and writes,
 * per kernel class, the summed device time in milliseconds and the number of launches
 * since recording started. */
td_status td_network_profile(td_network* net, int32_t enable, double* ms, int64_t* launches);

/* Algorithmic work per shot of one decoding call, per kernel class (arrays of TD_K_COUNT),
 * from the network's static bond dimensions (an upper bound where truncation keeps fewer):
 * bytes = minimum device-memory traffic (each tensor a kernel must read or write, once);
 * flops = multiply-adds x 2 of the contractions, plus textbook counts for the dense
 * factorisations (symmetric eigensolver with vectors 9n^3; SVD of m x n, m >= n, with both
 * factors 4m^2 n + 8m n^2 + 9n^3 in the truncation cores; the zip-up cuts need the singular
 * values and the left factor only: 6m n^2 + 11n^3, or 2n m^2 + 11m^3 for m < n).  fp64_flops = the part of flops done in FP64. */
td_status td_network_get_work(const td_network* net, double* bytes, double* flops, double* fp64_flops);

/* Measurement helper for roofline denominators (no counterpart in the paper): the fused
 * multiply-add throughput of the current GPU's CUDA cores in FP64 (fp64 != 0) or FP32, in
 * TFLOP/s (2 flops per FMA), from one timed launch (CUDA events on `stream`) of eight
 * independent FMA chains of `iters` steps per thread, eight 256-thread blocks per SM, after
 * an untimed one.  Synchronous; allocates a small output buffer.  Errors: TD_ERR_INVALID
 * (null tflops, iters < 1), TD_ERR_CUDA. */
td_status td_measure_fma_peak(int32_t fp64, int32_t iters, double* tflops, void* stream);

/* Release the network and its device workspace (NULL is a no-op).  The caller must
 * ensure no enqueued work still uses it. */
void td_free_network(td_network* net);

/* Message of the last failed call on this thread ("" if none). */
const char* td_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TD_H_ */
