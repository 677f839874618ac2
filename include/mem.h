/* mem.h -- C ABI of the GB300 matrix-element-method integrator (libmem.so).
 *
 * The library computes, for each collision event X, the matrix-element-method
 * probability density of Sec. 1 of arXiv:1407.7595 (Eq. "mem_def" convolved
 * with the transfer functions as in the p_hat equation that follows it, and in
 * the form of Eq. "integrand" of Sec. 3):
 *
 *   p_hat(X) = (1/N_perm) sum_perm int dY  sum_flavour |M|^2(Y) f1(x1) f2(x2)
 *              / (|q1||q2|) dPhi_n(q1+q2; Y) T(X|Y)
 *
 * as a Monte Carlo integral (Sec. 2, Eq. "sum", with its error estimate) over
 * the unmeasured degrees of freedom, importance-sampled with a VEGAS grid
 * (Sec. 2) that is refined on the device. Every integrand evaluation runs in
 * hand-written sm_103a CUDA; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Every call returns a mem_status; on failure mem_last_error() gives a
 *    thread-local message. Per-event problems go to ev_status and do not fail
 *    the call.
 *  - Handles (mem_process, mem_events) are owned by the library; release them
 *    with mem_destroy. Arrays passed in are owned by the caller.
 *  - Output arrays may be host or device memory (detected per pointer). With
 *    device outputs the call is asynchronous on `stream`; with host outputs
 *    it synchronises `stream` before returning.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Work runs on the CUDA device current on the calling thread.
 */
#ifndef MEM_H
#define MEM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MEM_OK = 0,
  MEM_ERR_INVALID_ARG = 1, /* a pointer, size or descriptor field is invalid */
  MEM_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  MEM_ERR_OOM = 3,         /* device allocation failed */
  MEM_ERR_NONFINITE = 4,   /* per event: some integrand values were not finite */
  MEM_NOT_CONVERGED = 5,   /* per event: the point cap was reached before the target */
  MEM_ERR_TIMEOUT = 6      /* a bounded device wait ran out */
} mem_status;

/* Processes (the |M|^2 of Eq. "mem_def"). */
enum {
  MEM_PROC_DY = 0,    /* q qbar -> photon/Z -> mu- mu+ ; 2 integration dims, 1 permutation */
  MEM_PROC_W = 1,     /* u dbar -> W+ -> e+ nu (or W-) ; 4 dims, 1 permutation */
  MEM_PROC_TTBAR = 2, /* gg, q qbar -> t tbar -> b l+ nu bbar d ubar ; 7 dims, 24 jet permutations */
  MEM_PROC_TTBAR_DILEP = 3, /* gg, q qbar -> t tbar -> b l+ nu bbar mu- nubar (Sec. 3-4, Eq.
                            * "dilepsolv": both neutrinos from the four virtualities and the
                            * visible pT imbalance, up to 4 solutions per point); 6 dims, 2 b-jet
                            * assignments. Records: objects 0 l+ (kind 4), 1 mu- (kind 1), 2 and 3
                            * the b jets (kind 5); leptons and jet directions exact, jet energies
                            * with the double Gaussian. Fixed-budget, adaptive-budget and batched
                            * integration and mem_eval_points; the learned-sampler calls reject it. */
  MEM_PROC_TTH_DILEP = 4   /* gg, q qbar -> t tbar H -> (b l+ nu)(bbar mu- nubar)(b bbar) (Sec. 3-4,
                            * Eq. "integrand" with Eq. "mhsolve"): 8 dims (b, bbar energies, W and
                            * top virtualities, the Higgs pair's f = E1 + E2 and m_H^2), 12 jet
                            * assignments. Records: objects 0 l+ (kind 4), 1 mu- (kind 1), 2..5 the
                            * b jets (kind 5). Needs mh, wh, mb in the process description.
                            * mem_integrate (fixed or adaptive budget), mem_integrate_batch and
                            * mem_eval_points (mem_integrate_noalloc rejects it: its kernels
                            * raise the per-thread stack limit, which reserves device memory;
                            * the first call on a device does that set-up, so it should come
                            * before any stream capture). */,
  MEM_PROC_TTBB_DILEP = 5  /* gg, q qbar -> t tbar b bbar -> (b l+ nu)(bbar mu- nubar) b bbar, the
                            * background of Sec. 3-4: the variables and 12 jet assignments of
                            * MEM_PROC_TTH_DILEP with the extra pair's mass mapped uniformly (no
                            * resonance); the pair's jets enter as (b, bbar) and (bbar, b). Same
                            * records and entry points as MEM_PROC_TTH_DILEP; its kernels also
                            * keep the colour matrices in constant memory. */
};

typedef struct mem_process mem_process; /* opaque, library-owned */
typedef struct mem_events mem_events;   /* opaque, library-owned device copy of events */

/* Physics parameters of a process (Sec. 1: |M|^2, PDFs f1, f2; sigma_i := 1).
 * Energies in GeV. PDFs are f(x) = A x^a (1-x)^b for quark, antiquark, gluon. */
typedef struct {
  int32_t kind;       /* MEM_PROC_* */
  int32_t reserved;   /* must be 0 */
  double sqrt_s;      /* collider energy */
  double mz, wz, mw, ww, mt, wt; /* masses and widths */
  double alpha, sw2, alpha_s;    /* e^2/4pi, sin^2(theta_W), g_s^2/4pi */
  double pdf_A[3], pdf_a[3], pdf_b[3];
  double mh, wh, mb;  /* Higgs mass and width, b mass in the b Yukawa (MEM_PROC_TTH_DILEP only) */
} mem_process_desc;

/* Transfer functions T(X|Y) (Sec. 1): delta functions for all directions and
 * the ttbar lepton energy; Gaussian lepton energies N(x; E, lep_rel E)
 * integrated over +-window_k sigma; double-Gaussian jet energies
 * (1-w) N(x; E, core E) + w N(x; E, tail E) integrated over
 * [x/jet_lo_div, min(x jet_hi_mul, sqrt_s/2)]; Gaussian missing-pT resolution
 * met_sigma per component, neutrino pT integrated over MET +- met_box_k sigma. */
typedef struct {
  double lep_rel, window_k;
  double jet_core, jet_tail, jet_tail_w, jet_lo_div, jet_hi_mul;
  double met_sigma, met_box_k;
} mem_tf_desc;

/* Schedule of one process group in mem_integrate_batch, as chosen by
 * mem_autotune or by hand; a field left 0 takes the mem_opts value (or its
 * default). */
typedef struct {
  int32_t n_adapt_iters;  /* VEGAS adaptation iterations */
  int32_t tiles_per_cta;  /* sampling tiles per persistent CTA and round (0 = 4) */
  uint64_t adapt_points;  /* points per item per adaptation iteration */
  uint64_t min_points;    /* points per event of the first frozen-grid round */
} mem_plan;

/* Integration options (NULL = defaults: fixed n_points per event, 5 VEGAS
 * adaptation iterations of min(2^14, n/8) points, alpha = 1.5). */
typedef struct {
  double target_rel_err;  /* > 0: adaptive budget -- keep adding frozen-grid points
                             until err/prob <= target or max_points (per event);
                             mem_integrate then runs the mem_integrate_batch schedule */
  uint64_t max_points;    /* cap per event in adaptive mode (0 = 2^24) */
  uint64_t min_points;    /* minimum per event in adaptive mode (0 = n_points) */
  int32_t n_adapt_iters;  /* VEGAS adaptation iterations, excluded from the estimate */
  int32_t flow_guided;    /* mem_integrate_flow: 1 = the VEGAS judge's grid starts from one
                             refinement with the flow pilot's per-bin sums of w^2 instead of
                             the uniform grid; must be 0 for every other entry point */
  uint64_t adapt_points;  /* points per item per adaptation iteration (0 = min(2^14, n/8)) */
  double alpha;           /* grid compression exponent (0 = 1.5) */
  const double* grid_in;  /* optional HOST array d x 129: starting grid shared by all items */
  uint64_t event_id_base; /* Philox counter id of event 0 (for sharded runs) */
  void* phase_events;     /* optional array of 4 cudaEvent_t recorded on `stream` before the
                             adaptation kernel, before the frozen-grid kernel, before the
                             finalisation kernel and after it (phase timing); NULL = none */
  double flow_screen;     /* mem_integrate_flow: after the flow pilot round an item goes to
                             the VEGAS judge when its flow variance per point exceeds
                             flow_screen * (event estimate)^2 / n_perm, or when the event
                             estimate is not positive (0 = 1.0; < 0: every item is judged) */
  double flow_cost;       /* mem_integrate_flow: time of a flow point relative to a VEGAS
                             point; the judge keeps the flow when
                             var_flow * flow_cost <= var_vegas (0 = 1.0) */
  const mem_plan* plans;  /* mem_integrate_batch: optional HOST array, one schedule per
                             group (NULL = the fields above for every group) */
  int32_t strat_points;   /* fixed-budget mem_integrate: 0 = plain sampling on the frozen
                             grid; k in [2, 64] = stratified sampling (Sec. 4): the map's
                             input cube is divided into n_s^d equal hypercubes, n_s the
                             largest side with k n_s^d <= the frozen-grid budget, with k
                             points in each (Philox index = phase start + c k + j for
                             point j of hypercube c, whose coordinates are the base-n_s
                             digits of c, dimension 0 least significant); estimate = mean
                             of the per-cube means, variance = sum of the per-cube sample
                             variances / k, over (n_s^d)^2. n_used then counts the points
                             actually used. Must be 0 in the adaptive mode. */
  int32_t reserved1;      /* must be 0 */
} mem_opts;

/* Number of integration dimensions / jet permutations of a process kind (-1 if invalid). */
int32_t mem_process_dims(int32_t kind);
int32_t mem_process_nperm(int32_t kind);

/* Validate a process description and copy it into a library-owned handle.
 * Errors: MEM_ERR_INVALID_ARG (NULL pointers, unknown kind, non-positive
 * masses/widths/energy, reserved != 0). */
mem_status mem_create_process(const mem_process_desc* desc, mem_process** out);

/* Tabulated parton densities (Sec. 3: PDF values stored on (x, Q) grids per
 * flavour and evaluated by bilinear interpolation) in place of the parametric
 * set of the descriptor. `table` (host, caller-owned, copied): 3 x n_q x n_x
 * float32, table[(t * n_q + j) * n_x + i] = f_t(x_i, Q_j) for t = quark,
 * antiquark, gluon (the flavour classes of the parametric set), at the nodes
 * ln x_i = lnx_min + i (lnx_max - lnx_min) / (n_x - 1) and
 * ln Q_j = lnq_min + j (lnq_max - lnq_min) / (n_q - 1), Q in GeV. Every
 * integrand of the process then takes f(x, Q) by bilinear interpolation in
 * (ln x, ln Q) between the four nodes around the point, with the factorisation
 * scale Q = sqrt(x1 x2 s) (the partonic invariant mass); outside the table the
 * edge cell continues linearly, negative values become 0, and f = 0 unless
 * 0 < x < 1. table = NULL restores the parametric set. Synchronous; affects
 * calls made after it returns (mem_integrate_noalloc takes a descriptor and
 * always uses the parametric set).
 * Errors: MEM_ERR_INVALID_ARG (invalid handle; n_x or n_q < 2 or
 * n_x n_q > 2^24; bounds not finite, not increasing, or lnx_max > 0; a
 * value negative or not finite), MEM_ERR_OOM, MEM_ERR_CUDA. */
mem_status mem_process_set_pdf_grid(mem_process* process, const float* table, int32_t n_x,
                                    int32_t n_q, double lnx_min, double lnx_max,
                                    double lnq_min, double lnq_max);

/* Copy n_events event records (32 float32 each, layout in the package's
 * synth module docs: 6 x (E, eta, phi, kind), MET x, y, n_obj, kind, ...)
 * into library-owned device memory. `records` is host memory if
 * records_on_device == 0, else device memory. The copy is enqueued on
 * `stream` and completes before the call returns.
 * Errors: MEM_ERR_INVALID_ARG (NULL, n_events < 1, records of another process
 * kind), MEM_ERR_OOM, MEM_ERR_CUDA. */
mem_status mem_upload_events(mem_process* proc, const float* records, int64_t n_events,
                             int32_t records_on_device, void* stream, mem_events** out);

/* Integrate every uploaded event with n_points integrand evaluations per
 * (event, jet permutation) item, Philox key `seed`. Writes per event:
 * prob (p_hat), err (MC standard error), n_used (evaluations, adaptation
 * included) and ev_status (MEM_OK, MEM_ERR_NONFINITE, MEM_NOT_CONVERGED).
 * Any of n_used / ev_status may be NULL. Each output holds n_events entries.
 * Errors: MEM_ERR_INVALID_ARG (NULL, n_points too small for the adaptation
 * plan or above 2^32, process mismatch), MEM_ERR_OOM, MEM_ERR_CUDA. */
mem_status mem_integrate(const mem_events* ev, const mem_process* proc, const mem_tf_desc* tf,
                         uint64_t n_points, uint64_t seed, const mem_opts* opts, double* prob,
                         double* err, uint64_t* n_used, int32_t* ev_status, void* stream);

/* Integrate several event sets (one mem_events per process; uneven dimensions,
 * permutation counts and budgets) to a target relative error in one call: the
 * per-event stop rule of the adaptive mode, err/prob <= opts->target_rel_err
 * (Sec. 2's MC error estimate; p_hat averaged over jet permutations, Sec. 4),
 * capped at opts->max_points per event (0 = 2^24) and starting from
 * opts->min_points (0 = 2^14) frozen-grid points per event after
 * opts->n_adapt_iters VEGAS iterations of opts->adapt_points points per item
 * (0 = 8192). Points are added in rounds that double each unconverged event's
 * budget; every round runs on the device and the whole schedule of all groups
 * is one CUDA graph (one forked stream per group). Outputs are concatenated
 * over the groups in order (sum of n_events entries each); ev_status is
 * MEM_OK (converged), MEM_NOT_CONVERGED (cap reached), MEM_ERR_NONFINITE or
 * MEM_ERR_INVALID_ARG (invalid record). Event ids in the Philox counter are
 * opts->event_id_base + the event's position in the concatenation. The call
 * returns when the work is complete. Errors: MEM_ERR_INVALID_ARG (NULL,
 * n_groups outside [1, 16], target_rel_err <= 0, grid_in given, budgets that do
 * not fit), MEM_ERR_OOM, MEM_ERR_CUDA. */
mem_status mem_integrate_batch(int32_t n_groups, const mem_events* const* events,
                               const mem_process* const* procs, const mem_tf_desc* const* tfs,
                               uint64_t seed, const mem_opts* opts, double* prob, double* err,
                               uint64_t* n_used, int32_t* ev_status, void* stream);

/* Autotuner of the batched schedule for one process: every candidate plan
 * (VEGAS adaptation of 2-5 iterations of 2048-8192 points per item; first
 * round 2^13-2^15 points per event; 2-8 sampling tiles per CTA) integrates
 * the given calibration events to opts->target_rel_err (cap opts->max_points)
 * with mem_integrate_batch, timed with CUDA events on `stream` (one warm-up,
 * best of two runs); the plan with the most converged events per second is
 * written to *best and its rate to *events_per_s (optional). The search is
 * two-staged (adaptation plan first, then first-round size and tiles) over a
 * fixed list; n_tried (optional) receives the number of plans timed.
 * Synchronous. Errors as mem_integrate_batch. */
mem_status mem_autotune(const mem_events* events, const mem_process* process,
                        const mem_tf_desc* tf, uint64_t seed, const mem_opts* opts,
                        mem_plan* best, double* events_per_s, int32_t* n_tried, void* stream);

/* Parton-level weights of semileptonic ttbar events (Sec. 4, "parton level"):
 * every final-state momentum is known, so every transfer function is a delta
 * function and nothing is integrated. Each record (uploaded with
 * mem_upload_events for the ttbar process) holds, as objects 0..5 with
 * (E [GeV], eta, phi, kind): the l+ (kind 4 or 2), two b quarks (kind 5), the
 * d and the ubar (kind 5) and the neutrino (kind 6); |eta| < 40.
 * For each of the two assignments of the b quarks (0: object 1 is the b and
 * object 2 the bbar; 1: the reverse) the weight is the density of Eq.
 * "mem_def" at these momenta: the final state is boosted transversely to zero
 * pT, which fixes x1 and x2 through its E + p_z and E - p_z; weight =
 * sum_flavours f(x1) f(x2) |M|^2 / (|q1||q2|) x (2 pi)^4 (2/s) x
 * prod_i 1/((2 pi)^3 2 E_i) over the six final-state particles (0 if x1 or x2
 * reaches 1).
 * Outputs (all host or all device memory, caller-owned): prob (n_events
 * doubles) = the mean over the two assignments; w_assign (NULL or 2 n_events
 * doubles, event-major) = the weight per assignment; ev_status (NULL or
 * n_events int32) = MEM_OK, or MEM_ERR_INVALID_ARG for a record whose object
 * kinds, energies or eta do not fit the layout above (its outputs are 0).
 * Asynchronous on `stream` with device outputs; synchronous with host outputs.
 * Errors: MEM_ERR_INVALID_ARG (NULL handle or prob, a process or events other
 * than ttbar, outputs mixing host and device memory, device outputs not aligned
 * to their element size), MEM_ERR_OOM, MEM_ERR_CUDA. */
mem_status mem_parton_weights(const mem_events* events, const mem_process* process, double* prob,
                              double* w_assign, int32_t* ev_status, void* stream);

/* Event discriminant (Sec. 3): D = log10(p_S / p_B) for each of n events, from
 * the probability densities of the same events under a signal and a background
 * hypothesis (e.g. two mem_integrate results), with the first-order error of
 * independent estimates sigma_D = sqrt((err_S/p_S)^2 + (err_B/p_B)^2) / ln 10.
 * Inputs prob_s, err_s, prob_b, err_b and outputs D, err_D (optional),
 * status (optional: MEM_OK, or MEM_ERR_INVALID_ARG where a density is not
 * > 0, with NaN outputs): n doubles (int32 for status) each, all host or all
 * device memory. Asynchronous on `stream` with device arrays.
 * Errors: MEM_ERR_INVALID_ARG (n < 1, NULL inputs or D, mixed memory kinds),
 * MEM_ERR_OOM, MEM_ERR_CUDA. */
mem_status mem_discriminant(int64_t n, const double* prob_s, const double* err_s,
                            const double* prob_b, const double* err_b, double* D, double* err_D,
                            int32_t* status, void* stream);

/* The colour matrices of the dilepton ttbb production terms (MEM_PROC_TTBB_DILEP):
 * K_nm = sum over external colours of conj(C_n) C_m for the 38 g g terms and the 7
 * q qbar terms, in the kernels' term order (see the header of csrc/mem_ttbb.cuh), as
 * interleaved (real, imaginary) float pairs, row major: kgg 38 x 38 x 2 and kqq
 * 7 x 7 x 2 floats of host memory, caller-owned. Host computation; no device needed.
 * Errors: MEM_ERR_INVALID_ARG (NULL pointers). */
mem_status mem_ttbb_colour_matrices(float* kgg, float* kqq);

/* The factors the ttbb kernels use for their colour sums: K = sum_k u_k u_k^dagger
 * for each colour matrix above, by pivoted Cholesky (K is a Gram matrix, so the
 * colour-summed square L^dagger K L of an amplitude vector L is sum_k |u_k^dagger L|^2
 * with rank(K) terms). Writes the rows conj(u_k), k < rank, as interleaved (real,
 * imaginary) float pairs, row major, the rows beyond the rank zero: ugg 38 x 38 x 2 and
 * uqq 7 x 7 x 2 floats, and ranks[2] (g g, q qbar); host memory, caller-owned. Host
 * computation; no device needed; no paper counterpart (a cheaper evaluation of the
 * same colour sums). Errors: MEM_ERR_INVALID_ARG (NULL pointers; or the factors do
 * not reproduce K to 1e-9 of its largest diagonal element). */
mem_status mem_ttbb_colour_factors(float* ugg, float* uqq, int32_t* ranks);

/* Working memory of mem_integrate_noalloc, fixed at build time (32 MiB per GPU). */
#define MEM_NOALLOC_SCRATCH_BYTES (32u << 20)

/* mem_integrate without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory
 * once they are running -- e.g. an online event selection inside a
 * data-acquisition process that reserves all GPU memory at start-up and
 * forbids per-batch allocations for predictable latency, or an application
 * that lends the library buffers from its own pool. It runs the same kernels
 * as mem_integrate with the default plan (5 VEGAS adaptation iterations of
 * min(2^14, n/8) points, alpha 1.5) and takes the process and transfer
 * functions by descriptor (no handles). `records` (n_events x 32 float32),
 * `prob`, `err` and `ev_status` (optional) must be plain DEVICE memory of the
 * current device (not host, pinned, managed or another GPU's memory; anything
 * else is rejected with MEM_ERR_INVALID_ARG before any launch); the call is
 * asynchronous on `stream` and copies nothing.
 * Working memory (grids, per-item constants, partial sums) is one static
 * device array of MEM_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * keeps until exit; a call needing more is rejected with MEM_ERR_INVALID_ARG
 * (about 2,400 Drell-Yan or W events at 2^20 points per event fit).
 * Set-up: the first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) and caches it; with CUDA's
 * lazy module loading that call, and the first launch of each kernel, also
 * loads the module and kernels, which reserves device memory. A caller that
 * may not allocate later makes one small call per process kind it will use
 * (e.g. 1 event, 16 points) at start-up, before it reserves its memory pool
 * and before any stream capture; later calls allocate nothing. Kinds 0-3 need
 * at most 1024 bytes of per-thread stack (callees included), the default limit,
 * so no launch grows the context's local memory; kinds 4 and 5 are rejected.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller.
 * Nothing in it needs clearing between calls: every region is written by the
 * call before the call reads it. */
mem_status mem_integrate_noalloc(const mem_process_desc* desc, const mem_tf_desc* tf,
                                 const float* records, int64_t n_events, uint64_t n_points,
                                 uint64_t seed, uint64_t event_id_base, double* prob,
                                 double* err, int32_t* ev_status, void* stream);

/* ---- learned importance sampler ------------------------------------------
 * An event-conditioned affine-coupling normalising flow on the unit cube that
 * replaces the VEGAS map (Sec. 2, importance sampling) for the ttbar
 * integrand: u ~ U(0,1)^7 -> logit -> 6 coupling layers (z_B <- z_B e^s + t,
 * (s, t) from a 128-128 ReLU MLP of z_A and 16 event features, s = 2 tanh(s_raw/2))
 * -> sigmoid. Its log-Jacobian is exact, so f(y)|dy/du| is an unbiased weight.
 * Hidden layers run on BF16 tensor cores with FP32 accumulation; FP32 master
 * parameters. Parameters use a flat FP32 layout: per layer k = 0..5 with
 * |A| = 4 (k even) or 3 (k odd) and |B| = 7 - |A|: W1a [|A|][128], W1c [16][128],
 * b1 [128], W2 [128][128], b2 [128], W3 [128][2|B|], b3 [2|B|]. */
typedef struct mem_flow mem_flow;

/* The dilepton neutrino solution of the integrand kernels (Sec. 3, Eq.
 * "dilepsolv": nu and nubar from the W+, W-, t and tbar virtualities and the
 * missing pT), exposed for parity tests like mem_eval_points. in: n x 22 HOST
 * doubles per system -- b, bbar, l+, mu- four-momenta (E, px, py, pz; GeV,
 * massless), MET x, y, q^2 of W+, W-, t, tbar (GeV^2). Writes nsol[n] (0..4), nu
 * [n][4][8] (per solution nu then nubar, GeV; unused slots 0) and jac [n][4]
 * (1 / |det d(q^2_W+, q^2_t, q^2_W-, q^2_tbar)/d(nu_x, nu_y, nu_z, nubar_z)|, GeV^-4):
 * the same double-float solver stages, checks and de-duplication as the
 * integrand (the inputs rounded to double-float, ~48 bits), one GPU thread per
 * system. Synchronous. Errors: MEM_ERR_INVALID_ARG (NULL, n < 1
 * or n > 2^24), MEM_ERR_CUDA. */
mem_status mem_dilep_solve(const double* in, int64_t n, int32_t* nsol, double* nu, double* jac);

/* Poll limit of every bounded tensor-core completion wait in the flow's
 * sampling kernels (mem_integrate_flow, mem_flow_eval_points) on the current
 * device; MEM_TC_WAIT_DEFAULT at load. A wait that reaches the limit gives up:
 * its CTA drains the products it has committed (a second bounded wait),
 * releases its tensor memory and stops, and the call returns MEM_ERR_TIMEOUT
 * with the context still usable. Lowering the limit (0 gives up at once) is a
 * test of that path; no paper counterpart. Synchronous; not to be called while
 * kernels of this library run.
 * Errors: MEM_ERR_CUDA. */
#define MEM_TC_WAIT_DEFAULT (1u << 20)
mem_status mem_set_tc_wait_limit(uint32_t polls);

/* Number of FP32 parameters of the flow. */
int64_t mem_flow_param_count(void);
/* Create a flow on the current device: random hidden weights (seeded), zero
 * output layers (the identity map). Release with mem_destroy. */
mem_status mem_flow_create(uint64_t seed, mem_flow** out);
/* Copy parameters in/out (host arrays of mem_flow_param_count() floats). */
mem_status mem_flow_set_params(mem_flow* flow, const float* params, int64_t n);
mem_status mem_flow_get_params(const mem_flow* flow, float* params, int64_t n);
/* Forward map of n points sharing one conditioning vector: cond (16 floats),
 * u (n x 7) -> y (n x 7) and log|dy/du| (n); all DEVICE arrays; synchronous. */
mem_status mem_flow_map(const mem_flow* flow, const float* cond, const float* u, int64_t n,
                        float* y, float* logj, void* stream);

/* Training data layout (all DEVICE arrays): n_items items of 128 samples, ys
 * [n_items][128][7] points in (0,1)^7, ws [n_items][128] weights normalised to
 * sum 1 per item, cs [n_items][16] conditioning. Loss of an item:
 * L = sum_i w_i log|dy/du|(y_i) = -sum_i w_i log q(y_i) (KL divergence from the
 * normalised integrand to the flow density, up to a constant).
 * mem_flow_grad: gradient of the summed loss over all items w.r.t. every
 * parameter (flat layout, HOST output of mem_flow_param_count() floats) and
 * the loss (host double); parameters unchanged.
 * mem_flow_train: n_steps Adam steps (beta 0.9/0.999) on minibatches of
 * batch_items items drawn by epochs of seeded permutations, gradient = mean
 * over the minibatch's items; loss_trace (HOST, n_steps floats, optional). */
mem_status mem_flow_grad(mem_flow* flow, const float* ys, const float* ws, const float* cs,
                         int64_t n_items, float* grad, double* loss, void* stream);
mem_status mem_flow_train(mem_flow* flow, const float* ys, const float* ws, const float* cs,
                          int64_t n_items, int32_t n_steps, int32_t batch_items, float lr,
                          uint64_t seed, float* loss_trace, void* stream);

/* Training set for the ttbar flow (Sec. 2: samples of the integrand drawn by
 * the VEGAS importance sampler). Every item (event, jet permutation) is
 * adapted as in mem_integrate (opts: n_adapt_iters, 0 = the uniform grid,
 * adapt_points, 0 = 8192, alpha; opts NULL = 5 x 8192, 1.5), then 128 points of the VEGAS stream that follow the
 * adaptation are drawn from its grid: ys = the points (kept inside
 * [2^-24, 1 - 2^-24]), ws = f J normalised to sum 1 over the item's 128 points
 * (per_event = 0) or over the event's 24 x 128 points (per_event = 1: items
 * weighted by their share of the event's estimate); 0 where the sum is 0.
 * cs = the item's 16 conditioning features (units of 100 GeV, frame rotated
 * to lepton phi = 0): lepton (px, pz); jets b, bbar, d, ubar of the
 * permutation, each (px, py, pz); missing pT (x, y). log_jv (optional) = log J
 * of the VEGAS map at each point, so that sum w log J is the training loss
 * that the VEGAS density itself would score. Outputs are DEVICE arrays laid out
 * as mem_flow_train reads them (n_items = n_events * 24).
 * MEM_ERR_INVALID_ARG for a process other than MEM_PROC_TTBAR. */
#define MEM_FLOW_SAMPLES_PER_ITEM 128
mem_status mem_flow_samples(const mem_events* events, const mem_process* process,
                            const mem_tf_desc* tf, uint64_t seed, const mem_opts* opts,
                            int32_t per_event, float* ys, float* ws, float* cs, float* log_jv,
                            void* stream);

/* Adaptive-budget ttbar integral with the flow as the importance sampler and
 * VEGAS as its fallback and judge. Round 0 (pilot): every item draws
 * ceil(min_points / 24) flow points (Philox stream 2). Items that the pilot
 * flags (opts->flow_screen) are adapted by VEGAS (n_adapt_iters x adapt_points,
 * defaults 5 x 8192); the variance of its last adaptation iteration is compared
 * with the flow's, and the lower (flow_cost-weighted) sampler integrates that item
 * from then on. Later rounds double the points of every item of every
 * unconverged event until err <= target_rel_err * prob or max_points (as
 * mem_integrate_batch). Samples of both samplers are pooled per item (both are
 * unbiased). n_used counts every evaluated point, adaptation included.
 * item_sampler (optional, n_events * 24 bytes, host or device, same kind as
 * prob): 0 flow, 1 flow kept by the judge, 2 VEGAS chosen by the judge.
 * Synchronous; target_rel_err must be > 0. */
mem_status mem_integrate_flow(const mem_events* events, const mem_process* process,
                              const mem_tf_desc* tf, const mem_flow* flow, uint64_t seed,
                              const mem_opts* opts, double* prob, double* err, uint64_t* n_used,
                              int32_t* ev_status, uint8_t* item_sampler, void* stream);

/* Flow-sampled points of one ttbar item (parity checks): points point0 ..
 * point0 + n - 1 of stream 2 for (seed, event_id, perm), record = one event
 * record (DEVICE); outputs the final logits z (n x 7 floats; the point is
 * y = 1 / (1 + exp(-z))), log|dy/du| (n floats) and the weight
 * prefactor * f(y) |dy/du| (n doubles), all DEVICE; synchronous. */
mem_status mem_flow_eval_points(const mem_process* process, const mem_tf_desc* tf,
                                const mem_flow* flow, const float* record, int32_t perm,
                                uint64_t seed, uint32_t event_id, uint32_t point0, int64_t n,
                                float* z, float* logj, double* w, void* stream);

/* Release a mem_process or mem_events handle (NULL is a no-op). Releasing a
 * process does not release events uploaded with it. */
void mem_destroy(void* handle);

/* Thread-local description of the last error ("" if none). */
const char* mem_last_error(void);

/* ---- parts of the hot path exposed for parity tests ---------------------- */

/* Integrand weight at points point0 .. point0+n-1 of item (event_index, perm)
 * on the given HOST grid (d x 129 doubles; NULL = uniform), using exactly the
 * generator, VEGAS map and integrand of mem_integrate, in FP32, times the
 * process's FP64 constant prefactor. w_out: n doubles, host or device. */
mem_status mem_eval_points(const mem_events* ev, const mem_process* proc, const mem_tf_desc* tf,
                           int64_t event_index, int32_t perm, uint64_t seed, uint64_t point0,
                           int64_t n, const double* grid, double* w_out, void* stream);

/* The device Philox4x32-10 stream (Salmon et al., SC'11): uniforms of
 * dimensions 0..d-1 for points point0.., counter (point, block<<8, event, perm).
 * out: n*d floats (row-major), host or device. */
mem_status mem_philox_uniforms(uint64_t seed, uint64_t event_id, int32_t perm, uint64_t point0,
                               int64_t n, int32_t d, float* out, void* stream);

/* Device VEGAS refinement (Sec. 2; Lepage 1978) of n_grids grids of d
 * dimensions: hist n_grids x d x 128 (accumulated squared weights), grid_in
 * and grid_out n_grids x d x 129 doubles, all HOST arrays. alpha = compression. */
mem_status mem_vegas_refine(int32_t n_grids, int32_t d, const double* hist,
                            const double* grid_in, double alpha, double* grid_out);

#ifdef __cplusplus
}
#endif
#endif
