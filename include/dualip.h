/*
 * dualip.h -- C ABI of a GB300-native (sm_103a) dual-gradient engine for the
 * ridge-regularised dual of matching linear programs (DuaLip-GPU technical
 * report, arXiv 2603.04621).
 *
 * The problem (Section 3.1, Eq. 1, with the matching structure of Section 3.2):
 *     min  c^T x   s.t.  A x <= b,  x_i in {x_i >= 0, sum_j x_ij <= 1} for every source i
 * where x has one variable per edge (i, j) and (A x)_j = sum_i a_ij x_ij
 * (Eq. 3, Definition 1 with one constraint family).  The library evaluates the
 * smoothed dual of Eq. 2,
 *     g(lambda) = min_{x in C} c^T x + (gamma/2) sum_e w_e x_e^2 + lambda^T (A x - b),
 * its Danskin gradient grad g(lambda) = A x*(lambda) - b (Section 3.1) with
 * x*(lambda) = Pi_C(-(A^T lambda + c) / gamma) computed per source, and runs
 * the dual ascent of Section 5 / Appendix B.  w_e = 1, or w_e = a_e^2 (1 where
 * a_e = 0) when primal scaling (Section 5.1, view (i) with v = |a|) is on.
 *
 * Conventions shared by every call:
 *  - Every entry point returns a dualip_status; nothing throws, aborts or traps.
 *    On failure dualip_last_error() returns a message for the calling thread.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work is ordered on that stream.
 *  - Pointers documented as "device" must be device (or managed) memory of the
 *    current CUDA device; "host" pointers are ordinary host memory (pinned
 *    host memory makes the copies asynchronous).
 *  - lambda and grad are always in the caller's destination numbering and
 *    original (unnormalised) coordinates.
 *  - A problem handle is not thread safe: calls on one handle must not overlap.
 */
#ifndef DUALIP_H
#define DUALIP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DUALIP_OK = 0,
  DUALIP_EINVAL = 1,        /* invalid argument or input data; nothing was changed */
  DUALIP_ENOMEM = 2,        /* a device or host allocation failed */
  DUALIP_ECUDA = 3,         /* a CUDA runtime call failed */
  DUALIP_ETIMEOUT = 4,      /* a bounded device-side wait gave up; results are invalid */
  DUALIP_EBUSY = 5,         /* the resource is in use (e.g. serving slots full) */
  DUALIP_ENOTCONVERGED = 6, /* dualip_solve stopped at max_iters before the tolerances */
  DUALIP_EDEVICE = 7,       /* a device-side consistency check failed */
  DUALIP_ECANCELED = 8      /* a serving request was cancelled */
} dualip_status;

typedef enum { DUALIP_EDGE_F32 = 0, DUALIP_EDGE_BF16 = 1 } dualip_edge_dtype;

/* The simple constraint set C of the primal (Section 3.2, Eqs. 4-5; Section
 * 4's projection maps, Section 6's batched projections):
 *   DUALIP_PROJ_SIMPLEX  each source's block in {x_i >= 0, sum_j x_ij <= 1}
 *   DUALIP_PROJ_BOX      every edge in [0, 1] (the unit-box clamp)
 * Box problems are evaluated and solved on their own handles; the batched and
 * serving forms and dualip_dual_grad_noalloc take simplex problems only. */
typedef enum { DUALIP_PROJ_SIMPLEX = 0, DUALIP_PROJ_BOX = 1 } dualip_projection;

/*
 * Source-major edge list (the paper's CSC tensor T of Section 6, "Sparse
 * tensor computation": one column per source i holding diag(D_i), so the
 * edges of a source are contiguous).
 *   num_sources  I >= 0
 *   num_edges    E >= 0; must equal src_offsets[I]
 *   num_dests    J >= 1
 *   src_offsets  [I+1] int64, src_offsets[0] = 0, nondecreasing; the edges of
 *                source i are src_offsets[i] .. src_offsets[i+1]-1
 *   dst          [E] int32, 0 <= dst[e] < J (repeated (i, j) pairs are separate variables)
 *   c            [E] float, cost of the edge (minimisation sign), finite
 *   a            [E] float, coefficient a_ij of the edge in row j of A, finite
 *   b            [J] float, budgets, finite
 *   inputs_on_device  0: the five arrays are host pointers; 1: device pointers
 *   storage      DUALIP_EDGE_F32 keeps c and a in FP32; DUALIP_EDGE_BF16 stores
 *                them as bfloat16 (round to nearest even) and computes in FP32
 *   primal_scaling  0: w_e = 1; 1: w_e = a_e^2 (1 where a_e = 0)
 *   projection   DUALIP_PROJ_SIMPLEX (0) or DUALIP_PROJ_BOX (1), see above
 *   num_families m >= 1 constraint families (Section 3.2, Definition 1: each
 *                source block stacks m diagonal blocks).  With m > 1, a holds
 *                m E floats, family-major (a[k E + e] is the coefficient of
 *                edge e in family k), and b holds m J floats; A then has
 *                m J rows, row k J + j, and lambda and grad of every call
 *                have m J entries in that order.  m > 1 needs FP32 storage;
 *                its pass is one warp per source without the lane-group
 *                tiling, and the batched, serving and allocation-free forms
 *                take one family only.
 * dualip_create copies everything into library-owned device memory; the
 * caller keeps ownership of its arrays and may free them on return.
 */
typedef struct {
  int64_t num_sources;
  int64_t num_edges;
  int32_t num_dests;
  const int64_t* src_offsets;
  const int32_t* dst;
  const float* c;
  const float* a;
  const float* b;
  int32_t inputs_on_device;
  int32_t storage;
  int32_t primal_scaling;
  int32_t projection;  /* dualip_projection: the simple constraint set C */
  int32_t num_families; /* m: constraint families (Definition 1); 0 or 1 = one */
} dualip_problem_desc;

/* Scalars of one dual evaluation, computed on the GPU in FP64 (Section 6: the
 * "local objective value and local regularization penalty"; Appendix A for
 * the infeasibility). */
typedef struct {
  double dual_obj;        /* g(lambda) of Eq. 2 */
  double primal_obj;      /* c^T x*(lambda) */
  double reg;             /* (gamma/2) sum_e w_e x_e^2 */
  double infeas_l2;       /* ||(A x* - b)_+||_2 */
  double lambda_dot_grad; /* lambda^T (A x* - b) */
} dualip_eval;

typedef struct dualip_problem dualip_problem;

/* Build a problem handle from a desc (validated: offsets, destination range,
 * finiteness).  Work is queued on `stream` and finished before return.
 * Errors: DUALIP_EINVAL (bad desc or data), DUALIP_ENOMEM, DUALIP_ECUDA.
 * On success *out owns device memory of about E * (4 + bytes of c and a)
 * + 12 I + 40 J bytes, plus 20 bytes per edge of hub sources (below); free it
 * with dualip_destroy.
 * Degree order: when the pass's lane-group cost model predicts at least 2%
 * fewer element slots for it, the sources are stored in order of increasing
 * degree.  Results do not depend on the stored order: A x and the objective
 * partials are exact fixed-point sums, and dualip_get_primal returns x in the
 * caller's edge order.
 * Segment classes: a source larger than a stage (3200 edges with FP32
 * storage, 4800 with BF16) is projected by a whole CTA; one of at least 16
 * stages (a hub source) by the whole grid, in a kernel of its own before
 * each pass, which keeps a candidate list of up to 16 bytes per edge of the
 * source in device memory (not for the unit box).  A hub source's edges are
 * stored in order of destination (4 bytes per edge keep the permutation;
 * sorting them takes a stream-ordered temporary of 12 bytes per hub edge and
 * a host pass over J per hub source), so that neighbouring lanes gather mu
 * from shared sectors; results do not depend on that order either. */
dualip_status dualip_create(const dualip_problem_desc* desc, void* stream, dualip_problem** out);

/* Release a handle (NULL is ignored).  Synchronises the handle's last stream. */
void dualip_destroy(dualip_problem* p);

/*
 * One dual-gradient evaluation (Section 3.1, Eq. 2 and Danskin's theorem):
 *   lambda  [J] float, device: dual point (any sign is accepted)
 *   gamma   ridge parameter, > 0
 *   grad    [J] float, device, written: A x*(lambda) - b
 *   out     host, may be NULL: the scalars of this evaluation; when non-NULL
 *           the call waits for `stream` to finish before returning
 * Errors: DUALIP_EINVAL (NULL handle/pointers, gamma <= 0 or not finite),
 * DUALIP_ECUDA, DUALIP_ETIMEOUT / DUALIP_EDEVICE (device-side check; the
 * outputs are then invalid).
 */
dualip_status dualip_dual_grad(dualip_problem* p, const float* lambda, double gamma, float* grad,
                               dualip_eval* out, void* stream);

/* Same as dualip_dual_grad, but never synchronises: the scalars are written
 * to `out_dev` (device, 5 doubles in dualip_eval order) and device-side error
 * reporting is deferred to dualip_check_device_status.  Safe to capture in a
 * CUDA graph. */
dualip_status dualip_dual_grad_async(dualip_problem* p, const float* lambda, double gamma,
                                     float* grad, double* out_dev, void* stream);

/* dualip_dual_grad with host buffers: copies lambda in and grad and the
 * scalars out inside the call (pinned host memory makes the copies fastest).
 * Waits for `stream`. */
dualip_status dualip_dual_grad_host(dualip_problem* p, const float* lambda_host, double gamma,
                                    float* grad_host, dualip_eval* out, void* stream);

/* The primal minimiser x*(lambda) of Section 3.1 for every edge, in the
 * caller's edge order:
 *   x  [E] float, device, written.  Other arguments as dualip_dual_grad.
 * For a problem stored in degree order it takes a stream-ordered temporary of
 * E floats and 16 bytes per source; with hub sources, one of E floats. */
dualip_status dualip_get_primal(dualip_problem* p, const float* lambda, double gamma, float* x,
                                void* stream);

/* Reads (and clears) the device-side error word of the handle; waits for
 * `stream`.  Returns DUALIP_OK, DUALIP_ETIMEOUT or DUALIP_EDEVICE. */
dualip_status dualip_check_device_status(dualip_problem* p, void* stream);

/* Kernel timing for measurement.  After dualip_profile_enable, each of the
 * next max_evals evaluations on the handle records CUDA events on its stream
 * around its three kernels (destination prologue, edge pass, destination
 * epilogue).  dualip_profile_collect waits for those events, returns the
 * summed durations in milliseconds and the number of evaluations recorded,
 * and turns recording off.  Errors: DUALIP_EINVAL, DUALIP_ENOMEM, DUALIP_ECUDA. */
dualip_status dualip_profile_enable(dualip_problem* p, int32_t max_evals);
dualip_status dualip_profile_collect(dualip_problem* p, double* ms_prologue, double* ms_pass,
                                     double* ms_epilogue, int32_t* count);

/* Sizes of a handle: I, J, E and the number of edge tiles of the pass. */
dualip_status dualip_get_info(const dualip_problem* p, int64_t* num_sources, int32_t* num_dests,
                              int64_t* num_edges, int64_t* num_tiles);

/*
 * Dual ascent (Section 5, Appendix B): accelerated projected ascent on the
 * Jacobi row-normalised dual (Section 5.1) with gamma continuation
 * gamma_k = max(gamma_final, gamma0 * 2^-floor(k / halve_every)) and the step
 * cap scaled in proportion to gamma (Section 5.1, "Regularization decay").
 * Step: eta_k = min(max_step * gamma_k / gamma0, secant estimate
 * ||y_k - y_{k-1}|| / ||G_k - G_{k-1}||), init_step right after a gamma
 * change; momentum restarts when gamma changes (restart_on_gamma_change) and,
 * with restart_on_decrease, whenever the dual objective at the evaluated
 * point is below that of the previous evaluation at the same gamma (an
 * adaptive restart; the secant estimate is kept).  The scalars are exact
 * fixed-point sums (objective partials) and fixed-order sums (per-row terms),
 * so the restart decisions, and the whole trajectory, repeat bit for bit.
 * Stopping, tested every check_every iterations at gamma_final:
 *   |lambda^T (A x - b)| / max(1, |p|, |g|) <= tol_gap  (p = c^T x + ridge term)
 *   ||(A x - b)_+||_2 / max(1, ||b||_2)     <= tol_infeas.
 */
typedef struct {
  double gamma0;            /* > 0 */
  double gamma_final;       /* > 0, <= gamma0 */
  int32_t halve_every;      /* iterations per halving of gamma; <= 0 keeps gamma0 */
  double max_step;          /* step cap at gamma0 (scaled by gamma_k / gamma0) */
  double init_step;         /* first step after a (re)start */
  int32_t max_iters;        /* >= 1 */
  double tol_gap;
  double tol_infeas;
  int32_t check_every;      /* >= 1; scalars are read back every check_every iterations */
  int32_t row_normalize;    /* 1: Jacobi row normalisation (default), 0: off */
  int32_t restart_on_gamma_change; /* 1 (default) */
  int32_t stop_on_tol;      /* 1: stop at the tolerances; 0: run exactly max_iters */
  int32_t use_graph;        /* 1: capture check_every iterations in one CUDA graph */
  int32_t restart_on_decrease; /* 1 (default): adaptive momentum restart, see above */
  int32_t resume;           /* 0 (default): start from lambda_inout; 1: continue the
                               handle's ascent (left by its last solve or by
                               dualip_solve_state_import) at its iteration k, with
                               its momentum, step history and gamma position;
                               lambda_inout is then only written */
} dualip_solve_opts;

typedef struct {
  int32_t iters;      /* evaluations performed */
  int32_t converged;  /* 1 if both tolerances held at a check */
  dualip_eval last;   /* scalars at the returned lambda */
  double gap_rel;
  double infeas_rel;
  double gamma;       /* gamma of the last evaluation */
} dualip_solve_result;

/* Fill opts with the defaults: gamma0 0.1, gamma_final 1e-3, halve_every 25,
 * max_step 10, init_step 1e-5, max_iters 5000, tolerances 1e-4,
 * check_every 10, row_normalize 1, restart 1, stop_on_tol 1, use_graph 1,
 * restart_on_decrease 1. */
void dualip_solve_opts_default(dualip_solve_opts* opts);

/*
 * Run the ascent from lambda_inout (device, [J], clamped at 0 on entry) and
 * write the last evaluated dual point back into it.  `trace` (device, may be
 * NULL) receives 8 doubles per iteration: gamma, g, p, infeas, gap_rel,
 * infeas_rel, step, lambda^T grad.  Returns DUALIP_OK when converged,
 * DUALIP_ENOTCONVERGED when max_iters ran out (result filled in both cases).
 */
dualip_status dualip_solve(dualip_problem* p, const dualip_solve_opts* opts, float* lambda_inout,
                           dualip_solve_result* result, double* trace, void* stream);

/*
 * Saved ascent, for the recurring solves of the paper's production setting
 * (Section 3: the same matching problem is solved again and again as its data
 * drift) and for pre-empting a solve: the state that dualip_solve leaves in a
 * handle (the normalised dual lambda', the extrapolated point y and the
 * previous one, the last two gradients, the row scale, the iteration counter
 * k that fixes gamma's place in the schedule, the momentum t, the step and
 * the last scalars) as an opaque host buffer of dualip_solve_state_size()
 * bytes; vectors are stored in the caller's destination numbering.
 *   export: needs a handle that has run dualip_solve (or imported a state);
 *           buffer (host) of at least the size; waits for `stream`.
 *   import: into a handle of a problem with the same J (normally the same
 *           problem, or its drifted data: same graph, new c, a or b); the next
 *           dualip_solve with opts.resume = 1 continues from it.  An ascent
 *           stopped after k iterations, exported, imported into a fresh handle
 *           of the same problem and resumed for n more iterations ends exactly
 *           (bit for bit) where k + n uninterrupted iterations end.
 * Errors: DUALIP_EINVAL (NULL pointers, small buffer, no state to export, a
 * buffer that is not a state or has another J), DUALIP_ENOMEM, DUALIP_ECUDA.
 */
dualip_status dualip_solve_state_size(const dualip_problem* p, int64_t* bytes);
dualip_status dualip_solve_state_export(dualip_problem* p, void* buffer, int64_t bytes,
                                        void* stream);
dualip_status dualip_solve_state_import(dualip_problem* p, const void* buffer, int64_t bytes,
                                        void* stream);

/*
 * Dual evaluation that allocates nothing (the paper has no counterpart; this
 * is for callers that cannot allocate device memory: a framework whose
 * caching allocator or pre-planned arena owns the device, a request path that
 * cannot take cudaMalloc's implicit synchronisation, a device that is nearly
 * full).  It needs no handle: it reads the caller's device arrays directly,
 * laid out as in dualip_problem_desc (FP32 c and a), and computes the same
 * grad and scalars as dualip_dual_grad.
 *   num_sources I >= 0; num_dests J, 1 <= J <= 1048576 (larger J: DUALIP_EINVAL)
 *   src_offsets [I+1], dst [E], c [E], a [E], b [J], lambda [J]: device, read only
 *   primal_scaling 0 / 1 as in dualip_problem_desc; gamma > 0
 *   grad [J] device, written; out_dev [5] device doubles in dualip_eval order
 * Scratch lives in one fixed __device__ array of about 8 MiB that every GPU
 * loading the library holds until exit.  The first call on a device looks up
 * that array's address and should come before any stream capture.  Every call
 * shares the array (it is cleared at the start of each call), so calls whose
 * work overlaps on the GPU race: serialise them.  Nothing is synchronised;
 * an edge whose destination is outside [0, J) is skipped and turns every
 * entry of grad and every scalar in out_dev into NaN.  The offsets are
 * trusted as given.  A x is summed with FP64 atomics in arrival order, so
 * repeated calls on the same inputs may differ in the last bits (the handle
 * path's A x is exact and reproducible).  The scratch address is looked up
 * once per device and process: do not call this entry point again after a
 * device reset (cudaDeviceReset or a primary-context reset) in that process.
 */
dualip_status dualip_dual_grad_noalloc(int64_t num_sources, int32_t num_dests,
                                       const int64_t* src_offsets, const int32_t* dst,
                                       const float* c, const float* a, const float* b,
                                       int32_t primal_scaling, const float* lambda, double gamma,
                                       float* grad, double* out_dev, void* stream);

/* ------------------------------------------------------------ batches ----
 * The batched form: several independent matching LPs evaluated, and solved,
 * by one launch of the pass per iteration (the paper batches the per-source
 * projections of one problem, Section 6; here whole problems are batched).
 * A batch is built from problem handles made by dualip_create, which keep
 * their own data; the batch only references them: destroy it before them,
 * and do not use a problem on its own while a batch call on it may run.
 * Every problem must use the same storage and primal_scaling.
 *
 * Joint vectors ("joint [sum J]") hold the problems' destination vectors back
 * to back in batch order, each in the caller's numbering: problem k's entries
 * start at J_0 + ... + J_{k-1}.
 */
typedef struct dualip_batch dualip_batch;

/* n >= 1 problems (host array of handles).  Tiles use the default shape (the
 * stage capacity: 3200 edges with FP32 storage, 4800 with BF16; 256 sources)
 * until dualip_batch_autotune picks another. */
dualip_status dualip_batch_create(int32_t n, dualip_problem* const* problems,
                                  dualip_batch** out);
void dualip_batch_destroy(dualip_batch* b);

/*
 * One evaluation of every problem, each at its own gamma, equal to what
 * dualip_dual_grad gives for it alone (the gradient, c^T x and the ridge
 * term bit for bit; g, the infeasibility and lambda^T (A x - b) up to the
 * order in which their per-row terms are summed).  Exception: a source of at
 * least 16 stages' edges, which alone goes to the multi-block class, is
 * projected in a batch by one CTA (the block class); its x then agrees
 * within rounding, not bit for bit.
 *   lambda [sum J] device joint, read; gammas [n] host; grad [sum J] device joint, written
 *   out [n] host (may be NULL): the scalars of each problem
 * Synchronises the stream.
 */
dualip_status dualip_batch_dual_grad(dualip_batch* b, const float* lambda, const double* gammas,
                                     float* grad, dualip_eval* out, void* stream);
/* Same, stream-ordered, scalars to out_dev ([5 n] device doubles, may be NULL). */
dualip_status dualip_batch_dual_grad_async(dualip_batch* b, const float* lambda,
                                           const double* gammas, float* grad, double* out_dev,
                                           void* stream);

/*
 * The ascent of dualip_solve for every problem at once, each with its own
 * gamma schedule, step, momentum and stopping test; a problem that has met
 * its tolerances (or its max_iters) stops being evaluated.
 *   opts: n_opts = 1 (shared) or n; check_every, row_normalize and use_graph
 *         are taken from opts[0]
 *   lambda_inout [sum J] device joint; results [n] host (may be NULL)
 * Returns DUALIP_ENOTCONVERGED if some problem ran out of iterations.
 */
dualip_status dualip_batch_solve(dualip_batch* b, const dualip_solve_opts* opts, int32_t n_opts,
                                 float* lambda_inout, dualip_solve_result* results, void* stream);

/* Tile shape autotuner: candidate (edges, sources) shapes are pruned by the
 * degree (segment length) histogram of the batch, each survivor is timed
 * over a few evaluations, and the fastest is kept; then the lean-window
 * policy (4-lane groups taking spans up to 64 or up to 80) is timed on it. */
typedef struct {
  int32_t n_candidates;
  int32_t chosen;              /* index of the shape kept */
  int32_t tile_edges[8];
  int32_t tile_sources[8];
  double ms[8];                /* mean evaluation time of each candidate shape */
  int64_t degree_hist[32];     /* sources with degree in [2^k, 2^(k+1)) (k = 0: 0 or 1) */
  int32_t lean80;              /* 1: 4-lane windows of up to 80 edges were kept (else 64) */
  int32_t pad;
  double ms_lean80;            /* the chosen shape timed with 80-edge windows */
} dualip_autotune_result;
dualip_status dualip_batch_autotune(dualip_batch* b, dualip_autotune_result* result, void* stream);
/* Kernel timing of the next max_evals batched evaluations, as for a problem
 * (dualip_profile_enable / _collect): prologue, pass and epilogue, in ms. */
dualip_status dualip_batch_profile_enable(dualip_batch* b, int32_t max_evals);
dualip_status dualip_batch_profile_collect(dualip_batch* b, double* ms_prologue, double* ms_pass,
                                           double* ms_epilogue, int32_t* count);
/* Explicit tile shape: 1 <= edges <= the stage capacity (3200 edges with
 * FP32 storage, 4800 with BF16), 1 <= sources <= 256. */
dualip_status dualip_batch_set_tile_shape(dualip_batch* b, int32_t edges, int32_t sources);
dualip_status dualip_batch_get_info(const dualip_batch* b, int32_t* n, int64_t* total_J,
                                    int64_t* total_E, int64_t* ntiles, int32_t* tile_edges,
                                    int32_t* tile_sources);

/* ------------------------------------------------------------ serving ----
 * A request loop (continuous batching) over the batched ascent.  Requests
 * (matching LPs with their solve options) are queued; one is admitted, in
 * arrival order, when a slot is free and its estimated device footprint fits
 * the HBM budget next to the problems already resident.  An admitted request
 * is built on the device (dualip_create, on its own stream, while the others
 * keep iterating) and joins the running ascent at the next chunk boundary
 * (every check_every iterations); its lambda, optimiser state and edges stay
 * on the device until it meets its tolerances or max_iters, then its lambda
 * goes to host memory and its memory is freed.  Requests with FP32 and BF16
 * storage (and with or without primal scaling) run in separate batches, one
 * after the other in every chunk.  A request's result is the one it gets
 * alone: its gradients are exact whatever shares the launch, and its step,
 * momentum and stopping test use its own quantities only.
 *
 * Footprint estimate (bytes): E (4 + bytes(c, a)) + 12 (I + 4) + 16 tiles
 * + 56 J, plus 12 E while host inputs are staged at creation.  A request
 * stored in degree order (see dualip_create) also holds 16 (I + 1) bytes of
 * source map during its creation, and one with hub sources 20 bytes per hub
 * edge (and 12 more while it is built); the estimate leaves these out.
 */
typedef struct dualip_server dualip_server;

typedef struct {
  int64_t hbm_budget_bytes;  /* > 0 */
  int32_t max_slots;         /* resident requests per storage kind, 1..1024 */
  int32_t check_every;       /* iterations per chunk (joins, exits, stopping tests), >= 1 */
} dualip_server_opts;

typedef enum {
  DUALIP_REQ_QUEUED = 0,   /* waiting for admission, or admitted and being built */
  DUALIP_REQ_RUNNING = 1,  /* built (its inputs copied): waiting to join, or iterating */
  DUALIP_REQ_DONE = 2,
  DUALIP_REQ_FAILED = 3
} dualip_request_state;

typedef struct {
  int32_t state;              /* dualip_request_state */
  int32_t status;             /* dualip_status of a failed request */
  dualip_solve_result result; /* valid when DONE */
  double t_submit, t_admit, t_done;  /* seconds since the server started (-1: not yet) */
  int64_t footprint_bytes;
  int32_t num_dests;
  int32_t pad;
} dualip_request_info;

typedef struct {
  int64_t submitted, queued, running, done, failed;
  int64_t resident_bytes, peak_resident_bytes;
  int64_t chunks;             /* chunk launches (each: check_every iterations of a batch) */
  int64_t slot_iterations;    /* iterations summed over requests */
  double busy_seconds;        /* time spent running chunks */
} dualip_server_stats;

dualip_status dualip_server_create(const dualip_server_opts* opts, dualip_server** out);
/* Queues a request.  The arrays of desc (host or device) must stay valid
 * until the request has left the QUEUED state; opts NULL = defaults. */
dualip_status dualip_server_submit(dualip_server* s, const dualip_problem_desc* desc,
                                   const dualip_solve_opts* opts, int64_t* ticket);
/* State of a request; lambda_out (host [J], may be NULL) receives its dual
 * point once DONE. */
dualip_status dualip_server_poll(dualip_server* s, int64_t ticket, dualip_request_info* info,
                                 float* lambda_out);
/* As poll, after waiting up to timeout_s for DONE or FAILED
 * (DUALIP_ETIMEOUT if neither came). */
dualip_status dualip_server_wait(dualip_server* s, int64_t ticket, double timeout_s,
                                 dualip_request_info* info, float* lambda_out);
dualip_status dualip_server_get_stats(dualip_server* s, dualip_server_stats* stats);
/* Cancels a request: one waiting for admission leaves the queue at once; one
 * being built or running leaves when its build ends or at the next chunk
 * boundary.  It ends FAILED with DUALIP_ECANCELED and no lambda.  A request
 * already DONE or FAILED is left as it is. */
dualip_status dualip_server_cancel(dualip_server* s, int64_t ticket);
/* Stops the loop; queued and running requests are dropped. */
void dualip_server_destroy(dualip_server* s);

/*
 * Fault injection from the host (for tests of the failure path; no device
 * fault is involved).  Sets, stream-ordered, a flag in the problem's device
 * status: the next evaluation's pass stops staging tiles and every bounded
 * device wait gives up at once, as a timed-out wait would, so the call that
 * reads the status returns DUALIP_ETIMEOUT.  Reading the status clears the
 * flag; the handle stays usable.
 */
dualip_status dualip_debug_abort_waits(dualip_problem* p, void* stream);

/* Message of the last failure on the calling thread ("" if none). */
const char* dualip_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DUALIP_H */
