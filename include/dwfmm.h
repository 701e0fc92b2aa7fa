/*
 * dwfmm.h -- C ABI of the GB300 dimension-weighted fast multipole method.
 *
 * Harbrecht, Multerer, Quizi, "The dimension weighted fast multipole method
 * for scattered data approximation" (arXiv 2402.09531).
 *
 * The library computes y = K_tilde x, the DW-FMM approximation of the dense
 * kernel matrix K = [phi(||x_i - x_j|| / sigma)] applied to R right-hand
 * sides (Sec. 5.2, Eq. (5.4)), and solves (K_tilde + lambda I) c = f by
 * conjugate gradients (Sec. 2, Eq. (2.2); Sec. 6.2).  Every numerical step
 * runs in CUDA kernels on one GPU; the host only validates arguments, sizes
 * allocations and sequences launches.
 *
 * Conventions shared by every entry point:
 *  - No exception crosses the ABI: every call returns a dwfmm_status.  A
 *    failed call leaves the plan in a state that dwfmm_plan_destroy accepts.
 *  - The caller owns every buffer it passes in, and the stream.  Pointers
 *    marked "host or device" may point to either; the library detects the
 *    kind with cudaPointerGetAttributes and stages host data through its own
 *    device buffers (copies are enqueued on the given stream).
 *  - The plan owns the tree-ordered copy of the sites, the interaction
 *    lists, the expansion data (nodes, V^{-1}) and all workspace.  It keeps
 *    no pointer given by the caller after a call returns.
 *  - A plan is used by one host thread and one stream at a time.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Calls return once the work is enqueued, except where
 *    stated (tree_build and solve synchronise the stream).
 *  - Matrices of right-hand sides are column-major N x R with a leading
 *    dimension ld >= N: entry (i, r) lives at x[r * ld + i], in the caller's
 *    site order.  Sites are row-major N x d with leading dimension ld >= d:
 *    coordinate k of site i lives at pts[i * ld + k].
 */
#ifndef DWFMM_H
#define DWFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DWFMM_OK = 0,
  DWFMM_ERR_INVALID_ARG = 1,   /* a NULL pointer, a size out of range, NaN/Inf sites */
  DWFMM_ERR_OOM = 2,           /* a device allocation failed */
  DWFMM_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  DWFMM_ERR_BREAKDOWN = 4,     /* CG: p^T (K_tilde + lambda I) p == 0 or not finite */
  DWFMM_ERR_NOT_CONVERGED = 5, /* CG: maxit reached before rtol */
  DWFMM_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
  DWFMM_ERR_STATE = 7,         /* call out of order (e.g. matvec before tree_build) */
  DWFMM_ERR_SINGULAR = 8       /* the Halton candidates were not unisolvent */
} dwfmm_status;

/* Radial kernels phi(r), evaluated at r = ||x - y||_2 / sigma.
 * Sec. 6.2 prints exp(+r); the positive definite exp(-r) is used (Def. 2.2). */
typedef enum {
  DWFMM_K_EXP = 0,       /* exp(-r) */
  DWFMM_K_MATERN32 = 1,  /* (1 + sqrt(3) r) exp(-sqrt(3) r) */
  DWFMM_K_GAUSS = 2      /* exp(-r^2 / 2) */
} dwfmm_kernel;

/* Arithmetic of the matvec.  FP64: every phase in float64.  FP32: near field
 * (P2P), couplings (M2L) and expansions in float32 with compensated
 * accumulation.  MIXED: FP32 with the near-field and M2L contractions
 * (targets x sources x right-hand sides) on the tensor cores when 9..16
 * right-hand sides are passed: TF32 with a hi/lo split of both operands and
 * three products (~2^-20 relative per term), FP32 accumulation, compensated
 * fold per source block.  The Gaussian takes that path in factored form
 * (exp(-|x-y|^2/(2 sigma^2)) as a product of per-site factors and
 * 2^(2 x'.y')) when |x|^2 log2(e) / (2 sigma^2) <= 30 over the sites'
 * bounding box, and the float32 CUDA-core path otherwise; results agree
 * to float32 accuracy either way.  CG dot products and vectors are float64
 * in every mode. */
typedef enum {
  DWFMM_P_FP64 = 0,
  DWFMM_P_FP32 = 1,
  DWFMM_P_MIXED = 2
} dwfmm_precision;

/* Rule for the weights omega_k of the index set Lambda (Sec. 4).
 *  INV_GAMMA:    omega_k = gamma_1 / gamma_k.
 *  PAPER_LOGRHO: Sec. 6.2, tau_k = 1 / (eta b_k) with b_k = 2 gamma_k,
 *                rho_k = e rho(tau_k) / rho(tau_1), omega_k = log rho_k,
 *                rho(tau) = 2 tau + sqrt(1 + 4 tau^2) (Lemma 4.1).
 *  EXPLICIT:     omega_k = weights[k]. */
typedef enum {
  DWFMM_W_INV_GAMMA = 0,
  DWFMM_W_PAPER_LOGRHO = 1,
  DWFMM_W_EXPLICIT = 2
} dwfmm_weight_rule;

/* Shape of the index set Lambda (the polynomial space of the expansion).
 *  TOTAL_DEGREE: sum_k omega_k alpha_k <= q, the weighted total degree set
 *                Lambda_{omega,q,d} of Sec. 4 (total degree interpolation
 *                for omega = 1, Sec. 6.1).
 *  TENSOR:       max_k omega_k alpha_k <= q, a tensor-product set; for
 *                omega = 1 the set ||alpha||_inf <= q of (q+1)^d indices
 *                that Sec. 6.1 compares against (tensor product
 *                interpolation).  No counterpart in the paper for omega != 1
 *                beyond the anisotropic reading of the same bound. */
typedef enum {
  DWFMM_I_TOTAL_DEGREE = 0,
  DWFMM_I_TENSOR = 1
} dwfmm_index_set;

/* Plan parameters.  All fields are read during dwfmm_plan_create only. */
typedef struct {
  int32_t d;                  /* dimension, 1..32 */
  int32_t kernel;             /* dwfmm_kernel */
  double sigma;               /* length scale, > 0 */
  const double* gamma;        /* host, d dimension weights gamma_k > 0 (Sec. 2, Eq. (2.3)) */
  int32_t weight_rule;        /* dwfmm_weight_rule */
  const double* weights;      /* host, d weights if EXPLICIT, else ignored */
  double q;                   /* degree of Lambda_{omega,q,d}, >= 0 (Sec. 4) */
  double eta;                 /* admissibility parameter, > 0 (Eq. (5.1)) */
  int32_t leaf_size;          /* max sites per leaf, 2..1024 (Sec. 5.1) */
  int32_t halton_candidates;  /* Halton candidates M; <= 0 selects max(2000, 10 n) (Sec. 5.4) */
  int32_t precision;          /* dwfmm_precision */
  int32_t max_rhs;            /* largest R passed to matvec/solve, 1..64 */
  int32_t index_set;          /* dwfmm_index_set; 0 (TOTAL_DEGREE) for the paper's method */
} dwfmm_config;

typedef struct dwfmm_plan_s* dwfmm_plan;

/* Create a plan: weights, the index set Lambda_{omega,q,d} (Sec. 4, enumerated
 * lexicographically in (alpha_1..alpha_d)), Halton candidates, approximate
 * Fekete nodes by greedy column-pivoted QR of the Vandermonde matrix on the
 * candidates (Sec. 5.4), V (Eq. (5.3)) and V^{-1} by Gauss-Jordan with
 * partial pivoting.  The candidate, QR and inversion steps run on the GPU in
 * float64.  Synchronises `stream`.  On success *out receives the plan.
 * Errors: INVALID_ARG (bad config), SINGULAR, OOM, CUDA. */
dwfmm_status dwfmm_plan_create(const dwfmm_config* cfg, void* stream, dwfmm_plan* out);

/* Replace the interpolation nodes by `nodes` (host, n x d row-major, in
 * [0,1]^d) and recompute V^{-1} on the GPU.  n must equal the index-set size.
 * Used to separate matvec parity from node-selection parity.  Must be called
 * before dwfmm_tree_build.  Synchronises `stream`. */
dwfmm_status dwfmm_plan_set_nodes(dwfmm_plan plan, const double* nodes, int64_t n, void* stream);

/* Build the cluster tree (Sec. 5.1: split along the longest bounding-box edge
 * into halves of ceil/floor size, the first half holding the sites smallest
 * by (x_k, position), stable), the far/near lists (Eq. (5.1): nu x nu' is far
 * iff admissible and its parent pair is not; near = non-admissible leaf
 * pairs; a pair at distance 0 is never admissible) and the per-cluster
 * expansion data.  `pts` (host or device) holds N x d sites, row-major with
 * leading dimension ld >= d; it is copied.  N = 0 is valid (matvec then does
 * nothing).  Replaces any previous tree.  Synchronises `stream`.
 * Errors: INVALID_ARG (NULL, ld < d, N < 0, non-finite site), OOM, CUDA. */
dwfmm_status dwfmm_tree_build(dwfmm_plan plan, const double* pts, int64_t n, int64_t ld,
                              void* stream);

/* y = K_tilde x for R = nrhs right-hand sides (Eq. (5.4), nested bases):
 * P2M, M2M, M2L, L2L, L2P on the far field plus the dense P2P near field.
 * x, y (host or device): float64, column-major N x R, leading dims ldx, ldy
 * >= N, caller's site order.  x and y must not overlap.  With device
 * pointers the call returns once the work is enqueued on `stream`; with a
 * host y it synchronises `stream` before returning.
 * Errors: STATE (no tree), INVALID_ARG (nrhs outside 1..max_rhs, ld < N,
 * NULL), CUDA. */
dwfmm_status dwfmm_matvec(dwfmm_plan plan, const double* x, double* y, int32_t nrhs,
                          int64_t ldx, int64_t ldy, void* stream);

/* Solve (K_tilde + lambda I) c = f for R = nrhs right-hand sides by
 * unpreconditioned conjugate gradients from c = 0 (Sec. 2 Eq. (2.2),
 * Sec. 6.2), float64 vectors and dot products, one CG per column.
 * Each column stops when its recurrence residual satisfies
 * ||r|| <= rtol ||f||.  For FP32/MIXED plans the solve runs iterative
 * refinement: the residual f - (K_tilde + lambda I) c is recomputed with the
 * float64 operator and an inner CG in the plan's precision corrects c, until
 * the float64 relative residual is <= rtol.  f, c (host or device):
 * float64, column-major N x R with leading dimension ld >= N.
 * iters_out (host, may be NULL): total CG iterations; relres_out (host, R
 * values, may be NULL): final true relative residual per column.
 * Synchronises `stream`.
 * Negative curvature (the compressed matrix can be mildly indefinite) does not
 * stop the iteration.  Errors: STATE, INVALID_ARG (lambda < 0, rtol <= 0,
 * maxit < 1), BREAKDOWN (p^T A p == 0 or not finite), NOT_CONVERGED, CUDA. */
dwfmm_status dwfmm_solve(dwfmm_plan plan, double lambda, const double* f, double* c,
                         int32_t nrhs, int64_t ld, double rtol, int32_t maxit,
                         int32_t* iters_out, double* relres_out, void* stream);

/* Incremental CG for many solves in flight (Sec. 2 Eq. (2.2), Sec. 6.2).
 * dwfmm_cg_begin starts one CG per column of f (device, column-major N x R,
 * leading dimension ld >= N; copied) on (K_tilde + lambda I) c = f from
 * c = 0; dwfmm_cg_step enqueues `iters` iterations on `stream` with every
 * scalar kept on the device (alpha, beta, per-column convergence
 * ||r|| <= rtol ||f|| and breakdown p^T A p == 0 are decided on the GPU), so
 * it never synchronises and solves on different plans and streams overlap;
 * the matvec uses the plan's precision.  dwfmm_cg_poll never blocks: *ready
 * = 1 once the work of the last dwfmm_cg_step (or dwfmm_batch_cg_step) since
 * the last dwfmm_cg_begin has finished (0 before the first), and then status
 * (R int32: 0 running, 1 converged, 2 breakdown), iters (R int32) and rr (R
 * doubles, ||r||^2) describe that point (any may be NULL).
 * dwfmm_cg_result copies the current c (host or device, ld >= N; a host
 * copy synchronises `stream`).  On a stream other than the legacy default
 * stream and with the phase timers off, dwfmm_cg_step captures its
 * iterations into a CUDA graph the second time it is called with the same
 * tree, R, lambda, iteration count and stream, and replays that graph from
 * then on (small problems are bound by the host's kernel-launch rate); the
 * first call with a new combination launches plainly, and so does every
 * call if a capture ever fails.  The results are identical either way.
 * Errors: STATE (no tree / no cg_begin), INVALID_ARG (f not a device buffer,
 * nrhs outside 1..max_rhs), CUDA. */
dwfmm_status dwfmm_cg_begin(dwfmm_plan plan, double lambda, const double* f, int32_t nrhs, int64_t ld,
                            double rtol, void* stream);
dwfmm_status dwfmm_cg_step(dwfmm_plan plan, int32_t iters, void* stream);
dwfmm_status dwfmm_cg_poll(dwfmm_plan plan, int32_t* ready, int32_t* status, int32_t* iters, double* rr);
dwfmm_status dwfmm_cg_result(dwfmm_plan plan, double* c, int64_t ld, void* stream);

/* r = f - (K_tilde + lambda I) c with the float64 operator whatever the
 * plan's precision (the outer residual of iterative refinement).  f, c, r:
 * host or device, column-major N x nrhs with leading dimension ld >= N; r
 * may be NULL.  relres (host, nrhs doubles, may be NULL) receives
 * ||r|| / ||f|| per column.  Synchronises `stream`. */
dwfmm_status dwfmm_residual(dwfmm_plan plan, double lambda, const double* f, const double* c, double* r,
                            int32_t nrhs, int64_t ld, double* relres, void* stream);

/* One step of iterative refinement with a minimal-residual step length (the
 * paper runs plain CG; this is the solver's own safeguard for reduced-
 * precision plans).  On entry r holds the float64 residual
 * f - (K_tilde + lambda I) c and delta a correction, typically an inner CG
 * solve of the plan's reduced-precision system with right-hand side r.  Per
 * column, a* = (r, A delta) / (A delta, A delta) with the float64 operator A
 * minimises ||r - a A delta||; the step is alpha = 1 (plain refinement)
 * when a* > 1/2, where that lowers the residual, else alpha = a* (0 when
 * A delta = 0 or a* is not finite).  Then c += alpha delta and
 * r -= alpha A delta, so the float64 residual never grows, also when the
 * float32 operator's error approaches lambda and the inner solve returns a
 * poor correction (plain refinement, c += delta, then diverges).  f, c, delta, r: host or device,
 * column-major N x nrhs, leading dimension ld >= N; c and r are updated in
 * place.  alpha and relres (host, nrhs doubles each, may be NULL) receive the
 * step lengths and ||r|| / ||f|| after the step.  Synchronises `stream`.
 * dwfmm_residual and dwfmm_refine use the incremental CG's scratch: call them
 * between solves (after dwfmm_cg_result, before the next dwfmm_cg_begin), not
 * between dwfmm_cg_step calls of one solve.  Errors: STATE (no tree),
 * INVALID_ARG (NULL buffer, ld < N, nrhs outside 1..max_rhs), CUDA. */
dwfmm_status dwfmm_refine(dwfmm_plan plan, double lambda, const double* f, double* c, const double* delta,
                          double* r, int32_t nrhs, int64_t ld, double* alpha, double* relres, void* stream);

/* The kernel interpolant at new points (Sec. 2: s_X(x) = sum_j alpha_j
 * K(x_j, x); Sec. 6.2 measures its prediction error at test points):
 * out(t, r) = sum_j phi(||x_t - x_j|| / sigma) c(j, r) for t < nt, evaluated
 * exactly (every target against every site, no compression) in the plan's
 * precision (float32 plans: d <= 20).  targets (host or device): nt x d
 * row-major, leading dimension ld_t >= d; c (host or device): column-major
 * N x nrhs, ld_c >= N, the caller's site order; out (host or device):
 * column-major nt x nrhs, ld_o >= nt.  Synchronises `stream`.
 * Errors: STATE (no tree), INVALID_ARG, OOM, CUDA, TIMEOUT. */
dwfmm_status dwfmm_evaluate(dwfmm_plan plan, const double* targets, int64_t nt, int64_t ld_t, const double* c,
                            int64_t ld_c, double* out, int64_t ld_o, int32_t nrhs, void* stream);

/* Batches: many uneven problems in one fused matvec (float32 plans).
 * dwfmm_batch_create groups `count` plans whose trees are built, with equal
 * kernel, index-set size |Lambda| and leaf block size (equal leaf_size and
 * N >= leaf_size), d <= 16 and precision FP32 or MIXED; nrhs[i] (1..16) is
 * the number of right-hand sides of problem i for every later call.  The
 * near field of all problems is one launch of the kernel-summation engine,
 * the couplings (M2L) of all problems another, the upward and downward
 * passes one launch per tree height/level; the launch shape of each of the
 * two fused launches (CTA width; one padded launch or one per right-hand-side
 * class) is chosen by timing every candidate on the batch's data, and the
 * whole sequence is captured as a CUDA graph.
 * The plans must stay alive and keep their trees while the batch exists.
 * Synchronises `stream` before it starts.
 * dwfmm_batch_matvec: y[i] = K_tilde_i x[i] for every problem, x[i] and y[i]
 * device buffers, column-major N_i x nrhs[i] with leading dimension N_i;
 * enqueued on `stream` (one graph launch).
 * dwfmm_batch_info: split (1 if the near field runs one launch per class),
 * tune_ms (2 doubles: near field + couplings at their best padded shapes, and
 * at their best shapes with per-class launches allowed) and the total number
 * of leaves; any output pointer may be NULL.
 * Errors: INVALID_ARG, STATE (a plan without a tree), OOM, CUDA. */
typedef struct dwfmm_batch_s* dwfmm_batch;
dwfmm_status dwfmm_batch_create(const dwfmm_plan* plans, const int32_t* nrhs, int32_t count, void* stream,
                                dwfmm_batch* out);
dwfmm_status dwfmm_batch_matvec(dwfmm_batch batch, const double* const* x, double* const* y, void* stream);
dwfmm_status dwfmm_batch_info(dwfmm_batch batch, int32_t* split, double* tune_ms, int64_t* leaves);

/* Launch shapes the batch's autotuner chose at creation (every candidate
 * timed on the batch's own data): shape[0] 1 if the near field runs one
 * launch per right-hand-side class, shape[1] its threads per CTA (each
 * thread owns 2 targets per pass: 32, 64, 96 or 128), shape[2], shape[3]
 * the same for the couplings (M2L).  `shape` is a host array of 4 int32.
 * Errors: INVALID_ARG (NULL batch or shape).  No counterpart in the paper. */
dwfmm_status dwfmm_batch_shape(dwfmm_batch batch, int32_t* shape);

/* Engines of a batch matvec.  0: the captured graph of launches described at
 * dwfmm_batch_create.  1: one persistent cooperative launch for the whole
 * matvec (every CTA resident; the phases separated by grid-wide barriers
 * whose waits are bounded: a wait that gives up ends the launch early and
 * raises the batch's device error flag instead of hanging; at creation that
 * makes the engine unavailable).  In it, CTAs that have finished their
 * share of a far-field phase (the upward pass by height, the couplings from
 * a work queue, the downward pass by level) take near-field target groups
 * from a second work queue while they wait, and all right-hand-side classes
 * share the queues; near-field and coupling target groups run on groups of
 * 32, 64 or 128 threads of a CTA.  Both engines sum every target in the same
 * order: their results are equal bit for bit.  When the batch's fused near
 * field and couplings take at least 2 ms (the launch tuner's time), creation
 * times the persistent engine at every near-field group width against the
 * graph (both without the gather and scatter) and uses the faster, if the
 * device can launch it and a stream capture holds it; smaller batches (a
 * serving loop rebuilds them often) start on the graph and tune the
 * persistent engine at the first request for it.
 * dwfmm_batch_engine: engine[0] the engine in use, engine[1] 1 if the
 *   persistent engine is available (0 also while it is not tuned); ms[0],
 *   ms[1] the best timed matvec of each engine (-1 if not timed);
 *   launch[0..2] the persistent launch's CTAs and the near-field and
 *   coupling group widths (0 if not available).  Host arrays of 2, 2 and 3
 *   elements.
 * dwfmm_batch_set_engine: selects engine 0 or 1 for later matvecs and
 *   batched CG steps; the first selection of 1 on a batch whose persistent
 *   engine is not tuned yet tunes it then (synchronising the device first:
 *   the timing runs use the batch's buffers); DWFMM_ERR_STATE if 1 is not
 *   available.
 * Errors: INVALID_ARG (NULL batch or output, engine outside 0..1).  No
 * counterpart in the paper (a scheduling choice). */
dwfmm_status dwfmm_batch_engine(dwfmm_batch batch, int32_t* engine, double* ms, int32_t* launch);
dwfmm_status dwfmm_batch_set_engine(dwfmm_batch batch, int32_t engine);

/* Batched CG (Sec. 2, Eq. (2.2); the CG of Sec. 6.2): `iters` iterations of
 * the incremental CG of every problem of the batch, each begun with
 * dwfmm_cg_begin on its plan (its own lambda, right-hand sides and rtol,
 * nrhs equal to the problem's batch nrhs).  Every iteration computes
 * Ap = K_tilde p of all problems as one fused batch matvec and updates all
 * problems' vectors with fused kernels; the per-column decisions are those of
 * dwfmm_cg_step (a column stops on convergence or breakdown, the others go
 * on).  Enqueued on `stream`; afterwards each plan's dwfmm_cg_poll and
 * dwfmm_cg_result read its state as after dwfmm_cg_step.  Inner products use
 * a fixed partition, so the result does not depend on timing.  Errors:
 * DWFMM_ERR_STATE if a plan has no CG begun, DWFMM_ERR_INVALID_ARG if its
 * right-hand-side count differs from the batch's. */
dwfmm_status dwfmm_batch_cg_step(dwfmm_batch batch, int32_t iters, void* stream);
dwfmm_status dwfmm_batch_destroy(dwfmm_batch batch);

/* Release every resource of the plan (NULL is accepted).  Synchronises the
 * plan's last stream first. */
dwfmm_status dwfmm_plan_destroy(dwfmm_plan plan);

/* Static description of a status code. */
const char* dwfmm_status_string(dwfmm_status s);

/* Message of the last failed call on this plan ("" if none). */
const char* dwfmm_last_error(dwfmm_plan plan);

/* Sizes: n_x = |Lambda|, n_far / n_near = block counts, depth = J.
 * Any output pointer may be NULL.  depth = -1 before tree_build. */
dwfmm_status dwfmm_plan_info(dwfmm_plan plan, int64_t* n_x, int64_t* n_far, int64_t* n_near,
                             int32_t* depth);

/* Which engine evaluated the near field N (Eq. (5.1)) in the plan's last
 * matvec (*engine, -1 before the first): 0 float64, one CTA per target leaf
 * over its near list; 1 float64, each unordered near pair of leaves once;
 * 2 float32 on the CUDA cores; 3 MIXED, contraction on the tensor cores (TF32
 * hi/lo, every ordered pair); 4 MIXED, each unordered near pair once, FP16
 * hi/lo on the tensor cores with fixed-point transposed sums; 5 as 4, with
 * the Gaussian's exponent 2x'.s' also on the tensor cores. */
dwfmm_status dwfmm_near_engine(dwfmm_plan plan, int32_t* engine);

/* Which engine ran the expansion phases (P2M, M2M, L2L, L2P and the V^{-T},
 * V^{-1} transforms of Sec. 5.2, Eq. (5.4)) in the plan's last matvec
 * (*engine, -1 before the first): 0 float64 CUDA cores; 1 float32 CUDA
 * cores; 2 MIXED on the tensor cores: basis values and right-hand sides
 * (scaled per column by a power of two) split into FP16 hi + lo,
 * hi*hi + hi*lo + lo*hi accumulated in FP32 by tcgen05.mma, per-cluster
 * contractions in 64-wide chunks folded in FP32, the transforms one GEMM per
 * tree level with the constant V^{-1} tile.  MIXED plans take engine 2 when
 * |Lambda| <= 128, leaves hold 128 or 256 sites and a multi-index has at
 * most 20 nonzero entries; otherwise engine 1.  Errors: INVALID_ARG. */
dwfmm_status dwfmm_far_engine(dwfmm_plan plan, int32_t* engine);

/* Which engine ran the couplings (M2L, Eq. (5.4): the far blocks S_{t,s}
 * applied to the node charges) in the plan's last matvec (*engine, -1 before
 * the first): 0 float64 CUDA cores; 1 float32 CUDA cores; 2 MIXED, every
 * ordered far pair, contraction on the tensor cores (TF32 hi/lo); 3 MIXED,
 * each unordered far pair (t, s > t) once on the symmetric tensor-core
 * engine of the near field (FP16 hi/lo, fixed-point transposed sums, node
 * sets padded to 128 slots).  For MIXED plans with 9..16 right-hand sides
 * the engine is the caller's choice (dwfmm_plan_set_m2l_engine) or, by
 * default, the faster of 2 and 3 as timed once per tree (engine 3 needs
 * |Lambda| <= 128 and a symmetric far list).  Errors: INVALID_ARG. */
dwfmm_status dwfmm_m2l_engine(dwfmm_plan plan, int32_t* engine);

/* Choose the M2L engine of MIXED matvecs with 9..16 right-hand sides:
 * -1 (the default) times engines 2 and 3 at the first such matvec of each
 * tree (before its near field starts, on the plan's moment buffer, zeroed)
 * and keeps the faster; 2 or 3 forces that engine (3 falls back to 2 where
 * it does not apply).  Both meet the float32 tolerance; engine 3 evaluates
 * each far pair once and is the more accurate.  Takes effect at the next
 * matvec.  Errors: INVALID_ARG (another value).  No counterpart in the
 * paper. */
dwfmm_status dwfmm_plan_set_m2l_engine(dwfmm_plan plan, int32_t engine);

/* The timing behind the default choice: ms[0] engine 3, ms[1] engine 2 (one
 * M2L each, -1 where not timed or not applicable).  `ms`: host, 2 doubles. */
dwfmm_status dwfmm_m2l_tune_ms(dwfmm_plan plan, double* ms);

/* Copy out plan data (host buffers, NULL to skip), for tests and tools:
 *  weights: d doubles; lam: n x d int32 multi-indices (row-major);
 *  nodes: n x d doubles; pivots: n int32 Halton indices (0-based, -1 if the
 *  nodes were set by dwfmm_plan_set_nodes); vinv: n x n doubles, row-major. */
dwfmm_status dwfmm_plan_export(dwfmm_plan plan, double* weights, int32_t* lam, double* nodes,
                               int32_t* pivots, double* vinv);

/* Copy out the tree (host buffers, NULL to skip): perm (N int64, tree
 * position -> caller index), begin/end (2^{J+1}-1 int64 each, heap order:
 * level j holds clusters 2^j-1 .. 2^{j+1}-2), lo/hi (clusters x d doubles). */
dwfmm_status dwfmm_tree_export(dwfmm_plan plan, int64_t* perm, int64_t* begin, int64_t* end,
                               double* lo, double* hi);

/* Copy out the lists (host buffers, NULL to skip): far (n_far x 2 int32
 * (target, source) cluster ids sorted by level, target, source) and near
 * (n_near x 2 int32, sorted by target, source). */
dwfmm_status dwfmm_lists_export(dwfmm_plan plan, int32_t* far, int32_t* near);

/* Phase timing.  With enable != 0 every later matvec records CUDA events on
 * the streams that launch each phase (enable = 1: the near field still runs
 * on its own stream, concurrently with the far field, as in production;
 * enable = 2: the near field runs on the caller's stream after the far field,
 * so each phase is timed alone).  dwfmm_phase_times returns, per phase,
 * the summed milliseconds since the last reset and the launch counts:
 * ms[0] gather, [1] P2M+M2M, [2] M2L, [3] L2L+L2P, [4] P2P, [5] scatter,
 * [6] whole matvec; launches[i] the number of kernel launches of phase i.
 * Reading the times synchronises the plan's streams. */
dwfmm_status dwfmm_set_profiling(dwfmm_plan plan, int32_t enable);
dwfmm_status dwfmm_phase_times(dwfmm_plan plan, double* ms, int64_t* launches, int32_t reset);

/* Exact direct sum y = K x over all N sites (no tree, no compression) that
 * allocates no memory: for callers that cannot call cudaMalloc, such as a
 * host application whose framework owns the device memory pool (its caching
 * allocator has reserved nearly all of it) or a latency-critical loop that
 * cannot take the device synchronisation of cudaMalloc/cudaFree.  The paper
 * has no counterpart of this entry point; it reuses the library's float32
 * near-field kernel on blocks of 256 sites.
 *
 * pts, x, y: device pointers (float64) of the current device (or managed
 * memory); unlike dwfmm_matvec this entry point does not stage host
 * buffers, and a host pointer returns DWFMM_ERR_INVALID_ARG.  pts is N x d
 * row-major (leading dimension ld_pts >= d); x and y are column-major
 * N x nrhs (leading dimensions ldx, ldy >= N).  Limits: N <= 8192,
 * 1 <= d <= 16, 1 <= nrhs <= 16; larger sizes return DWFMM_ERR_INVALID_ARG.
 * The result is float32-accurate (relative error ~1e-7); a bounded
 * shared-memory wait that gave up writes NaN into y.
 *
 * All intermediates live in one fixed device array of about 1.6 MB inside
 * the library, which every GPU that loads the library keeps until the
 * process exits.  The first call on each device sets kernel attributes and
 * looks up that array's device address (no allocation); make that first
 * call before any stream capture: a first call made while `stream` is
 * capturing returns DWFMM_ERR_STATE.  Later calls outside capture look the
 * address up again.  The array is shared by all calls on a device and keeps
 * the last call's contents; each call rewrites what it reads, so calls
 * ordered on one stream are safe, but calls whose work overlaps on the GPU
 * (e.g. on unsynchronised streams) race on it.  Work is enqueued on
 * `stream`; the call does not synchronise. */
dwfmm_status dwfmm_direct_sum_noalloc(int32_t kernel, double sigma, const double* pts, int64_t n,
                                      int32_t d, int64_t ld_pts, const double* x, double* y,
                                      int32_t nrhs, int64_t ldx, int64_t ldy, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DWFMM_H */
