/*
 * fmmpc.h -- C ABI of the GB300 FMM-BEM preconditioner library (libfmmpc.so).
 *
 * Method: Ibeid, Yokota, Pestana and Keyes, "Fast Multipole Preconditioners for Sparse
 * Matrices Arising from Elliptic Equations" (arXiv:1308.3339).  A Krylov solve of the
 * 5-point finite-difference Poisson system -lap u = f on a square, u = g on its boundary
 * (Sec. 2.1, Eqs. e:p and e:axb), preconditioned by z = P^{-1} r: a free-space Laplace
 * FMM over every grid node (Sec. 5) plus a boundary-element correction that enforces
 * z = 0 on the boundary (Sec. 3.2 Fig. f:flow_chart, Sec. 4.1 Eqs. e:ubound/e:uinter).
 *
 * Conventions for every call:
 *  - Grid vectors are FP64, row-major [n_rhs][ny][nx] with x fastest, in the natural
 *    (not Morton) order, interior nodes only: node (i, j), 0-based, sits at
 *    (x0 + (i+1) h, y0 + (j+1) h) with h = (x1 - x0) / (nx + 1).
 *  - Boundary data g is FP64 [n_rhs][4 n]: the Dirichlet values at the stencil neighbours
 *    outside the interior block, in the order bottom (x increasing), right (y increasing),
 *    top (x decreasing), left (y decreasing).  Corners are never used.
 *  - "_dev" pointers are device memory owned by the caller; the library never frees or
 *    keeps them past the call.  "_host" pointers are host memory (pinned or pageable).
 *  - The handle owns every internal buffer (tree, lists, expansions, BEM inverse, Krylov
 *    basis, graphs) and its CUDA stream binding; one handle is used by one host thread
 *    at a time.  Calls are stream-ordered on the handle's stream; fmmpc_apply returns
 *    without synchronising, fmmpc_solve returns after its convergence test.
 *  - Return value: FMMPC_OK (0) or a negative FMMPC_ERR_* code; no exception or abort
 *    crosses the ABI.  fmmpc_last_error() gives a message for the last failure.
 */
#ifndef FMMPC_H
#define FMMPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMMPC_OK 0
#define FMMPC_ERR_INVALID (-1)       /* bad argument or unsupported grid */
#define FMMPC_ERR_OOM (-2)           /* device or host allocation failed */
#define FMMPC_ERR_CUDA (-3)          /* a CUDA call failed */
#define FMMPC_ERR_NOT_CONVERGED (-4) /* solve stopped at maxit above rtol */
#define FMMPC_ERR_NAN (-5)           /* NaN or Inf met in a residual norm */
#define FMMPC_ERR_TIMEOUT (-6)       /* a bounded device wait ran out */
#define FMMPC_ERR_UNSUPPORTED (-7)   /* valid request this build does not implement */

/* FMM arithmetic inside the preconditioner.  The Krylov recurrences, inner products,
 * residual checks and the boundary-element solve are FP64 in every mode. */
#define FMMPC_PREC_FP64 0       /* FMM in FP64 on CUDA cores (plain FP64 form) */
#define FMMPC_PREC_FP32 1       /* FMM in FP32 on CUDA cores (plain FP32 form) */
#define FMMPC_PREC_MIXED_BF16 2 /* FP32 P2P/expansions, M2L on tensor cores in BF16, FP32 accumulate */
#define FMMPC_PREC_MIXED_TF32 3 /* FP32 P2P/expansions, M2L on tensor cores in TF32, FP32 accumulate */
/* In the mixed forms the volume-to-volume M2L (Sec. 5.3 item 3) of every level >= 2 runs as
 * a lattice convolution on the tensor cores: the leading multipoles and their translation
 * columns are split hi + lo, so the apply stays within ~1e-4 of the FP64 FMM (p <= 15;
 * larger p keeps the FP32 CUDA-core M2L).  Boundary-source M2L stays on CUDA cores. */

#define FMMPC_CG 0
#define FMMPC_GMRES 1
#define FMMPC_FGMRES 2

typedef struct fmmpc_handle fmmpc_handle;

/* Square grid of nx = ny interior nodes on [x0, x1] x [y0, y1] with x1-x0 = y1-y0. */
typedef struct {
  int32_t nx, ny;
  double x0, y0, x1, y1;
} fmmpc_grid;

/* p: expansion order, coefficients n = 0..p-1 (Sec. 5.3); p must be one of 4, 6, 8, 10, 12, 16
 *   (the kernels are compiled for these orders; any other value is rejected with _INVALID).
 * leaf_max: the tree splits a cell at its centre lines while it holds more than leaf_max
 *   nodes (Sec. 5.1); the grid must stay divisible down to the leaf (nx = m 2^L) and the
 *   leaf side m must be 4, 8 or 16.
 * theta: MAC (R_A + R_B) < theta |c_A - c_B| of the dual tree traversal (Sec. 5.2), R the
 *   half-diagonal; 0 < theta < 1, taken as the rational round(1000 theta)/1000.
 * precision: FMMPC_PREC_*.  n_rhs: largest number of right-hand sides per call.
 * autotune: 0 = use p and leaf_max as given; see fmmpc_autotune for the tuner. */
typedef struct {
  int32_t p;
  int32_t leaf_max;
  double theta;
  int32_t precision;
  int32_t n_rhs;
  int32_t autotune;
} fmmpc_params;

/* method: FMMPC_CG | FMMPC_GMRES | FMMPC_FGMRES; restart: Krylov basis size m of
 * (F)GMRES(m); maxit: cap on preconditioner applications; rtol: stop when the relative
 * residual ||b - A u|| / ||b|| <= rtol (Sec. 6 stops at a relative-residual drop).
 * use_graphs: how the iteration is driven.
 *   0: a host loop; every kernel launched one by one, and the host reads the Hessenberg
 *      column (or the CG scalars) after every step to decide convergence.
 *   1: the same host loop, each preconditioner application replayed from its CUDA graph.
 *   2: the whole solve is one CUDA graph launched once: set-up, a conditional WHILE node
 *      whose body is one Arnoldi step (or one CG iteration), and the final true residual.
 *      The Givens rotations, the residual estimate, the convergence decision and the back
 *      substitution run on the device and set the loop's condition; the loop is bounded by
 *      maxit.  The host waits once, for the report.  Graphs are kept per (method, restart,
 *      n_rhs, g present) and rebuilt when the workspace grows. */
typedef struct {
  int32_t method;
  int32_t restart;
  int32_t maxit;
  double rtol;
  int32_t use_graphs;
} fmmpc_solve_opts;

/* Per-solve report.  rel_res is the true residual recomputed in FP64 at the end
 * (largest over right-hand sides); iters the preconditioner applications of the
 * slowest right-hand side; status FMMPC_OK or FMMPC_ERR_NOT_CONVERGED / _NAN. */
typedef struct {
  int32_t iters;
  double rel_res;
  double t_setup_ms;
  double t_solve_ms;
  int32_t status;
} fmmpc_solve_info;

/* Set-up, the analogue of the paper's PCSetUp (Sec. 7.1): Morton keys and radix sort
 * of the nodes, quadtree (Sec. 5.1), dual-tree-traversal interaction lists (Sec. 5.2),
 * translation tables, boundary elements and the FP64 inverse of the single-layer BEM
 * matrix (Sec. 4.3), workspace.  stream: a cudaStream_t (NULL = legacy default stream)
 * on which every later call of this handle runs.  On success *out owns all of it and
 * must be released with fmmpc_destroy.  Errors: _INVALID (grid/params), _OOM, _CUDA. */
int fmmpc_create(fmmpc_handle **out, const fmmpc_grid *g, const fmmpc_params *prm, void *stream);

/* Preconditioner action z = P^{-1} r (Sec. 3.2, PCApply): for each right-hand side,
 * (1) FMM volume potential V r of Eq. e:volume_integral at the nodes and at the boundary
 * collocation points, (2) q = S^{-1}(-(V r)|_Gamma), Eq. e:ubound with z = 0 on Gamma,
 * (3) z = V r + int_Gamma q G, Eq. e:uinter.  r_dev, z_dev: [n_rhs][ny][nx] FP64
 * device, not aliased; 1 <= n_rhs <= params.n_rhs.  Asynchronous on the handle stream. */
int fmmpc_apply(fmmpc_handle *h, const double *r_dev, double *z_dev, int32_t n_rhs);

/* Same as fmmpc_apply with host buffers: copies r in, applies, copies z out and
 * synchronises the stream before returning. */
int fmmpc_apply_host(fmmpc_handle *h, const double *r_host, double *z_host, int32_t n_rhs);

/* Parts of the apply, for testing each stage against the oracle.  part:
 *  0 full P^{-1} r (as fmmpc_apply);
 *  1 V r at the nodes: the volume FMM alone, Eq. e:volume_integral, no boundary term;
 *  2 the near-field (P2P) part of V r alone, in physical units;
 *  3 V r at the N_Gamma = 4n collocation points (out holds [n_rhs][4n] values);
 *  4 q = S^{-1}(-(V r)|_Gamma), the boundary density of Eq. e:ubound ([n_rhs][4n]). */
int fmmpc_apply_part(fmmpc_handle *h, int32_t part, const double *r_dev, double *out_dev,
                     int32_t n_rhs);

/* The boundary-integral solution of -lap u = f in the square, u = g on its boundary
 * (Sec. 4.1): q = du/dn from Eq. e:ubound, S q = (1/2 I + K) g - (V f)|_Gamma, then
 * Eq. e:uinter at the nodes, u = V f + int_Gamma q G - int_Gamma g dG/dn (V f by the FMM;
 * the double-layer term -D g through the boundary tree with the element ends as point
 * sources of weight +-i g, and closed-form element integrals next to the boundary).  This
 * is the preconditioner's own construction with the boundary values kept: with g = 0 it is
 * fmmpc_apply.  Constant elements make it first-order accurate in h (Sec. 6.2).
 * f_dev, u_dev: [n_rhs][ny][nx] FP64 device (distinct); g_dev: [n_rhs][4n] FP64 device,
 * the Dirichlet values at the 4n element midpoints (the collocation points: side length
 * / n apart from half an element past each corner), in the order bottom (x increasing),
 * right (y increasing), top (x decreasing), left (y decreasing).  The boundary solve is
 * FP64 in every form.  Uses the single-layer equations whatever fmmpc_set_bem_form set.
 * Asynchronous on the handle's stream.  Errors: _INVALID. */
int fmmpc_apply_bc(fmmpc_handle *h, const double *f_dev, const double *g_dev, double *u_dev, int32_t n_rhs);

/* The transpose of the preconditioner, rb = P^{-T} zb: the gradient of a loss of z = P^{-1} r
 * with respect to the source weights r, given its gradient zb with respect to z.  With
 * P^{-1} = V - S_OG S^{-1} V_GO (Sec. 3.2, Eqs. e:ubound and e:uinter with z = 0 on Gamma):
 * P^{-T} = V - V_GO^T S^{-T} S_OG^T, V symmetric.  The FMM-transpose pass runs the apply's
 * volume FMM on zb, takes the element integrals of that potential over the 4n boundary
 * elements (S_OG^T zb: the local expansions integrated in closed form, closed-form log
 * integrals next to the boundary), applies S^{-T} (the side-DFT blocks transposed, FP64;
 * formed on first use), and sums the resulting point sources at the collocation points
 * back into the nodes through the boundary FMM tree (V_GO^T).  Accurate to the FMM
 * truncation against the exact transpose.  zb_dev, rb_dev: [n_rhs][ny][nx] FP64 device,
 * distinct.  Single-layer form only (_UNSUPPORTED after fmmpc_set_bem_form(DOUBLE_LAYER)).
 * Errors: _INVALID, _UNSUPPORTED. */
int fmmpc_apply_transpose(fmmpc_handle *h, const double *zb_dev, double *rb_dev, int32_t n_rhs);

/* Boundary correction of the preconditioner.
 *  FMMPC_BEM_SINGLE_LAYER (default): the paper's, Eq. e:ubound with z = 0 on Gamma, a
 *    first-kind single-layer system S q = -(V r)|_Gamma, then z = V r + int_Gamma q G.
 *  FMMPC_BEM_DOUBLE_LAYER: a second-kind double-layer correction with the same continuum
 *    limit, (-1/2 I + K) mu = -(V r)|_Gamma, then z = V r + int_Gamma mu dG/dn (its inverse
 *    formed on first selection, like S's, from the side-DFT blocks).  fmmpc_apply_part
 *    part 4 then returns mu.
 * Captured apply and solve graphs of the other form are dropped.  Errors: _INVALID. */
#define FMMPC_BEM_SINGLE_LAYER 0
#define FMMPC_BEM_DOUBLE_LAYER 1
int fmmpc_set_bem_form(fmmpc_handle *h, int32_t form);

/* y = A x with zero boundary values: the operator chosen by fmmpc_set_operator (the
 * five-point stencil of Eq. e:axb by default). */
int fmmpc_spmv(fmmpc_handle *h, const double *x_dev, double *y_dev, int32_t n_rhs);

/* Krylov solve of A u = b with b = f + (boundary values g of the stencil neighbours)/h^2
 * (Sec. 3.1, Eq. e:axb), right-preconditioned by P^{-1} (Sec. 3.2), FP64 recurrences.
 * f_dev [n_rhs][ny][nx]; g_dev [n_rhs][4n] or NULL for g = 0; u_dev holds the initial
 * iterate on entry (zeros for the paper's setting) and the solution on exit.  info may
 * be NULL.  Returns FMMPC_OK when every right-hand side met rtol, FMMPC_ERR_NOT_CONVERGED
 * when one stopped at maxit (u_dev still holds the last iterate), FMMPC_ERR_NAN. */
int fmmpc_solve(fmmpc_handle *h, const double *f_dev, const double *g_dev, double *u_dev,
                int32_t n_rhs, const fmmpc_solve_opts *opts, fmmpc_solve_info *info);

/* fmmpc_solve with host buffers (copies in, solves, copies u out). */
int fmmpc_solve_host(fmmpc_handle *h, const double *f_host, const double *g_host,
                     double *u_host, int32_t n_rhs, const fmmpc_solve_opts *opts,
                     fmmpc_solve_info *info);

/* Sizes of the set-up, for buffer allocation by fmmpc_export callers.  what:
 *  0 L (leaf level), 1 leaf side m, 2 #M2L pairs, 3 #P2P pairs, 4 #M2L volume-boundary
 *  pairs, 5 #P2P volume-boundary pairs, 6 N_Gamma, 7 #cells (all levels), 8 #nodes,
 *  9 distinct P2P leaf offsets, 10 kernel launches of the last apply, 11 device bytes
 *  held by the handle, 12 device error flags of the tensor-core kernels (non-zero: a
 *  bounded wait gave up; bits 0-7 P2P, 8-15 M2L; synchronises), 13 1 if the near field
 *  runs on the tensor cores, 14 tensor-core M2L: 0 off, 1 TF32, 2 BF16. */
int fmmpc_query(const fmmpc_handle *h, int32_t what, int64_t *value);

/* Copies an internal array of the set-up to host memory dst (bytes = capacity).  what:
 *  0 Morton keys u32 [N] (natural order); 1 permutation i32 [N] (Morton position ->
 *  natural index); 2 cell starts i32 [#cells]; 3 M2L list i32 [#][3] (level, target,
 *  source); 4 P2P list i32 [#][2]; 5 volume-boundary M2L list i32 [#][3] (level, volume
 *  cell, boundary cell); 6 volume-boundary P2P list i32 [#][2].  Lists are in canonical
 *  (level, target, source) order.  Errors: _INVALID if bytes is too small. */
int fmmpc_export(fmmpc_handle *h, int32_t what, void *dst, int64_t bytes);

/* Near-field engine: 0 (the default) the tensor-core lattice P2P where the grid allows it
 * (8x8 leaves, at least 128 leaves per row, FP32 or mixed precision; three FP16 products
 * per pair with each source leaf's weights scaled by a power of two, FP32-accurate in every
 * single-precision form), 1 the CUDA-core kernel. */
int fmmpc_set_p2p_engine(fmmpc_handle *h, int32_t engine);

/* Operator of the Krylov solves, fmmpc_spmv and the right-hand side folding (the
 * preconditioner stays the constant-coefficient FMM-BEM P of the handle):
 *  FMMPC_OP_FD5 (default): the five-point stencil (1/h^2)(4 u_ij - neighbours), Eq. e:axb.
 *  FMMPC_OP_FD5_VAR: -div(a grad u) (Sec. 2.1 Eq. e:p with a variable diffusion
 *    coefficient, Sec. 4.4 and Sec. 6.4), five-point flux form: the coefficient of the face
 *    between two nodes is the mean of a at the two nodes.  a_dev: FP64 device array of
 *    (n+2)^2 values at the nodes of the full grid including the boundary ring, row-major,
 *    interior node (i, j) at (j+1)(n+2) + (i+1); copied by the call (the caller keeps
 *    ownership).  Boundary data g enters through the face coefficient.  Sec. 6.4
 *    preconditions this operator with the constant-coefficient P, as here.
 *  FMMPC_OP_Q1: the Q1 bilinear finite-element stiffness of -lap, the paper's
 *    discretisation (Sec. 6.1): 8/3 on the diagonal, -1/3 for the eight neighbours; the
 *    right-hand side is the lumped load b = h^2 f; the preconditioner acts on M^{-1} r, M
 *    the consistent Q1 mass matrix (the finite-element function of the residual), through
 *    tridiagonal solves along the rows and columns.  Boundary data is rejected (_INVALID):
 *    the nine-point stencil would need the corner values.
 * a_dev is ignored unless op = FMMPC_OP_FD5_VAR.  Errors: _INVALID. */
#define FMMPC_OP_FD5 0
#define FMMPC_OP_FD5_VAR 1
#define FMMPC_OP_Q1 2
int fmmpc_set_operator(fmmpc_handle *h, int32_t op, const double *a_dev);

/* on = 1 (the default): fmmpc_apply records its kernels once per distinct (r, z, n_rhs)
 * into a CUDA graph on an internal stream and replays it (ordered after and before the
 * handle's stream with events); on = 0: launches the kernels one by one.  Either way,
 * with stage timing off, the full apply runs the tensor-core near field, the volume M2L
 * and the near-boundary correction on three further internal streams, forked and joined
 * with events, so they overlap the boundary chain; the result is the same bit for bit as
 * with the stages in order on one stream.  fmmpc_solve follows its own opts.use_graphs
 * instead.  Up to 64 graphs are kept per handle. */
int fmmpc_set_graphs(fmmpc_handle *h, int32_t on);

/* Per-stage timing of fmmpc_apply with CUDA events recorded on the handle's stream; with
 * timing on, the apply runs its stages in order on that one stream (no overlap).
 * fmmpc_set_timing(h, 1) creates the events and turns recording on for every stage; 2
 * records only the four events around the M2L (stage 5) and P2P (stage 9) kernels, so the
 * rest of the apply runs without event records; 0 turns recording off.
 * fmmpc_get_timing synchronises the stream and writes the durations in milliseconds of
 * the stages of the last apply into ms[0 .. min(cap, count)), *count = 11 stages:
 *  0 weight image, 1 P2M + M2M (Sec. 5.3 items 1-2), 2 collocation pass (M2L to boundary
 *  cells, local expansions and near field at the collocation points), 3 BEM solve (FP64,
 *  or two-word FP32 in the single-precision forms), 4 boundary multipoles, 5 M2L (item 3;
 *  with the tensor-core M2L its volume part only), 6 boundary-source M2L with the
 *  tensor-core M2L (kept apart, added by the downward pass), 7 L2L (item 4; only for trees
 *  of fewer than three levels, else part of stage 10), 8 near-boundary element integrals,
 *  9 P2P near field (item 5, Eq. e:volume_integral), 10 L2L + L2P + the final sum.
 * A stage that did not run reports 0.  Errors: _INVALID if timing is off. */
int fmmpc_set_timing(fmmpc_handle *h, int32_t on);
int fmmpc_get_timing(fmmpc_handle *h, float *ms, int32_t cap, int32_t *count);

/* Near field of the volume operator without any device allocation.
 *
 * This computes the same quantity as fmmpc_apply_part(h, 2, ...): the part of V r that
 * the dual tree traversal assigns to direct P2P interactions between leaves, in physical
 * units, FP32 arithmetic, one right-hand side.  The grid rules are those of fmmpc_create
 * (n interior nodes per side, a power of two, leaf side 4, 8 or 16 from leaf_max, MAC
 * parameter theta) on a square of side length `side`.  r_dev and out_dev are [n][n] FP64
 * device buffers owned by the caller; the call is asynchronous on `stream`.
 *
 * It exists for callers that must not allocate device memory: code running inside a
 * framework whose memory pool already owns the device memory (a cudaMalloc there can fail
 * or fragment the pool), code that records work while a stream is being captured, and
 * latency-bound loops that cannot afford cudaMalloc's implicit synchronisation.  Instead
 * of handle-owned buffers it uses one static device array of 4,194,304 FP32 values
 * (16 MiB) that every GPU loading this library holds until the process exits.  It holds
 * the log table and the zero-padded weight image; grids needing more (e.g. n = 2048 with
 * 8x8 leaves) are rejected with FMMPC_ERR_INVALID and a message, before any GPU work.
 * n = 1024 with 8x8 leaves and theta = 0.4 is the largest grid that fits.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current, and so does the first call after the device's context was made
 * anew (cudaDeviceReset reloads the module); make those calls before any stream capture.
 * All calls
 * share the one array and it keeps the last call's contents; each call rewrites the table
 * and the whole padded image, so nothing stale is read.  Calls that overlap on the GPU
 * (on different streams, or from several host threads) race on the array and must be
 * serialised by the caller.  No cudaMalloc, cudaFree or allocating library routine is
 * called; the kernel's shared-memory limit is raised when this call needs more, never
 * lowered.  Errors: _INVALID (arguments, size), _UNSUPPORTED (theta so small that the stencil
 * radius passes 15 leaves, or a source tile beyond one block's shared memory; both found
 * before any GPU work is queued), _CUDA; message via fmmpc_last_error(NULL).  The paper has no counterpart of this entry point. */
int fmmpc_near_field_noalloc(int32_t n, double side, int32_t leaf_max, double theta,
                             const double *r_dev, double *out_dev, void *stream);

/* Releases every resource of the handle (NULL is allowed). */
void fmmpc_destroy(fmmpc_handle *h);

/* One candidate of the autotuner. */
typedef struct {
  int32_t leaf_max;
  int32_t p;
  double rel_err;   /* relative L2 difference of its apply from the FP64 p = 16 apply */
  double solve_ms;  /* measured time-to-solution (0 when the gate failed) */
  int32_t iters;
  int32_t ok;       /* 1 if within the gate and converged */
} fmmpc_tune_entry;

/* Autotuner: picks leaf_max in {16, 64, 256} and p in {6, 8, 10, 12} by measured
 * time-to-solution of opts on the right-hand side f_dev ([ny][nx] FP64, device), among
 * the candidates whose preconditioner apply is within relative L2 error tol of an FP64
 * p = 16 reference apply (accuracy traded for speed as in Sec. 6.2, Fig. f:convergence;
 * the paper fixes p and theta by hand, Sec. 7.1).  base supplies theta, precision and
 * n_rhs.  *best receives the chosen parameters; report (capacity cap, may be NULL) the
 * candidates, *count their number.  Results are cached per (grid, precision, n_rhs, tol)
 * in the process; a report request bypasses the cache.  fmmpc_create with
 * params.autotune = 1 runs this on a synthetic smooth right-hand side with tol = 1e-5.
 * Allocates and frees temporary handles.  Errors: _INVALID (no candidate passed). */
int fmmpc_autotune(const fmmpc_grid *g, const fmmpc_params *base, const fmmpc_solve_opts *opts,
                   const double *f_dev, double tol, void *stream, fmmpc_params *best,
                   fmmpc_tune_entry *report, int32_t cap, int32_t *count);

/* Batches of independent problems of uneven size, solved together. */
typedef struct fmmpc_batch fmmpc_batch;

/* One handle per grid (each on its own internal stream, ordered after `stream`), with
 * params shared; params.autotune = 1 tunes leaf size and p per distinct grid. */
int fmmpc_create_batched(fmmpc_batch **out, int32_t nprob, const fmmpc_grid *grids,
                         const fmmpc_params *prm, void *stream);

/* FGMRES(m) on every problem in lockstep: each Arnoldi step launches all active
 * problems' preconditioner applies (CUDA graphs on their streams, running concurrently),
 * SpMVs and orthogonalisations, then synchronises once for the whole batch; converged
 * problems drop out.  f_dev[i], u_dev[i] (initial iterate in, solution out) and g_dev[i]
 * (NULL array or entries for g = 0) are device pointers of problem i's grid.  infos[i]
 * receives each problem's report.  Returns FMMPC_OK when all converged, otherwise the
 * first failing status.  opts->method must be FMMPC_FGMRES. */
int fmmpc_solve_batched(fmmpc_batch *b, const double *const *f_dev, const double *const *g_dev,
                        double *const *u_dev, const fmmpc_solve_opts *opts,
                        fmmpc_solve_info *infos);

/* fmmpc_query on problem prob of the batch; what = 100 gives its expansion order p. */
int fmmpc_batch_query(const fmmpc_batch *b, int32_t prob, int32_t what, int64_t *value);
const char *fmmpc_batch_last_error(const fmmpc_batch *b);
void fmmpc_destroy_batched(fmmpc_batch *b);

/* Message of the last failed call on h (or of the last failed fmmpc_create when h is
 * NULL).  The string lives until the next call on the same handle. */
const char *fmmpc_last_error(const fmmpc_handle *h);

/* Library build identification ("fmmpc <version> sm_103a"). */
const char *fmmpc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FMMPC_H */
