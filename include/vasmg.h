/*
 * vasmg.h -- C ABI of the GB300 (sm_103a) V-ASMG-preconditioned CG library.
 *
 * The library solves A U = F (Sec. 1, eq. (equ)) where A is the stiffness
 * matrix of P1 (linear Lagrange) finite elements for isotropic linear
 * elasticity in 2D or 3D (Sec. 2, eq. (prob) and the block form of A), with
 * PCG (Alg. 2) preconditioned by one V-cycle (Alg. 3, applied recursively) of
 * the vertex-based auxiliary space multigrid of Sec. 3: a region quadtree /
 * octree over the mesh vertices (Sec. 3.1.1), coarser grids by merging the
 * deepest cells (Sec. 3.1.2), bilinear / trilinear transfers (Sec. 3.2,
 * eq. (wkl)), Galerkin coarse operators (eq. (R), (Ac)), multicolour block
 * Gauss-Seidel smoothing (Sec. 2.1, Alg. 1) and a direct solve on the
 * coarsest grid (Sec. 3, Step 2.3).
 *
 * Conventions
 *  - Every function returns VASMG_OK (0) on success, VASMG_NOT_CONVERGED (+1)
 *    when PCG hit max_iters (U then holds the last iterate), or a negative
 *    VASMG_ERR_* code.  No C++ exception crosses this boundary.
 *  - Degree of freedom numbering is vertex-interleaved: dof = vertex*dim + c.
 *  - Problem arrays are host memory owned by the caller; vasmg_setup copies
 *    them and keeps nothing that points into them.  The handle owns all device
 *    memory of one hierarchy until vasmg_destroy.
 *  - Vector arguments (F, U, x, y) may be host or device pointers (copies use
 *    unified addressing, cudaMemcpyDefault).  They are FP64 arrays of length
 *    n = dim * n_vertices unless stated otherwise.
 *  - All device work of a handle runs on options.stream (NULL = the legacy
 *    default stream).  One thread may use a handle at a time.
 *  - A device wait inside a kernel that gives up returns VASMG_ERR_TIMEOUT;
 *    the context stays usable.
 */
#ifndef VASMG_H
#define VASMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  VASMG_OK = 0,
  VASMG_NOT_CONVERGED = 1,
  VASMG_PENDING = 2,                 /* vasmg_server_poll: the request is not done yet */
  VASMG_ERR_INVALID_ARG = -1,
  VASMG_ERR_DEGENERATE_ELEMENT = -2, /* an element has zero (or non-finite) measure */
  VASMG_ERR_OOM = -3,
  VASMG_ERR_CUDA = -4,
  VASMG_ERR_BREAKDOWN = -5,          /* p^T q <= 0 or NaN inside PCG */
  VASMG_ERR_TIMEOUT = -6,            /* a bounded device wait gave up */
  VASMG_ERR_UNSUPPORTED = -7
};

/* Precision of the V-cycle.  The outer CG (SpMV, dot products, updates) and
 * the coarsest factorisation are always FP64. */
enum {
  VASMG_FP64 = 0,                    /* V-cycle in FP64 storage and arithmetic */
  VASMG_FP32_VCYCLE = 1,             /* operators, transfers, vectors FP32 */
  VASMG_FP32_VCYCLE_BF16_SMOOTH = 2  /* as FP32, with operator values stored BF16 */
};

typedef struct vasmg_ctx* vasmg_handle;

/* The problem statement of Sec. 2: vertices, P1 simplices, Lame parameters
 * (mu = E/(2(1+nu)), lambda = E nu/((1+nu)(1-2nu))) and Dirichlet data. */
typedef struct {
  int32_t dim;                 /* 2 or 3 */
  int64_t n_vertices;
  const double* coords;        /* [n_vertices*dim], vertex-major */
  int64_t n_elements;
  const int32_t* elements;     /* [n_elements*(dim+1)], 0-based vertex ids */
  const double* lambda;        /* [n_elements] or NULL -> lambda_const */
  const double* mu;            /* [n_elements] or NULL -> mu_const */
  double lambda_const, mu_const;
  int64_t n_dirichlet;
  const int64_t* dirichlet_dofs;   /* [n_dirichlet], dof = vertex*dim + component */
  const double* dirichlet_values;  /* [n_dirichlet] or NULL -> homogeneous */
} vasmg_problem;

typedef struct {
  int32_t leaf_threshold;      /* a region-tree cell splits when it holds more
                                  vertices than this (Sec. 3.1.1 Step 2: 4 in
                                  2D); default 4 in 2D, 8 in 3D */
  int32_t n_pre, n_post;       /* smoothing sweeps; only 1, 1 is supported */
  int32_t precision;           /* VASMG_FP64 | VASMG_FP32_VCYCLE | ..._BF16_SMOOTH */
  int64_t coarse_max_dofs;     /* 0: coarsen to the root cell (Sec. 3.1.2);
                                  else stop at the first level with at most this
                                  many dofs (<= 4096) */
  int32_t max_iters;           /* PCG iteration cap, default 1000 */
  int32_t use_graph;           /* 1: one CUDA graph per solve (device-side loop) */
  int32_t max_ctas;            /* 0: the sweep launches use every CTA slot the
                                  device can hold at once; > 0: at most this
                                  many, so that handles whose caps add up to at
                                  most the device's capacity can solve
                                  concurrently (vasmg_solve_batch, the server) */
  int32_t dense_coarse;        /* FP32-vector modes only.  1 (default): the
                                  V-cycle from the first small level k whose
                                  order n_k fits (n_k^2 <= tail CTAs * 640^2)
                                  down to the coarsest is precomputed at setup
                                  as one dense n_k x n_k matrix (the cycle
                                  applied to the unit vectors) and applied as
                                  one matrix-vector product: the same linear
                                  operator up to FP32 rounding.  0: run the
                                  recursion.  Ignored by VASMG_FP64. */
  int32_t autotune;            /* 1 (default): at setup, time each region
                                  level's sweeps with 4, 8, 16 and 32 lanes per
                                  row and keep the fastest.  The lane count
                                  changes the order of additions within a row,
                                  so the choice is cached per level signature
                                  (dim, precision, vertices, blocks) for the
                                  process: handles of the same problem give the
                                  same bits.  0: lanes per row by rule from the
                                  mean row length. */
  void* stream;                /* cudaStream_t used for all device work */
  int32_t cycle;               /* coarse corrections per level, gamma: 1 (default)
                                  the V-cycle of Alg. 3, 2 the W-cycle of Fig. 2
                                  (every level above the second-coarsest solves
                                  its coarse problem by two cycles, the second on
                                  the updated coarse residual), up to 4.  gamma >= 2
                                  runs every level with per-level launches (no
                                  cluster tail, no dense level) */
  int32_t additive;            /* 1: the preconditioner is the additive form of
                                  Sec. 4, B = S + P B_1 P^T: S one forward and one
                                  backward multicolour sweep from zero on the fine
                                  level, B_1 the cycle above from level 1 (the
                                  coarsest solve when level 1 is the coarsest);
                                  0 (default): the cycle from the fine level */
} vasmg_options;

typedef struct {
  int32_t iterations;          /* number of products A p (Alg. 2) */
  double rel_res;              /* ||r_k|| / ||F|| of the recursive residual */
  double setup_ms, solve_ms;   /* wall-clock of vasmg_setup / vasmg_solve */
  int32_t n_levels;            /* fine level + coarse levels */
  double op_complexity;        /* sum_l nnzb_l / nnzb_0 */
  double* res_history;         /* caller-owned host array or NULL */
  int32_t res_history_cap;
} vasmg_stats;

/* Fill *out with the defaults for dim (2 or 3). */
int vasmg_default_options(int dim, vasmg_options* out);

/* Assemble A (Sec. 2), impose Dirichlet rows, build the region tree, the
 * coarse grids, transfers and Galerkin operators (Sec. 3), colour every level,
 * and factor the coarsest operator -- all on the device.  Returns
 * VASMG_ERR_DEGENERATE_ELEMENT if an element has zero measure,
 * VASMG_ERR_INVALID_ARG for out-of-range ids or sizes. */
int vasmg_setup(const vasmg_problem* problem, const vasmg_options* options, vasmg_handle* out);

/* New material data or new Dirichlet values for the same mesh and the same
 * set of Dirichlet dofs, reusing the hierarchy.  The region tree, coarse
 * grids and transfers (Sec. 3.1, 3.2), the sparsity patterns, colourings,
 * renumbering and the solve engine's layout depend only on the mesh and on
 * which dofs are constrained; only values are recomputed: the assembly
 * (Sec. 2), the Dirichlet lift, the Galerkin products (eq. (Ac)), the
 * diagonal inverses and the coarsest Cholesky factor.
 *   lambda, mu        [n_elements] host arrays, or NULL for lambda_const /
 *                     mu_const on every element
 *   dirichlet_values  [n_dirichlet] host array in the order of the dofs given
 *                     to vasmg_setup, or NULL to keep the current values
 * Later solves give what a fresh vasmg_setup with the new data would give.
 * VASMG_ERR_INVALID_ARG for a NULL handle or non-finite parameters. */
int vasmg_update_data(vasmg_handle h, const double* lambda, const double* mu, double lambda_const, double mu_const,
                      const double* dirichlet_values);

/* F = consistent load of a constant body force f (Sec. 2, F_1, F_2):
 * F_i += f |K| / (dim+1) over the elements K containing vertex i.
 * body_force: host [dim].  F: host or device [n]. */
int vasmg_assemble_load(vasmg_handle h, const double* body_force, double* F);

/* PCG (Alg. 2) with the V-ASMG V-cycle as preconditioner, U0 = 0, until
 * ||F - A U|| / ||F|| < tol (Sec. 5, item (3)).  F: [n], entries at Dirichlet
 * dofs are ignored; U: [n] output, Dirichlet values written in.  st may be
 * NULL.  Returns VASMG_OK, VASMG_NOT_CONVERGED or an error. */
int vasmg_solve(vasmg_handle h, const double* F, double* U, double tol, vasmg_stats* st);

/* k right-hand sides on one hierarchy: k independent PCG solves (Alg. 2 with
 * the V-cycle of Alg. 3) of A U_i = F_i, each to tol, advanced together.  In
 * the FP32-vector modes every kernel of an iteration reads the operators once
 * for up to 8 right-hand sides (the sweeps, residuals and transfers apply each
 * block or weight to all of them; the FP64 SpMV to 4 at a time), so the
 * iterations cost less than k separate ones.  Each right-hand side follows
 * exactly the arithmetic of vasmg_solve: U_i, its iteration count and its
 * residual history are bitwise those of vasmg_solve(h, F[i], U[i], tol, ...);
 * a right-hand side that has converged keeps its iterate while the others go
 * on.  The paper solves one right-hand side at a time; this is the same solve
 * batched.
 *   F, U  arrays of k pointers to [n] doubles (host or device)
 *   st    NULL or an array of k stats (solve_ms is the whole call's)
 * With VASMG_FP64 the k solves run one after another.  The first call with a
 * given number of right-hand sides (rounded up to 2, 4 or 8 per pass) builds
 * that pass's vectors and graph.  Returns the most severe status. */
int vasmg_solve_multi(vasmg_handle h, int32_t k, const double* const* F, double* const* U, double tol,
                      vasmg_stats* st);
/* (With vasmg_options.cycle > 1 or .additive, the k solves also run one after
 * another.) */

/* Solve k independent systems (uneven sizes allowed, 2D and 3D mixed), each
 * to tol, sharing the device; h[i] may repeat.  st may be NULL or an array of
 * k stats.
 *
 * When the handles are distinct, on the current device, set up with one
 * FP32-vector precision (VASMG_FP32_VCYCLE or ..._BF16_SMOOTH) and the plain
 * V-cycle, the k PCG solves advance together with one launch per level and
 * phase for all of them: each region level's forward sweeps, residuals,
 * restrictions, prolongations and backward sweeps of every handle in one
 * launch (a CTA per region of each), every handle's small levels in one
 * launch (a thread-block cluster each), and every CG kernel for all handles
 * in one launch.  A level's regions of all handles must be resident at once:
 * handles whose regions (vasmg_options.max_ctas, as set up) do not fit the
 * device together run in successive groups of such launches.
 *
 * Otherwise the solves run concurrently, one host thread and one stream per
 * handle, in groups whose sweep grids fit the device together; handles set
 * up with max_ctas = 0 then run one at a time, and a handle that appears
 * twice runs in two different groups.
 *
 * Either way each result is the one vasmg_solve gives alone (the same
 * arithmetic for every row and reduction).  vasmg_last_launch_count of each
 * handle reports the batch's launches.  Returns the most severe status. */
int vasmg_solve_batch(int32_t k, const vasmg_handle* h, const double* const* F, double* const* U, double tol,
                      vasmg_stats* st);

/* ------------------------------------------------------------------ serving
 *
 * A request server for many independent problems (the paper has no
 * counterpart; it solves one system at a time).  Requests (one mesh, 1..n
 * right-hand sides) queue in arrival order.  `slots` worker threads each take
 * the next request once its estimated device footprint fits the memory
 * budget left (the head request is admitted alone if it fits nowhere), set up
 * its hierarchy on the slot's own stream, keep it resident while solving every
 * right-hand side, write U and release the memory.  Requests on different
 * slots overlap on the device; every handle's sweep grids are capped to a
 * share of the device so that all running sweeps stay resident together.
 * Each result equals what vasmg_setup + vasmg_solve give for that request
 * alone. */
typedef struct vasmg_server vasmg_server;

typedef struct {
  int32_t slots;               /* requests on the device at once; default 4 */
  int32_t precision;           /* V-cycle precision; default VASMG_FP32_VCYCLE */
  int32_t max_iters;           /* default 1000 */
  double tol;                  /* relative residual; default 1e-6 */
  int64_t memory_budget;       /* device bytes for admitted requests; 0: half
                                  the free device memory at creation */
  int32_t batch;               /* 0 (default): each slot solves its request's
                                  right-hand sides itself, all of them in one
                                  vasmg_solve_multi.  1: the slots set up the
                                  hierarchies, and one executor advances the
                                  solves of every request ready at the time
                                  together, one right-hand side of each per
                                  round, with vasmg_solve_batch (one launch per
                                  level and phase for all of them) */
} vasmg_server_opts;

typedef struct {
  int32_t status;              /* VASMG_OK, VASMG_NOT_CONVERGED or the error of
                                  the request's setup or solve */
  int32_t n_rhs;
  int32_t iterations;          /* summed over the right-hand sides */
  int32_t max_iterations;
  double max_rel_res;
  double queue_ms;             /* submit -> admitted */
  double setup_ms;
  double solve_ms;             /* all right-hand sides */
  double latency_ms;           /* submit -> done */
  int64_t footprint_bytes;     /* the admission estimate */
} vasmg_request_stats;

int vasmg_server_default_opts(vasmg_server_opts* out);

/* Start the worker threads on the current device. */
int vasmg_server_create(const vasmg_server_opts* opts, vasmg_server** out);

/* Queue one request.  The problem arrays and F[0..n_rhs) (host, [n] each) are
 * copied before the call returns; U[0..n_rhs) are caller-owned host arrays of
 * [n] doubles that the server writes when the request completes, and that
 * must stay valid until vasmg_server_poll reports it done.  *ticket names the
 * request. */
int vasmg_server_submit(vasmg_server* s, const vasmg_problem* problem, int32_t n_rhs, const double* const* F,
                        double* const* U, uint64_t* ticket);

/* Wait up to wait_ms milliseconds (< 0: without limit) for a request.
 * Returns VASMG_PENDING if it is still queued or running, VASMG_OK once it is
 * done (st, if not NULL, receives its statistics and the ticket is released),
 * VASMG_ERR_INVALID_ARG for an unknown ticket. */
int vasmg_server_poll(vasmg_server* s, uint64_t ticket, int32_t wait_ms, vasmg_request_stats* st);

/* Finish every queued request, stop the workers and free the server. */
int vasmg_server_destroy(vasmg_server* s);

/* Number of levels (fine + coarse). */
int vasmg_num_levels(vasmg_handle h);

/* Vertices, off-diagonal-inclusive block count and colour count of a level. */
int vasmg_level_info(vasmg_handle h, int32_t level, int64_t* n_vertices, int64_t* nnzb, int32_t* n_colours);

/* Export selectors for vasmg_export (all in canonical order: level 0 =
 * input vertex ids, level >= 1 = ascending lattice key). */
enum {
  VASMG_EXPORT_MORTON = 0,       /* u64[n_vertices] Morton keys of the quantised coordinates */
  VASMG_EXPORT_LEAF = 1,         /* i64[2*n_vertices] (depth, cell key) of each vertex's leaf */
  VASMG_EXPORT_CELLS = 3,        /* i64[2*ncells] (depth, cell key) of the cells of a level >= 1 */
  VASMG_EXPORT_LATTICE = 4,      /* u64[nv_l] lattice-corner keys of a level >= 1 */
  VASMG_EXPORT_P_RP = 5,         /* i64[nv_l+1] interpolation rows (level l -> l+1) */
  VASMG_EXPORT_P_CI = 6,         /* i32[nnz] */
  VASMG_EXPORT_P_W = 7,          /* f64[nnz] */
  VASMG_EXPORT_A_RP = 8,         /* i64[nv_l+1] operator block pattern (with diagonal) */
  VASMG_EXPORT_A_CI = 9,         /* i32[nnzb] */
  VASMG_EXPORT_A_V = 10,         /* f64[nnzb*dim*dim] row-major blocks (FP64 values) */
  VASMG_EXPORT_DEAD = 11,        /* u8[nv_l*dim] 1 = dof removed (Dirichlet / empty column) */
  VASMG_EXPORT_COLOUR = 12,      /* i32[nv_l] */
  VASMG_EXPORT_DINV = 13,        /* f64[nv_l*dim*dim] inverses of the diagonal blocks */
  VASMG_EXPORT_BOX = 14,         /* f64[2] bounding square (m, M) */
  VASMG_EXPORT_LIFT = 15,        /* f64[n] A u_D of the Dirichlet data */
  VASMG_EXPORT_VOL = 16,         /* f64[n_elements] element measures */
  VASMG_EXPORT_DENSE = 17,       /* i64[2] (k, n_k) of the dense level, (-1, 0) if none (level ignored) */
  VASMG_EXPORT_LANES = 18,       /* i32[n_levels] lanes per row of each level's region sweeps, 0 for the
                                    levels the tail launch runs (level ignored) */
  VASMG_EXPORT_STAGED = 19       /* i64[5] the staged copies a 3D region level's sweeps stream (forward slots,
                                    lower-part blocks, backward slots, whole-row blocks, bytes per slot);
                                    zeros where the sweeps read the operator in place */
};

/* Copy an exported array to host buffer buf (NULL: only report the size).
 * *bytes receives the byte count. */
int vasmg_export(vasmg_handle h, int32_t what, int32_t level, void* buf, int64_t* bytes);

/* Single steps of the hot path, for parity testing: all vectors FP64 in
 * canonical order, device or host pointers.
 *   VASMG_OP_MATVEC      y = A_l x (level 0: the FP64 operator of the outer CG;
 *                        level > 0: the V-cycle operator, in its precision)
 *   VASMG_OP_SMOOTH_FWD  y = one forward multicolour sweep from x = 0 on A_l y = x
 *   VASMG_OP_SMOOTH_BWD  y = one backward sweep on A_l y = x from y's input value
 *   VASMG_OP_RESIDUAL    y = r after a zero-start forward sweep on A_l z = x
 *   VASMG_OP_RESTRICT    y = R x (level l -> l+1, y has nv_{l+1}*dim entries)
 *   VASMG_OP_PROLONG     y += P x (level l+1 -> l, x has nv_{l+1}*dim entries)
 *   VASMG_OP_COARSE      y = A_L^{-1} x on the coarsest level (Cholesky)
 *   VASMG_OP_VCYCLE      y = M x, one cycle (V, or gamma of vasmg_options.cycle) from level l down
 *   VASMG_OP_PRECOND     y = B x, the preconditioner PCG applies (the options' cycle from level 0,
 *                        or the additive form); level must be 0 */
enum {
  VASMG_OP_MATVEC = 0,
  VASMG_OP_SMOOTH_FWD = 1,
  VASMG_OP_SMOOTH_BWD = 2,
  VASMG_OP_RESIDUAL = 3,
  VASMG_OP_RESTRICT = 4,
  VASMG_OP_PROLONG = 5,
  VASMG_OP_COARSE = 6,
  VASMG_OP_VCYCLE = 7,
  VASMG_OP_PRECOND = 8
};
int vasmg_apply(vasmg_handle h, int32_t op, int32_t level, const double* x, double* y);

/* Coarsest-level solve x = A_L^{-1} b that allocates nothing.
 *
 * The paper has no counterpart: this is a library-level variant of
 * vasmg_apply(h, VASMG_OP_COARSE, ...), which stages its vectors through
 * device buffers it allocates on every call.  Use this entry point where the
 * caller cannot allocate device memory during the call: a server whose
 * device memory is budgeted per request (an allocation could push it over its
 * budget or wait on the allocator's lock), or a latency-bound loop that must
 * not enter the allocator.
 *
 * b, x    device (or managed) pointers on the handle's device, [n] doubles
 *         each, n = dim * (vertices of the coarsest level), canonical order
 *         (dof = vertex*dim + component), as for VASMG_OP_COARSE.  b and x
 *         may be the same buffer.  The library cannot check their length.
 * stream  cudaStream_t to run on (NULL: the legacy default stream).
 *
 * The device current at the call must be the one that was current at
 * vasmg_setup (the factor lives there).  The work runs asynchronously on
 * `stream`; the call returns once it is enqueued.  It reads the handle's FP64
 * Cholesky factor (every precision mode keeps one) and uses a scratch array of
 * VASMG_NOALLOC_MAX_DOFS doubles (32 KiB) in the library's static device
 * memory, which every device that loads the library holds until the process
 * exits.  Nothing in that scratch needs to start at zero: each call writes
 * every entry it reads, and the array keeps the last call's values.
 *
 * The scratch is shared by every call on the device, so two calls whose
 * kernels overlap on the GPU (e.g. issued on different streams without
 * ordering) race and give wrong results; order such calls on one stream or
 * with events.  vasmg_update_data waits for the last call's kernel before it
 * rewrites the factor; a call issued after vasmg_update_data returns sees the
 * new factor.  The first call on a device (and again after the device's
 * context was reset) looks up the scratch address with cudaGetSymbolAddress,
 * which may load the library's device code; make that first call before
 * capturing a stream that will contain later calls.
 *
 * Returns VASMG_ERR_INVALID_ARG for NULL pointers, for b or x not in device
 * memory of the handle's device, when another device is current, or when n
 * exceeds VASMG_NOALLOC_MAX_DOFS (the detail string is not updated on this
 * path: that would allocate host memory); VASMG_ERR_CUDA if a CUDA call
 * fails. */
#define VASMG_NOALLOC_MAX_DOFS 4096
int vasmg_coarse_solve_noalloc(vasmg_handle h, const double* b, double* x, void* stream);

/* Timing helper: launch kernel class `which` (VASMG_KERNEL_*) `reps` times on
 * the handle's stream between two CUDA events; *ms = mean per launch and
 * *bytes = algorithmic bytes that one launch moves. */
enum {
  VASMG_KERNEL_SPMV64 = 0,       /* level-0 FP64 SpMV (SELL-32) */
  VASMG_KERNEL_SWEEP = 1,        /* one backward multicolour sweep of level `level` */
  VASMG_KERNEL_VCYCLE = 2,       /* one V-cycle from level 0 */
  VASMG_KERNEL_DOWN = 3,         /* pre-smooth + residual + restriction of level `level` */
  VASMG_KERNEL_UP = 4,           /* prolongation + post-smooth of level `level` */
  VASMG_KERNEL_FWD_SWEEP = 5,    /* one forward multicolour sweep from zero of level `level` */
  VASMG_KERNEL_RESIDUAL = 6,     /* r = b - A x after the forward sweep, level `level` */
  VASMG_KERNEL_RESTRICT = 7,     /* b_{l+1} = R r_l */
  VASMG_KERNEL_PROLONG = 8,      /* x_l += P x_{l+1} */
  VASMG_KERNEL_TAIL = 9          /* the V-cycle of all levels from `level` down, in the
                                    single cluster launch that runs the small levels */
};
int vasmg_time_kernel(vasmg_handle h, int32_t which, int32_t level, int32_t reps, double* ms, double* bytes);

/* As vasmg_time_kernel for the kernels of vasmg_solve_multi with k = 2, 4 or
 * 8 right-hand sides per launch (VASMG_KERNEL_SPMV64, _SWEEP, _VCYCLE,
 * _FWD_SWEEP, _RESIDUAL, _RESTRICT, _PROLONG, _TAIL; FP32-vector modes only,
 * else VASMG_ERR_UNSUPPORTED).  *bytes counts the operator arrays once and
 * every vector entry once per right-hand side (0 for the tail). */
int vasmg_time_kernel_multi(vasmg_handle h, int32_t which, int32_t level, int32_t k, int32_t reps, double* ms,
                            double* bytes);

/* Measured FP64 FMA throughput of the current device, the arithmetic roof of
 * the FP64 kernels (the outer CG's SpMV): a kernel of independent FMA chains
 * on every SM, timed with CUDA events (one warm-up launch, five timed).
 * *tflops = 2 * FMAs / time / 1e12; *ms (may be NULL) = one launch.  The
 * paper has no counterpart (measurement hook). */
int vasmg_probe_fp64_rate(double* tflops, double* ms);

/* Kernels launched by the last vasmg_solve (for accounting). */
int64_t vasmg_last_launch_count(vasmg_handle h);

int vasmg_destroy(vasmg_handle h);

const char* vasmg_error_string(int code);

/* Human-readable detail of the last error raised on the calling thread. */
const char* vasmg_last_error_detail(void);

/* Failure detection without a fault: runs the bounded wait of the sweep
 * kernels (the neighbour-region stage wait) in one CTA on its own stream,
 * against a stage word that nothing publishes.  The wait gives up after its
 * iteration limit (about 0.1-1 s), raises the abort flag and returns, so the
 * call returns VASMG_ERR_TIMEOUT and the context stays usable; *elapsed_ms
 * (may be NULL) receives the kernel's duration.  VASMG_OK would mean the wait
 * was satisfied, which cannot happen. */
int vasmg_probe_wait_timeout(double* elapsed_ms);

#ifdef __cplusplus
}
#endif

#endif /* VASMG_H */
