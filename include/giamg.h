/*
 * giamg.h -- C ABI of the GB300 GIAMG solver: geometrically informed algebraic multigrid
 * preconditioned conjugate gradients for assembled high-order (nodal GLL, hexahedral) finite
 * element systems, after arXiv 2512.15121.
 *
 * The problem statement follows the paper: the caller hands over an assembled symmetric
 * positive definite matrix A (Eq. 1, Ax = b) and the element-to-dof map ("l2g") whose column
 * order implies the basis order inside each element (Sec. 2.1 and the appendix, Eq. 8:
 * local index (p+1)^2 i + (p+1) j + k, i along x).  Nothing else about the geometry is needed;
 * nodal coordinates may be passed for validation only.
 *
 * Setup builds the hierarchy on the GPU: p-coarsening p -> p/2 -> ... -> 1 by element-local
 * interpolation (Algorithms 2-4 and 7), then h-coarsening by smoothed aggregation (Sec. 2.5)
 * while a level has more than coarse_max rows, Galerkin coarse operators R A P with R = P^T
 * (Sec. 2), Jacobi-Chebyshev smoother bounds, and a dense Cholesky factor of the coarsest
 * level.  A solve runs preconditioned CG with one V-cycle (Algorithm 1) per iteration.
 *
 * Conventions for every entry point:
 *   - Return value: GIAMG_OK (0) or a negative GIAMG_ERR_* code; giamg_last_error() then holds
 *     a one-line description (per calling thread).  Nothing is thrown; no call aborts.
 *   - Ownership: the caller owns every array it passes.  The library copies what it keeps
 *     (host mode) or reads device arrays without retaining them (device mode); the handle owns
 *     all device memory it allocates until giamg_free.
 *   - Pointers: with options.device_ptrs == 0 all vector/matrix arguments are host pointers;
 *     with device_ptrs == 1 they are device pointers on the handle's device.  Scalar outputs
 *     (iters, relres, sizes) are always host pointers.
 *   - Streams: all work is ordered on the stream given to giamg_setup (NULL = legacy default
 *     stream).  Calls that return host scalars synchronise that stream before returning.
 *   - Threads: a handle is not thread-safe; distinct handles are independent.
 *   - Layouts: CSR with int64 row pointers, int32 column indices ascending within each row,
 *     float64 values.  Vectors are contiguous float64.  Multi-RHS blocks are row-major n x m.
 */
#ifndef GIAMG_H
#define GIAMG_H

#include <stdint.h>

#if defined(__GNUC__)
#define GIAMG_API __attribute__((visibility("default")))
#else
#define GIAMG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GIAMG_OK = 0,
  GIAMG_ERR_ARG = -1,        /* invalid argument (NULL pointer, size, option, level index) */
  GIAMG_ERR_ORDER = -2,      /* element orders not uniform, or outside 1..GIAMG_MAX_ORDER */
  GIAMG_ERR_MAP = -3,        /* element map out of range or inconsistent with A's pattern / coords */
  GIAMG_ERR_OOM = -4,        /* device or host allocation failed */
  GIAMG_ERR_CUDA = -5,       /* a CUDA runtime call failed (message carries the CUDA error) */
  GIAMG_ERR_NOT_SPD = -6,    /* non-positive diagonal or Cholesky pivot */
  GIAMG_ERR_BREAKDOWN = -7,  /* CG breakdown: p^T A p <= 0, r^T z <= 0 or a NaN */
  GIAMG_ERR_MAXITER = -8,    /* max_iter reached above rtol; the outputs are still valid */
  GIAMG_ERR_TIMEOUT = -9     /* a bounded device-side wait expired */
};

enum { GIAMG_LEVEL_P = 0, GIAMG_LEVEL_H = 1, GIAMG_LEVEL_COARSEST = 2 };
#define GIAMG_MAX_ORDER 12

typedef struct giamg_hierarchy* giamg_handle;

typedef struct {
  int cheb_degree;        /* Chebyshev degree k for pre- and post-smoothing (Sec. 2).  Default 3
                             (Table 1 uses 3 for the Helmholtz operator; Sec. 3.2 uses 2). */
  double cheb_lo;         /* smoothing interval [cheb_lo, cheb_hi] * rho_hat of D^-1 A; 0.1 */
  double cheb_hi;         /* 1.1 */
  int lanczos_steps;      /* Lanczos steps for rho_hat; 20 */
  int coarse_max;         /* h-coarsen while a level has more rows than this; 500 */
  int max_levels;         /* 16 */
  double strength_theta;  /* 0: structural strength graph (bit-exact hierarchy); > 0 keeps
                             |a_ij| >= theta sqrt(a_ii a_jj) */
  int precision;          /* 0: FP64 V-cycle in PCG; 1: FP32 V-cycle in FP64 flexible CG */
  int max_iter;           /* 1000 */
  int force_iters;        /* 0, or run exactly this many iterations (parity tests) */
  int device_ptrs;        /* 0: host arrays; 1: device arrays (e.g. torch tensors) */
  int hash_kind;          /* node hash of MIS-2 / Lanczos start: 0 SplitMix64-based, 1 identity */
  int compress_patterns;  /* 1 (default): detect rows that repeat one of a few offset patterns
                             (stored as a template id instead of column indices) and groups of rows
                             with identical column sets (x gathered once per group); detection is
                             exact, plain CSR otherwise; 0: plain CSR everywhere */
  int autotune;           /* 1: after setup, time the finest level's row-kernel variants (CSR,
                             row patterns, hybrid, vector hybrid, sliced; several threads per row)
                             inside the solve -- 3 forced CG iterations per candidate and
                             precision on a fixed right-hand side, the faster of two runs -- and
                             keep the fastest per precision (operators of at least 2^20
                             nonzeros); 0 (default): the variants measured best inside the solve
                             (FP64: the sliced form on levels of at least 2^18 rows; FP32: the
                             vector hybrid where there are at least 4096 groups of 16 or more rows
                             averaging 192 or more columns, else the sliced form on levels of at
                             least 2^18 rows; on smaller levels FP32 rows on row patterns and FP64
                             rows on CSR) */
  int row_form;           /* force the row-kernel form: 0 automatic, 1 CSR, 2 row patterns, 3 row
                             groups, 4 hybrid (groups of at least 16 rows by the group kernel, the
                             other rows by the row-pattern kernel), 5 vector hybrid (the big
                             groups' values from a group-major copy with rows padded to 16 bytes,
                             read with 16-byte loads: FP32 one warp per row, FP64 4 lanes per row
                             and 8 rows of a group per warp), 6 sliced (every row in slices of
                             32 rows of equal length, one lane per row, values interleaved by
                             column and read with 16-byte loads, columns from the row group's
                             list); each falls back to CSR where the form is not available */
  int row_threads;        /* force threads per row (4, 8, 16, 32); 0 automatic */
  int prefetch_rows;      /* row-pattern kernels: every block prefetches into L2 the values of the
                             block this many rows ahead; 0 off, -1 (default) automatic */
  int row_chains;         /* row-pattern kernels: independent load chains per thread (2, 4, 8);
                             0 (default) automatic */
  int graphs;             /* 1 (default): a solve runs the whole PCG loop as one CUDA graph whose
                             convergence test runs on the device, captured at the second solve
                             of a shape (precision; number of right-hand sides) so one-off shapes
                             pay no capture; 2: captured at the first solve; 0: a host loop with
                             one synchronisation per iteration.  All give the same iterations
                             and bits.  The host loop is used while profiling or when
                             force_iters > max_iter. */
  int p_schedule;         /* order sequence of the p-levels: 0 (default) halving, q = p/2 (odd p:
                             its largest proper divisor); 1 by one, q = p - 1; 2 by two,
                             q = p - 2 (at least 1).  When p/q is not whole, coarse nodes are
                             numbered by their nearest fine nodes (ties: the smaller global id) */
  int basis;              /* element basis of A and elem_dof: 0 (default) nodal, Lagrange on the
                             GLL points (interpolation between orders, Algorithm 7's nodal form);
                             1 modal hierarchical, local 1D index 0 and p the vertex modes,
                             1..p-1 the bubble modes of degree 2..p (the paper's setting: the
                             coarse space keeps the modes of degree <= q, Algorithm 2's prefix,
                             and P is the injection, Algorithm 7 with values 1).  Elements must
                             share one orientation; coords must be NULL */
} giamg_options;

/* Fill *opt with the defaults listed above. */
GIAMG_API void giamg_default_options(giamg_options* opt);

/* Build the hierarchy (Sec. 2; Algorithms 2-4, 7; Sec. 2.5).
 *   n, row_ptr[n+1], col_idx[nnz], val[nnz]: A, symmetric positive definite, columns ascending.
 *     Dirichlet rows, if any, are identity rows whose columns have been removed elsewhere.
 *   n_elem, elem_dof[n_elem][(p+1)^3]: element-to-dof map, entries in [0, n).
 *   elem_order[n_elem]: polynomial order of each element; all equal (GIAMG_ERR_ORDER if not).
 *     With p = 1 there is no p-level and elem_dof may be NULL.
 *   coords[n][3]: nodal coordinates or NULL; when given, every element's nodes must be the
 *     trilinear image of the GLL tensor points (1e-8 of the element size), else GIAMG_ERR_MAP.
 *   opt: options (NULL = defaults).  cuda_stream: a cudaStream_t or NULL; with device_ptrs
 *     the inputs are read on this stream, so they may still be in flight on it at the call.
 *   *out: the new handle.  Every element pair (a, b) must be present in A's pattern unless
 *   one of the two rows is a Dirichlet identity row (GIAMG_ERR_MAP otherwise). */
GIAMG_API int giamg_setup(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                int32_t n_elem, const int32_t* elem_dof, const int32_t* elem_order,
                const double* coords, const giamg_options* opt, void* cuda_stream,
                giamg_handle* out);

/* Solve A x = b by PCG with one V-cycle per iteration (Sec. 2), x0 = 0 (Sec. 3.1), stopping
 * when ||r||_2 / ||b||_2 <= rtol on the recursive residual, or after force_iters iterations
 * when that option is set.  x: output (n).  *iters: iterations done; *relres: final relative
 * residual.  GIAMG_ERR_MAXITER leaves a valid x. */
GIAMG_API int giamg_solve(giamg_handle h, const double* b, double* x, double rtol, int* iters, double* relres);

/* giamg_solve with the precision (0 FP64, 1 FP32 V-cycle + flexible CG) and force_iters chosen
 * per call instead of from the handle's options. */
GIAMG_API int giamg_solve_ex(giamg_handle h, int precision, int force_iters, const double* b, double* x,
                   double rtol, int* iters, double* relres);

/* giamg_solve enqueued on the handle's stream without any host synchronisation (the solve of
 * Algorithm 1's PCG loop as one CUDA graph with its stopping rule on the device).  Needs
 * device_ptrs = 1 and graphs != 0; force_iters and max_iter from the options (force_iters <=
 * max_iter).
 *   b, x: device arrays of n values (caller-owned; b may be reused once the stream passes the call).
 *   iters, relres, status: device pointers (each may be NULL) written when the stream reaches the
 *     end of the solve: the iteration count, ||r||/||b|| (0 for b = 0), and GIAMG_OK,
 *     GIAMG_ERR_MAXITER or GIAMG_ERR_BREAKDOWN with the rules of giamg_solve.
 * The caller synchronises the stream before reading them.  The first call for a precision
 * captures the graph, which synchronises the stream once.  The return value reports argument
 * and launch errors only.  giamg_solve_stats keeps the true residual of an asynchronous solve
 * but not its history. */
GIAMG_API int giamg_solve_async(giamg_handle h, int precision, const double* b, double* x, double rtol, int* iters,
                                double* relres, int* status);

/* The multi-right-hand-side solves of several hierarchies at once, for a server whose requests
 * for different operators are ready together: every phase of an iteration (the outer product and
 * CG updates, each V-cycle level's smoother steps, residual, transfers and coarsest solve) is ONE
 * kernel launch over all hierarchies that take part in it, each hierarchy's share of the grid
 * being the grid of its own launch, so each hierarchy's results are bit for bit those of
 * giamg_solve_batch with the same arguments (FP32 V-cycle in FP64 flexible CG, precision 1,
 * independent columns).  No counterpart in the paper (a serving feature).
 *   count: number of hierarchies; handles[count]: distinct handles on one device, each with
 *     device_ptrs = 1; work runs on handles[0]'s stream (the other handles' streams are
 *     synchronised first).
 *   m[count]: right-hand sides per hierarchy (1..32); B[i], X[i]: device arrays, row-major
 *     n_i x m[i] (caller-owned).
 *   iters, relres: host arrays of sum(m) entries, hierarchy after hierarchy (NULL to skip);
 *   status[count] (NULL to skip): GIAMG_OK, GIAMG_ERR_MAXITER or GIAMG_ERR_BREAKDOWN per hierarchy.
 * The return value reports argument and CUDA errors only; the call synchronises the stream. */
GIAMG_API int giamg_solve_grouped(int count, const giamg_handle* handles, const int* m, const double* const* B,
                                  double* const* X, double rtol, int* iters, double* relres, int* status);

/* m independent solves A X_j = B_j sharing every matrix pass (multi-right-hand-side PCG: one
 * CG recurrence per column, each with its own alpha, beta and stopping test; the products and
 * the V-cycle work on all columns at once, so the matrix is read once per m solves).
 *   B, X: row-major n x m (the m values of a row are contiguous), 1 <= m <= 32.
 *   iters[m], relres[m]: per-column iterations and final relative residuals (host arrays).
 * Columns stop independently; GIAMG_ERR_MAXITER if any column misses rtol. */
GIAMG_API int giamg_solve_batch(giamg_handle h, int m, const double* B, double* X, double rtol, int* iters,
                                double* relres);
GIAMG_API int giamg_solve_batch_ex(giamg_handle h, int precision, int force_iters, int m, const double* B, double* X,
                                   double rtol, int* iters, double* relres);

/* The m right-hand sides as one block in block PCG (O'Leary, "The block conjugate gradient
 * algorithm and related methods", 1980), preconditioned by the V-cycle of Algorithm 1: one
 * Krylov space shared by all columns, m x m coefficient matrices per iteration, X0 = 0:
 *   Q = A P;  G = P^T Q;  alpha = G^+ (P^T R);  X += P alpha;  R -= Q alpha;
 *   Z = M R;  beta = -G^+ (Q^T Z);  P = Z + P beta   (P0 = Z0 = M B).
 * beta keeps P A-conjugate to the previous block for a fixed or a varying (FP32) V-cycle.
 * G^+: G scaled to unit diagonal and factored by Cholesky in index order; a direction with
 * pivot <= 1e-10 (dependent, duplicate or zero columns) is dropped from alpha and beta.
 *   precision: 0 FP64 V-cycle, 1 FP32 V-cycle; everything else is FP64.
 *   B, X: row-major n x m, 1 <= m <= 32 (host or device per device_ptrs; caller-owned).
 *   iters[m]: the block iteration count (the same for every column); relres[m]: per column.
 *   force_iters > 0: exactly that many iterations, rtol ignored.
 * The iteration stops when every column has ||r_j|| <= rtol ||b_j||.  GIAMG_ERR_MAXITER when
 * max_iter is reached first (X valid); GIAMG_ERR_BREAKDOWN on NaN, or when every direction is
 * dropped while a column is above rtol. */
GIAMG_API int giamg_solve_block(giamg_handle h, int precision, int force_iters, int m, const double* B, double* X,
                                double rtol, int* iters, double* relres);

/* After a solve: relative residual history hist[0..min(len, iters+1)) of the recursive
 * residual, and the true relative residual ||b - A x|| / ||b|| recomputed in FP64. */
GIAMG_API int giamg_solve_stats(giamg_handle h, double* hist, int len, double* true_relres);

/* Hierarchy inspection (used by the bit-exact structure tests). */
GIAMG_API int giamg_num_levels(giamg_handle h, int* n_levels);
/* kind: GIAMG_LEVEL_*; n, nnz of A_l; order: p of a p-level (0 for aggregated levels);
 * p_nnz / n_next: size of the prolongation to level l+1 (0 on the coarsest level). */
GIAMG_API int giamg_level_info(giamg_handle h, int level, int* kind, int64_t* n, int64_t* nnz, int* order,
                     int64_t* p_nnz, int64_t* n_next);
/* Copy A_l to caller arrays sized from giamg_level_info (row_ptr n+1, col_idx/val nnz; any may
 * be NULL), and the aggregate id of every row of an h-level (NULL to skip).  Host pointers
 * unless device_ptrs is set. */
GIAMG_API int giamg_export_level(giamg_handle h, int level, int64_t* row_ptr, int32_t* col_idx, double* val,
                       int32_t* aggregates);
/* Copy the assembled prolongation P_l (n x n_next, p_nnz entries) built during setup. */
GIAMG_API int giamg_export_prolongation(giamg_handle h, int level, int64_t* row_ptr, int32_t* col_idx,
                              double* val);
/* Row-pattern compression of A_l: number of templates and of stored offsets (0, 0 when the
 * level uses plain CSR). */
GIAMG_API int giamg_level_templates(giamg_handle h, int level, int64_t* n_templates, int64_t* n_offsets);
/* Row-kernel variant used on A_l for precision 0 (FP64) or 1 (FP32): threads per row and the
 * form (*pattern: 0 CSR, 1 row patterns, 2 row groups with identical column sets, 3 hybrid of
 * big row groups and row patterns, 4 vector hybrid, 5 sliced), chosen by the setup-time tuner
 * when autotune is set. */
GIAMG_API int giamg_level_kernel(giamg_handle h, int level, int precision, int* threads_per_row, int* pattern);
/* Switch the row kernel of level `level` for precision 0 (FP64) or 1 (FP32) after setup: form 0
 * the default rule, 1..6 as the row_form option (CSR, row patterns, row groups, hybrid, vector
 * hybrid, sliced), threads 0 (automatic) or 4, 8, 16, 32 threads per row where the form has a
 * choice.  Builds the value copy the form reads and releases copies no longer read; a form that
 * does not apply to the level falls back to the default kernel (giamg_level_kernel reports what
 * runs).  Results change only by rounding.  Synchronises the handle's stream; captured solve
 * graphs are dropped and recaptured.  Used by the in-solve tuners (Python tune.py). */
GIAMG_API int giamg_set_row_kernel(giamg_handle h, int level, int precision, int form, int threads);
/* Rows per work item of the multi-right-hand-side FP32 products on `level` (giamg_solve_batch):
 * 1 one row per warp, 2 two rows of one row group per warp sharing every gathered row of X
 * (needs row groups), 0 automatic (2 when more than 16 columns).  Results of a column do not
 * depend on the choice beyond rounding.  Synchronises the stream; batch graphs are dropped. */
GIAMG_API int giamg_set_batch_rows(giamg_handle h, int level, int rows_per_item);
/* Largest Ritz value rho_hat of D^-1/2 A_l D^-1/2 used by the level's smoother. */
GIAMG_API int giamg_level_rho(giamg_handle h, int level, double* rho_hat);
/* Change the degree k of every level's Chebyshev smoother (Sec. 2) after setup: the hierarchy
 * and the Lanczos bounds are kept, only the polynomial's coefficients change, so the result is
 * the handle giamg_setup would have built with cheb_degree = degree.  degree in [1, 64]
 * (GIAMG_ERR_ARG otherwise).  Synchronises the handle's stream first. */
GIAMG_API int giamg_set_cheb_degree(giamg_handle h, int degree);

/* Single steps of the solve, on the handle's stream (parity tests call these):
 *   giamg_apply_vcycle: z = V(r), Algorithm 1 from the finest level (precision 0 / 1).
 *   giamg_level_spmv:   y = A_l x.
 *   giamg_level_spmv32: y = A_l x with A_l's FP32 values, FP32 x and y and FP32 accumulation: the
 *                       product of the FP32 V-cycle, through the level's FP32 row kernel.
 *   giamg_level_smooth: Chebyshev smoothing of A_l x = b in place (x_is_zero: x enters as 0).
 *   giamg_level_restrict: r_c = R_l r_f (R = P^T; element form on p-levels).
 *   giamg_level_prolong:  x_f += P_l e_c (element form on p-levels).
 *   giamg_coarse_solve:  x = A_L^-1 r on the coarsest level (Cholesky triangular solves).
 * The V-cycle applies A_L^-1 as a dense matrix formed at setup from the Cholesky factor by the
 * same triangular solves on the unit vectors. */
GIAMG_API int giamg_apply_vcycle(giamg_handle h, int precision, const double* r, double* z);
GIAMG_API int giamg_level_spmv(giamg_handle h, int level, const double* x, double* y);
GIAMG_API int giamg_level_spmv32(giamg_handle h, int level, const float* x, float* y);
GIAMG_API int giamg_level_smooth(giamg_handle h, int level, const double* b, double* x, int x_is_zero);
GIAMG_API int giamg_level_restrict(giamg_handle h, int level, const double* r_f, double* r_c);
GIAMG_API int giamg_level_prolong(giamg_handle h, int level, const double* e_c, double* x_f);
GIAMG_API int giamg_coarse_solve(giamg_handle h, const double* r, double* x);
/*   giamg_level_residual: r = b - A_l x (the residual step of Algorithm 1, FP64). */
GIAMG_API int giamg_level_residual(giamg_handle h, int level, const double* b, const double* x, double* r);

/* Single steps of the FP32 V-cycle (precision 1), through the same kernels it launches: A_l's
 * FP32 values, the FP32 diagonal inverse, FP32 interpolation tables and FP32 vectors with FP32
 * accumulation.  Vectors are float32 (host or device per device_ptrs, caller-owned; lengths n_l of
 * the level, n_next for the coarse side of a transfer, n_L for the coarsest level).
 *   giamg_level_residual32: r = b - A_l x.
 *   giamg_level_smooth32:   Chebyshev smoothing of A_l x = b in place (Sec. 2's smoother with the
 *                           level's coefficients rounded to FP32; x_is_zero: x enters as 0).
 *   giamg_level_restrict32: r_c = R_l r_f (element form on p-levels, Algorithm 7's P transposed).
 *   giamg_level_prolong32:  x_f += P_l e_c (element form on p-levels).
 *   giamg_coarse_solve32:   x = A_L^-1 r on the coarsest level as the FP32 V-cycle applies it: r
 *                           widened to FP64, the dense A_L^-1 formed at setup, x rounded to FP32.
 * GIAMG_ERR_ARG for a level index out of range, a coarsest level passed to a transfer or to the
 * smoother, or NULL vectors. */
GIAMG_API int giamg_level_residual32(giamg_handle h, int level, const float* b, const float* x, float* r);
GIAMG_API int giamg_level_smooth32(giamg_handle h, int level, const float* b, float* x, int x_is_zero);
GIAMG_API int giamg_level_restrict32(giamg_handle h, int level, const float* r_f, float* r_c);
GIAMG_API int giamg_level_prolong32(giamg_handle h, int level, const float* e_c, float* x_f);
GIAMG_API int giamg_coarse_solve32(giamg_handle h, const float* r, float* x);

/* Switch the pointer mode of later calls on this handle (0 host arrays, 1 device arrays). */
GIAMG_API int giamg_set_device_ptrs(giamg_handle h, int device_ptrs);

/* Opt-in timers (CUDA events around the launches of each category, on the handle's stream):
 *   0 CSR row kernels of the finest level inside the V-cycle (smoother steps, residual)
 *   1 CSR row kernels of the coarser levels   2 transfers   3 coarsest solve   4 vectors
 *   5 the outer CG product q = A p
 * giamg_profile_enable resets the records; giamg_profile_read synchronises the stream and
 * returns, for one category, the summed kernel time (ms), the number of timed launches and the
 * algorithmic bytes those launches must move (matrix values, indices and row pointers once,
 * each vector once). */
GIAMG_API int giamg_profile_enable(giamg_handle h, int enable);
GIAMG_API int giamg_profile_read(giamg_handle h, int category, double* total_ms, int64_t* launches,
                                 double* bytes);

/* Number of kernels this library has launched in the process so far (all handles). */
GIAMG_API int giamg_launch_count(int64_t* count);

/* The true relative residual ||b - A x||_2 / ||b||_2 on the finest level, computed without
 * allocating any memory (the paper has no counterpart; this is a service for callers).
 * Callers that cannot call cudaMalloc -- code whose device memory is owned by another allocator
 * that has reserved the GPU, or a loop that must keep a fixed memory footprint -- get the same
 * number as giamg_solve_stats, which allocates a small buffer on every call.
 *   b, x: device arrays of the handle's n on the handle's device (always device pointers, whatever
 *     device_ptrs says); host memory or another device's memory is refused with GIAMG_ERR_ARG.
 *   *true_relres: host output.  Work runs on the handle's stream, which is synchronised; the
 *     handle's device is made current for the call and the caller's device restored after it.
 * The partial sums live in a static 1 MiB device array that every GPU loading the library holds
 * until the process exits; matrices with more than 16,777,216 rows are rejected with
 * GIAMG_ERR_ARG.  giamg_setup loads that array (and this call's kernels) on the handle's device
 * and looks up its device address, so the array exists once setup has returned and no call here
 * loads or allocates anything, its first one included.  All calls on one device share the array,
 * so calls that overlap on the same GPU race; each call writes every entry it reads, so nothing
 * needs clearing. */
GIAMG_API int giamg_true_relres_noalloc(giamg_handle h, const double* b, const double* x, double* true_relres);

/* Release the handle and all of its device memory.  NULL is accepted. */
GIAMG_API int giamg_free(giamg_handle h);

/* Last error message of the calling thread ("" if none). */
GIAMG_API const char* giamg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
