/*
 * oracle.h -- plain, slow, FP64 CPU oracle of the GIAMG-preconditioned CG solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this code.  The CUDA library never calls it, and it never calls the CUDA
 * library; the two share no source.
 *
 * Every function follows one step of the paper (arXiv 2512.15121) and says which:
 *   Algorithm 1  the V-cycle                         orc_vcycle
 *   Algorithm 2  extract the next level's dofs       orc_extract_next_dof
 *   Algorithm 3  collect and sort them               orc_dof_next
 *   Algorithm 4  next-level element map              orc_l2g_next
 *   Algorithm 7  prolongation (nodal footnote)       orc_comp_prol
 *   Sec. 2       Galerkin coarse operator RAP        orc_spgemm / orc_transpose
 *   Sec. 2.5     smoothed aggregation (MIS, SPAI)    orc_mis2 / orc_aggregate / orc_sa_prolongation
 *   Sec. 2       Jacobi-Chebyshev smoother           orc_cheb
 *   Sec. 2       coarsest direct solve (Cholesky)    orc_cholesky / orc_chol_solve
 *   Sec. 2       PCG with one V-cycle per iteration  orc_solve
 * Parity pins: see the tests (GLL values of Fig. 1, Table 1's 27/343 coarsest level, closed
 * forms, brute force on small graphs, dense solves).  Algorithms 5-6 (the MPI renumbering)
 * have no counterpart on one process.
 */
#ifndef GIAMG_ORACLE_H
#define GIAMG_ORACLE_H
#include <stdint.h>

#define ORC_MAXP 12

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_ORDER = -2, ORC_ERR_MAP = -3, ORC_ERR_OOM = -4,
       ORC_ERR_NOT_SPD = -6, ORC_ERR_BREAKDOWN = -7, ORC_ERR_MAXITER = -8 };
enum { ORC_KIND_P = 0, ORC_KIND_H = 1, ORC_KIND_COARSEST = 2 };

typedef struct {
  int64_t n, m;        /* rows, columns */
  int64_t* rp;         /* [n+1] */
  int32_t* ci;         /* [nnz], ascending in each row */
  double* v;           /* [nnz] */
} orc_csr;

typedef struct {
  int cheb_degree;       /* k, pre and post */
  double cheb_lo, cheb_hi; /* interval [lo, hi] * rho_hat */
  int lanczos_steps;
  int coarse_max;        /* h-coarsen while n > coarse_max */
  int max_levels;
  double strength_theta; /* 0: structural strength graph */
  int hash_kind;         /* 0: SplitMix64-based hash; 1: identity hash h(i) = i */
  int p_schedule;        /* 0: halving (q = p/2, odd p: largest proper divisor), 1: q = p - 1,
                            2: q = p - 2 (at least 1) */
  int basis;             /* 0: nodal GLL Lagrange basis; 1: modal (hierarchical) basis, local 1D
                            index 0 and p the vertex modes, 1..p-1 the bubbles of degree 2..p */
} orc_options;

typedef struct orc_hier orc_hier;

void orc_default_options(orc_options* o);

/* ---- building blocks (exported for the pins) ---- */
uint32_t orc_hash(int kind, int64_t i);
void orc_gll_nodes(int p, double* xi);
int orc_next_order(int p);
int orc_next_order_sched(int p, int schedule);
/* fine local index (per direction) that labels coarse local index s (0..q) of an order-q
   element inside an order-p one: s p / q when that is whole, else the nearer index; *tie is set
   when s p / q lies half way (both neighbours then label it, see orc_coarse_anchor) */
int orc_anchor_index(int p, int q, int s, int* tie);
void orc_p1d(int p, int q, double* tab /* [(p+1)][(q+1)] */);
/* the 1D prolongation table of a basis: orc_p1d for the nodal basis; for the modal basis the
   injection P1D[a][b] = 1 when fine mode a is coarse mode b (a = b for b < q, a = p for b = q) */
void orc_p1d_basis(int p, int q, int basis, double* tab);
int orc_spgemm(const orc_csr* A, const orc_csr* B, orc_csr* C);
int orc_transpose(const orc_csr* A, orc_csr* T);
void orc_csr_free(orc_csr* A);
int orc_mis2(int64_t n, const int64_t* rp, const int32_t* ci, int hash_kind, uint8_t* in_set,
             int* rounds);
int orc_aggregate(int64_t n, const int64_t* rp, const int32_t* ci, const uint8_t* in_set,
                  int32_t* agg, int64_t* n_agg);
int orc_sa_prolongation_csr(const orc_csr* A, const int32_t* agg, int64_t n_agg, orc_csr* P);
double orc_lanczos_rho(const orc_csr* A, int steps, int hash_kind);
double orc_tridiag_max_eig(int m, const double* alpha, const double* beta);
int orc_cholesky(int n, double* a /* in: SPD, row-major; out: L in the lower triangle */);
void orc_chol_solve(int n, const double* L, const double* b, double* x);
void orc_spmv(const orc_csr* A, const double* x, double* y);

/* ---- hierarchy ---- */
int orc_setup(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, int32_t n_elem,
              const int32_t* elem_dof, int p, const orc_options* opt, orc_hier** out);
int orc_num_levels(const orc_hier* h);
int orc_level_info(const orc_hier* h, int l, int* kind, int64_t* n, int64_t* nnz, int* order,
                   int64_t* p_nnz, int64_t* n_next);
int orc_export_level(const orc_hier* h, int l, int64_t* rp, int32_t* ci, double* v, int32_t* agg);
int orc_export_prolongation(const orc_hier* h, int l, int64_t* rp, int32_t* ci, double* v);
int orc_level_extra(const orc_hier* h, int l, double* rho_hat, int32_t* l2g /* or NULL */);
void orc_free(orc_hier* h);

/* z = V(r), one V-cycle (Algorithm 1) from the finest level; precision 0 = FP64, 1 = FP32 levels */
int orc_vcycle(orc_hier* h, int precision, const double* r, double* z);
/* single steps on level l (FP64) */
int orc_level_spmv(orc_hier* h, int l, const double* x, double* y);
int orc_level_cheb(orc_hier* h, int l, const double* b, double* x, int x_is_zero);
int orc_level_restrict(orc_hier* h, int l, const double* rf, double* rc);
int orc_level_prolong(orc_hier* h, int l, const double* ec, double* xf);
int orc_coarse_solve(orc_hier* h, const double* r, double* x);
int orc_level_residual(orc_hier* h, int l, const double* b, const double* x, double* r);
/* single steps of the FP32 V-cycle (orc_vcycle with precision 1): FP32 copies of A_l, D^-1, P_l
   and R_l, FP32 vectors and accumulation; the coarsest solve in FP64 on the widened right-hand
   side, rounded back to FP32 */
int orc_level_spmv32(orc_hier* h, int l, const float* x, float* y);
int orc_level_residual32(orc_hier* h, int l, const float* b, const float* x, float* r);
int orc_level_cheb32(orc_hier* h, int l, const float* b, float* x, int x_is_zero);
int orc_level_restrict32(orc_hier* h, int l, const float* rf, float* rc);
int orc_level_prolong32(orc_hier* h, int l, const float* ec, float* xf);
int orc_coarse_solve32(orc_hier* h, const float* r, float* x);

/* PCG (flexible=0) or flexible CG (flexible=1) with one V-cycle per iteration, x0 = 0.
   force_iters > 0 runs exactly that many iterations.  hist[0..iters] receives the relative
   residual of the recursive residual (may be NULL). */
int orc_solve(orc_hier* h, const double* b, double* x, double rtol, int max_iter, int force_iters,
              int precision, int flexible, int* iters, double* relres, double* hist);

int orc_num_threads(void);
void orc_set_num_threads(int n);
#endif
