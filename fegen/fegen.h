/*
 * fegen.h -- seeded synthetic finite-element inputs (mesh, element map, assembled CSR system,
 * right-hand sides).  See fegen.c.  This is input generation only: the multigrid method, its
 * oracle and the CUDA library each live elsewhere and share no code with this file.
 */
#ifndef FEGEN_H
#define FEGEN_H
#include <stdint.h>

#define FEGEN_MAXP 12
#define FEGEN_MAXQ 16

enum { FEGEN_MESH_UNIFORM = 0, FEGEN_MESH_JITTER = 1, FEGEN_MESH_GRADED = 2 };
enum { FEGEN_BASIS_NODAL = 0, FEGEN_BASIS_MODAL = 1 };
enum { FEGEN_RHS_NONE = 0, FEGEN_RHS_MANUFACTURED = 1, FEGEN_RHS_FOURIER = 2, FEGEN_RHS_ONE = 3 };

typedef struct {
  int nx, ny, nz;        /* elements per direction (x slowest in the element index) */
  int p;                 /* uniform polynomial order, 1..FEGEN_MAXP */
  int nq;                /* Gauss-Legendre points per direction; 0 means p + 2 */
  int mesh_kind;         /* FEGEN_MESH_* */
  double jitter;         /* interior vertex jitter as a fraction of h (uniform in [-j h, j h]) */
  uint64_t mesh_seed;
  double grade_first;    /* graded mesh: thickness of the first z layer; 0 means 1 / (10 nz) */
  int kappa_kind;        /* 0: kappa = 1; 1: kappa = 1 + 0.5 sin(2 pi x); 2: kappa = 0 */
  double lambda;         /* zeroth-order coefficient */
  int dirichlet;         /* 1: homogeneous Dirichlet on all six faces, eliminated symmetrically */
  int rhs_kind;          /* unused by fegen_create; the caller passes the kind to fegen_rhs */
  uint64_t rhs_seed;
  uint64_t perm_seed;    /* 0: natural global numbering; else a seeded random relabelling */
  uint64_t sym_seed;     /* 0: structured local order; else a seeded cube symmetry per element */
  int basis;             /* FEGEN_BASIS_NODAL: Lagrange on the GLL points; FEGEN_BASIS_MODAL: the
                            hierarchical modes -- 1D local index 0 and p the vertex modes (1 - x)/2
                            and (1 + x)/2, index a in 1..p-1 the bubble of degree a + 1,
                            (1 - x)(1 + x)/4 P^(1,1)_(a-1)(x); elements must share one orientation
                            (no sym_seed), as the odd bubbles change sign under reflection */
} fegen_params;

typedef struct fegen_ctx fegen_ctx;

void fegen_default_params(fegen_params* p);
int fegen_create(const fegen_params* prm, fegen_ctx** out);
void fegen_sizes(const fegen_ctx* c, int64_t* n, int64_t* nnz, int32_t* n_elem, int32_t* nloc);
int fegen_fill(fegen_ctx* c, int64_t* row_ptr, int32_t* col, double* val, int32_t* elem_dof,
               double* coords, uint8_t* boundary);
int fegen_rhs(fegen_ctx* c, int kind, uint64_t seed, double* b);
double fegen_l2_error(const fegen_ctx* c, const double* uh);
double fegen_u_manufactured(const double x[3]);
void fegen_free(fegen_ctx* c);
int fegen_num_threads(void);
/* n-point Gauss-Legendre rule on [-1, 1] (1 <= n <= 64), nodes ascending; 0 or -1 on bad n */
int fegen_gauss_rule(int n, double* x, double* w);
/* the 64 coefficients of the Fourier right-hand side of `seed`, index (k1-1)*16 + (k2-1)*4 + (k3-1) */
void fegen_fourier_coef(uint64_t seed, double* coef);

#endif
