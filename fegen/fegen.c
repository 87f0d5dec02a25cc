/*
 * fegen.c -- seeded synthetic finite-element inputs for the GIAMG solver and its oracle.
 *
 * This module plays the part of the finite-element library that, in the paper, assembles the
 * global matrix and hands over the element-to-dof map (Sec. 2, "Required geometric
 * information"; the paper uses Nektar++ for this).  It holds no step of the multigrid method:
 * it builds
 *   - structured hexahedral meshes of the unit cube (uniform, interior vertices jittered, or
 *     graded towards z = 0),
 *   - nodal Gauss-Lobatto-Legendre (GLL) tensor-product elements of order p with the element
 *     local ordering (p+1)^2 i + (p+1) j + k, i along x (appendix, Eq. 8),
 *   - the assembled CSR matrix of  -div(kappa grad u) + lambda u = f  (Eq. 2 with a variable
 *     coefficient), Gauss-Legendre quadrature, symmetric elimination of homogeneous Dirichlet
 *     conditions on all faces,
 *   - right-hand sides: the manufactured solution of Sec. 3.1 (Eqs. 3-4, sign fixed for
 *     -lap u + lambda u = f) or smooth random Fourier fields.
 * Both the CUDA library and the CPU oracle receive these arrays as inputs; neither links this
 * file, and this file links neither of them.
 *
 * Determinism: every floating-point sum has a fixed order that does not depend on the number
 * of threads (entries are summed over elements in ascending element order).  Compile with
 * -ffp-contract=off so that x86 and Arm builds produce identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "fegen.h"

#define FG_PI 3.14159265358979323846

/* ---------------------------------------------------------------- random numbers */
/* SplitMix64 output function applied to a counter: a stateless generator. */
static uint64_t fg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static uint64_t fg_rand(uint64_t seed, uint64_t ctr) {
  return fg_mix64(seed * 0xD1B54A32D192ED03ULL + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}
/* uniform in [0,1) with 53 random bits */
static double fg_unif(uint64_t seed, uint64_t ctr) {
  return (double)(fg_rand(seed, ctr) >> 11) * (1.0 / 9007199254740992.0);
}
/* standard normal by Box-Muller from two counters */
static double fg_normal(uint64_t seed, uint64_t ctr) {
  double u1 = 1.0 - fg_unif(seed, 2 * ctr);     /* (0,1] */
  double u2 = fg_unif(seed, 2 * ctr + 1);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * FG_PI * u2);
}

/* ---------------------------------------------------------------- 1D rules */
/* Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence. */
static void fg_legendre(int n, double x, double* pn, double* pnm1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  *pn = p1; *pnm1 = p0;
}

/* GLL nodes of order p on [-1,1]: the endpoints and the zeros of P_p'.  Newton iteration on
   (1-x^2) P_p'(x) = p (P_{p-1}(x) - x P_p(x)); the left half is computed and mirrored so the
   set is exactly symmetric, with an exact 0 in the middle for even p. */
static void fg_gll_nodes(int p, double* x) {
  x[0] = -1.0; x[p] = 1.0;
  for (int j = 1; j <= p / 2; ++j) {
    double t = -cos(FG_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double pn, pnm1;
      fg_legendre(p, t, &pn, &pnm1);
      /* g(t) = P_{p-1} - t P_p ; g'(t) = P_{p-1}' - P_p - t P_p'.
         Use the identities (1-t^2) P_n' = n (P_{n-1} - t P_n). */
      double dpn = p * (pnm1 - t * pn) / (1.0 - t * t);
      double pnm2 = 0.0, dummy;
      fg_legendre(p - 1, t, &dummy, &pnm2);
      double dpnm1 = (p - 1) * (pnm2 - t * pnm1) / (1.0 - t * t);
      double g = pnm1 - t * pn;
      double dg = dpnm1 - pn - t * dpn;
      double dt = g / dg;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    x[j] = t;
    x[p - j] = -t;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
}

/* Gauss-Legendre rule with n points on [-1,1] (exact for degree 2n-1). */
static void fg_gauss(int n, double* x, double* w) {
  for (int j = 0; j < (n + 1) / 2; ++j) {
    double t = -cos(FG_PI * (j + 0.75) / (n + 0.5));
    double pn = 0, pnm1 = 0;
    for (int it = 0; it < 100; ++it) {
      fg_legendre(n, t, &pn, &pnm1);
      double dp = n * (pnm1 - t * pn) / (1.0 - t * t);
      double dt = pn / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    fg_legendre(n, t, &pn, &pnm1);
    double dp = n * (pnm1 - t * pn) / (1.0 - t * t);
    x[j] = t; x[n - 1 - j] = -t;
    w[j] = w[n - 1 - j] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
  if (n % 2 == 1) {
    double pn, pnm1;
    fg_legendre(n, 0.0, &pn, &pnm1);
    double dp = n * pnm1;
    x[n / 2] = 0.0;
    w[n / 2] = 2.0 / (dp * dp);
  }
}

/* Lagrange basis on nodes xi[0..p] and its derivative, evaluated at t. */
static double fg_lagrange(int p, const double* xi, int a, double t) {
  double v = 1.0;
  for (int m = 0; m <= p; ++m)
    if (m != a) v *= (t - xi[m]) / (xi[a] - xi[m]);
  return v;
}
static double fg_lagrange_d(int p, const double* xi, int a, double t) {
  double s = 0.0;
  for (int k = 0; k <= p; ++k) {
    if (k == a) continue;
    double v = 1.0 / (xi[a] - xi[k]);
    for (int m = 0; m <= p; ++m)
      if (m != a && m != k) v *= (t - xi[m]) / (xi[a] - xi[m]);
    s += v;
  }
  return s;
}

/* Jacobi polynomial P_n^(a,b)(x) by its three-term recurrence. */
static double fg_jacobi(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int k = 2; k <= n; ++k) {
    const double c = 2.0 * k + a + b;
    const double a1 = 2.0 * k * (k + a + b) * (c - 2.0);
    const double a2 = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b);
    const double a3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
    const double p2 = (a2 * p1 - a3 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}
/* hierarchical 1D modes at local index m of order p, and their derivatives */
static double fg_modal(int p, int m, double x) {
  if (m == 0) return 0.5 * (1.0 - x);
  if (m == p) return 0.5 * (1.0 + x);
  return 0.25 * (1.0 - x) * (1.0 + x) * fg_jacobi(m - 1, 1.0, 1.0, x);
}
static double fg_modal_d(int p, int m, double x) {
  if (m == 0) return -0.5;
  if (m == p) return 0.5;
  /* d/dx P_n^(1,1) = (n + 3)/2 P_(n-1)^(2,2) */
  const int n = m - 1;
  const double dp = n > 0 ? 0.5 * (n + 3.0) * fg_jacobi(n - 1, 2.0, 2.0, x) : 0.0;
  return -0.5 * x * fg_jacobi(n, 1.0, 1.0, x) + 0.25 * (1.0 - x) * (1.0 + x) * dp;
}

/* ---------------------------------------------------------------- context */
struct fegen_ctx {
  fegen_params prm;
  int p, n1, nloc, nq;
  int nx, ny, nz;
  int64_t N, nnz;
  int32_t n_elem;
  int64_t N1x, N1y, N1z;       /* nodes per direction */
  double *vx, *vy, *vz;         /* vertex coordinates, (nx+1)(ny+1)(nz+1) each */
  double xi[FEGEN_MAXP + 1];    /* GLL nodes */
  double qx[FEGEN_MAXQ], qw[FEGEN_MAXQ];
  double B[FEGEN_MAXQ * (FEGEN_MAXP + 1)], D[FEGEN_MAXQ * (FEGEN_MAXP + 1)];
  int64_t* perm;                /* structured id -> output id (NULL: identity) */
  uint8_t* sym;                 /* per-element index symmetry (0..47) or NULL */
  int32_t* l2g;                 /* [n_elem][nloc] output ids, structured local order */
  uint8_t* bnd;                 /* [N] by output id */
  int64_t* inc_ptr;             /* node -> (element, local) incidences, ascending element */
  int32_t* inc_e;
  int32_t* inc_a;
  int64_t* row_cnt;
  double* Ke;                   /* [n_elem][nloc][nloc] element matrices, structured order */
  double* be;                   /* [n_elem][nloc] element load vectors (current rhs) */
};

static int fg_sym_map(int s, int n1, int a) {
  /* a = (i, j, k) in the element's local frame; return the structured local index.
     s in [0,48): s % 6 picks an axis permutation, s / 6 picks reflections. */
  static const int perms[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
  int c[3] = {a / (n1 * n1), (a / n1) % n1, a % n1};
  int r = s / 6;
  const int* pm = perms[s % 6];
  int o[3];
  for (int d = 0; d < 3; ++d) {
    int v = c[pm[d]];
    if (r & (1 << d)) v = n1 - 1 - v;
    o[d] = v;
  }
  return (o[0] * n1 + o[1]) * n1 + o[2];
}

static void fg_vertex(const fegen_ctx* c, int ex, int ey, int ez, double v[8][3]) {
  int64_t Vy = c->ny + 1, Vz = c->nz + 1;
  for (int cx = 0; cx < 2; ++cx)
    for (int cy = 0; cy < 2; ++cy)
      for (int cz = 0; cz < 2; ++cz) {
        int64_t vid = ((int64_t)(ex + cx) * Vy + (ey + cy)) * Vz + (ez + cz);
        int id = (cx * 2 + cy) * 2 + cz;
        v[id][0] = c->vx[vid]; v[id][1] = c->vy[vid]; v[id][2] = c->vz[vid];
      }
}

/* trilinear map and its Jacobian J[d][r] = dx_d / dxi_r at reference point (s,t,u) */
static void fg_map(const double v[8][3], double s, double t, double u, double x[3], double J[3][3]) {
  double L[2][3] = {{(1 - s) / 2, (1 - t) / 2, (1 - u) / 2}, {(1 + s) / 2, (1 + t) / 2, (1 + u) / 2}};
  double dL[2] = {-0.5, 0.5};
  for (int d = 0; d < 3; ++d) {
    x[d] = 0; J[d][0] = J[d][1] = J[d][2] = 0;
  }
  for (int cx = 0; cx < 2; ++cx)
    for (int cy = 0; cy < 2; ++cy)
      for (int cz = 0; cz < 2; ++cz) {
        int id = (cx * 2 + cy) * 2 + cz;
        double n = L[cx][0] * L[cy][1] * L[cz][2];
        double n0 = dL[cx] * L[cy][1] * L[cz][2];
        double n1 = L[cx][0] * dL[cy] * L[cz][2];
        double n2 = L[cx][0] * L[cy][1] * dL[cz];
        for (int d = 0; d < 3; ++d) {
          x[d] += n * v[id][d];
          J[d][0] += n0 * v[id][d];
          J[d][1] += n1 * v[id][d];
          J[d][2] += n2 * v[id][d];
        }
      }
}

static double fg_kappa(int kind, const double x[3]) {
  if (kind == 1) return 1.0 + 0.5 * sin(2.0 * FG_PI * x[0]);
  if (kind == 2) return 0.0; /* pure mass matrix (used by a test) */
  return 1.0;
}

/* source term for the manufactured u = sin(pi x) sin(pi y) sin(pi z) of Eq. 4 */
static double fg_f_manufactured(int kappa_kind, double lambda, const double x[3]) {
  double sx = sin(FG_PI * x[0]), sy = sin(FG_PI * x[1]), sz = sin(FG_PI * x[2]);
  double u = sx * sy * sz;
  double k = fg_kappa(kappa_kind, x);
  double f = (3.0 * FG_PI * FG_PI * k + lambda) * u;
  if (kappa_kind == 1)
    f -= FG_PI * FG_PI * cos(2.0 * FG_PI * x[0]) * cos(FG_PI * x[0]) * sy * sz;
  return f;
}
double fegen_u_manufactured(const double x[3]) {
  return sin(FG_PI * x[0]) * sin(FG_PI * x[1]) * sin(FG_PI * x[2]);
}
/* smooth random field: sum over k1,k2,k3 = 1..4 of c_k sin(k1 pi x) sin(k2 pi y) sin(k3 pi z) */
static double fg_f_fourier(const double* coef, const double x[3]) {
  double sx[4], sy[4], sz[4];
  for (int k = 0; k < 4; ++k) {
    sx[k] = sin((k + 1) * FG_PI * x[0]);
    sy[k] = sin((k + 1) * FG_PI * x[1]);
    sz[k] = sin((k + 1) * FG_PI * x[2]);
  }
  double f = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) f += coef[(a * 4 + b) * 4 + c] * sx[a] * sy[b] * sz[c];
  return f;
}

/* C[a][b] += sum_q W[q] X1[q1][a1] Y1[q1][b1] X2[q2][a2] Y2[q2][b2] X3[q3][a3] Y3[q3][b3]
   with a = (a1 n1 + a2) n1 + a3, by three one-dimensional contractions. */
static void fg_contract(int nq, int n1, const double* W, const double* X1, const double* Y1,
                        const double* X2, const double* Y2, const double* X3, const double* Y3,
                        double* T1, double* T2, double* C) {
  int n2 = n1 * n1, nl = n2 * n1;
  /* T1[q1][q2][a3][b3] */
  for (int q1 = 0; q1 < nq; ++q1)
    for (int q2 = 0; q2 < nq; ++q2) {
      const double* w = W + (q1 * nq + q2) * nq;
      double* t = T1 + (size_t)(q1 * nq + q2) * n2;
      for (int a3 = 0; a3 < n1; ++a3)
        for (int b3 = 0; b3 < n1; ++b3) {
          double s = 0.0;
          for (int q3 = 0; q3 < nq; ++q3) s += w[q3] * X3[q3 * n1 + a3] * Y3[q3 * n1 + b3];
          t[a3 * n1 + b3] = s;
        }
    }
  /* T2[q1][a2][b2][a3 b3] */
  for (int q1 = 0; q1 < nq; ++q1)
    for (int a2 = 0; a2 < n1; ++a2)
      for (int b2 = 0; b2 < n1; ++b2) {
        double* t2 = T2 + (((size_t)q1 * n1 + a2) * n1 + b2) * n2;
        for (int m = 0; m < n2; ++m) t2[m] = 0.0;
        for (int q2 = 0; q2 < nq; ++q2) {
          double f = X2[q2 * n1 + a2] * Y2[q2 * n1 + b2];
          const double* t1 = T1 + (size_t)(q1 * nq + q2) * n2;
          for (int m = 0; m < n2; ++m) t2[m] += f * t1[m];
        }
      }
  /* C */
  for (int a1 = 0; a1 < n1; ++a1)
    for (int b1 = 0; b1 < n1; ++b1)
      for (int q1 = 0; q1 < nq; ++q1) {
        double f = X1[q1 * n1 + a1] * Y1[q1 * n1 + b1];
        for (int a2 = 0; a2 < n1; ++a2)
          for (int b2 = 0; b2 < n1; ++b2) {
            const double* t2 = T2 + (((size_t)q1 * n1 + a2) * n1 + b2) * n2;
            for (int a3 = 0; a3 < n1; ++a3) {
              double* crow = C + (size_t)((a1 * n1 + a2) * n1 + a3) * nl + (b1 * n1 + b2) * n1;
              const double* tr = t2 + a3 * n1;
              for (int b3 = 0; b3 < n1; ++b3) crow[b3] += f * tr[b3];
            }
          }
      }
}

/* Element matrix and geometric data of element e (structured local order). */
static void fg_element(const fegen_ctx* c, int32_t e, double* Ke, double* W, double* T1, double* T2) {
  int nq = c->nq, n1 = c->n1, nl = c->nloc, nq3 = nq * nq * nq;
  int ex = e / (c->ny * c->nz), ey = (e / c->nz) % c->ny, ez = e % c->nz;
  double v[8][3];
  fg_vertex(c, ex, ey, ez, v);
  /* W holds 7 weight arrays: G00 G01 G02 G11 G12 G22 and the mass weight */
  for (int q1 = 0; q1 < nq; ++q1)
    for (int q2 = 0; q2 < nq; ++q2)
      for (int q3 = 0; q3 < nq; ++q3) {
        int q = (q1 * nq + q2) * nq + q3;
        double x[3], J[3][3];
        fg_map(v, c->qx[q1], c->qx[q2], c->qx[q3], x, J);
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        double Ji[3][3]; /* inverse of J: Ji[r][d] = dxi_r / dx_d */
        Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        double wdet = c->qw[q1] * c->qw[q2] * c->qw[q3] * fabs(det);
        double k = fg_kappa(c->prm.kappa_kind, x) * wdet;
        int m = 0;
        for (int r = 0; r < 3; ++r)
          for (int s = r; s < 3; ++s) {
            double g = 0.0;
            for (int d = 0; d < 3; ++d) g += Ji[r][d] * Ji[s][d];
            W[(size_t)m * nq3 + q] = k * g;
            ++m;
          }
        W[(size_t)6 * nq3 + q] = c->prm.lambda * wdet;
      }
  memset(Ke, 0, sizeof(double) * (size_t)nl * nl);
  const double* B = c->B;
  const double* D = c->D;
  int m = 0;
  for (int r = 0; r < 3; ++r)
    for (int s = r; s < 3; ++s) {
      const double* Wrs = W + (size_t)m * nq3;
      /* term (r,s) and, off the diagonal, its transpose (s,r) */
      for (int tr = 0; tr < (r == s ? 1 : 2); ++tr) {
        int rr = tr ? s : r, ss = tr ? r : s;
        fg_contract(nq, n1, Wrs, rr == 0 ? D : B, ss == 0 ? D : B, rr == 1 ? D : B, ss == 1 ? D : B,
                    rr == 2 ? D : B, ss == 2 ? D : B, T1, T2, Ke);
      }
      ++m;
    }
  if (c->prm.lambda != 0.0) fg_contract(nq, n1, W + (size_t)6 * nq3, B, B, B, B, B, B, T1, T2, Ke);
  /* the (r,s) and (s,r) contractions round differently: average so K_e is exactly symmetric */
  for (int a = 0; a < nl; ++a)
    for (int b = a + 1; b < nl; ++b) {
      double v = 0.5 * (Ke[(size_t)a * nl + b] + Ke[(size_t)b * nl + a]);
      Ke[(size_t)a * nl + b] = v;
      Ke[(size_t)b * nl + a] = v;
    }
}

/* element load vector for the current rhs kind */
static void fg_element_load(const fegen_ctx* c, int32_t e, int kind, const double* coef, double* be, double* F) {
  int nq = c->nq, n1 = c->n1, nl = c->nloc;
  int ex = e / (c->ny * c->nz), ey = (e / c->nz) % c->ny, ez = e % c->nz;
  double v[8][3];
  fg_vertex(c, ex, ey, ez, v);
  for (int q1 = 0; q1 < nq; ++q1)
    for (int q2 = 0; q2 < nq; ++q2)
      for (int q3 = 0; q3 < nq; ++q3) {
        double x[3], J[3][3];
        fg_map(v, c->qx[q1], c->qx[q2], c->qx[q3], x, J);
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        double f;
        if (kind == FEGEN_RHS_MANUFACTURED) f = fg_f_manufactured(c->prm.kappa_kind, c->prm.lambda, x);
        else if (kind == FEGEN_RHS_FOURIER) f = fg_f_fourier(coef, x);
        else f = 1.0;
        F[(q1 * nq + q2) * nq + q3] = c->qw[q1] * c->qw[q2] * c->qw[q3] * fabs(det) * f;
      }
  for (int a = 0; a < nl; ++a) {
    int a1 = a / (n1 * n1), a2 = (a / n1) % n1, a3 = a % n1;
    double s = 0.0;
    for (int q1 = 0; q1 < nq; ++q1)
      for (int q2 = 0; q2 < nq; ++q2) {
        double b12 = c->B[q1 * n1 + a1] * c->B[q2 * n1 + a2];
        for (int q3 = 0; q3 < nq; ++q3) s += F[(q1 * nq + q2) * nq + q3] * b12 * c->B[q3 * n1 + a3];
      }
    be[a] = s;
  }
}

static int fg_cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

void fegen_default_params(fegen_params* p) {
  memset(p, 0, sizeof(*p));
  p->nx = p->ny = p->nz = 4;
  p->p = 4;
  p->nq = 0;
  p->mesh_kind = FEGEN_MESH_UNIFORM;
  p->jitter = 0.2;
  p->mesh_seed = 1;
  p->kappa_kind = 0;
  p->lambda = 1.0;
  p->dirichlet = 1;
  p->rhs_kind = FEGEN_RHS_MANUFACTURED;
  p->rhs_seed = 1000;
}

/* geometric ratio r with h0 (1 + r + ... + r^{n-1}) = 1 */
static double fg_grade_ratio(int n, double h0) {
  if (fabs(h0 * n - 1.0) < 1e-15) return 1.0;
  double lo = 1.0 + 1e-12, hi = 10.0;
  if (h0 * n > 1.0) { lo = 1e-6; hi = 1.0 - 1e-12; }
  for (int it = 0; it < 200; ++it) {
    double r = 0.5 * (lo + hi), s = 0.0, t = 1.0;
    for (int k = 0; k < n; ++k) { s += t; t *= r; }
    if (h0 * s > 1.0) hi = r; else lo = r;
  }
  return 0.5 * (lo + hi);
}

int fegen_create(const fegen_params* prm, fegen_ctx** out) {
  *out = NULL;
  if (prm->p < 1 || prm->p > FEGEN_MAXP || prm->nx < 1 || prm->ny < 1 || prm->nz < 1) return -1;
  if (prm->basis != FEGEN_BASIS_NODAL && prm->basis != FEGEN_BASIS_MODAL) return -1;
  if (prm->basis == FEGEN_BASIS_MODAL && prm->sym_seed) return -1;
  fegen_ctx* c = (fegen_ctx*)calloc(1, sizeof(fegen_ctx));
  if (!c) return -4;
  c->prm = *prm;
  c->p = prm->p;
  c->n1 = prm->p + 1;
  c->nloc = c->n1 * c->n1 * c->n1;
  c->nq = prm->nq > 0 ? prm->nq : prm->p + 2;
  if (c->nq > FEGEN_MAXQ) { free(c); return -1; }
  c->nx = prm->nx; c->ny = prm->ny; c->nz = prm->nz;
  c->N1x = (int64_t)c->nx * c->p + 1;
  c->N1y = (int64_t)c->ny * c->p + 1;
  c->N1z = (int64_t)c->nz * c->p + 1;
  c->N = c->N1x * c->N1y * c->N1z;
  c->n_elem = c->nx * c->ny * c->nz;
  int p = c->p, n1 = c->n1, nl = c->nloc;

  /* vertices */
  int64_t Vx = c->nx + 1, Vy = c->ny + 1, Vz = c->nz + 1, nv = Vx * Vy * Vz;
  c->vx = (double*)malloc(sizeof(double) * nv);
  c->vy = (double*)malloc(sizeof(double) * nv);
  c->vz = (double*)malloc(sizeof(double) * nv);
  double zr = 1.0, z0 = 1.0 / c->nz;
  if (prm->mesh_kind == FEGEN_MESH_GRADED) {
    z0 = prm->grade_first > 0 ? prm->grade_first : 1.0 / (10.0 * c->nz);
    zr = fg_grade_ratio(c->nz, z0);
  }
  for (int64_t ix = 0; ix < Vx; ++ix)
    for (int64_t iy = 0; iy < Vy; ++iy)
      for (int64_t iz = 0; iz < Vz; ++iz) {
        int64_t vid = (ix * Vy + iy) * Vz + iz;
        double x = (double)ix / c->nx, y = (double)iy / c->ny, z = (double)iz / c->nz;
        if (prm->mesh_kind == FEGEN_MESH_GRADED) {
          double s = 0.0, t = z0;
          for (int64_t k = 0; k < iz; ++k) { s += t; t *= zr; }
          z = iz == c->nz ? 1.0 : s;
        }
        int interior = ix > 0 && ix < c->nx && iy > 0 && iy < c->ny && iz > 0 && iz < c->nz;
        if (prm->mesh_kind == FEGEN_MESH_JITTER && interior) {
          x += (2.0 * fg_unif(prm->mesh_seed, 3 * vid + 0) - 1.0) * prm->jitter / c->nx;
          y += (2.0 * fg_unif(prm->mesh_seed, 3 * vid + 1) - 1.0) * prm->jitter / c->ny;
          z += (2.0 * fg_unif(prm->mesh_seed, 3 * vid + 2) - 1.0) * prm->jitter / c->nz;
        }
        c->vx[vid] = x; c->vy[vid] = y; c->vz[vid] = z;
      }

  /* 1D tables */
  fg_gll_nodes(p, c->xi);
  fg_gauss(c->nq, c->qx, c->qw);
  for (int q = 0; q < c->nq; ++q)
    for (int a = 0; a < n1; ++a) {
      if (prm->basis == FEGEN_BASIS_MODAL) {
        c->B[q * n1 + a] = fg_modal(p, a, c->qx[q]);
        c->D[q * n1 + a] = fg_modal_d(p, a, c->qx[q]);
      } else {
        c->B[q * n1 + a] = fg_lagrange(p, c->xi, a, c->qx[q]);
        c->D[q * n1 + a] = fg_lagrange_d(p, c->xi, a, c->qx[q]);
      }
    }

  /* numbering: structured id s = (I N1y + J) N1z + K, output id = perm[s] */
  if (prm->perm_seed) {
    c->perm = (int64_t*)malloc(sizeof(int64_t) * c->N);
    for (int64_t i = 0; i < c->N; ++i) c->perm[i] = i;
    for (int64_t i = c->N - 1; i > 0; --i) {
      int64_t j = (int64_t)(fg_rand(prm->perm_seed, (uint64_t)i) % (uint64_t)(i + 1));
      int64_t t = c->perm[i]; c->perm[i] = c->perm[j]; c->perm[j] = t;
    }
  }
  if (prm->sym_seed) {
    c->sym = (uint8_t*)malloc(c->n_elem);
    for (int32_t e = 0; e < c->n_elem; ++e) c->sym[e] = (uint8_t)(fg_rand(prm->sym_seed, (uint64_t)e) % 48);
  }
  c->l2g = (int32_t*)malloc(sizeof(int32_t) * (size_t)c->n_elem * nl);
  c->bnd = (uint8_t*)calloc((size_t)c->N, 1);
  for (int32_t e = 0; e < c->n_elem; ++e) {
    int ex = e / (c->ny * c->nz), ey = (e / c->nz) % c->ny, ez = e % c->nz;
    for (int a = 0; a < nl; ++a) {
      int i = a / (n1 * n1), j = (a / n1) % n1, k = a % n1;
      int64_t I = (int64_t)ex * p + i, J = (int64_t)ey * p + j, K = (int64_t)ez * p + k;
      int64_t s = (I * c->N1y + J) * c->N1z + K;
      int64_t g = c->perm ? c->perm[s] : s;
      c->l2g[(size_t)e * nl + a] = (int32_t)g;
      if (I == 0 || I == c->N1x - 1 || J == 0 || J == c->N1y - 1 || K == 0 || K == c->N1z - 1)
        c->bnd[g] = prm->dirichlet ? 1 : 0;
    }
  }
  /* incidences, ascending element */
  c->inc_ptr = (int64_t*)calloc((size_t)c->N + 1, sizeof(int64_t));
  for (size_t t = 0; t < (size_t)c->n_elem * nl; ++t) c->inc_ptr[c->l2g[t] + 1]++;
  for (int64_t i = 0; i < c->N; ++i) c->inc_ptr[i + 1] += c->inc_ptr[i];
  c->inc_e = (int32_t*)malloc(sizeof(int32_t) * (size_t)c->n_elem * nl);
  c->inc_a = (int32_t*)malloc(sizeof(int32_t) * (size_t)c->n_elem * nl);
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->N);
    memcpy(fill, c->inc_ptr, sizeof(int64_t) * (size_t)c->N);
    for (int32_t e = 0; e < c->n_elem; ++e)
      for (int a = 0; a < nl; ++a) {
        int32_t g = c->l2g[(size_t)e * nl + a];
        c->inc_e[fill[g]] = e;
        c->inc_a[fill[g]] = a;
        fill[g]++;
      }
    free(fill);
  }
  /* row counts */
  c->row_cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->N);
  int64_t nnz = 0;
#pragma omp parallel reduction(+ : nnz)
  {
    int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)c->N);
    for (int64_t i = 0; i < c->N; ++i) mark[i] = -1;
#pragma omp for schedule(dynamic, 256)
    for (int64_t g = 0; g < c->N; ++g) {
      int64_t cnt = 0;
      if (c->bnd[g]) cnt = 1;
      else
        for (int64_t t = c->inc_ptr[g]; t < c->inc_ptr[g + 1]; ++t) {
          const int32_t* row = c->l2g + (size_t)c->inc_e[t] * nl;
          for (int b = 0; b < nl; ++b) {
            int32_t col = row[b];
            if (c->bnd[col] || mark[col] == (int32_t)g) continue;
            mark[col] = (int32_t)g;
            ++cnt;
          }
        }
      c->row_cnt[g] = cnt;
      nnz += cnt;
    }
    free(mark);
  }
  c->nnz = nnz;

  /* element matrices (only needed by interior rows; all are computed) */
  c->Ke = (double*)malloc(sizeof(double) * (size_t)c->n_elem * nl * nl);
  if (!c->Ke) { fegen_free(c); return -4; }
#pragma omp parallel
  {
    int nq = c->nq;
    double* W = (double*)malloc(sizeof(double) * 7 * nq * nq * nq);
    double* T1 = (double*)malloc(sizeof(double) * nq * nq * n1 * n1);
    double* T2 = (double*)malloc(sizeof(double) * nq * n1 * n1 * n1 * n1);
#pragma omp for schedule(dynamic, 1)
    for (int32_t e = 0; e < c->n_elem; ++e) fg_element(c, e, c->Ke + (size_t)e * nl * nl, W, T1, T2);
    free(W); free(T1); free(T2);
  }
  *out = c;
  return 0;
}

void fegen_sizes(const fegen_ctx* c, int64_t* n, int64_t* nnz, int32_t* n_elem, int32_t* nloc) {
  if (n) *n = c->N;
  if (nnz) *nnz = c->nnz;
  if (n_elem) *n_elem = c->n_elem;
  if (nloc) *nloc = c->nloc;
}

/* Fill the CSR matrix (columns ascending; each entry summed over elements in ascending
   element order), the element map (element local order, with the optional per-element
   symmetries), the nodal coordinates and the boundary flags.  Any output may be NULL. */
int fegen_fill(fegen_ctx* c, int64_t* row_ptr, int32_t* col, double* val, int32_t* elem_dof,
               double* coords, uint8_t* boundary) {
  int nl = c->nloc, n1 = c->n1, p = c->p;
  if (row_ptr) {
    row_ptr[0] = 0;
    for (int64_t g = 0; g < c->N; ++g) row_ptr[g + 1] = row_ptr[g] + c->row_cnt[g];
  }
  if (row_ptr && col) {
#pragma omp parallel
    {
      int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)c->N);
      int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)c->N);
      for (int64_t i = 0; i < c->N; ++i) mark[i] = -1;
#pragma omp for schedule(dynamic, 256)
      for (int64_t g = 0; g < c->N; ++g) {
        int32_t* cg = col + row_ptr[g];
        if (c->bnd[g]) {
          cg[0] = (int32_t)g;
          if (val) val[row_ptr[g]] = 1.0;
          continue;
        }
        int64_t cnt = 0;
        for (int64_t t = c->inc_ptr[g]; t < c->inc_ptr[g + 1]; ++t) {
          const int32_t* row = c->l2g + (size_t)c->inc_e[t] * nl;
          for (int b = 0; b < nl; ++b) {
            int32_t cc = row[b];
            if (c->bnd[cc] || mark[cc] == (int32_t)g) continue;
            mark[cc] = (int32_t)g;
            cg[cnt++] = cc;
          }
        }
        qsort(cg, (size_t)cnt, sizeof(int32_t), fg_cmp_i32);
        if (!val) continue;
        double* vg = val + row_ptr[g];
        for (int64_t t = 0; t < cnt; ++t) { pos[cg[t]] = (int32_t)t; vg[t] = 0.0; }
        for (int64_t t = c->inc_ptr[g]; t < c->inc_ptr[g + 1]; ++t) {
          int32_t e = c->inc_e[t];
          int a = c->inc_a[t];
          const int32_t* row = c->l2g + (size_t)e * nl;
          const double* K = c->Ke + ((size_t)e * nl + a) * nl;
          for (int b = 0; b < nl; ++b) {
            int32_t cc = row[b];
            if (c->bnd[cc]) continue;
            vg[pos[cc]] += K[b];
          }
        }
      }
      free(mark); free(pos);
    }
  }
  if (elem_dof) {
    for (int32_t e = 0; e < c->n_elem; ++e)
      for (int a = 0; a < nl; ++a) {
        int s = c->sym ? fg_sym_map(c->sym[e], n1, a) : a;
        elem_dof[(size_t)e * nl + a] = c->l2g[(size_t)e * nl + s];
      }
  }
  if (coords) {
    for (int32_t e = 0; e < c->n_elem; ++e) {
      int ex = e / (c->ny * c->nz), ey = (e / c->nz) % c->ny, ez = e % c->nz;
      double v[8][3];
      fg_vertex(c, ex, ey, ez, v);
      for (int a = 0; a < nl; ++a) {
        int i = a / (n1 * n1), j = (a / n1) % n1, k = a % n1;
        double x[3], J[3][3];
        fg_map(v, c->xi[i], c->xi[j], c->xi[k], x, J);
        int32_t g = c->l2g[(size_t)e * nl + a];
        coords[3 * (int64_t)g + 0] = x[0];
        coords[3 * (int64_t)g + 1] = x[1];
        coords[3 * (int64_t)g + 2] = x[2];
      }
    }
  }
  if (boundary) memcpy(boundary, c->bnd, (size_t)c->N);
  (void)p;
  return 0;
}

/* Right-hand side b_a = sum over elements of the quadrature of f phi_a (ascending element),
   zero on Dirichlet dofs.  kind: FEGEN_RHS_*; seed selects the Fourier coefficients. */
int fegen_rhs(fegen_ctx* c, int kind, uint64_t seed, double* b) {
  int nl = c->nloc, nq = c->nq;
  double coef[64];
  for (int k = 0; k < 64; ++k) coef[k] = fg_normal(seed, (uint64_t)k);
  double* be = (double*)malloc(sizeof(double) * (size_t)c->n_elem * nl);
  if (!be) return -4;
#pragma omp parallel
  {
    double* F = (double*)malloc(sizeof(double) * nq * nq * nq);
#pragma omp for schedule(dynamic, 4)
    for (int32_t e = 0; e < c->n_elem; ++e) fg_element_load(c, e, kind, coef, be + (size_t)e * nl, F);
    free(F);
  }
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < c->N; ++g) {
    double s = 0.0;
    if (!c->bnd[g])
      for (int64_t t = c->inc_ptr[g]; t < c->inc_ptr[g + 1]; ++t) s += be[(size_t)c->inc_e[t] * nl + c->inc_a[t]];
    b[g] = s;
  }
  free(be);
  return 0;
}

/* L2 norm of (u_h - u) over the mesh, u the manufactured solution, u_h the nodal field. */
double fegen_l2_error(const fegen_ctx* c, const double* uh) {
  int nl = c->nloc, nq = c->nq, n1 = c->n1;
  double total = 0.0;
  double* part = (double*)calloc((size_t)c->n_elem, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
  for (int32_t e = 0; e < c->n_elem; ++e) {
    int ex = e / (c->ny * c->nz), ey = (e / c->nz) % c->ny, ez = e % c->nz;
    double v[8][3];
    fg_vertex(c, ex, ey, ez, v);
    const int32_t* row = c->l2g + (size_t)e * nl;
    double s = 0.0;
    for (int q1 = 0; q1 < nq; ++q1)
      for (int q2 = 0; q2 < nq; ++q2)
        for (int q3 = 0; q3 < nq; ++q3) {
          double x[3], J[3][3];
          fg_map(v, c->qx[q1], c->qx[q2], c->qx[q3], x, J);
          double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
          double uhq = 0.0;
          for (int a = 0; a < nl; ++a) {
            int a1 = a / (n1 * n1), a2 = (a / n1) % n1, a3 = a % n1;
            uhq += uh[row[a]] * c->B[q1 * n1 + a1] * c->B[q2 * n1 + a2] * c->B[q3 * n1 + a3];
          }
          double d = uhq - fegen_u_manufactured(x);
          s += c->qw[q1] * c->qw[q2] * c->qw[q3] * fabs(det) * d * d;
        }
    part[e] = s;
  }
  for (int32_t e = 0; e < c->n_elem; ++e) total += part[e];
  free(part);
  return sqrt(total);
}

void fegen_free(fegen_ctx* c) {
  if (!c) return;
  free(c->vx); free(c->vy); free(c->vz);
  free(c->perm); free(c->sym); free(c->l2g); free(c->bnd);
  free(c->inc_ptr); free(c->inc_e); free(c->inc_a); free(c->row_cnt);
  free(c->Ke); free(c->be);
  free(c);
}

int fegen_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* The n-point Gauss-Legendre rule of the assembly (nodes ascending), exposed for its tests. */
int fegen_gauss_rule(int n, double* x, double* w) {
  if (n < 1 || n > 64 || !x || !w) return -1;
  fg_gauss(n, x, w);
  return 0;
}

/* The 64 coefficients c_k (k = (k1 - 1) 16 + (k2 - 1) 4 + (k3 - 1)) of the Fourier right-hand
   side drawn from `seed`, as fegen_rhs uses them; exposed for its tests. */
void fegen_fourier_coef(uint64_t seed, double* coef) {
  for (int k = 0; k < 64; ++k) coef[k] = fg_normal(seed, (uint64_t)k);
}
