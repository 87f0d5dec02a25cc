/*
 * oracle.c -- plain FP64 CPU oracle of GIAMG-preconditioned CG (arXiv 2512.15121).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU-baseline leg of
 * the benchmark, never by the CUDA library.  It shares no source with the library.
 *
 * Written for clarity, not speed: every step is the plain definition or the paper's algorithm
 * in the paper's order.  The only concessions to size are OpenMP pragmas on loops over rows
 * whose iterations are independent; every floating-point reduction runs in a fixed order
 * (dot products over fixed 4096-row blocks, summed in block order), so results do not depend
 * on the thread count.  Build with -ffp-contract=off so x86 and Arm builds agree bit for bit.
 *
 * Readings where the paper is silent (kept identical in the CUDA library):
 *   - p schedule: q = p/2 for even p, else the largest proper divisor of p, down to 1.
 *   - coarse dofs of a nodal element: coarse node (i,j,k) inherits the id of fine node
 *     (ri, rj, rk), r = p/q (Algorithm 2's index rule with the stride r).
 *   - prolongation values: Lagrange interpolation of the order-q basis at the order-p GLL
 *     nodes (Algorithm 7's nodal footnote); the row of a fine dof takes its values from the
 *     first element (ascending) that contains it; exact zeros are not stored.
 *   - h-coarsening: MIS-2 by synchronous max rounds over (state, hash, index) tuples on the
 *     structural graph, aggregates by distance, SPAI-0 smoothing  P = T - M A T.
 *   - smoother: Chebyshev of degree k on D^-1 A over [lo, hi] * rho_hat, rho_hat the largest
 *     Ritz value of Lanczos on D^-1/2 A D^-1/2.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_BLOCK 4096

/* ======================================================================= utilities */
uint32_t orc_hash(int kind, int64_t i) {
  if (kind == 1) return (uint32_t)i;
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ULL + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (uint32_t)(z >> 32);
}

void orc_csr_free(orc_csr* A) {
  free(A->rp); free(A->ci); free(A->v);
  A->rp = NULL; A->ci = NULL; A->v = NULL;
  A->n = A->m = 0;
}

static int64_t orc_nnz(const orc_csr* A) { return A->rp ? A->rp[A->n] : 0; }

/* blocked dot product: fixed 4096-row blocks, partial sums added in block order */
static double orc_dot(int64_t n, const double* x, const double* y) {
  int64_t nb = (n + ORC_BLOCK - 1) / ORC_BLOCK;
  double* part = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nb; ++b) {
    int64_t lo = b * ORC_BLOCK, hi = lo + ORC_BLOCK < n ? lo + ORC_BLOCK : n;
    double s = 0.0;
    for (int64_t i = lo; i < hi; ++i) s += x[i] * y[i];
    part[b] = s;
  }
  double s = 0.0;
  for (int64_t b = 0; b < nb; ++b) s += part[b];
  free(part);
  return s;
}

void orc_spmv(const orc_csr* A, const double* x, double* y) {
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t) s += A->v[t] * x[A->ci[t]];
    y[i] = s;
  }
}

static void orc_spmv32(int64_t n, const int64_t* rp, const int32_t* ci, const float* v, const float* x,
                       float* y) {
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) s += v[t] * x[ci[t]];
    y[i] = s;
  }
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* ======================================================================= 1D rules */
/* GLL nodes of order p: -1, 1 and the zeros of the derivative of the Legendre polynomial
   P_p.  Newton's method on P_p', with P_p' and P_p'' from the recurrences
   P_{k+1} = ((2k+1) x P_k - k P_{k-1}) / (k+1) and P_{k+1}' = P_{k-1}' + (2k+1) P_k,
   P_{k+1}'' = P_{k-1}'' + (2k+1) P_k'; started from -cos(pi j / p), stopped at |step| < 1e-15.
   The left half is mirrored, and the middle node is exactly 0 for even p. */
void orc_gll_nodes(int p, double* xi) {
  xi[0] = -1.0;
  xi[p] = 1.0;
  for (int j = 1; j <= p / 2; ++j) {
    double x = -cos(ORC_PI * (double)j / (double)p);
    for (int it = 0; it < 200; ++it) {
      /* values, first and second derivatives for k = 0, 1 */
      double P0 = 1.0, P1 = x, d0 = 0.0, d1 = 1.0, s0 = 0.0, s1 = 0.0;
      for (int k = 1; k < p; ++k) {
        double P2 = ((2.0 * k + 1.0) * x * P1 - k * P0) / (k + 1.0);
        double d2 = d0 + (2.0 * k + 1.0) * P1;
        double s2 = s0 + (2.0 * k + 1.0) * d1;
        P0 = P1; P1 = P2; d0 = d1; d1 = d2; s0 = s1; s1 = s2;
      }
      double step = d1 / s1;
      x -= step;
      if (fabs(step) < 1e-15) break;
    }
    xi[j] = x;
    xi[p - j] = -x;
  }
  if (p % 2 == 0) xi[p / 2] = 0.0;
}

/* p schedule (reading): q = p/2 for even p, else the largest proper divisor of p. */
int orc_next_order(int p) {
  if (p <= 1) return 1;
  if (p % 2 == 0) return p / 2;
  for (int d = p / 2; d >= 1; --d)
    if (p % d == 0) return d;
  return 1;
}

/* Modal (hierarchical) bases: the order-q modes are the order-p modes of degree <= q, so the
   paper's prefix extraction (Algorithm 2) keeps them and Algorithm 7 puts a 1 at each: coarse 1D
   mode b is fine mode b for b < q (vertex mode at -1, bubbles of degree 2..q) and fine mode p for
   b = q (vertex mode at +1). */
static int orc_modal_index(int p, int q, int b) { return b == q ? p : b; }

void orc_p1d_basis(int p, int q, int basis, double* tab) {
  if (basis != 1) {
    orc_p1d(p, q, tab);
    return;
  }
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= q; ++b) tab[a * (q + 1) + b] = a == orc_modal_index(p, q, b) ? 1.0 : 0.0;
}

/* The other p schedules (the paper compares coarsening by one and by two, Sec. 3.2). */
int orc_next_order_sched(int p, int schedule) {
  if (p <= 1) return 1;
  if (schedule == 1) return p - 1;
  if (schedule == 2) return p > 2 ? p - 2 : 1;
  return orc_next_order(p);
}

/* Labels of coarse nodes by fine nodes (Algorithm 2, generalised to any q < p).  With r = p/q
   whole, coarse node s is labelled by fine node r s.  Otherwise by the fine node nearest to the
   fraction s p / q of the edge; when s p / q is half way between two fine nodes, both are
   candidates and orc_coarse_anchor keeps the one with the smaller global id, a choice that does
   not depend on how an element is oriented (reflecting an edge maps the two candidates onto
   each other).  Since p / q > 1, different coarse nodes never share a candidate. */
int orc_anchor_index(int p, int q, int s, int* tie) {
  const int f = (s * p) / q, rem = (s * p) % q;
  *tie = 0;
  if (rem == 0) return f;
  if (2 * rem < q) return f;
  if (2 * rem > q) return f + 1;
  *tie = 1;
  return f;  /* candidates f and f + 1 */
}

/* the fine dof labelling coarse local node (i, j, k): the smallest global id among the
   candidates of the three directions */
static int32_t orc_coarse_anchor(int p, int q, int basis, const int32_t* df_arr, int i, int j, int k) {
  const int n1 = p + 1;
  if (basis == 1)
    return df_arr[(n1 * n1) * orc_modal_index(p, q, i) + n1 * orc_modal_index(p, q, j) + orc_modal_index(p, q, k)];
  int ti, tj, tk;
  const int ai = orc_anchor_index(p, q, i, &ti), aj = orc_anchor_index(p, q, j, &tj), ak = orc_anchor_index(p, q, k, &tk);
  int32_t best = INT32_MAX;
  for (int di = 0; di <= ti; ++di)
    for (int dj = 0; dj <= tj; ++dj)
      for (int dk = 0; dk <= tk; ++dk) {
        const int32_t g = df_arr[(n1 * n1) * (ai + di) + n1 * (aj + dj) + (ak + dk)];
        if (g < best) best = g;
      }
  return best;
}

/* P1D[a][b] = l_b^(q)(xi_a^(p)): order-q Lagrange basis on the order-q GLL nodes evaluated at
   the order-p GLL nodes, product formula multiplied in ascending m. */
void orc_p1d(int p, int q, double* tab) {
  double xp[ORC_MAXP + 1], xq[ORC_MAXP + 1];
  orc_gll_nodes(p, xp);
  orc_gll_nodes(q, xq);
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= q; ++b) {
      double v = 1.0;
      for (int m = 0; m <= q; ++m)
        if (m != b) v = v * ((xp[a] - xq[m]) / (xq[b] - xq[m]));
      tab[a * (q + 1) + b] = v;
    }
}

/* ======================================================================= sparse products */
/* C = A B.  Pattern: the symbolic union over the inner index (no value-based dropping), columns
   ascending.  Values: each entry summed over the inner index k in ascending order, starting
   from 0, one product a_ik * b_kj rounded then added at a time. */
int orc_spgemm(const orc_csr* A, const orc_csr* B, orc_csr* C) {
  if (A->m != B->n) return ORC_ERR_ARG;
  int64_t n = A->n, m = B->m;
  C->n = n; C->m = m;
  C->rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!C->rp) return ORC_ERR_OOM;
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int err = 0;
#pragma omp parallel
  {
    int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    if (!mark) err = 1;
    for (int64_t j = 0; mark && j < m; ++j) mark[j] = -1;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      if (!mark) continue;
      int64_t c = 0;
      for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t) {
        int32_t k = A->ci[t];
        for (int64_t u = B->rp[k]; u < B->rp[k + 1]; ++u) {
          int32_t j = B->ci[u];
          if (mark[j] != i) { mark[j] = i; ++c; }
        }
      }
      cnt[i] = c;
    }
    free(mark);
  }
  if (err) { free(cnt); return ORC_ERR_OOM; }
  C->rp[0] = 0;
  for (int64_t i = 0; i < n; ++i) C->rp[i + 1] = C->rp[i] + cnt[i];
  free(cnt);
  int64_t nnz = C->rp[n];
  C->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  C->v = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!C->ci || !C->v) return ORC_ERR_OOM;
#pragma omp parallel
  {
    int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    double* acc = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; ++j) mark[j] = -1;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      int32_t* ci = C->ci + C->rp[i];
      int64_t c = 0;
      for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t) {
        int32_t k = A->ci[t];
        for (int64_t u = B->rp[k]; u < B->rp[k + 1]; ++u) {
          int32_t j = B->ci[u];
          if (mark[j] != i) { mark[j] = i; ci[c++] = j; acc[j] = 0.0; }
        }
      }
      qsort(ci, (size_t)c, sizeof(int32_t), cmp_i32);
      for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t) {
        int32_t k = A->ci[t];
        double a = A->v[t];
        for (int64_t u = B->rp[k]; u < B->rp[k + 1]; ++u) {
          double prod = a * B->v[u];
          acc[B->ci[u]] = acc[B->ci[u]] + prod;
        }
      }
      double* cv = C->v + C->rp[i];
      for (int64_t t = 0; t < c; ++t) cv[t] = acc[ci[t]];
    }
    free(mark); free(acc);
  }
  return ORC_OK;
}

/* T = A^T by a stable counting sort: row i of A contributes in ascending i, so every row of
   T has ascending columns. */
int orc_transpose(const orc_csr* A, orc_csr* T) {
  int64_t n = A->n, m = A->m, nnz = orc_nnz(A);
  T->n = m; T->m = n;
  T->rp = (int64_t*)calloc((size_t)m + 1, sizeof(int64_t));
  T->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  T->v = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!T->rp || !T->ci || !T->v) return ORC_ERR_OOM;
  for (int64_t t = 0; t < nnz; ++t) T->rp[A->ci[t] + 1]++;
  for (int64_t j = 0; j < m; ++j) T->rp[j + 1] += T->rp[j];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  memcpy(fill, T->rp, sizeof(int64_t) * (size_t)m);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int64_t d = fill[A->ci[t]]++;
      T->ci[d] = (int32_t)i;
      T->v[d] = A->v[t];
    }
  free(fill);
  return ORC_OK;
}

/* ======================================================================= p-coarsening */
/* Algorithm 2 with nodal labels: the coarse local node (i,j,k), i,j,k <= q, is labelled by the
   fine node of orc_coarse_anchor ((ri, rj, rk) when r = p/q is whole); the labels are copied in
   coarse local order. */
static void orc_extract_next_dof(int p, int q, int basis, const int32_t* df_arr, int32_t* dc_arr) {
  int c = 0;
  for (int i = 0; i <= q; ++i)
    for (int j = 0; j <= q; ++j)
      for (int k = 0; k <= q; ++k) dc_arr[c++] = orc_coarse_anchor(p, q, basis, df_arr, i, j, k);
}

/* Algorithm 3: collect the retained fine dofs over all elements (skipping those already
   collected), then sort.  Membership is kept in a flag array over the fine dofs. */
static int32_t* orc_dof_next(int64_t n_f, int32_t n_elem, int p, int q, int basis, const int32_t* l2g, int64_t* n_c) {
  int nlf = (p + 1) * (p + 1) * (p + 1), nlc = (q + 1) * (q + 1) * (q + 1);
  uint8_t* in = (uint8_t*)calloc((size_t)n_f, 1);
  int32_t* collect = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_f);
  int32_t* dc = (int32_t*)malloc(sizeof(int32_t) * (size_t)nlc);
  int64_t c = 0;
  for (int32_t e = 0; e < n_elem; ++e) {
    orc_extract_next_dof(p, q, basis, l2g + (size_t)e * nlf, dc);
    for (int d = 0; d < nlc; ++d) {
      if (in[dc[d]]) continue;
      in[dc[d]] = 1;
      collect[c++] = dc[d];
    }
  }
  qsort(collect, (size_t)c, sizeof(int32_t), cmp_i32);
  free(in); free(dc);
  *n_c = c;
  return collect;
}

/* Algorithm 4: l2g_next(e, dof) = hash_l2g(extracted fine dof), hash_l2g the position of a
   fine dof in the sorted collect array. */
static int32_t* orc_l2g_next(int64_t n_f, int32_t n_elem, int p, int q, int basis, const int32_t* l2g,
                             const int32_t* collect, int64_t n_c) {
  int nlf = (p + 1) * (p + 1) * (p + 1), nlc = (q + 1) * (q + 1) * (q + 1);
  int32_t* hash = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_f);
  for (int64_t i = 0; i < n_f; ++i) hash[i] = -1;
  for (int64_t c = 0; c < n_c; ++c) hash[collect[c]] = (int32_t)c;
  int32_t* nxt = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_elem * nlc);
  int32_t* dc = (int32_t*)malloc(sizeof(int32_t) * (size_t)nlc);
  for (int32_t e = 0; e < n_elem; ++e) {
    orc_extract_next_dof(p, q, basis, l2g + (size_t)e * nlf, dc);
    for (int d = 0; d < nlc; ++d) nxt[(size_t)e * nlc + d] = hash[dc[d]];
  }
  free(hash); free(dc);
  return nxt;
}

typedef struct { int32_t row, col, elem; double val; } orc_coo;

/* Algorithm 7, nodal form: every element appends (fine dof, coarse dof, interpolation value)
   for every fine local node a and coarse local node b with a non-zero value
   P1D[a1][b1] * P1D[a2][b2] * P1D[a3][b3] (multiplied left to right); the list is sorted by
   (row, column) and duplicates are removed keeping the first element's entry.  The sort is a
   stable bucket sort by row followed by a stable insertion sort by column inside each row. */
static int orc_comp_prol(int64_t n_f, int64_t n_c, int32_t n_elem, int p, int q, int basis, const int32_t* l2g,
                         const int32_t* l2g_next, orc_csr* P, double* max_dup_diff) {
  int n1 = p + 1, m1 = q + 1, nlf = n1 * n1 * n1, nlc = m1 * m1 * m1;
  double tab[(ORC_MAXP + 1) * (ORC_MAXP + 1)];
  orc_p1d_basis(p, q, basis, tab);
  /* count entries per row */
  int64_t* cnt = (int64_t*)calloc((size_t)n_f + 1, sizeof(int64_t));
  for (int32_t e = 0; e < n_elem; ++e)
    for (int a = 0; a < nlf; ++a) {
      int a1 = a / (n1 * n1), a2 = (a / n1) % n1, a3 = a % n1;
      int c = 0;
      for (int b = 0; b < nlc; ++b) {
        int b1 = b / (m1 * m1), b2 = (b / m1) % m1, b3 = b % m1;
        double v = tab[a1 * m1 + b1] * tab[a2 * m1 + b2] * tab[a3 * m1 + b3];
        if (v != 0.0) ++c;
      }
      cnt[l2g[(size_t)e * nlf + a] + 1] += c;
    }
  for (int64_t i = 0; i < n_f; ++i) cnt[i + 1] += cnt[i];
  int64_t total = cnt[n_f];
  orc_coo* coo = (orc_coo*)malloc(sizeof(orc_coo) * (size_t)(total > 0 ? total : 1));
  if (!coo) { free(cnt); return ORC_ERR_OOM; }
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_f);
  memcpy(fill, cnt, sizeof(int64_t) * (size_t)n_f);
  for (int32_t e = 0; e < n_elem; ++e)
    for (int a = 0; a < nlf; ++a) {
      int a1 = a / (n1 * n1), a2 = (a / n1) % n1, a3 = a % n1;
      int32_t row = l2g[(size_t)e * nlf + a];
      for (int b = 0; b < nlc; ++b) {
        int b1 = b / (m1 * m1), b2 = (b / m1) % m1, b3 = b % m1;
        double v = tab[a1 * m1 + b1] * tab[a2 * m1 + b2] * tab[a3 * m1 + b3];
        if (v == 0.0) continue;
        orc_coo en = {row, l2g_next[(size_t)e * nlc + b], e, v};
        coo[fill[row]++] = en;
      }
    }
  free(fill);
  /* per row: stable insertion sort by column, drop duplicates keeping the first */
  P->n = n_f; P->m = n_c;
  P->rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_f + 1));
  int64_t* keep = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_f + 1));
  double dmax = 0.0;
#pragma omp parallel for schedule(dynamic, 256) reduction(max : dmax)
  for (int64_t i = 0; i < n_f; ++i) {
    orc_coo* r = coo + cnt[i];
    int64_t len = cnt[i + 1] - cnt[i];
    for (int64_t s = 1; s < len; ++s) {
      orc_coo x = r[s];
      int64_t t = s - 1;
      while (t >= 0 && r[t].col > x.col) { r[t + 1] = r[t]; --t; }
      r[t + 1] = x;
    }
    int64_t k = 0;
    for (int64_t s = 0; s < len; ++s) {
      if (k > 0 && r[k - 1].col == r[s].col) {
        double d = fabs(r[k - 1].val - r[s].val);
        if (d > dmax) dmax = d;
        continue;
      }
      r[k++] = r[s];
    }
    keep[i] = k;
  }
  P->rp[0] = 0;
  for (int64_t i = 0; i < n_f; ++i) P->rp[i + 1] = P->rp[i] + keep[i];
  int64_t nnz = P->rp[n_f];
  P->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  P->v = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  for (int64_t i = 0; i < n_f; ++i)
    for (int64_t s = 0; s < keep[i]; ++s) {
      P->ci[P->rp[i] + s] = coo[cnt[i] + s].col;
      P->v[P->rp[i] + s] = coo[cnt[i] + s].val;
    }
  free(keep); free(cnt); free(coo);
  if (max_dup_diff) *max_dup_diff = dmax;
  return ORC_OK;
}

/* ======================================================================= h-coarsening */
enum { ST_OUT = 0, ST_UND = 1, ST_IN = 2 };

/* tuple order (state, hash, index), compared lexicographically */
static int orc_tuple_gt(int sa, uint32_t ha, int64_t a, int sb, uint32_t hb, int64_t b) {
  if (sa != sb) return sa > sb;
  if (ha != hb) return ha > hb;
  return a > b;
}

/* MIS-2 by synchronous rounds (after Bell, Dalton and Olson 2012).  Every round takes, for
   each node, the largest (state, hash, index) tuple of its closed distance-2 neighbourhood as
   two distance-1 max passes over the previous round's states; an undecided node that is its
   own maximum joins the set, an undecided node whose maximum is in the set leaves.  The graph
   (rp, ci) holds the off-diagonal neighbours and must be symmetric. */
int orc_mis2(int64_t n, const int64_t* rp, const int32_t* ci, int hash_kind, uint8_t* in_set, int* rounds) {
  int* st = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int* st2 = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  uint32_t* h = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  int64_t* m1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) { st[i] = ST_UND; h[i] = orc_hash(hash_kind, i); }
  int r = 0;
  for (;;) {
    int64_t und = 0;
    for (int64_t i = 0; i < n; ++i) und += st[i] == ST_UND;
    if (!und) break;
    ++r;
    /* pass 1: m1[i] = argmax over the closed neighbourhood of i */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int64_t best = i;
      for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
        int64_t j = ci[t];
        if (orc_tuple_gt(st[j], h[j], j, st[best], h[best], best)) best = j;
      }
      m1[i] = best;
    }
    /* pass 2 and the state update */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int64_t best = m1[i];
      for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
        int64_t j = m1[ci[t]];
        if (orc_tuple_gt(st[j], h[j], j, st[best], h[best], best)) best = j;
      }
      int s = st[i];
      if (s == ST_UND) {
        if (best == i) s = ST_IN;
        else if (st[best] == ST_IN) s = ST_OUT;
      }
      st2[i] = s;
    }
    memcpy(st, st2, sizeof(int) * (size_t)n);
  }
  for (int64_t i = 0; i < n; ++i) in_set[i] = st[i] == ST_IN;
  free(st); free(st2); free(h); free(m1);
  if (rounds) *rounds = r;
  return ORC_OK;
}

/* Aggregates from an MIS-2: roots numbered in ascending index order; phase 1, every node
   next to a root joins it (the root is unique); phase 2, every remaining node joins the
   aggregate of the phase-1 neighbour with the smallest aggregate id. */
int orc_aggregate(int64_t n, const int64_t* rp, const int32_t* ci, const uint8_t* in_set, int32_t* agg,
                  int64_t* n_agg) {
  int32_t* a1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t na = 0;
  for (int64_t i = 0; i < n; ++i) a1[i] = in_set[i] ? (int32_t)na++ : -1;
  int bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (in_set[i]) continue;
    int32_t g = -1;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
      if (in_set[ci[t]]) {
        if (g >= 0 && a1[ci[t]] != g) bad = 1;
        g = a1[ci[t]];
      }
    a1[i] = g;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (a1[i] >= 0) { agg[i] = a1[i]; continue; }
    int32_t g = -1;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
      int32_t c = a1[ci[t]];
      if (c >= 0 && (g < 0 || c < g)) g = c;
    }
    if (g < 0) bad = 1;
    agg[i] = g;
  }
  free(a1);
  *n_agg = na;
  return bad ? ORC_ERR_ARG : ORC_OK;
}

/* strength graph: off-diagonal pattern of A; with theta > 0 only |a_ij| >= theta sqrt(a_ii a_jj) */
static void orc_strength(const orc_csr* A, double theta, int64_t** grp, int32_t** gci) {
  int64_t n = A->n;
  double* diag = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    diag[i] = 0.0;
    for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t)
      if (A->ci[t] == i) diag[i] = A->v[t];
  }
  int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  rp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int32_t j = A->ci[t];
      if (j == i) continue;
      if (theta > 0.0 && !(fabs(A->v[t]) >= theta * sqrt(diag[i] * diag[j]))) continue;
      ++c;
    }
    rp[i + 1] = rp[i] + c;
  }
  int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = rp[i];
    for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int32_t j = A->ci[t];
      if (j == i) continue;
      if (theta > 0.0 && !(fabs(A->v[t]) >= theta * sqrt(diag[i] * diag[j]))) continue;
      ci[c++] = j;
    }
  }
  free(diag);
  *grp = rp; *gci = ci;
}

/* Smoothed aggregation prolongation P = T - M A T, T[i, agg(i)] = 1, M = diag(a_ii / sum_j a_ij^2)
   (SPAI-0).  Pattern: that of A T united with that of T; no dropping.  A row without off-diagonal
   entries (a Dirichlet identity row: an isolated node, its own aggregate) is not smoothed, M_ii =
   0: SPAI-0 would give it M_ii = 1/a_ii and so an all-zero column of P. */
static int orc_sa_prolongation(const orc_csr* A, const int32_t* agg, int64_t n_agg, orc_csr* P) {
  int64_t n = A->n;
  orc_csr T = {n, n_agg, NULL, NULL, NULL};
  T.rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  T.ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  T.v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i <= n; ++i) T.rp[i] = i;
  for (int64_t i = 0; i < n; ++i) { T.ci[i] = agg[i]; T.v[i] = 1.0; }
  orc_csr AT;
  int rc = orc_spgemm(A, &T, &AT);
  if (rc) { orc_csr_free(&T); return rc; }
  /* union with T (T's entry is already in A T when a_ii is stored; kept general) */
  P->n = n; P->m = n_agg;
  P->rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  P->rp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int found = 0;
    for (int64_t t = AT.rp[i]; t < AT.rp[i + 1]; ++t) found |= AT.ci[t] == agg[i];
    P->rp[i + 1] = P->rp[i] + (AT.rp[i + 1] - AT.rp[i]) + (found ? 0 : 1);
  }
  P->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P->rp[n] > 0 ? P->rp[n] : 1));
  P->v = (double*)malloc(sizeof(double) * (size_t)(P->rp[n] > 0 ? P->rp[n] : 1));
  for (int64_t i = 0; i < n; ++i) {
    double diag = 0.0, ss = 0.0;
    int coupled = 0;
    for (int64_t t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      ss = ss + A->v[t] * A->v[t];
      if (A->ci[t] == i) diag = A->v[t];
      else coupled = 1;
    }
    double mi = coupled ? diag / ss : 0.0;
    int inserted = 0;
    for (int64_t t = AT.rp[i]; t < AT.rp[i + 1]; ++t) inserted |= AT.ci[t] == agg[i];
    int64_t d = P->rp[i];
    for (int64_t t = AT.rp[i]; t < AT.rp[i + 1]; ++t) {
      int32_t j = AT.ci[t];
      if (!inserted && agg[i] < j) { P->ci[d] = agg[i]; P->v[d] = 1.0; ++d; inserted = 1; }
      double tij = j == agg[i] ? 1.0 : 0.0;
      P->ci[d] = j;
      P->v[d] = tij - mi * AT.v[t];
      ++d;
    }
    if (!inserted) { P->ci[d] = agg[i]; P->v[d] = 1.0; }
  }
  orc_csr_free(&T);
  orc_csr_free(&AT);
  return ORC_OK;
}

int orc_sa_prolongation_csr(const orc_csr* A, const int32_t* agg, int64_t n_agg, orc_csr* P) {
  return orc_sa_prolongation(A, agg, n_agg, P);
}

/* ======================================================================= smoother */
/* largest eigenvalue of the symmetric tridiagonal matrix (alpha on the diagonal, beta off it)
   by bisection on the Sturm count */
double orc_tridiag_max_eig(int m, const double* alpha, const double* beta) {
  double lo = alpha[0], hi = alpha[0];
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i < m - 1 ? fabs(beta[i]) : 0.0);
    if (alpha[i] - r < lo) lo = alpha[i] - r;
    if (alpha[i] + r > hi) hi = alpha[i] + r;
  }
  for (int it = 0; it < 200; ++it) {
    double x = 0.5 * (lo + hi);
    if (x <= lo || x >= hi) break;
    /* number of eigenvalues below x */
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      d = alpha[i] - x - (i > 0 ? beta[i - 1] * beta[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++cnt;
    }
    if (cnt == m) hi = x; else lo = x;
  }
  return hi;
}

/* rho_hat: largest Ritz value of `steps` Lanczos steps (no reorthogonalisation) on
   D^-1/2 A D^-1/2 from v_i = 1 + (hash(i) mod 1024) / 1024, normalised. */
double orc_lanczos_rho(const orc_csr* A, int steps, int hash_kind) {
  int64_t n = A->n;
  double* dsq = (double*)malloc(sizeof(double) * (size_t)n);
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  double* vp = (double*)calloc((size_t)n, sizeof(double));
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t u = A->rp[i]; u < A->rp[i + 1]; ++u)
      if (A->ci[u] == i) d = A->v[u];
    dsq[i] = 1.0 / sqrt(d);
    v[i] = 1.0 + (double)(orc_hash(hash_kind, i) % 1024u) / 1024.0;
  }
  double nv = sqrt(orc_dot(n, v, v));
  for (int64_t i = 0; i < n; ++i) v[i] = v[i] / nv;
  int m = steps < n ? steps : (int)n;
  double* al = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double* be = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double bprev = 0.0;
  int used = 0;
  for (int j = 0; j < m; ++j) {
    for (int64_t i = 0; i < n; ++i) t[i] = dsq[i] * v[i];
    orc_spmv(A, t, w);
    for (int64_t i = 0; i < n; ++i) w[i] = dsq[i] * w[i] - bprev * vp[i];
    double a = orc_dot(n, w, v);
    for (int64_t i = 0; i < n; ++i) w[i] = w[i] - a * v[i];
    double b = sqrt(orc_dot(n, w, w));
    al[j] = a;
    be[j] = b;
    used = j + 1;
    if (j == m - 1 || b <= 1e-14 * fabs(a)) break;
    for (int64_t i = 0; i < n; ++i) { vp[i] = v[i]; v[i] = w[i] / b; }
    bprev = b;
  }
  double rho = orc_tridiag_max_eig(used, al, be);
  free(dsq); free(v); free(vp); free(w); free(t); free(al); free(be);
  return rho;
}

/* ======================================================================= coarsest */
/* dense right-looking Cholesky, row-major n x n; L is left in the lower triangle */
int orc_cholesky(int n, double* a) {
  for (int k = 0; k < n; ++k) {
    double d = a[(size_t)k * n + k];
    if (!(d > 0.0)) return ORC_ERR_NOT_SPD;
    d = sqrt(d);
    a[(size_t)k * n + k] = d;
    for (int i = k + 1; i < n; ++i) a[(size_t)i * n + k] = a[(size_t)i * n + k] / d;
    for (int j = k + 1; j < n; ++j)
      for (int i = j; i < n; ++i) a[(size_t)i * n + j] = a[(size_t)i * n + j] - a[(size_t)i * n + k] * a[(size_t)j * n + k];
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) a[(size_t)i * n + j] = 0.0;
  return ORC_OK;
}

/* L L^T x = b by forward then backward substitution */
void orc_chol_solve(int n, const double* L, const double* b, double* x) {
  double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s = s - L[(size_t)i * n + k] * y[k];
    y[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s = s - L[(size_t)k * n + i] * x[k];
    x[i] = s / L[(size_t)i * n + i];
  }
  free(y);
}

/* ======================================================================= hierarchy */
typedef struct {
  int kind, order;
  orc_csr A, P, R;          /* P: n x n_next prolongation to this level; R = P^T */
  int32_t* agg;             /* h-levels: aggregate of each row */
  int32_t* l2g;             /* p-levels (orders >= 1 reached by p-coarsening): element map */
  double* dinv;
  double rho;
  double* L;                /* coarsest: Cholesky factor, n x n */
  /* FP32 copies for the mixed-precision V-cycle */
  float *A32, *P32, *R32, *dinv32;
  /* work */
  double *x, *b, *r, *d;
  float *x32, *b32, *r32, *d32;
} orc_level;

struct orc_hier {
  orc_options opt;
  int nlev;
  orc_level lev[64];
  int32_t n_elem;
  double max_dup_diff;
};

void orc_default_options(orc_options* o) {
  o->cheb_degree = 3;
  o->cheb_lo = 0.1;
  o->cheb_hi = 1.1;
  o->lanczos_steps = 20;
  o->coarse_max = 500;
  o->max_levels = 16;
  o->strength_theta = 0.0;
  o->hash_kind = 0;
  o->p_schedule = 0;
  o->basis = 0;
}

static int orc_copy_csr(int64_t n, int64_t m, const int64_t* rp, const int32_t* ci, const double* v, orc_csr* A) {
  A->n = n; A->m = m;
  int64_t nnz = rp[n];
  A->rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  A->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  A->v = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!A->rp || !A->ci || !A->v) return ORC_ERR_OOM;
  memcpy(A->rp, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(A->ci, ci, sizeof(int32_t) * (size_t)nnz);
  memcpy(A->v, v, sizeof(double) * (size_t)nnz);
  return ORC_OK;
}

static float* orc_to_f32(const double* v, int64_t n) {
  float* o = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) o[i] = (float)v[i];
  return o;
}

/* Galerkin coarse operator A_c = R (A P) with R = P^T */
static int orc_galerkin(const orc_csr* A, const orc_csr* P, orc_csr* R, orc_csr* Ac) {
  orc_csr AP;
  int rc = orc_spgemm(A, P, &AP);
  if (rc) return rc;
  rc = orc_transpose(P, R);
  if (rc) { orc_csr_free(&AP); return rc; }
  rc = orc_spgemm(R, &AP, Ac);
  orc_csr_free(&AP);
  return rc;
}

int orc_setup(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, int32_t n_elem,
              const int32_t* elem_dof, int p, const orc_options* opt, orc_hier** out) {
  *out = NULL;
  if (n <= 0 || !rp || !ci || !v || opt->cheb_degree < 1) return ORC_ERR_ARG;
  if (p < 1 || p > ORC_MAXP) return ORC_ERR_ORDER;
  int nlf0 = (p + 1) * (p + 1) * (p + 1);
  if (p > 1) {
    if (n_elem <= 0 || !elem_dof) return ORC_ERR_MAP;
    for (size_t t = 0; t < (size_t)n_elem * nlf0; ++t)
      if (elem_dof[t] < 0 || elem_dof[t] >= n) return ORC_ERR_MAP;
  }
  orc_hier* h = (orc_hier*)calloc(1, sizeof(orc_hier));
  h->opt = *opt;
  h->n_elem = n_elem;
  int rc = orc_copy_csr(n, n, rp, ci, v, &h->lev[0].A);
  if (rc) { orc_free(h); return rc; }
  h->lev[0].order = p;
  if (p > 1) {
    h->lev[0].l2g = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_elem * nlf0);
    memcpy(h->lev[0].l2g, elem_dof, sizeof(int32_t) * (size_t)n_elem * nlf0);
  }
  h->nlev = 1;
  /* p-coarsening: Algorithms 2-4 and 7, then the Galerkin product, until order 1 */
  while (h->lev[h->nlev - 1].order > 1 && h->nlev < opt->max_levels) {
    orc_level* f = &h->lev[h->nlev - 1];
    orc_level* c = &h->lev[h->nlev];
    int pf = f->order, q = orc_next_order_sched(pf, opt->p_schedule);
    int64_t n_c;
    int32_t* collect = orc_dof_next(f->A.n, n_elem, pf, q, opt->basis, f->l2g, &n_c);
    c->l2g = orc_l2g_next(f->A.n, n_elem, pf, q, opt->basis, f->l2g, collect, n_c);
    free(collect);
    double dd = 0.0;
    rc = orc_comp_prol(f->A.n, n_c, n_elem, pf, q, opt->basis, f->l2g, c->l2g, &f->P, &dd);
    if (rc) { orc_free(h); return rc; }
    if (dd > h->max_dup_diff) h->max_dup_diff = dd;
    rc = orc_galerkin(&f->A, &f->P, &f->R, &c->A);
    if (rc) { orc_free(h); return rc; }
    f->kind = ORC_KIND_P;
    c->order = q;
    h->nlev++;
  }
  /* h-coarsening by smoothed aggregation (Sec. 2.5) while the level is large */
  while (h->lev[h->nlev - 1].A.n > opt->coarse_max && h->nlev < opt->max_levels) {
    orc_level* f = &h->lev[h->nlev - 1];
    int64_t *grp; int32_t* gci;
    orc_strength(&f->A, opt->strength_theta, &grp, &gci);
    uint8_t* in_set = (uint8_t*)malloc((size_t)f->A.n);
    orc_mis2(f->A.n, grp, gci, opt->hash_kind, in_set, NULL);
    int32_t* agg = (int32_t*)malloc(sizeof(int32_t) * (size_t)f->A.n);
    int64_t n_agg = 0;
    rc = orc_aggregate(f->A.n, grp, gci, in_set, agg, &n_agg);
    free(grp); free(gci); free(in_set);
    if (rc || (double)n_agg > 0.9 * (double)f->A.n) { free(agg); break; }
    rc = orc_sa_prolongation(&f->A, agg, n_agg, &f->P);
    if (rc) { free(agg); orc_free(h); return rc; }
    orc_level* c = &h->lev[h->nlev];
    rc = orc_galerkin(&f->A, &f->P, &f->R, &c->A);
    if (rc) { free(agg); orc_free(h); return rc; }
    f->agg = agg;
    f->kind = ORC_KIND_H;
    c->order = 0;
    h->nlev++;
  }
  /* coarsest level: dense Cholesky */
  orc_level* cl = &h->lev[h->nlev - 1];
  cl->kind = ORC_KIND_COARSEST;
  {
    int64_t nc = cl->A.n;
    if (nc > 20000) { orc_free(h); return ORC_ERR_ARG; }
    cl->L = (double*)calloc((size_t)(nc * nc), sizeof(double));
    for (int64_t i = 0; i < nc; ++i)
      for (int64_t t = cl->A.rp[i]; t < cl->A.rp[i + 1]; ++t) cl->L[i * nc + cl->A.ci[t]] = cl->A.v[t];
    rc = orc_cholesky((int)nc, cl->L);
    if (rc) { orc_free(h); return rc; }
  }
  /* smoother data and work vectors */
  for (int l = 0; l < h->nlev; ++l) {
    orc_level* L = &h->lev[l];
    int64_t nl = L->A.n;
    L->dinv = (double*)malloc(sizeof(double) * (size_t)nl);
    for (int64_t i = 0; i < nl; ++i) {
      double d = 0.0;
      for (int64_t t = L->A.rp[i]; t < L->A.rp[i + 1]; ++t)
        if (L->A.ci[t] == i) d = L->A.v[t];
      if (!(d > 0.0)) { orc_free(h); return ORC_ERR_NOT_SPD; }
      L->dinv[i] = 1.0 / d;
    }
    if (L->kind != ORC_KIND_COARSEST) L->rho = orc_lanczos_rho(&L->A, opt->lanczos_steps, opt->hash_kind);
    L->x = (double*)calloc((size_t)nl, sizeof(double));
    L->b = (double*)calloc((size_t)nl, sizeof(double));
    L->r = (double*)calloc((size_t)nl, sizeof(double));
    L->d = (double*)calloc((size_t)nl, sizeof(double));
    L->A32 = orc_to_f32(L->A.v, orc_nnz(&L->A));
    L->dinv32 = (float*)malloc(sizeof(float) * (size_t)nl);
    for (int64_t i = 0; i < nl; ++i) L->dinv32[i] = (float)L->dinv[i];
    if (L->kind != ORC_KIND_COARSEST) {
      L->P32 = orc_to_f32(L->P.v, orc_nnz(&L->P));
      L->R32 = orc_to_f32(L->R.v, orc_nnz(&L->R));
    }
    L->x32 = (float*)calloc((size_t)nl, sizeof(float));
    L->b32 = (float*)calloc((size_t)nl, sizeof(float));
    L->r32 = (float*)calloc((size_t)nl, sizeof(float));
    L->d32 = (float*)calloc((size_t)nl, sizeof(float));
  }
  *out = h;
  return ORC_OK;
}

int orc_num_levels(const orc_hier* h) { return h->nlev; }

int orc_level_info(const orc_hier* h, int l, int* kind, int64_t* n, int64_t* nnz, int* order, int64_t* p_nnz,
                   int64_t* n_next) {
  if (l < 0 || l >= h->nlev) return ORC_ERR_ARG;
  const orc_level* L = &h->lev[l];
  if (kind) *kind = L->kind;
  if (n) *n = L->A.n;
  if (nnz) *nnz = orc_nnz(&L->A);
  if (order) *order = L->order;
  if (p_nnz) *p_nnz = L->kind == ORC_KIND_COARSEST ? 0 : orc_nnz(&L->P);
  if (n_next) *n_next = L->kind == ORC_KIND_COARSEST ? 0 : L->P.m;
  return ORC_OK;
}

int orc_export_level(const orc_hier* h, int l, int64_t* rp, int32_t* ci, double* v, int32_t* agg) {
  if (l < 0 || l >= h->nlev) return ORC_ERR_ARG;
  const orc_level* L = &h->lev[l];
  int64_t nnz = orc_nnz(&L->A);
  if (rp) memcpy(rp, L->A.rp, sizeof(int64_t) * (size_t)(L->A.n + 1));
  if (ci) memcpy(ci, L->A.ci, sizeof(int32_t) * (size_t)nnz);
  if (v) memcpy(v, L->A.v, sizeof(double) * (size_t)nnz);
  if (agg && L->agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->A.n);
  return ORC_OK;
}

int orc_export_prolongation(const orc_hier* h, int l, int64_t* rp, int32_t* ci, double* v) {
  if (l < 0 || l >= h->nlev || h->lev[l].kind == ORC_KIND_COARSEST) return ORC_ERR_ARG;
  const orc_level* L = &h->lev[l];
  int64_t nnz = orc_nnz(&L->P);
  if (rp) memcpy(rp, L->P.rp, sizeof(int64_t) * (size_t)(L->P.n + 1));
  if (ci) memcpy(ci, L->P.ci, sizeof(int32_t) * (size_t)nnz);
  if (v) memcpy(v, L->P.v, sizeof(double) * (size_t)nnz);
  return ORC_OK;
}

int orc_level_extra(const orc_hier* h, int l, double* rho_hat, int32_t* l2g) {
  if (l < 0 || l >= h->nlev) return ORC_ERR_ARG;
  const orc_level* L = &h->lev[l];
  if (rho_hat) *rho_hat = L->rho;
  if (l2g && L->l2g && L->order >= 1) {
    int n1 = L->order + 1;
    memcpy(l2g, L->l2g, sizeof(int32_t) * (size_t)h->n_elem * n1 * n1 * n1);
  }
  return ORC_OK;
}

void orc_free(orc_hier* h) {
  if (!h) return;
  for (int l = 0; l < 64; ++l) {
    orc_level* L = &h->lev[l];
    orc_csr_free(&L->A); orc_csr_free(&L->P); orc_csr_free(&L->R);
    free(L->agg); free(L->l2g); free(L->dinv); free(L->L);
    free(L->A32); free(L->P32); free(L->R32); free(L->dinv32);
    free(L->x); free(L->b); free(L->r); free(L->d);
    free(L->x32); free(L->b32); free(L->r32); free(L->d32);
  }
  free(h);
}

/* ======================================================================= V-cycle */
/* Chebyshev smoothing of degree k on level L (Saad, Iterative Methods, Alg. 12.1, with the
   Jacobi preconditioner): theta = (b+a)/2, delta = (b-a)/2, sigma = theta/delta,
   rho_0 = 1/sigma; d = D^-1 r / theta, x += d; then for s = 1..k-1
   rho_s = 1/(2 sigma - rho_{s-1}), d = rho_s rho_{s-1} d + (2 rho_s / delta) D^-1 r, x += d,
   with r = b - A x recomputed before every step.  With x = 0 the first residual is b. */
static void orc_cheb(orc_hier* h, orc_level* L, const double* b, double* x, int x_is_zero) {
  int64_t n = L->A.n;
  int k = h->opt.cheb_degree;
  double lo = h->opt.cheb_lo * L->rho, hi = h->opt.cheb_hi * L->rho;
  double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  double* r = L->r;
  double* d = L->d;
  if (x_is_zero) memcpy(r, b, sizeof(double) * (size_t)n);
  else {
    orc_spmv(&L->A, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  }
  for (int64_t i = 0; i < n; ++i) {
    d[i] = L->dinv[i] * r[i] / theta;
    x[i] = x_is_zero ? d[i] : x[i] + d[i];
  }
  for (int s = 1; s < k; ++s) {
    orc_spmv(&L->A, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double rho_new = 1.0 / (2.0 * sigma - rho);
    double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
    for (int64_t i = 0; i < n; ++i) {
      d[i] = c1 * d[i] + c2 * L->dinv[i] * r[i];
      x[i] = x[i] + d[i];
    }
    rho = rho_new;
  }
}

static void orc_cheb32(orc_hier* h, orc_level* L, const float* b, float* x, int x_is_zero) {
  int64_t n = L->A.n;
  int k = h->opt.cheb_degree;
  double lo = h->opt.cheb_lo * L->rho, hi = h->opt.cheb_hi * L->rho;
  double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  float* r = L->r32;
  float* d = L->d32;
  float it = (float)(1.0 / theta);
  if (x_is_zero) memcpy(r, b, sizeof(float) * (size_t)n);
  else {
    orc_spmv32(n, L->A.rp, L->A.ci, L->A32, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  }
  for (int64_t i = 0; i < n; ++i) {
    d[i] = L->dinv32[i] * r[i] * it;
    x[i] = x_is_zero ? d[i] : x[i] + d[i];
  }
  for (int s = 1; s < k; ++s) {
    orc_spmv32(n, L->A.rp, L->A.ci, L->A32, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double rho_new = 1.0 / (2.0 * sigma - rho);
    float c1 = (float)(rho_new * rho), c2 = (float)(2.0 * rho_new / delta);
    for (int64_t i = 0; i < n; ++i) {
      d[i] = c1 * d[i] + c2 * L->dinv32[i] * r[i];
      x[i] = x[i] + d[i];
    }
    rho = rho_new;
  }
}

/* Algorithm 1 on level l: the coarsest level is solved directly; otherwise presmooth, form
   the residual, restrict it (p- or h-transfer: both are R = P^T here), recurse, interpolate
   the error, correct, postsmooth.  x enters as zero on every level. */
static void orc_vcycle_level(orc_hier* h, int l, const double* b, double* x) {
  orc_level* L = &h->lev[l];
  int64_t n = L->A.n;
  if (L->kind == ORC_KIND_COARSEST) {
    orc_chol_solve((int)n, L->L, b, x);
    return;
  }
  orc_level* C = &h->lev[l + 1];
  orc_cheb(h, L, b, x, 1);                       /* presmooth */
  orc_spmv(&L->A, x, L->r);                      /* residual */
  for (int64_t i = 0; i < n; ++i) L->r[i] = b[i] - L->r[i];
  orc_spmv(&L->R, L->r, C->b);                   /* restrict */
  orc_vcycle_level(h, l + 1, C->b, C->x);        /* recurse */
  orc_spmv(&L->P, C->x, L->r);                   /* interpolate the error */
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + L->r[i]; /* correct */
  orc_cheb(h, L, b, x, 0);                       /* postsmooth */
}

/* FP32 steps of Algorithm 1: the coarsest solve in FP64 on the widened right-hand side, rounded
   back to FP32; the residual r = b - A x; the correction x += P e (t: an n-vector of scratch) */
static void orc_coarse32(orc_level* L, const float* b, float* x) {
  int64_t n = L->A.n;
  double* bd = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* xd = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  for (int64_t i = 0; i < n; ++i) bd[i] = (double)b[i];
  orc_chol_solve((int)n, L->L, bd, xd);
  for (int64_t i = 0; i < n; ++i) x[i] = (float)xd[i];
  free(bd); free(xd);
}
static void orc_residual32(orc_level* L, const float* b, const float* x, float* r) {
  int64_t n = L->A.n;
  orc_spmv32(n, L->A.rp, L->A.ci, L->A32, x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
}
static void orc_correct32(orc_level* L, const float* e, float* x, float* t) {
  orc_spmv32(L->P.n, L->P.rp, L->P.ci, L->P32, e, t);
  for (int64_t i = 0; i < L->A.n; ++i) x[i] = x[i] + t[i];
}

static void orc_vcycle_level32(orc_hier* h, int l, const float* b, float* x) {
  orc_level* L = &h->lev[l];
  if (L->kind == ORC_KIND_COARSEST) {
    orc_coarse32(L, b, x);
    return;
  }
  orc_level* C = &h->lev[l + 1];
  orc_cheb32(h, L, b, x, 1);                                       /* presmooth */
  orc_residual32(L, b, x, L->r32);                                 /* residual */
  orc_spmv32(L->R.n, L->R.rp, L->R.ci, L->R32, L->r32, C->b32);    /* restrict */
  orc_vcycle_level32(h, l + 1, C->b32, C->x32);                    /* recurse */
  orc_correct32(L, C->x32, x, L->r32);                             /* interpolate and correct */
  orc_cheb32(h, L, b, x, 0);                                       /* postsmooth */
}

int orc_vcycle(orc_hier* h, int precision, const double* r, double* z) {
  orc_level* L = &h->lev[0];
  int64_t n = L->A.n;
  if (precision == 0) {
    orc_vcycle_level(h, 0, r, z);
  } else {
    for (int64_t i = 0; i < n; ++i) L->b32[i] = (float)r[i];
    orc_vcycle_level32(h, 0, L->b32, L->x32);
    for (int64_t i = 0; i < n; ++i) z[i] = (double)L->x32[i];
  }
  return ORC_OK;
}

int orc_level_spmv(orc_hier* h, int l, const double* x, double* y) {
  if (l < 0 || l >= h->nlev) return ORC_ERR_ARG;
  orc_spmv(&h->lev[l].A, x, y);
  return ORC_OK;
}
int orc_level_cheb(orc_hier* h, int l, const double* b, double* x, int x_is_zero) {
  if (l < 0 || l >= h->nlev || h->lev[l].kind == ORC_KIND_COARSEST) return ORC_ERR_ARG;
  orc_cheb(h, &h->lev[l], b, x, x_is_zero);
  return ORC_OK;
}
int orc_level_restrict(orc_hier* h, int l, const double* rf, double* rc) {
  if (l < 0 || l >= h->nlev || h->lev[l].kind == ORC_KIND_COARSEST) return ORC_ERR_ARG;
  orc_spmv(&h->lev[l].R, rf, rc);
  return ORC_OK;
}
int orc_level_prolong(orc_hier* h, int l, const double* ec, double* xf) {
  if (l < 0 || l >= h->nlev || h->lev[l].kind == ORC_KIND_COARSEST) return ORC_ERR_ARG;
  orc_level* L = &h->lev[l];
  double* t = (double*)malloc(sizeof(double) * (size_t)L->A.n);
  orc_spmv(&L->P, ec, t);
  for (int64_t i = 0; i < L->A.n; ++i) xf[i] = xf[i] + t[i];
  free(t);
  return ORC_OK;
}
int orc_coarse_solve(orc_hier* h, const double* r, double* x) {
  orc_level* L = &h->lev[h->nlev - 1];
  orc_chol_solve((int)L->A.n, L->L, r, x);
  return ORC_OK;
}
int orc_level_residual(orc_hier* h, int l, const double* b, const double* x, double* r) {
  if (l < 0 || l >= h->nlev) return ORC_ERR_ARG;
  orc_level* L = &h->lev[l];
  orc_spmv(&L->A, x, r);
  for (int64_t i = 0; i < L->A.n; ++i) r[i] = b[i] - r[i];
  return ORC_OK;
}

/* single steps of the FP32 V-cycle: the same functions orc_vcycle(precision = 1) applies */
int orc_level_spmv32(orc_hier* h, int l, const float* x, float* y) {
  if (l < 0 || l >= h->nlev) return ORC_ERR_ARG;
  orc_level* L = &h->lev[l];
  orc_spmv32(L->A.n, L->A.rp, L->A.ci, L->A32, x, y);
  return ORC_OK;
}
int orc_level_residual32(orc_hier* h, int l, const float* b, const float* x, float* r) {
  if (l < 0 || l >= h->nlev) return ORC_ERR_ARG;
  orc_residual32(&h->lev[l], b, x, r);
  return ORC_OK;
}
int orc_level_cheb32(orc_hier* h, int l, const float* b, float* x, int x_is_zero) {
  if (l < 0 || l >= h->nlev || h->lev[l].kind == ORC_KIND_COARSEST) return ORC_ERR_ARG;
  orc_cheb32(h, &h->lev[l], b, x, x_is_zero);
  return ORC_OK;
}
int orc_level_restrict32(orc_hier* h, int l, const float* rf, float* rc) {
  if (l < 0 || l >= h->nlev || h->lev[l].kind == ORC_KIND_COARSEST) return ORC_ERR_ARG;
  orc_level* L = &h->lev[l];
  orc_spmv32(L->R.n, L->R.rp, L->R.ci, L->R32, rf, rc);
  return ORC_OK;
}
int orc_level_prolong32(orc_hier* h, int l, const float* ec, float* xf) {
  if (l < 0 || l >= h->nlev || h->lev[l].kind == ORC_KIND_COARSEST) return ORC_ERR_ARG;
  orc_level* L = &h->lev[l];
  float* t = (float*)malloc(sizeof(float) * (size_t)(L->A.n > 0 ? L->A.n : 1));
  orc_correct32(L, ec, xf, t);
  free(t);
  return ORC_OK;
}
int orc_coarse_solve32(orc_hier* h, const float* r, float* x) {
  orc_coarse32(&h->lev[h->nlev - 1], r, x);
  return ORC_OK;
}

/* ======================================================================= PCG */
/* Preconditioned CG with one V-cycle per iteration and x0 = 0 (Sec. 2 and Sec. 3.1).  The
   relative residual is ||r_k||_2 / ||b||_2 of the recursive residual.  flexible = 1 takes the
   Polak-Ribiere form beta = <z_{k+1}, r_{k+1} - r_k> / <z_k, r_k> (Notay 2000), used with the
   FP32 V-cycle. */
int orc_solve(orc_hier* h, const double* b, double* x, double rtol, int max_iter, int force_iters,
              int precision, int flexible, int* iters, double* relres, double* hist) {
  orc_level* L0 = &h->lev[0];
  int64_t n = L0->A.n;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  double* rold = flexible ? (double*)malloc(sizeof(double) * (size_t)n) : NULL;
  for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
  double bnorm = sqrt(orc_dot(n, b, b));
  int status = ORC_OK, it = 0;
  double rr = 1.0;
  if (hist) hist[0] = bnorm > 0.0 ? 1.0 : 0.0;
  if (bnorm == 0.0) {
    rr = 0.0;
    goto done;
  }
  orc_vcycle(h, precision, r, z);
  memcpy(p, z, sizeof(double) * (size_t)n);
  double rho = orc_dot(n, r, z);
  int limit = force_iters > 0 ? force_iters : max_iter;
  while (it < limit) {
    orc_spmv(&L0->A, p, q);
    double pq = orc_dot(n, p, q);
    if (!(pq > 0.0) || !(rho > 0.0)) { status = ORC_ERR_BREAKDOWN; break; }
    double alpha = rho / pq;
    if (flexible) memcpy(rold, r, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      x[i] = x[i] + alpha * p[i];
      r[i] = r[i] - alpha * q[i];
    }
    ++it;
    rr = sqrt(orc_dot(n, r, r)) / bnorm;
    if (hist) hist[it] = rr;
    if (force_iters <= 0 && rr <= rtol) break;
    if (it == limit) break;
    orc_vcycle(h, precision, r, z);
    double rho_new;
    if (flexible) {
      for (int64_t i = 0; i < n; ++i) rold[i] = r[i] - rold[i];
      rho_new = orc_dot(n, z, r);
      double beta = orc_dot(n, z, rold) / rho;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    } else {
      rho_new = orc_dot(n, r, z);
      double beta = rho_new / rho;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    rho = rho_new;
  }
  if (status == ORC_OK && force_iters <= 0 && rr > rtol) status = ORC_ERR_MAXITER;
done:
  if (iters) *iters = it;
  if (relres) *relres = rr;
  free(r); free(z); free(p); free(q); free(rold);
  return status;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* thread count of the OpenMP row loops (the results do not depend on it); no effect without OpenMP */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
