// batch_kernels.cu -- kernels of the multi-right-hand-side solve: m independent CG recurrences
// (m <= 32) that share every matrix pass.  Blocks of vectors are row-major n x m, so the m
// values of one row are contiguous.
//
//   SpMM row kernels: G = next power of two >= m lanes per row, lane j holds column j; each
//     nonzero (value, column) is loaded once per row and applied to the m gathered values
//     X[col * m + j] (one coalesced segment), so the matrix is read once per m solves.  FP32
//     with m > 16 (the V-cycle of a wide batch): two rows of one row group per warp, so each
//     gathered X row serves both (bat_pairs).
//   p-transfers: the element contractions of the single-vector path with a column index.
//   coarsest solve: X = A^-1 B with the dense inverse.
//   CG updates and dot products per column, reduced in a fixed order (reproducible bits).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace giamg {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t work, int per_block) {
  return (unsigned)std::max<int64_t>((work + per_block - 1) / per_block, 1);
}
inline unsigned vec_grid(int64_t n) {
  return (unsigned)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 16);
}

enum BatchMode { kSpmm = 0, kResid = 1, kBatCheb = 2, kAdd = 3 };

// One row per group of G lanes; lane j < m owns column j.  PAT: columns from the row's template.
//
// Every kernel body below takes the block index and the grid size as arguments (vb, nvb): the
// standalone kernels pass blockIdx.x and gridDim.x, the grouped kernels (several hierarchies in
// one launch) the block's index and count within its hierarchy's share of the grid, so a
// hierarchy's arithmetic -- reduction partitions included -- is the same alone and in a group.
template <int G, typename V, int MODE, bool PAT>
__device__ __forceinline__ void bat_rows_body(int64_t vb, int64_t n, int m, const int64_t* __restrict__ rp,
                                              const int32_t* __restrict__ ci, const int32_t* __restrict__ obase,
                                              const int32_t* __restrict__ toff, const V* __restrict__ val,
                                              const V* __restrict__ X, const V* __restrict__ B, V* __restrict__ Y,
                                              V* __restrict__ D, const V* __restrict__ dinv, V c1, V c2) {
  const int64_t gt = vb * blockDim.x + threadIdx.x;
  const int64_t row = gt / G;
  const int j = threadIdx.x % G;
  if (row >= n || j >= m) return;
  const int64_t s = rp[row], e = rp[row + 1];
  V acc0 = 0, acc1 = 0;
  if (PAT) {
    const int32_t* __restrict__ off = toff + obase[row];
    const V* __restrict__ xr = X + row * m + j;
    const int len = (int)(e - s);
    int k = 0;
    for (; k + 1 < len; k += 2) {
      acc0 = fma(__ldg(val + s + k), xr[(int64_t)__ldg(off + k) * m], acc0);
      acc1 = fma(__ldg(val + s + k + 1), xr[(int64_t)__ldg(off + k + 1) * m], acc1);
    }
    if (k < len) acc0 = fma(__ldg(val + s + k), xr[(int64_t)__ldg(off + k) * m], acc0);
  } else {
    const V* __restrict__ xc = X + j;
    int64_t t = s;
    for (; t + 1 < e; t += 2) {
      acc0 = fma(__ldg(val + t), xc[(int64_t)__ldg(ci + t) * m], acc0);
      acc1 = fma(__ldg(val + t + 1), xc[(int64_t)__ldg(ci + t + 1) * m], acc1);
    }
    if (t < e) acc0 = fma(__ldg(val + t), xc[(int64_t)__ldg(ci + t) * m], acc0);
  }
  const V acc = acc0 + acc1;
  const int64_t o = row * m + j;
  if (MODE == kSpmm) {
    Y[o] = acc;
  } else if (MODE == kAdd) {
    Y[o] += acc;
  } else if (MODE == kResid) {
    Y[o] = B[o] - acc;
  } else {
    const V r = B[o] - acc;
    const V dn = (c1 == V(0) ? V(0) : c1 * D[o]) + c2 * dinv[row] * r;
    D[o] = dn;
    Y[o] = X[o] + dn;
  }
}
template <int G, typename V, int MODE, bool PAT>
__global__ void __launch_bounds__(kThreads)
    bat_rows(int64_t n, int m, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
             const int32_t* __restrict__ obase, const int32_t* __restrict__ toff,
             const V* __restrict__ val, const V* __restrict__ X, const V* __restrict__ B, V* __restrict__ Y,
             V* __restrict__ D, const V* __restrict__ dinv, V c1, V c2) {
  bat_rows_body<G, V, MODE, PAT>(blockIdx.x, n, m, rp, ci, obase, toff, val, X, B, Y, D, dinv, c1, c2);
}

// FP32, m > 16 columns: one warp per work item of two rows of one row group (or one row), lane j
// owning column j.  The two rows have the same columns (the group's column list), so each
// gathered X row (128 bytes) serves both; values are those of each row's CSR entries.  The
// products are summed in bat_rows' order (even and odd entries in two chains).
template <int MODE>
__device__ __forceinline__ void bat_pairs_body(int64_t vblock, int64_t n_items, const int32_t* __restrict__ ia,
                                               const int32_t* __restrict__ ib, const int32_t* __restrict__ ig,
                                               const int64_t* __restrict__ gptr, const int32_t* __restrict__ gcol,
                                               const int64_t* __restrict__ rp, int m, const float* __restrict__ val,
                                               const float* __restrict__ X, const float* __restrict__ B,
                                               float* __restrict__ Y, float* __restrict__ D,
                                               const float* __restrict__ dinv, float c1, float c2) {
  const int64_t item = vblock * (kThreads / 32) + (threadIdx.x >> 5);
  const int j = threadIdx.x & 31;
  if (item >= n_items || j >= m) return;
  const int64_t ra = ia[item], rb = ib[item], g = ig[item];
  const int64_t c0 = gptr[g];
  const int len = (int)(gptr[g + 1] - c0);
  const int32_t* __restrict__ cols = gcol + c0;
  const float* __restrict__ va = val + rp[ra];
  const float* __restrict__ vb = val + rp[rb >= 0 ? rb : ra];
  const float* __restrict__ xc = X + j;
  float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
  int k = 0;
  if (rb >= 0) {
    for (; k + 1 < len; k += 2) {
      const float x0 = xc[(int64_t)__ldg(cols + k) * m], x1 = xc[(int64_t)__ldg(cols + k + 1) * m];
      a0 = fmaf(__ldg(va + k), x0, a0);
      a1 = fmaf(__ldg(va + k + 1), x1, a1);
      b0 = fmaf(__ldg(vb + k), x0, b0);
      b1 = fmaf(__ldg(vb + k + 1), x1, b1);
    }
    if (k < len) {
      const float x0 = xc[(int64_t)__ldg(cols + k) * m];
      a0 = fmaf(__ldg(va + k), x0, a0);
      b0 = fmaf(__ldg(vb + k), x0, b0);
    }
  } else {
    for (; k + 1 < len; k += 2) {
      a0 = fmaf(__ldg(va + k), xc[(int64_t)__ldg(cols + k) * m], a0);
      a1 = fmaf(__ldg(va + k + 1), xc[(int64_t)__ldg(cols + k + 1) * m], a1);
    }
    if (k < len) a0 = fmaf(__ldg(va + k), xc[(int64_t)__ldg(cols + k) * m], a0);
  }
  auto finish = [&](int64_t row, float acc) {
    const int64_t o = row * m + j;
    if (MODE == kSpmm) {
      Y[o] = acc;
    } else if (MODE == kAdd) {
      Y[o] += acc;
    } else if (MODE == kResid) {
      Y[o] = B[o] - acc;
    } else {
      const float r = B[o] - acc;
      const float dn = (c1 == 0.f ? 0.f : c1 * D[o]) + c2 * dinv[row] * r;
      D[o] = dn;
      Y[o] = X[o] + dn;
    }
  };
  finish(ra, a0 + a1);
  if (rb >= 0) finish(rb, b0 + b1);
}
template <int MODE>
__global__ void __launch_bounds__(kThreads)
    bat_pairs(int64_t n_items, const int32_t* __restrict__ ia, const int32_t* __restrict__ ib,
              const int32_t* __restrict__ ig, const int64_t* __restrict__ gptr, const int32_t* __restrict__ gcol,
              const int64_t* __restrict__ rp, int m, const float* __restrict__ val, const float* __restrict__ X,
              const float* __restrict__ B, float* __restrict__ Y, float* __restrict__ D,
              const float* __restrict__ dinv, float c1, float c2) {
  bat_pairs_body<MODE>(blockIdx.x, n_items, ia, ib, ig, gptr, gcol, rp, m, val, X, B, Y, D, dinv, c1, c2);
}

template <int G, typename V, int MODE, bool PAT>
void launch_g(const DCSR& A, int m, const V* val, const V* X, const V* B, V* Y, V* D, const V* dinv, V c1, V c2,
              cudaStream_t s) {
  bat_rows<G, V, MODE, PAT><<<grid_for(A.n * G, kThreads), kThreads, 0, s>>>(
      A.n, m, A.rp.get(), A.ci.get(), A.pat.obase.get(), A.pat.toff.get(), val, X, B, Y, D, dinv, c1, c2);
  note_launch();
}

template <typename V, int MODE>
void launch_bat(const DCSR& A, int m, const V* val, const V* X, const V* B, V* Y, V* D, const V* dinv, V c1, V c2,
                cudaStream_t s) {
  if (A.n == 0) return;
  const bool own = val == (sizeof(V) == 8 ? (const V*)A.v.get() : (const V*)A.v32.get());
  const bool pat = own && A.pat.on;
  if constexpr (sizeof(V) == 4) {
    const bool pairs = A.batch_rows == 2 || (A.batch_rows == 0 && m > 16);
    if (pat && A.grp.pon && pairs) {
      bat_pairs<MODE><<<grid_for(A.grp.n_items * 32, kThreads), kThreads, 0, s>>>(
          A.grp.n_items, A.grp.item_a.get(), A.grp.item_b.get(), A.grp.item_g.get(), A.grp.gptr.get(),
          A.grp.gcol.get(), A.rp.get(), m, val, X, B, Y, D, dinv, c1, c2);
      note_launch();
      GIAMG_CUDA(cudaGetLastError());
      return;
    }
  }
  const int G = m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : m <= 16 ? 16 : 32;
#define BAT_CASE(GG)                                                              \
  case GG:                                                                        \
    if (pat) launch_g<GG, V, MODE, true>(A, m, val, X, B, Y, D, dinv, c1, c2, s); \
    else launch_g<GG, V, MODE, false>(A, m, val, X, B, Y, D, dinv, c1, c2, s);    \
    break;
  switch (G) {
    BAT_CASE(1)
    BAT_CASE(2)
    BAT_CASE(4)
    BAT_CASE(8)
    BAT_CASE(16)
    BAT_CASE(32)
  }
#undef BAT_CASE
  GIAMG_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ element transfers, m columns
// The single-vector contractions with the column as the fastest index of every work array.
template <typename V>
__device__ __forceinline__ void bp_prolong_body(int64_t vb, int p, int q, int m, const int32_t* __restrict__ l2g,
                                                const uint8_t* __restrict__ own, const int32_t* __restrict__ l2g_c,
                                                const V* __restrict__ p1d, const V* __restrict__ ec,
                                                V* __restrict__ xf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int n1 = p + 1, m1 = q + 1;
  const int nlf = n1 * n1 * n1, nlc = m1 * m1 * m1;
  V* T = sm;                      // n1 * m1
  V* u = T + n1 * m1;             // nlc * m
  V* t1 = u + nlc * m;            // m1 * m1 * n1 * m
  V* t2 = t1 + m1 * m1 * n1 * m;  // m1 * n1 * n1 * m
  const int64_t e = vb;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n1 * m1; i += nt) T[i] = p1d[i];
  for (int i = tid; i < nlc * m; i += nt) {
    const int b = i / m, j = i % m;
    u[i] = ec[(int64_t)l2g_c[(int64_t)e * nlc + b] * m + j];
  }
  __syncthreads();
  for (int i = tid; i < m1 * m1 * n1 * m; i += nt) {
    const int j = i % m, w = i / m, a3 = w % n1, b12 = w / n1;
    V s = 0;
    for (int b3 = 0; b3 < m1; ++b3) s += T[a3 * m1 + b3] * u[(b12 * m1 + b3) * m + j];
    t1[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < m1 * n1 * n1 * m; i += nt) {
    const int j = i % m, w = i / m, a3 = w % n1, a2 = (w / n1) % n1, b1 = w / (n1 * n1);
    V s = 0;
    for (int b2 = 0; b2 < m1; ++b2) s += T[a2 * m1 + b2] * t1[((b1 * m1 + b2) * n1 + a3) * m + j];
    t2[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < nlf * m; i += nt) {
    const int j = i % m, a = i / m;
    const int64_t slot = (int64_t)e * nlf + a;
    if (!own[slot]) continue;
    const int a23 = a % (n1 * n1), a1 = a / (n1 * n1);
    V s = 0;
    for (int b1 = 0; b1 < m1; ++b1) s += T[a1 * m1 + b1] * t2[(b1 * n1 * n1 + a23) * m + j];
    xf[(int64_t)l2g[slot] * m + j] += s;
  }
}
template <typename V>
__global__ void bp_prolong_kernel(int32_t n_elem, int p, int q, int m, const int32_t* __restrict__ l2g,
                                  const uint8_t* __restrict__ own, const int32_t* __restrict__ l2g_c,
                                  const V* __restrict__ p1d, const V* __restrict__ ec, V* __restrict__ xf) {
  bp_prolong_body<V>(blockIdx.x, p, q, m, l2g, own, l2g_c, p1d, ec, xf);
}

template <typename V>
__device__ __forceinline__ void bp_restrict_body(int64_t vb, int p, int q, int m, const int32_t* __restrict__ l2g,
                                                 const uint8_t* __restrict__ own, const V* __restrict__ p1d,
                                                 const V* __restrict__ rf, V* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int n1 = p + 1, m1 = q + 1;
  const int nlf = n1 * n1 * n1, nlc = m1 * m1 * m1;
  V* T = sm;                      // n1 * m1
  V* v = T + n1 * m1;             // nlf * m
  V* t1 = v + nlf * m;            // n1 * n1 * m1 * m
  V* t2 = t1 + n1 * n1 * m1 * m;  // n1 * m1 * m1 * m
  const int64_t e = vb;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n1 * m1; i += nt) T[i] = p1d[i];
  for (int i = tid; i < nlf * m; i += nt) {
    const int a = i / m, j = i % m;
    const int64_t slot = (int64_t)e * nlf + a;
    v[i] = own[slot] ? rf[(int64_t)l2g[slot] * m + j] : V(0);
  }
  __syncthreads();
  for (int i = tid; i < n1 * n1 * m1 * m; i += nt) {
    const int j = i % m, w = i / m, b3 = w % m1, a12 = w / m1;
    V s = 0;
    for (int a3 = 0; a3 < n1; ++a3) s += T[a3 * m1 + b3] * v[(a12 * n1 + a3) * m + j];
    t1[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < n1 * m1 * m1 * m; i += nt) {
    const int j = i % m, w = i / m, b3 = w % m1, b2 = (w / m1) % m1, a1 = w / (m1 * m1);
    V s = 0;
    for (int a2 = 0; a2 < n1; ++a2) s += T[a2 * m1 + b2] * t1[((a1 * n1 + a2) * m1 + b3) * m + j];
    t2[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < nlc * m; i += nt) {
    const int j = i % m, b = i / m;
    const int b23 = b % (m1 * m1), b1 = b / (m1 * m1);
    V s = 0;
    for (int a1 = 0; a1 < n1; ++a1) s += T[a1 * m1 + b1] * t2[(a1 * m1 * m1 + b23) * m + j];
    part[((int64_t)e * nlc + b) * m + j] = s;
  }
}
template <typename V>
__global__ void bp_restrict_kernel(int32_t n_elem, int p, int q, int m, const int32_t* __restrict__ l2g,
                                   const uint8_t* __restrict__ own, const V* __restrict__ p1d,
                                   const V* __restrict__ rf, V* __restrict__ part) {
  bp_restrict_body<V>(blockIdx.x, p, q, m, l2g, own, p1d, rf, part);
}

template <typename V>
__device__ __forceinline__ void bp_gather_body(int64_t vb, int64_t nc, int m, const int64_t* __restrict__ ptr,
                                               const int32_t* __restrict__ slot, const V* __restrict__ part,
                                               V* __restrict__ rc) {
  const int64_t g = vb * blockDim.x + threadIdx.x;
  if (g >= nc * m) return;
  const int64_t c = g / m;
  const int j = (int)(g % m);
  V s = 0;
  for (int64_t t = ptr[c]; t < ptr[c + 1]; ++t) s += part[(int64_t)slot[t] * m + j];
  rc[g] = s;
}
template <typename V>
__global__ void bp_gather_kernel(int64_t nc, int m, const int64_t* __restrict__ ptr, const int32_t* __restrict__ slot,
                                 const V* __restrict__ part, V* __restrict__ rc) {
  bp_gather_body<V>(blockIdx.x, nc, m, ptr, slot, part, rc);
}

template <typename V>
size_t bprolong_smem(int p, int q, int m) {
  const int n1 = p + 1, m1 = q + 1;
  return sizeof(V) * ((size_t)n1 * m1 + (size_t)m * (m1 * m1 * m1 + m1 * m1 * n1 + m1 * n1 * n1));
}
template <typename V>
size_t brestrict_smem(int p, int q, int m) {
  const int n1 = p + 1, m1 = q + 1;
  return sizeof(V) * ((size_t)n1 * m1 + (size_t)m * (n1 * n1 * n1 + n1 * n1 * m1 + n1 * m1 * m1));
}

// ------------------------------------------------------------------ coarsest solve, vectors
template <typename V>
__device__ __forceinline__ void bat_inverse_body(int64_t vb, const double* __restrict__ Ainv, int64_t nc, int m,
                                                 const V* __restrict__ B, V* __restrict__ X) {
  const int64_t g = vb * blockDim.x + threadIdx.x;
  if (g >= nc * m) return;
  const int64_t row = g / m;
  const int j = (int)(g % m);
  double s = 0.0;
  for (int64_t k = 0; k < nc; ++k) s += Ainv[row * nc + k] * (double)B[k * m + j];
  X[g] = (V)s;
}
template <typename V>
__global__ void bat_inverse_apply(const double* __restrict__ Ainv, int64_t nc, int m, const V* __restrict__ B,
                                  V* __restrict__ X) {
  bat_inverse_body<V>(blockIdx.x, Ainv, nc, m, B, X);
}

template <typename V>
__device__ __forceinline__ void bat_cheb_first_body(int64_t vb, int64_t nvb, int64_t n, int m, const V* __restrict__ B,
                                                    const V* __restrict__ dinv, V c2, V* __restrict__ X,
                                                    V* __restrict__ D) {
  for (int64_t i = vb * blockDim.x + threadIdx.x; i < n * m; i += nvb * blockDim.x) {
    const V v = c2 * dinv[i / m] * B[i];
    D[i] = v;
    X[i] = v;
  }
}
template <typename V>
__global__ void bat_cheb_first(int64_t n, int m, const V* __restrict__ B, const V* __restrict__ dinv, V c2,
                               V* __restrict__ X, V* __restrict__ D) {
  bat_cheb_first_body<V>(blockIdx.x, gridDim.x, n, m, B, dinv, c2, X, D);
}

// Batched CG scalars, one entry per column.
struct BatchScalars {
  double rho[32], pq[32], alpha[32], beta[32], rr[32], bb[32];
  int status[32], active[32];
  double tol2;  // rtol^2, and whether the iteration count is forced: written before each solve
  int force;
  int pad;
};

__device__ __forceinline__ void bat_init_body(int64_t vb, int64_t nvb, int64_t n, int m, const double* __restrict__ B,
                                              double* __restrict__ X, double* __restrict__ R, double* partial) {
  __shared__ double sh[32 * 32];
  const int l = threadIdx.x & 31;
  double s = 0.0;
  const int64_t rows_per_block = (n + nvb - 1) / nvb;
  const int64_t r0 = vb * rows_per_block, r1 = min(n, r0 + rows_per_block);
  for (int64_t i = r0 + (threadIdx.x >> 5); i < r1; i += blockDim.x >> 5) {
    if (l < m) {
      const double b = B[i * m + l];
      X[i * m + l] = 0.0;
      R[i * m + l] = b;
      s += b * b;
    }
  }
  column_block_sum(s, m, sh, partial + vb * 32);
}
__global__ void __launch_bounds__(kRedThreads) bat_init(int64_t n, int m, const double* __restrict__ B,
                                                        double* __restrict__ X, double* __restrict__ R,
                                                        double* partial) {
  bat_init_body(blockIdx.x, gridDim.x, n, m, B, X, R, partial);
}

// <r_j, z_j> and, for flexible CG, <z_j, r_j - rold_j>
__device__ __forceinline__ void bat_dot_rz_body(int64_t vb, int64_t nvb, int64_t n, int m, const double* __restrict__ R,
                                                const double* __restrict__ Z, const double* __restrict__ Rold,
                                                int flexible, double* partial) {
  __shared__ double sh[32 * 32];
  const int l = threadIdx.x & 31;
  double s0 = 0.0, s1 = 0.0;
  const int64_t rows_per_block = (n + nvb - 1) / nvb;
  const int64_t r0 = vb * rows_per_block, r1 = min(n, r0 + rows_per_block);
  for (int64_t i = r0 + (threadIdx.x >> 5); i < r1; i += blockDim.x >> 5) {
    if (l < m) {
      const double z = Z[i * m + l], r = R[i * m + l];
      s0 += r * z;
      if (flexible) s1 += z * (r - Rold[i * m + l]);
    }
  }
  column_block_sum(s0, m, sh, partial + vb * 32);
  column_block_sum(s1, m, sh, partial + (nvb + vb) * 32);
}
__global__ void __launch_bounds__(kRedThreads) bat_dot_rz(int64_t n, int m, const double* __restrict__ R,
                                                          const double* __restrict__ Z,
                                                          const double* __restrict__ Rold, int flexible,
                                                          double* partial) {
  bat_dot_rz_body(blockIdx.x, gridDim.x, n, m, R, Z, Rold, flexible, partial);
}

__device__ __forceinline__ void bat_dot_body(int64_t vb, int64_t nvb, int64_t n, int m, const double* __restrict__ P,
                                             const double* __restrict__ Q, double* partial) {
  __shared__ double sh[32 * 32];
  const int l = threadIdx.x & 31;
  double s = 0.0;
  const int64_t rows_per_block = (n + nvb - 1) / nvb;
  const int64_t r0 = vb * rows_per_block, r1 = min(n, r0 + rows_per_block);
  for (int64_t i = r0 + (threadIdx.x >> 5); i < r1; i += blockDim.x >> 5)
    if (l < m) s += P[i * m + l] * Q[i * m + l];
  column_block_sum(s, m, sh, partial + vb * 32);
}
__global__ void __launch_bounds__(kRedThreads) bat_dot(int64_t n, int m, const double* __restrict__ P,
                                                       const double* __restrict__ Q, double* partial) {
  bat_dot_body(blockIdx.x, gridDim.x, n, m, P, Q, partial);
}

// Column sums of the block partials, by all kFinishThreads threads of the block: warp w sums the
// partials of blocks w, w + 32, ... in order, then lane j of warp 0 adds the 32 warp sums in warp
// order (a fixed order for a fixed grid: bitwise reproducible).  The result is valid in warp 0.
constexpr int kFinishThreads = 1024;
__device__ double column_total(const double* partial, int blocks, double (*sh)[33]) {
  const int j = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double s = 0.0;
  for (int b = w; b < blocks; b += nw) s += partial[(int64_t)b * 32 + j];
  sh[w][j] = s;
  __syncthreads();
  double t = 0.0;
  if (w == 0)
    for (int k = 0; k < nw; ++k) t += sh[k][j];
  __syncthreads();
  return t;
}

__device__ __forceinline__ void bat_finish_bb_body(BatchScalars* sc, const double* partial, int blocks,
                                                                 int m) {
  __shared__ double sh[32][33];
  const int j = threadIdx.x;
  const double v = column_total(partial, blocks, sh);
  if (j >= m) return;
  sc->bb[j] = v;
  sc->rr[j] = v;
  sc->status[j] = 0;
  sc->active[j] = v > 0.0 ? 1 : 0;
}
__global__ void __launch_bounds__(kFinishThreads) bat_finish_bb(BatchScalars* sc, const double* partial, int blocks, int m) { bat_finish_bb_body(sc, partial, blocks, m); }

__device__ __forceinline__ void bat_finish_rz_body(BatchScalars* sc, const double* partial, int blocks,
                                                                 int m, int first, int flexible) {
  __shared__ double sh[32][33];
  const int j = threadIdx.x;
  const double rz = column_total(partial, blocks, sh);
  const double zd = column_total(partial + (int64_t)blocks * 32, blocks, sh);
  if (j >= m) return;
  if (!sc->active[j]) {
    sc->beta[j] = 0.0;
    return;
  }
  if (!(rz > 0.0) && sc->status[j] == 0) sc->status[j] = GIAMG_ERR_BREAKDOWN;
  sc->beta[j] = first ? 0.0 : (flexible ? zd : rz) / sc->rho[j];
  sc->rho[j] = rz;
}
__global__ void __launch_bounds__(kFinishThreads) bat_finish_rz(BatchScalars* sc, const double* partial, int blocks, int m, int first, int flexible) { bat_finish_rz_body(sc, partial, blocks, m, first, flexible); }

__device__ __forceinline__ void bat_finish_pq_body(BatchScalars* sc, const double* partial, int blocks,
                                                                 int m) {
  __shared__ double sh[32][33];
  const int j = threadIdx.x;
  const double pq = column_total(partial, blocks, sh);
  if (j >= m) return;
  sc->pq[j] = pq;
  if (!sc->active[j]) {
    sc->alpha[j] = 0.0;
    return;
  }
  if (!(pq > 0.0) && sc->status[j] == 0) sc->status[j] = GIAMG_ERR_BREAKDOWN;
  sc->alpha[j] = sc->rho[j] / pq;
}
__global__ void __launch_bounds__(kFinishThreads) bat_finish_pq(BatchScalars* sc, const double* partial, int blocks, int m) { bat_finish_pq_body(sc, partial, blocks, m); }

// after the update: record ||r_j||^2 and retire columns that reached the tolerance
__device__ __forceinline__ void bat_finish_rr_body(BatchScalars* sc, const double* partial, int blocks,
                                                                 int m) {
  __shared__ double sh[32][33];
  const int j = threadIdx.x;
  const double rr = column_total(partial, blocks, sh);
  if (j >= m) return;
  if (!sc->active[j]) return;
  sc->rr[j] = rr;
  if (!(rr == rr) && sc->status[j] == 0) sc->status[j] = GIAMG_ERR_BREAKDOWN;
  if (sc->status[j] != 0 || (!sc->force && rr <= sc->tol2 * sc->bb[j])) sc->active[j] = 0;
}
__global__ void __launch_bounds__(kFinishThreads) bat_finish_rr(BatchScalars* sc, const double* partial, int blocks, int m) { bat_finish_rr_body(sc, partial, blocks, m); }

// The loop captured as a CUDA graph: per-column iteration counts (a column counts the iterations
// it entered active), and the loop condition (some column active, the limit not reached, no
// breakdown) set on the graph's conditional handles.
__global__ void bat_graph_start(const BatchScalars* __restrict__ sc, int m, BatchGraphState* __restrict__ st,
                                cudaGraphConditionalHandle first, cudaGraphConditionalHandle loop) {
  int any = 0;
  for (int j = 0; j < m; ++j) {
    st->its[j] = 0;
    st->was[j] = sc->active[j];
    any |= st->was[j];
  }
  st->it = 0;
  st->breakdown = 0;
  const unsigned go = (any && st->limit > 0) ? 1u : 0u;
  cudaGraphSetConditional(first, go);
  cudaGraphSetConditional(loop, go);
}
__global__ void bat_graph_check(const BatchScalars* __restrict__ sc, int m, BatchGraphState* __restrict__ st,
                                cudaGraphConditionalHandle loop, cudaGraphConditionalHandle more) {
  const int it = st->it + 1;
  st->it = it;
  int any = 0, bd = 0;
  for (int j = 0; j < m; ++j) {
    if (st->was[j]) st->its[j] = it;
    st->was[j] = sc->active[j];
    any |= st->was[j];
    bd |= sc->status[j] != 0;
  }
  st->breakdown = bd;
  const unsigned cont = (any && it < st->limit && !bd) ? 1u : 0u;
  cudaGraphSetConditional(loop, cont);
  cudaGraphSetConditional(more, cont);
}

__device__ __forceinline__ void bat_update_p_body(int64_t vb, int64_t nvb, int64_t n, int m, const double* __restrict__ Z,
                                                  double* __restrict__ P, const BatchScalars* __restrict__ sc,
                                                  int first) {
  for (int64_t i = vb * blockDim.x + threadIdx.x; i < n * m; i += nvb * blockDim.x) {
    const int j = (int)(i % m);
    if (!sc->active[j]) continue;
    P[i] = first ? Z[i] : Z[i] + sc->beta[j] * P[i];
  }
}
__global__ void bat_update_p(int64_t n, int m, const double* __restrict__ Z, double* __restrict__ P,
                             const BatchScalars* __restrict__ sc, int first) {
  bat_update_p_body(blockIdx.x, gridDim.x, n, m, Z, P, sc, first);
}

__device__ __forceinline__ void bat_update_xr_body(int64_t vb, int64_t nvb, int64_t n, int m, const double* __restrict__ P,
                                                   const double* __restrict__ Q, double* __restrict__ X,
                                                   double* __restrict__ R, double* __restrict__ Rold, int flexible,
                                                   const BatchScalars* __restrict__ sc, double* partial) {
  __shared__ double sh[32 * 32];
  const int l = threadIdx.x & 31;
  const bool act = l < m && sc->active[l];
  const double alpha = act ? sc->alpha[l] : 0.0;
  double s = 0.0;
  const int64_t rows_per_block = (n + nvb - 1) / nvb;
  const int64_t r0 = vb * rows_per_block, r1 = min(n, r0 + rows_per_block);
  for (int64_t i = r0 + (threadIdx.x >> 5); i < r1; i += blockDim.x >> 5) {
    if (act) {
      const int64_t o = i * m + l;
      const double ri = R[o];
      if (flexible) Rold[o] = ri;
      X[o] = X[o] + alpha * P[o];
      const double rn = ri - alpha * Q[o];
      R[o] = rn;
      s += rn * rn;
    }
  }
  column_block_sum(s, m, sh, partial + vb * 32);
}
__global__ void __launch_bounds__(kRedThreads) bat_update_xr(int64_t n, int m, const double* __restrict__ P,
                                                             const double* __restrict__ Q, double* __restrict__ X,
                                                             double* __restrict__ R, double* __restrict__ Rold,
                                                             int flexible, const BatchScalars* __restrict__ sc,
                                                             double* partial) {
  bat_update_xr_body(blockIdx.x, gridDim.x, n, m, P, Q, X, R, Rold, flexible, sc, partial);
}

template <typename T, typename U>
__device__ __forceinline__ void bat_convert_body(int64_t vb, int64_t nvb, int64_t count, const T* __restrict__ x,
                                                 U* __restrict__ y) {
  for (int64_t i = vb * blockDim.x + threadIdx.x; i < count; i += nvb * blockDim.x) y[i] = (U)x[i];
}
template <typename T, typename U>
__global__ void bat_convert(int64_t count, const T* __restrict__ x, U* __restrict__ y) {
  bat_convert_body<T, U>(blockIdx.x, gridDim.x, count, x, y);
}

constexpr int kBatBlocks = 1024;

// ------------------------------------------------------------------ grouped kernels
// Several hierarchies' work of one phase in one launch: block b belongs to hierarchy i with
// start[i] <= b < start[i + 1] and runs that hierarchy's body with block index b - start[i] in a
// grid of start[i + 1] - start[i] blocks -- the grid its standalone launch would have -- so every
// hierarchy computes exactly what it computes alone.  The descriptors travel as kernel arguments.
template <class Args>
struct GroupLaunch {
  int count;
  int start[kGroupMax + 1];
  Args a[kGroupMax];
};
__device__ __forceinline__ int group_of_block(const int* start, int count, int b) {
  int i = 0;
  while (i + 1 < count && b >= start[i + 1]) ++i;
  return i;
}

template <typename V, int MODE>
__global__ void __launch_bounds__(kThreads) grp_rows_kernel(const GroupLaunch<GrpRowsArgs> P) {
  const int i = group_of_block(P.start, P.count, blockIdx.x);
  const GrpRowsArgs& a = P.a[i];
  const int64_t vb = (int64_t)blockIdx.x - P.start[i];
  const V* val = (const V*)a.val;
  const V* X = (const V*)a.X;
  const V* B = (const V*)a.B;
  V* Y = (V*)a.Y;
  V* D = (V*)a.D;
  const V* dinv = (const V*)a.dinv;
  const V c1 = (V)a.c1, c2 = (V)a.c2;
  if constexpr (sizeof(V) == 4) {
    if (a.pairs) {
      bat_pairs_body<MODE>(vb, a.n_items, a.ia, a.ib, a.ig, a.gptr, a.gcol, a.rp, a.m, val, X, B, Y, D, dinv, c1, c2);
      return;
    }
  }
#define GRP_ROWS_CASE(GG)                                                                                        \
  case GG:                                                                                                       \
    if (a.pat) bat_rows_body<GG, V, MODE, true>(vb, a.n, a.m, a.rp, a.ci, a.obase, a.toff, val, X, B, Y, D, dinv, c1, c2); \
    else bat_rows_body<GG, V, MODE, false>(vb, a.n, a.m, a.rp, a.ci, a.obase, a.toff, val, X, B, Y, D, dinv, c1, c2); \
    break;
  switch (a.G) {
    GRP_ROWS_CASE(1)
    GRP_ROWS_CASE(2)
    GRP_ROWS_CASE(4)
    GRP_ROWS_CASE(8)
    GRP_ROWS_CASE(16)
    GRP_ROWS_CASE(32)
  }
#undef GRP_ROWS_CASE
}

template <typename V>
__global__ void grp_restrict_kernel(const GroupLaunch<GrpTransferArgs> P) {
  const int i = group_of_block(P.start, P.count, blockIdx.x);
  const GrpTransferArgs& a = P.a[i];
  bp_restrict_body<V>((int64_t)blockIdx.x - P.start[i], a.p, a.q, a.m, a.l2g, a.own, (const V*)a.p1d,
                      (const V*)a.in, (V*)a.part);
}
template <typename V>
__global__ void grp_gather_kernel(const GroupLaunch<GrpTransferArgs> P) {
  const int i = group_of_block(P.start, P.count, blockIdx.x);
  const GrpTransferArgs& a = P.a[i];
  bp_gather_body<V>((int64_t)blockIdx.x - P.start[i], a.n_next, a.m, a.cptr, a.cinc, (const V*)a.part, (V*)a.out);
}
template <typename V>
__global__ void grp_prolong_kernel(const GroupLaunch<GrpTransferArgs> P) {
  const int i = group_of_block(P.start, P.count, blockIdx.x);
  const GrpTransferArgs& a = P.a[i];
  bp_prolong_body<V>((int64_t)blockIdx.x - P.start[i], a.p, a.q, a.m, a.l2g, a.own, a.l2g_c, (const V*)a.p1d,
                     (const V*)a.in, (V*)a.out);
}

// vector phases: op selects the body; a, b, c, d, e the operands in the order of the standalone call
enum GrpVecOp { kGvInverse32 = 0, kGvChebFirst32, kGvTo32, kGvTo64, kGvInit, kGvDotRz, kGvDot, kGvUpdateXr, kGvUpdateP,
                kGvFinishBb, kGvFinishRz, kGvFinishPq, kGvFinishRr };
template <int OP>
__global__ void __launch_bounds__(kFinishThreads) grp_vec_kernel(const GroupLaunch<GrpVecArgs> P) {
  const int i = group_of_block(P.start, P.count, blockIdx.x);
  const GrpVecArgs& a = P.a[i];
  const int64_t vb = (int64_t)blockIdx.x - P.start[i], nvb = (int64_t)P.start[i + 1] - P.start[i];
  BatchScalars* sc = (BatchScalars*)a.sc;
  if (OP == kGvInverse32) bat_inverse_body<float>(vb, (const double*)a.a, a.n, a.m, (const float*)a.b, (float*)a.c);
  if (OP == kGvChebFirst32)
    bat_cheb_first_body<float>(vb, nvb, a.n, a.m, (const float*)a.a, (const float*)a.b, (float)a.v, (float*)a.c,
                               (float*)a.d);
  if (OP == kGvTo32) bat_convert_body<double, float>(vb, nvb, a.n, (const double*)a.a, (float*)a.c);
  if (OP == kGvTo64) bat_convert_body<float, double>(vb, nvb, a.n, (const float*)a.a, (double*)a.c);
  if (OP == kGvInit) bat_init_body(vb, nvb, a.n, a.m, (const double*)a.a, (double*)a.c, (double*)a.d, a.partial);
  if (OP == kGvDotRz)
    bat_dot_rz_body(vb, nvb, a.n, a.m, (const double*)a.a, (const double*)a.b, (const double*)a.e, a.flag1, a.partial);
  if (OP == kGvDot) bat_dot_body(vb, nvb, a.n, a.m, (const double*)a.a, (const double*)a.b, a.partial);
  if (OP == kGvUpdateXr)
    bat_update_xr_body(vb, nvb, a.n, a.m, (const double*)a.a, (const double*)a.b, (double*)a.c, (double*)a.d,
                       (double*)a.e, a.flag1, sc, a.partial);
  if (OP == kGvUpdateP) bat_update_p_body(vb, nvb, a.n, a.m, (const double*)a.a, (double*)a.c, sc, a.flag1);
  if (OP == kGvFinishBb) bat_finish_bb_body(sc, a.partial, kBatBlocks, a.m);
  if (OP == kGvFinishRz) bat_finish_rz_body(sc, a.partial, kBatBlocks, a.m, a.flag1, a.flag2);
  if (OP == kGvFinishPq) bat_finish_pq_body(sc, a.partial, kBatBlocks, a.m);
  if (OP == kGvFinishRr) bat_finish_rr_body(sc, a.partial, kBatBlocks, a.m);
}

}  // namespace

// ================================================================== launchers
void bat_rows_launch64(const DCSR& A, int m, int mode, const double* val, const double* X, const double* B, double* Y,
                       double* D, const double* dinv, double c1, double c2, cudaStream_t s) {
  switch (mode) {
    case kSpmm: launch_bat<double, kSpmm>(A, m, val, X, B, Y, D, dinv, c1, c2, s); break;
    case kResid: launch_bat<double, kResid>(A, m, val, X, B, Y, D, dinv, c1, c2, s); break;
    case kBatCheb: launch_bat<double, kBatCheb>(A, m, val, X, B, Y, D, dinv, c1, c2, s); break;
    default: launch_bat<double, kAdd>(A, m, val, X, B, Y, D, dinv, c1, c2, s); break;
  }
}
void bat_rows_launch32(const DCSR& A, int m, int mode, const float* val, const float* X, const float* B, float* Y,
                       float* D, const float* dinv, float c1, float c2, cudaStream_t s) {
  switch (mode) {
    case kSpmm: launch_bat<float, kSpmm>(A, m, val, X, B, Y, D, dinv, c1, c2, s); break;
    case kResid: launch_bat<float, kResid>(A, m, val, X, B, Y, D, dinv, c1, c2, s); break;
    case kBatCheb: launch_bat<float, kBatCheb>(A, m, val, X, B, Y, D, dinv, c1, c2, s); break;
    default: launch_bat<float, kAdd>(A, m, val, X, B, Y, D, dinv, c1, c2, s); break;
  }
}

template <typename V>
static void bp_restrict_t(const Level& L, int m, const V* rf, V* rc, const V* p1d, V* part, cudaStream_t s) {
  const size_t sm = brestrict_smem<V>(L.p, L.q, m);
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(bp_restrict_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)); });
  GIAMG_CHECK(sm <= 200 * 1024, GIAMG_ERR_ARG, "batched restriction: too many columns for the element order");
  { bp_restrict_kernel<V><<<(unsigned)L.n_elem, 256, sm, s>>>(L.n_elem, L.p, L.q, m, L.l2g.get(), L.own.get(), p1d, rf, part); note_launch(); }
  { bp_gather_kernel<V><<<grid_for(L.n_next * m, 256), 256, 0, s>>>(L.n_next, m, L.cinc_ptr.get(), L.cinc.get(), part, rc); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
template <typename V>
static void bp_prolong_t(const Level& L, int m, const V* ec, V* xf, const V* p1d, cudaStream_t s) {
  const size_t sm = bprolong_smem<V>(L.p, L.q, m);
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(bp_prolong_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)); });
  GIAMG_CHECK(sm <= 200 * 1024, GIAMG_ERR_ARG, "batched prolongation: too many columns for the element order");
  { bp_prolong_kernel<V><<<(unsigned)L.n_elem, 256, sm, s>>>(L.n_elem, L.p, L.q, m, L.l2g.get(), L.own.get(), L.l2g_c.get(), p1d, ec, xf); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_p_restrict(const Level& L, int m, const double* rf, double* rc, double* part, cudaStream_t s) {
  bp_restrict_t<double>(L, m, rf, rc, L.p1d.get(), part, s);
}
void bat_p_restrict32(const Level& L, int m, const float* rf, float* rc, float* part, cudaStream_t s) {
  bp_restrict_t<float>(L, m, rf, rc, L.p1d32.get(), part, s);
}
void bat_p_prolong(const Level& L, int m, const double* ec, double* xf, cudaStream_t s) {
  bp_prolong_t<double>(L, m, ec, xf, L.p1d.get(), s);
}
void bat_p_prolong32(const Level& L, int m, const float* ec, float* xf, cudaStream_t s) {
  bp_prolong_t<float>(L, m, ec, xf, L.p1d32.get(), s);
}
void bat_inverse(const double* Ainv, int64_t nc, int m, const double* B, double* X, cudaStream_t s) {
  { bat_inverse_apply<double><<<grid_for(nc * m, 256), 256, 0, s>>>(Ainv, nc, m, B, X); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_inverse32(const double* Ainv, int64_t nc, int m, const float* B, float* X, cudaStream_t s) {
  { bat_inverse_apply<float><<<grid_for(nc * m, 256), 256, 0, s>>>(Ainv, nc, m, B, X); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_cheb_first64(int64_t n, int m, const double* B, const double* dinv, double c2, double* X, double* D, cudaStream_t s) {
  { bat_cheb_first<double><<<vec_grid(n * m), 256, 0, s>>>(n, m, B, dinv, c2, X, D); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_cheb_first32(int64_t n, int m, const float* B, const float* dinv, float c2, float* X, float* D, cudaStream_t s) {
  { bat_cheb_first<float><<<vec_grid(n * m), 256, 0, s>>>(n, m, B, dinv, c2, X, D); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_to32(int64_t count, const double* x, float* y, cudaStream_t s) {
  { bat_convert<double, float><<<vec_grid(count), 256, 0, s>>>(count, x, y); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_to64(int64_t count, const float* x, double* y, cudaStream_t s) {
  { bat_convert<float, double><<<vec_grid(count), 256, 0, s>>>(count, x, y); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

size_t batch_scalars_bytes() { return sizeof(BatchScalars); }
int batch_reduction_blocks() { return kBatBlocks; }

void bat_pcg_init(int64_t n, int m, const double* B, double* X, double* R, double* partial, void* sc, cudaStream_t s) {
  { bat_init<<<kBatBlocks, kRedThreads, 0, s>>>(n, m, B, X, R, partial); note_launch(); }
  { bat_finish_bb<<<1, kFinishThreads, 0, s>>>((BatchScalars*)sc, partial, kBatBlocks, m); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_pcg_rz(int64_t n, int m, const double* R, const double* Z, const double* Rold, int flexible, int first,
                double* partial, void* sc, cudaStream_t s) {
  { bat_dot_rz<<<kBatBlocks, kRedThreads, 0, s>>>(n, m, R, Z, Rold, flexible, partial); note_launch(); }
  { bat_finish_rz<<<1, kFinishThreads, 0, s>>>((BatchScalars*)sc, partial, kBatBlocks, m, first, flexible); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_pcg_update_p(int64_t n, int m, const double* Z, double* P, const void* sc, int first, cudaStream_t s) {
  { bat_update_p<<<vec_grid(n * m), 256, 0, s>>>(n, m, Z, P, (const BatchScalars*)sc, first); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_pcg_pq(int64_t n, int m, const double* P, const double* Q, double* partial, void* sc, cudaStream_t s) {
  { bat_dot<<<kBatBlocks, kRedThreads, 0, s>>>(n, m, P, Q, partial); note_launch(); }
  { bat_finish_pq<<<1, kFinishThreads, 0, s>>>((BatchScalars*)sc, partial, kBatBlocks, m); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_pcg_update_xr(int64_t n, int m, const double* P, const double* Q, double* X, double* R, double* Rold,
                       int flexible, double* partial, void* sc, cudaStream_t s) {
  { bat_update_xr<<<kBatBlocks, kRedThreads, 0, s>>>(n, m, P, Q, X, R, Rold, flexible, (const BatchScalars*)sc, partial); note_launch(); }
  { bat_finish_rr<<<1, kFinishThreads, 0, s>>>((BatchScalars*)sc, partial, kBatBlocks, m); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
// ------------------------------------------------------------------ grouped launches
namespace {
template <class Args, class Kernel>
void launch_grouped(const std::vector<Args>& ops, const std::vector<int64_t>& blocks, Kernel k, int threads,
                    size_t smem, cudaStream_t s) {
  for (size_t c0 = 0; c0 < ops.size(); c0 += kGroupMax) {
    const size_t c1 = std::min(ops.size(), c0 + kGroupMax);
    GroupLaunch<Args> P{};
    P.count = (int)(c1 - c0);
    int64_t tot = 0;
    for (size_t i = c0; i < c1; ++i) {
      P.start[i - c0] = (int)tot;
      P.a[i - c0] = ops[i];
      tot += blocks[i];
    }
    P.start[c1 - c0] = (int)tot;
    GIAMG_CHECK(tot < INT32_MAX, GIAMG_ERR_ARG, "grouped launch: too many blocks");
    if (tot > 0) {
      k<<<(unsigned)tot, threads, smem, s>>>(P);
      note_launch();
    }
  }
  GIAMG_CUDA(cudaGetLastError());
}
}  // namespace

GrpRowsArgs grp_rows_args(const DCSR& A, int m, const void* val, const void* X, const void* B, void* Y, void* D,
                          const void* dinv, double c1, double c2, bool fp32) {
  GrpRowsArgs a{};
  const bool own = fp32 ? val == (const void*)A.v32.get() : val == (const void*)A.v.get();
  a.n = A.n;
  a.m = m;
  a.pat = own && A.pat.on;
  a.pairs = fp32 && a.pat && A.grp.pon && (A.batch_rows == 2 || (A.batch_rows == 0 && m > 16));
  a.G = m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : m <= 16 ? 16 : 32;
  a.rp = A.rp.get();
  a.ci = A.ci.get();
  a.obase = A.pat.obase.get();
  a.toff = A.pat.toff.get();
  a.n_items = A.grp.n_items;
  a.ia = A.grp.item_a.get();
  a.ib = A.grp.item_b.get();
  a.ig = A.grp.item_g.get();
  a.gptr = A.grp.gptr.get();
  a.gcol = A.grp.gcol.get();
  a.val = val;
  a.X = X;
  a.B = B;
  a.Y = Y;
  a.D = D;
  a.dinv = dinv;
  a.c1 = c1;
  a.c2 = c2;
  return a;
}

template <typename V>
static void grp_rows_t(int mode, const std::vector<GrpRowsArgs>& ops, cudaStream_t s) {
  std::vector<GrpRowsArgs> act;
  std::vector<int64_t> blocks;
  for (const GrpRowsArgs& a : ops) {
    if (a.n == 0) continue;
    act.push_back(a);
    blocks.push_back(a.pairs ? grid_for(a.n_items * 32, kThreads) : grid_for(a.n * a.G, kThreads));
  }
  switch (mode) {
    case kSpmm: launch_grouped(act, blocks, grp_rows_kernel<V, kSpmm>, kThreads, 0, s); break;
    case kResid: launch_grouped(act, blocks, grp_rows_kernel<V, kResid>, kThreads, 0, s); break;
    case kBatCheb: launch_grouped(act, blocks, grp_rows_kernel<V, kBatCheb>, kThreads, 0, s); break;
    default: launch_grouped(act, blocks, grp_rows_kernel<V, kAdd>, kThreads, 0, s); break;
  }
}
void grp_rows64(int mode, const std::vector<GrpRowsArgs>& ops, cudaStream_t s) { grp_rows_t<double>(mode, ops, s); }
void grp_rows32(int mode, const std::vector<GrpRowsArgs>& ops, cudaStream_t s) { grp_rows_t<float>(mode, ops, s); }

GrpTransferArgs grp_transfer_args(const Level& L, int m, const float* in, float* out, float* part) {
  GrpTransferArgs a{};
  a.p = L.p;
  a.q = L.q;
  a.m = m;
  a.n_elem = L.n_elem;
  a.n_next = L.n_next;
  a.l2g = L.l2g.get();
  a.own = L.own.get();
  a.l2g_c = L.l2g_c.get();
  a.p1d = L.p1d32.get();
  a.cptr = L.cinc_ptr.get();
  a.cinc = L.cinc.get();
  a.in = in;
  a.out = out;
  a.part = part;
  return a;
}
void grp_p_restrict32(const std::vector<GrpTransferArgs>& ops, cudaStream_t s) {
  std::vector<int64_t> eb, gb;
  size_t sm = 0;
  for (const GrpTransferArgs& a : ops) {
    eb.push_back(a.n_elem);
    gb.push_back(grid_for(a.n_next * a.m, 256));
    sm = std::max(sm, brestrict_smem<float>(a.p, a.q, a.m));
  }
  GIAMG_CHECK(sm <= 200 * 1024, GIAMG_ERR_ARG, "grouped restriction: too many columns for the element order");
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(grp_restrict_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)); });
  launch_grouped(ops, eb, grp_restrict_kernel<float>, 256, sm, s);
  launch_grouped(ops, gb, grp_gather_kernel<float>, 256, 0, s);
}
void grp_p_prolong32(const std::vector<GrpTransferArgs>& ops, cudaStream_t s) {
  std::vector<int64_t> eb;
  size_t sm = 0;
  for (const GrpTransferArgs& a : ops) {
    eb.push_back(a.n_elem);
    sm = std::max(sm, bprolong_smem<float>(a.p, a.q, a.m));
  }
  GIAMG_CHECK(sm <= 200 * 1024, GIAMG_ERR_ARG, "grouped prolongation: too many columns for the element order");
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(grp_prolong_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)); });
  launch_grouped(ops, eb, grp_prolong_kernel<float>, 256, sm, s);
}

void grp_vec(int op, const std::vector<GrpVecArgs>& ops, cudaStream_t s) {
  std::vector<int64_t> blocks;
  int threads = 256;
  for (const GrpVecArgs& a : ops) {
    switch (op) {
      case kGvInverse32: blocks.push_back(grid_for(a.n * a.m, 256)); break;
      case kGvChebFirst32: case kGvUpdateP: blocks.push_back(vec_grid(a.n * a.m)); break;
      case kGvTo32: case kGvTo64: blocks.push_back(vec_grid(a.n)); break;
      case kGvInit: case kGvDotRz: case kGvDot: case kGvUpdateXr: blocks.push_back(kBatBlocks); break;
      default: blocks.push_back(1); threads = kFinishThreads; break;
    }
  }
  if (op == kGvInit || op == kGvDotRz || op == kGvDot || op == kGvUpdateXr) threads = kRedThreads;
  switch (op) {
#define GV(OP) case OP: launch_grouped(ops, blocks, grp_vec_kernel<OP>, threads, 0, s); break;
    GV(kGvInverse32) GV(kGvChebFirst32) GV(kGvTo32) GV(kGvTo64) GV(kGvInit) GV(kGvDotRz) GV(kGvDot) GV(kGvUpdateXr)
    GV(kGvUpdateP) GV(kGvFinishBb) GV(kGvFinishRz) GV(kGvFinishPq) GV(kGvFinishRr)
#undef GV
    default: GIAMG_CHECK(false, GIAMG_ERR_ARG, "grouped vector phase out of range");
  }
}

void bat_graph_start_launch(const void* sc, int m, BatchGraphState* st, cudaGraphConditionalHandle first,
                            cudaGraphConditionalHandle loop, cudaStream_t s) {
  { bat_graph_start<<<1, 1, 0, s>>>((const BatchScalars*)sc, m, st, first, loop); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void bat_graph_check_launch(const void* sc, int m, BatchGraphState* st, cudaGraphConditionalHandle loop,
                            cudaGraphConditionalHandle more, cudaStream_t s) {
  { bat_graph_check<<<1, 1, 0, s>>>((const BatchScalars*)sc, m, st, loop, more); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

}  // namespace giamg
