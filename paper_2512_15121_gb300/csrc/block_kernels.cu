// block_kernels.cu -- block CG (O'Leary 1980) on m <= 32 right-hand sides sharing one Krylov
// space.  Blocks are row-major n x m (the m values of a row contiguous), as in the independent
// multi-right-hand-side solve, whose SpMM, V-cycle, initialisation and loop control it shares.
//
// One iteration, with A-conjugate directions:
//   Q = A P;  G = P^T Q, C = P^T R            (blk_gram, two products from one pass over P)
//   alpha = G^+ C                            (blk_coef mode 0: scaled Cholesky with dropping)
//   X += P alpha;  R -= Q alpha;  ||r_j||^2  (blk_update_xr)
//   Z = M R;  E = Q^T Z;  beta = -G^+ E      (blk_gram, blk_coef mode 1)
//   P = Z + P beta                           (blk_update_p)
// G^+: S = diag(G)^-1/2, Cholesky of S G S (lower triangle) in index order; a direction whose
// pivot is <= kBlockDropTol, or whose diagonal is not positive, is dropped (zero rows of alpha
// and beta), so equal, dependent or zero columns leave the search space unchanged.
//
// X, R, Q and the solution of the m x m systems are FP64.  With the FP64 V-cycle the Gram
// products and P beta are FP64 too; the row kernels are then bound by the FP64 pipe (m FMAs per
// value), not by HBM: per row, 2 m^2 FMAs for the two Gram products, 2 m^2 for X and R, m^2
// for P.  With the FP32 V-cycle the Gram products and P beta take FP32 arithmetic (FP64
// accumulation across 32-row chunks), as the V-cycle itself does: they only steer the search
// directions and step lengths, while X, R and Q = A P stay FP64 and consistent with each other;
// the drop threshold is then kBlockDropTol32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.cuh"

namespace giamg {

namespace {

constexpr int kGramThreads = 256;
constexpr int kGramBlocks = 2 * 152;  // fixed: the partial sums are reduced in block order
constexpr int kGramRows = 32;         // rows staged in shared memory per pass
constexpr int kRowBlocks = 1024;      // fixed grid of the row-update kernels (per-column partials)

// Partial Gram products Lf^T R1 (and Lf^T R2) over the block's contiguous slab of rows.  Thread
// (ty, tx) of the 16 x 16 grid owns entries (2ty + i, 2tx + j), i, j in {0, 1}; entries with an
// index >= m read the zero padding of the staging tiles and are never used.  T = float: the
// operands are rounded to FP32 when staged and each 32-row chunk is summed in FP32 with FMAs,
// then added to FP64 accumulators (one FP64 add per 32 products).
template <int NR, typename T>
__global__ void __launch_bounds__(kGramThreads) gram_kernel(int64_t n, int m, const double* __restrict__ Lf,
                                                            const double* __restrict__ R1,
                                                            const double* __restrict__ R2,
                                                            double* __restrict__ partial) {
  using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  __shared__ __align__(16) T sL[kGramRows * 32];
  __shared__ __align__(16) T sR[NR][kGramRows * 32];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  for (int e = t; e < kGramRows * 32; e += kGramThreads) {
    sL[e] = T(0);
#pragma unroll
    for (int o = 0; o < NR; ++o) sR[o][e] = T(0);
  }
  double acc[NR][2][2];
#pragma unroll
  for (int o = 0; o < NR; ++o) acc[o][0][0] = acc[o][0][1] = acc[o][1][0] = acc[o][1][1] = 0.0;
  const int64_t rows_per_block = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block, r1 = min(n, r0 + rows_per_block);
  __syncthreads();
  for (int64_t c0 = r0; c0 < r1; c0 += kGramRows) {
    const int cnt = (int)min((int64_t)kGramRows, r1 - c0);
    const int tot = cnt * m;  // the chunk is contiguous: rows c0 .. c0 + cnt - 1, m values each
    const double* gl = Lf + c0 * m;
    const double* g1 = R1 + c0 * m;
    const double* g2 = NR > 1 ? R2 + c0 * m : nullptr;
    for (int e = t; e < tot; e += kGramThreads) {
      const int r = e / m, c = e - r * m;
      sL[r * 32 + c] = (T)gl[e];
      sR[0][r * 32 + c] = (T)g1[e];
      if (NR > 1) sR[NR - 1][r * 32 + c] = (T)g2[e];
    }
    __syncthreads();
    T ch[NR][2][2];
#pragma unroll
    for (int o = 0; o < NR; ++o) ch[o][0][0] = ch[o][0][1] = ch[o][1][0] = ch[o][1][1] = T(0);
    for (int r = 0; r < cnt; ++r) {
      const T2 a = *reinterpret_cast<const T2*>(&sL[r * 32 + 2 * ty]);
#pragma unroll
      for (int o = 0; o < NR; ++o) {
        const T2 b = *reinterpret_cast<const T2*>(&sR[o][r * 32 + 2 * tx]);
        ch[o][0][0] = fma(a.x, b.x, ch[o][0][0]);
        ch[o][0][1] = fma(a.x, b.y, ch[o][0][1]);
        ch[o][1][0] = fma(a.y, b.x, ch[o][1][0]);
        ch[o][1][1] = fma(a.y, b.y, ch[o][1][1]);
      }
    }
#pragma unroll
    for (int o = 0; o < NR; ++o)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[o][i][j] += (double)ch[o][i][j];
    __syncthreads();
  }
  double* out = partial + (int64_t)blockIdx.x * NR * 1024;
#pragma unroll
  for (int o = 0; o < NR; ++o)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) out[o * 1024 + (2 * ty + i) * 32 + 2 * tx + j] = acc[o][i][j];
}

// out[e] = sum over blocks of partial[b][e], blocks in order: each of the 8 warps sums a
// contiguous range of blocks for 32 entries, then the warp sums are added in warp order.
__global__ void __launch_bounds__(256) gram_finish(const double* __restrict__ partial, int blocks, int entries,
                                                   double* __restrict__ out) {
  __shared__ double sh[8][32];
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + l;
  const int per = (blocks + 7) / 8;
  const int b0 = w * per, b1 = min(blocks, b0 + per);
  double s = 0.0;
  for (int b = b0; b < b1; ++b) s += partial[(int64_t)b * entries + e];
  sh[w][l] = s;
  __syncthreads();
  if (w == 0) {
    double tsum = 0.0;
    for (int k = 0; k < 8; ++k) tsum += sh[k][l];
    out[e] = tsum;
  }
}

// The m x m part of an iteration, one block of 32 x 32 threads.  Mode 0: factor G = gram[0]
// (scaled, dropping dependent directions) and alpha = G^+ gram[1].  Mode 1: beta = -G^+ gram[0]
// with the stored factor.
__global__ void __launch_bounds__(1024) coef_kernel(int m, int mode, BlockState* __restrict__ st, double tau) {
  __shared__ double g[32][33];
  __shared__ double y[32][33];
  __shared__ double s[32];
  __shared__ int keep[32];
  const int i = threadIdx.x >> 5, j = threadIdx.x & 31;
  if (mode == 0) {
    if (threadIdx.x < 32) {
      const int a = threadIdx.x;
      const double d = a < m ? st->gram[0][a * 32 + a] : 0.0;
      const bool k = a < m && d > 0.0 && d < INFINITY;
      keep[a] = k ? 1 : 0;
      s[a] = k ? 1.0 / sqrt(d) : 0.0;
    }
    __syncthreads();
    g[i][j] = (i < m && j <= i) ? s[i] * st->gram[0][i * 32 + j] * s[j] : 0.0;
    __syncthreads();
    // right-looking Cholesky of the lower triangle, one column at a time
    for (int k = 0; k < m; ++k) {
      if (threadIdx.x == 0 && keep[k]) {
        const double piv = g[k][k];
        if (piv > tau) {
          g[k][k] = sqrt(piv);
        } else {
          keep[k] = 0;
          s[k] = 0.0;
        }
      }
      __syncthreads();
      if (keep[k]) {
        if (j == k && i > k && i < m) g[i][k] = g[i][k] / g[k][k];
        __syncthreads();
        if (i > k && i < m && j > k && j <= i) g[i][j] = g[i][j] - g[i][k] * g[j][k];
      } else if (j == k) {
        g[i][k] = 0.0;
      }
      __syncthreads();
    }
    st->L[i * 32 + j] = (keep[i] && j <= i) ? g[i][j] : 0.0;
    if (threadIdx.x < 32) {
      st->s[threadIdx.x] = s[threadIdx.x];
      st->keep[threadIdx.x] = keep[threadIdx.x];
    }
    if (threadIdx.x == 0) {
      int r = 0;
      for (int a = 0; a < m; ++a) r += keep[a];
      st->rank = r;
    }
  } else {
    g[i][j] = st->L[i * 32 + j];
    if (threadIdx.x < 32) {
      s[threadIdx.x] = st->s[threadIdx.x];
      keep[threadIdx.x] = st->keep[threadIdx.x];
    }
  }
  __syncthreads();
  // right-hand sides: column c of gram[1] (alpha) or gram[0] (beta), scaled by S
  const double* Y = st->gram[mode == 0 ? 1 : 0];
  y[i][j] = (i < m && j < m) ? s[i] * Y[i * 32 + j] : 0.0;
  __syncthreads();
  if (threadIdx.x < m) {
    const int c = threadIdx.x;
    for (int r = 0; r < m; ++r) {  // L z = S y
      if (!keep[r]) {
        y[r][c] = 0.0;
        continue;
      }
      double v = y[r][c];
      for (int k = 0; k < r; ++k)
        if (keep[k]) v -= g[r][k] * y[k][c];
      y[r][c] = v / g[r][r];
    }
    for (int r = m - 1; r >= 0; --r) {  // L^T w = z
      if (!keep[r]) continue;
      double v = y[r][c];
      for (int k = r + 1; k < m; ++k)
        if (keep[k]) v -= g[k][r] * y[k][c];
      y[r][c] = v / g[r][r];
    }
  }
  __syncthreads();
  double* out = mode == 0 ? st->alpha : st->beta;
  const double v = (i < m && j < m) ? s[i] * y[i][j] : 0.0;
  out[i * 32 + j] = mode == 0 ? v : -v;
}

// X += P alpha, R -= Q alpha: one warp per row, lane c owns column c and holds column c of
// alpha; the row's P and Q values are broadcast by shuffles.  Per-column ||r||^2 partials.
__global__ void __launch_bounds__(kRedThreads) update_xr_kernel(int64_t n, int m, const double* __restrict__ P,
                                                                const double* __restrict__ Q, double* __restrict__ X,
                                                                double* __restrict__ R,
                                                                const BlockState* __restrict__ st,
                                                                double* __restrict__ partial) {
  __shared__ double sh[32 * 32];
  const int l = threadIdx.x & 31;
  const bool lane = l < m;
  double al[32];
#pragma unroll
  for (int a = 0; a < 32; ++a) al[a] = (lane && a < m) ? st->alpha[a * 32 + l] : 0.0;
  double sum = 0.0;
  const int64_t rows_per_block = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block, r1 = min(n, r0 + rows_per_block);
  for (int64_t i = r0 + (threadIdx.x >> 5); i < r1; i += blockDim.x >> 5) {
    const int64_t o = i * m + l;
    const double p = lane ? P[o] : 0.0, q = lane ? Q[o] : 0.0;
    double dx = 0.0, dr = 0.0;
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      if (a < m) {
        const double pa = __shfl_sync(0xffffffffu, p, a), qa = __shfl_sync(0xffffffffu, q, a);
        dx = fma(pa, al[a], dx);
        dr = fma(qa, al[a], dr);
      }
    }
    if (lane) {
      X[o] = X[o] + dx;
      const double rn = R[o] - dr;
      R[o] = rn;
      sum += rn * rn;
    }
  }
  column_block_sum(sum, m, sh, partial + (int64_t)blockIdx.x * 32);
}

// ||r_j||^2 in block order; a column stays active until it meets the tolerance (or, with a
// forced count, while it is non-zero); NaN, or no direction left while a column is active, is a
// breakdown.
__global__ void __launch_bounds__(1024) finish_rr_kernel(BatchScalarsHost* sc, const BlockState* st,
                                                         const double* partial, int blocks, int m) {
  // warp w sums blocks w, w + 32, ... in order; lane j of warp 0 adds the warp sums in order
  __shared__ double sh[32][33];
  const int j = threadIdx.x & 31, w = threadIdx.x >> 5;
  double part = 0.0;
  for (int b = w; b < blocks; b += 32) part += partial[(int64_t)b * 32 + j];
  sh[w][j] = part;
  __syncthreads();
  if (w != 0 || j >= m) return;
  double rr = 0.0;
  for (int k = 0; k < 32; ++k) rr += sh[k][j];
  sc->rr[j] = rr;
  const bool open = sc->bb[j] > 0.0 && (sc->force || !(rr <= sc->tol2 * sc->bb[j]));
  sc->active[j] = open ? 1 : 0;
  if (sc->status[j] == 0 && (!(rr == rr) || (open && st->rank == 0))) sc->status[j] = GIAMG_ERR_BREAKDOWN;
}

// P = Z + P beta (first: P = Z), one warp per row as in update_xr_kernel.  T = float: the sum
// P beta is taken in FP32 from rounded operands and added to Z in FP64.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) update_p_kernel(int64_t n, int m, const double* __restrict__ Z,
                                                               double* __restrict__ P,
                                                               const BlockState* __restrict__ st, int first) {
  const int l = threadIdx.x & 31;
  const bool lane = l < m;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (first) {
    for (int64_t i = w0; i < n; i += warps)
      if (lane) P[i * m + l] = Z[i * m + l];
    return;
  }
  T be[32];
#pragma unroll
  for (int a = 0; a < 32; ++a) be[a] = (lane && a < m) ? (T)st->beta[a * 32 + l] : T(0);
  for (int64_t i = w0; i < n; i += warps) {
    const int64_t o = i * m + l;
    const T p = lane ? (T)P[o] : T(0);
    T d = T(0);
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      if (a < m) d = fma(__shfl_sync(0xffffffffu, p, a), be[a], d);
    }
    if (lane) P[o] = Z[o] + (double)d;
  }
}

}  // namespace

int block_gram_blocks() { return kGramBlocks; }

void blk_gram(int64_t n, int m, const double* Lf, const double* R1, const double* R2, int fp32, double* partial,
              BlockState* st, cudaStream_t s) {
  const int nr = R2 ? 2 : 1;
  if (nr == 2 && fp32) {
    gram_kernel<2, float><<<kGramBlocks, kGramThreads, 0, s>>>(n, m, Lf, R1, R2, partial);
  } else if (nr == 2) {
    gram_kernel<2, double><<<kGramBlocks, kGramThreads, 0, s>>>(n, m, Lf, R1, R2, partial);
  } else if (fp32) {
    gram_kernel<1, float><<<kGramBlocks, kGramThreads, 0, s>>>(n, m, Lf, R1, nullptr, partial);
  } else {
    gram_kernel<1, double><<<kGramBlocks, kGramThreads, 0, s>>>(n, m, Lf, R1, nullptr, partial);
  }
  note_launch();
  { gram_finish<<<nr * 1024 / 32, 256, 0, s>>>(partial, kGramBlocks, nr * 1024, &st->gram[0][0]); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void blk_coef(int m, int mode, double tau, BlockState* st, cudaStream_t s) {
  { coef_kernel<<<1, 1024, 0, s>>>(m, mode, st, tau); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void blk_update_xr(int64_t n, int m, const double* P, const double* Q, double* X, double* R, const BlockState* st,
                   double* partial, void* sc, cudaStream_t s) {
  { update_xr_kernel<<<kRowBlocks, kRedThreads, 0, s>>>(n, m, P, Q, X, R, st, partial); note_launch(); }
  { finish_rr_kernel<<<1, 1024, 0, s>>>((BatchScalarsHost*)sc, st, partial, kRowBlocks, m); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void blk_update_p(int64_t n, int m, const double* Z, double* P, const BlockState* st, int first, int fp32,
                  cudaStream_t s) {
  if (fp32) {
    update_p_kernel<float><<<kRowBlocks, kRedThreads, 0, s>>>(n, m, Z, P, st, first);
  } else {
    update_p_kernel<double><<<kRowBlocks, kRedThreads, 0, s>>>(n, m, Z, P, st, first);
  }
  note_launch();
  GIAMG_CUDA(cudaGetLastError());
}

}  // namespace giamg
