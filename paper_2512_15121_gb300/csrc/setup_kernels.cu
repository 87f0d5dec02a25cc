// setup_kernels.cu -- hierarchy construction on the GPU (Sec. 2, Algorithms 2-4 and 7,
// Sec. 2.5): p-level dof selection and element maps by mark + prefix sum, the assembled
// prolongation, Galerkin products R A P by a two-phase SpGEMM, MIS-2 aggregation with the
// smoothed prolongation P = T - M A T, and the Chebyshev bound by Lanczos.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace giamg {

namespace {

inline unsigned blocks_for(int64_t work, int per_block, int64_t cap = (int64_t)1 << 30) {
  int64_t g = (work + per_block - 1) / per_block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ================================================================== scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total) {
  // sh: 32 entries
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sh[lane] = s;
  }
  __syncthreads();
  const int64_t warp_off = w > 0 ? sh[w - 1] : 0;
  if (total) *total = sh[nw - 1];
  const int64_t r = warp_off + x - v;
  __syncthreads();
  return r;
}

template <typename T>
__global__ void scan_tile_sums(const T* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += (int64_t)in[base + k];
  int64_t tot;
  block_exclusive_scan(s, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void scan_tile_apply(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                                int64_t* __restrict__ out) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  int64_t tot;
  int64_t pre = block_exclusive_scan(s, sh, &tot) + offs[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = pre;
    pre += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = pre;
}

// exclusive scan with out[n] = total
template <typename T>
void scan_impl(const T* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n == 0) {
    GIAMG_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return;
  }
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  DBuf<int64_t> sums, offs;
  sums.alloc(nt, s);
  offs.alloc(nt + 1, s);
  if (nt == 1) {
    GIAMG_CUDA(cudaMemsetAsync(offs.get(), 0, sizeof(int64_t), s));
  } else {
    { scan_tile_sums<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, sums.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
    scan_impl<int64_t>(sums.get(), offs.get(), nt, s);
  }
  { scan_tile_apply<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, offs.get(), out); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

// ================================================================== radix sort (stable, LSD, 4-bit digits)
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;

__global__ void radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int64_t n_tiles,
                           int64_t* __restrict__ hist) {
  __shared__ int cnt[16];
  if (threadIdx.x < 16) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)threadIdx.x * kRadixItems;
  for (int k = 0; k < kRadixItems; ++k)
    if (base + k < n) atomicAdd(&cnt[(keys[base + k] >> shift) & 15], 1);
  __syncthreads();
  if (threadIdx.x < 16) hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void radix_scatter(const uint32_t* __restrict__ kin, const int64_t* __restrict__ iin, int64_t n, int shift,
                              int64_t n_tiles, const int64_t* __restrict__ offs, uint32_t* __restrict__ kout,
                              int64_t* __restrict__ iout) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)threadIdx.x * kRadixItems;
  uint32_t k[kRadixItems];
  int dg[kRadixItems];
  int c[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) c[d] = 0;
#pragma unroll
  for (int t = 0; t < kRadixItems; ++t) {
    const bool ok = base + t < n;
    k[t] = ok ? kin[base + t] : 0u;
    dg[t] = ok ? (int)((k[t] >> shift) & 15) : -1;
#pragma unroll
    for (int d = 0; d < 16; ++d) c[d] += (dg[t] == d);
  }
  int64_t pos[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) {
    const int64_t pre = block_exclusive_scan(c[d], sh, nullptr);
    pos[d] = offs[(int64_t)d * n_tiles + blockIdx.x] + pre;
  }
#pragma unroll
  for (int t = 0; t < kRadixItems; ++t) {
    if (dg[t] < 0) continue;
    int64_t p = 0;
#pragma unroll
    for (int d = 0; d < 16; ++d)
      if (dg[t] == d) p = pos[d]++;
    kout[p] = k[t];
    iout[p] = iin[base + t];
  }
}

__global__ void iota64(int64_t* x, int64_t n) { GRID_STRIDE(i, n) x[i] = i; }

// ================================================================== transpose
__global__ void expand_rows(const int64_t* __restrict__ rp, int64_t n, int32_t* __restrict__ row_of) {
  GRID_STRIDE(i, n) {
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) row_of[t] = (int32_t)i;
  }
}
__global__ void count_cols(const int32_t* __restrict__ ci, int64_t nnz, int32_t* __restrict__ cnt) {
  GRID_STRIDE(t, nnz) atomicAdd(&cnt[ci[t]], 1);
}
__global__ void gather_transpose(const int64_t* __restrict__ idx, int64_t nnz, const int32_t* __restrict__ row_of,
                                 const double* __restrict__ v, int32_t* __restrict__ tci, double* __restrict__ tv) {
  GRID_STRIDE(t, nnz) {
    const int64_t s = idx[t];
    tci[t] = row_of[s];
    tv[t] = v[s];
  }
}
__global__ void cols_as_keys(const int32_t* __restrict__ ci, int64_t nnz, uint32_t* __restrict__ k) {
  GRID_STRIDE(t, nnz) k[t] = (uint32_t)ci[t];
}

// ================================================================== SpGEMM
constexpr int kHashCap = 2048;    // per-warp hash table slots
constexpr int kMaxUnique = 1024;  // rows with more distinct columns take the fallback path
constexpr int kSymWarps = 4;
constexpr int kNumWarps = 4;

__device__ __forceinline__ uint32_t hslot(int32_t key) { return ((uint32_t)key * 2654435761u) >> 21; }  // 11 bits

// insert key into the warp's table; returns 1 if new, 0 if present, -1 if the table is full
__device__ __forceinline__ int hinsert(int32_t* tab, int32_t key) {
  uint32_t s = hslot(key);
  for (int probe = 0; probe < kHashCap; ++probe) {
    const int32_t prev = atomicCAS(&tab[s], -1, key);
    if (prev == -1) return 1;
    if (prev == key) return 0;
    s = (s + 1) & (kHashCap - 1);
  }
  return -1;
}
__device__ __forceinline__ int hfind(const int32_t* tab, int32_t key) {
  uint32_t s = hslot(key);
  for (int probe = 0; probe < kHashCap; ++probe) {
    const int32_t k = tab[s];
    if (k == key) return (int)s;
    if (k == -1) return -1;
    s = (s + 1) & (kHashCap - 1);
  }
  return -1;
}

__global__ void __launch_bounds__(kSymWarps * 32) spgemm_symbolic(int64_t n, const int64_t* __restrict__ arp,
                                                                  const int32_t* __restrict__ aci,
                                                                  const int64_t* __restrict__ brp,
                                                                  const int32_t* __restrict__ bci,
                                                                  int32_t* __restrict__ cnt) {
  __shared__ int32_t table[kSymWarps][kHashCap];
  __shared__ int32_t uc[kSymWarps];
  __shared__ int32_t ovf[kSymWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * kSymWarps + w;
  if (row >= n) return;
  int32_t* tab = table[w];
  for (int i = lane; i < kHashCap; i += 32) tab[i] = -1;
  if (lane == 0) { uc[w] = 0; ovf[w] = 0; }
  __syncwarp();
  for (int64_t t = arp[row]; t < arp[row + 1]; ++t) {
    const int32_t k = aci[t];
    const int64_t b0 = brp[k], b1 = brp[k + 1];
    for (int64_t u = b0 + lane; u < b1; u += 32) {
      const int r = hinsert(tab, bci[u]);
      if (r == 1) atomicAdd(&uc[w], 1);
      if (r < 0) ovf[w] = 1;
    }
    __syncwarp();
    if (uc[w] > kMaxUnique || ovf[w]) break;
  }
  __syncwarp();
  if (lane == 0) cnt[row] = (uc[w] > kMaxUnique || ovf[w]) ? -1 : uc[w];
}

struct NumSmem {
  int32_t tab[kHashCap];
  int32_t sorted[kMaxUnique];
  double acc[kHashCap];
  int32_t count;
};
struct FillSmem {  // the pattern pass of the grouped product: no sums
  int32_t tab[kHashCap];
  int32_t sorted[kMaxUnique];
  int32_t count;
};

__global__ void __launch_bounds__(kNumWarps * 32) spgemm_numeric(int64_t n, const int64_t* __restrict__ arp,
                                                                 const int32_t* __restrict__ aci,
                                                                 const double* __restrict__ av,
                                                                 const int64_t* __restrict__ brp,
                                                                 const int32_t* __restrict__ bci,
                                                                 const double* __restrict__ bv,
                                                                 const int32_t* __restrict__ cnt,
                                                                 const int64_t* __restrict__ crp,
                                                                 int32_t* __restrict__ cci, double* __restrict__ cv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NumSmem* all = reinterpret_cast<NumSmem*>(smem_raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * kNumWarps + w;
  if (row >= n || cnt[row] < 0) return;
  NumSmem& S = all[w];
  for (int i = lane; i < kHashCap; i += 32) {
    S.tab[i] = -1;
    S.acc[i] = 0.0;
  }
  if (lane == 0) S.count = 0;
  __syncwarp();
  // distinct columns
  for (int64_t t = arp[row]; t < arp[row + 1]; ++t) {
    const int32_t k = aci[t];
    for (int64_t u = brp[k] + lane; u < brp[k + 1]; u += 32) hinsert(S.tab, bci[u]);
  }
  __syncwarp();
  for (int i = lane; i < kHashCap; i += 32) {
    const int32_t key = S.tab[i];
    if (key >= 0) S.sorted[atomicAdd(&S.count, 1)] = key;
  }
  __syncwarp();
  const int u = S.count;
  int np2 = 1;
  while (np2 < u) np2 <<= 1;
  for (int i = u + lane; i < np2; i += 32) S.sorted[i] = INT32_MAX;
  __syncwarp();
  // bitonic sort of the distinct columns
  for (int kk = 2; kk <= np2; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < np2; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = S.sorted[i], b = S.sorted[ixj];
          const bool up = (i & kk) == 0;
          if ((a > b) == up) {
            S.sorted[i] = b;
            S.sorted[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
  }
  // values: inner index ascending, one rounded product then one rounded sum at a time
  for (int64_t t = arp[row]; t < arp[row + 1]; ++t) {
    const int32_t k = aci[t];
    const double a = av[t];
    for (int64_t q = brp[k] + lane; q < brp[k + 1]; q += 32) {
      const int s = hfind(S.tab, bci[q]);
      S.acc[s] = __dadd_rn(S.acc[s], __dmul_rn(a, bv[q]));
    }
    __syncwarp();
  }
  const int64_t base = crp[row];
  for (int i = lane; i < u; i += 32) {
    const int32_t key = S.sorted[i];
    cci[base + i] = key;
    cv[base + i] = S.acc[hfind(S.tab, key)];
  }
}

// Fallback for rows with many distinct columns: one CTA per row with a dense marker and
// accumulator over all columns (global scratch per CTA slot).
__global__ void spgemm_fallback(const int32_t* __restrict__ rows, int64_t n_rows, int64_t m,
                                const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                const double* __restrict__ av, const int64_t* __restrict__ brp,
                                const int32_t* __restrict__ bci, const double* __restrict__ bv, int phase,
                                int32_t* __restrict__ cnt, const int64_t* __restrict__ crp, int32_t* __restrict__ cci,
                                double* __restrict__ cv, int64_t* __restrict__ mark_all, double* __restrict__ acc_all) {
  __shared__ int64_t sh[32];
  int64_t* mark = mark_all + (int64_t)blockIdx.x * m;
  double* acc = acc_all + (int64_t)blockIdx.x * m;
  for (int64_t it = blockIdx.x; it < n_rows; it += gridDim.x) {
    const int64_t row = rows[it];
    const int64_t tag = 2 * row + phase;
    for (int64_t t = arp[row]; t < arp[row + 1]; ++t) {
      const int32_t k = aci[t];
      for (int64_t u = brp[k] + threadIdx.x; u < brp[k + 1]; u += blockDim.x) mark[bci[u]] = tag;
    }
    __syncthreads();
    int64_t running = 0;
    for (int64_t j0 = 0; j0 < m; j0 += blockDim.x) {
      const int64_t j = j0 + threadIdx.x;
      const int f = (j < m && mark[j] == tag) ? 1 : 0;
      int64_t tot;
      const int64_t pre = block_exclusive_scan(f, sh, &tot);
      if (phase == 1 && f) {
        cci[crp[row] + running + pre] = (int32_t)j;
        acc[j] = 0.0;
      }
      running += tot;
    }
    if (phase == 0) {
      if (threadIdx.x == 0) cnt[row] = (int32_t)running;
      __syncthreads();
      continue;
    }
    __syncthreads();
    for (int64_t t = arp[row]; t < arp[row + 1]; ++t) {
      const int32_t k = aci[t];
      const double a = av[t];
      for (int64_t q = brp[k] + threadIdx.x; q < brp[k + 1]; q += blockDim.x)
        acc[bci[q]] = __dadd_rn(acc[bci[q]], __dmul_rn(a, bv[q]));
      __syncthreads();
    }
    for (int64_t i = threadIdx.x; i < running; i += blockDim.x) cv[crp[row] + i] = acc[cci[crp[row] + i]];
    __syncthreads();
  }
}

__global__ void list_overflow(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ rows,
                              int32_t* __restrict__ n_rows) {
  GRID_STRIDE(i, n) {
    if (cnt[i] < 0) rows[atomicAdd(n_rows, 1)] = (int32_t)i;
  }
}

__global__ void to32v(const double* __restrict__ x, float* __restrict__ y, int64_t n) { GRID_STRIDE(i, n) y[i] = (float)x[i]; }

// ================================================================== diagonal, Lanczos
__global__ void diag_inv_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ v, double* __restrict__ dinv, float* __restrict__ dinv32,
                                double* __restrict__ diag_out, int* __restrict__ bad) {
  GRID_STRIDE(i, n) {
    double d = 0.0;
    int64_t lo = rp[i], hi = rp[i + 1];
    while (lo < hi) {  // binary search for the diagonal
      const int64_t mid = (lo + hi) >> 1;
      if (ci[mid] < i) lo = mid + 1;
      else hi = mid;
    }
    if (lo < rp[i + 1] && ci[lo] == i) d = v[lo];
    if (!(d > 0.0)) {
      atomicAdd(bad, 1);
      d = 1.0;
    }
    if (dinv) dinv[i] = 1.0 / d;
    if (dinv32) dinv32[i] = (float)(1.0 / d);
    if (diag_out) diag_out[i] = d;
  }
}

__device__ __forceinline__ uint32_t dev_hash(int kind, int64_t i) {
  if (kind == 1) return (uint32_t)i;
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ULL + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (uint32_t)(z >> 32);
}

__global__ void lanczos_start(int64_t n, int kind, const double* __restrict__ diag, double* __restrict__ v,
                              double* __restrict__ dsq) {
  GRID_STRIDE(i, n) {
    v[i] = 1.0 + (double)(dev_hash(kind, i) % 1024u) / 1024.0;
    dsq[i] = 1.0 / sqrt(diag[i]);
  }
}
__global__ void vmul(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  GRID_STRIDE(i, n) c[i] = a[i] * b[i];
}
__global__ void vscale(int64_t n, double* __restrict__ x, const double* __restrict__ s, int invert) {
  const double f = invert ? 1.0 / *s : *s;
  GRID_STRIDE(i, n) x[i] = x[i] * f;
}
// w = dsq * w - bprev * vp
__global__ void lanczos_w(int64_t n, const double* __restrict__ dsq, double* __restrict__ w, double bprev,
                          const double* __restrict__ vp) {
  GRID_STRIDE(i, n) w[i] = dsq[i] * w[i] - bprev * vp[i];
}
__global__ void lanczos_orth(int64_t n, double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ a) {
  const double al = *a;
  GRID_STRIDE(i, n) w[i] = w[i] - al * v[i];
}
__global__ void lanczos_next(int64_t n, double* __restrict__ v, double* __restrict__ vp, const double* __restrict__ w,
                             double beta) {
  GRID_STRIDE(i, n) {
    vp[i] = v[i];
    v[i] = w[i] / beta;
  }
}

// ================================================================== p-level construction
// The fine node labelling coarse local node (i, j, k) of element e (Algorithm 2 with nodal
// labels, any q < p).  Per direction, coarse index s is labelled by fine index s p / q when that
// is whole (r = p/q whole: the node (ri, rj, rk)), else by the nearer fine index; at exactly half
// way both neighbours are candidates, and the candidate with the smallest global id wins -- the
// same node seen from every element sharing it, whatever its orientation.  p / q > 1 keeps the
// candidates of different coarse nodes apart.
__device__ __forceinline__ int anchor_axis(int p, int q, int s, int& ties) {
  const int f = (s * p) / q, rem = (s * p) % q;
  ties = (rem != 0 && 2 * rem == q) ? 1 : 0;
  return (rem != 0 && 2 * rem > q) ? f + 1 : f;
}
// Modal (hierarchical) basis: the order-q modes are the order-p modes of degree <= q (Algorithm 2's
// prefix): coarse 1D mode s is fine mode s for s < q and the vertex mode p for s = q.
__device__ __forceinline__ int modal_axis(int p, int q, int s) { return s == q ? p : s; }

__device__ __forceinline__ int32_t coarse_anchor(const int32_t* __restrict__ le, int p, int q, int modal, int i, int j,
                                                 int k) {
  const int n1 = p + 1;
  if (modal) return le[(n1 * n1) * modal_axis(p, q, i) + n1 * modal_axis(p, q, j) + modal_axis(p, q, k)];
  int ti, tj, tk;
  const int ai = anchor_axis(p, q, i, ti), aj = anchor_axis(p, q, j, tj), ak = anchor_axis(p, q, k, tk);
  int32_t best = le[(n1 * n1) * ai + n1 * aj + ak];
  for (int di = 0; di <= ti; ++di)
    for (int dj = 0; dj <= tj; ++dj)
      for (int dk = 0; dk <= tk; ++dk) best = min(best, le[(n1 * n1) * (ai + di) + n1 * (aj + dj) + (ak + dk)]);
  return best;
}
__global__ void mark_anchors(int32_t n_elem, int p, int q, int modal, const int32_t* __restrict__ l2g,
                             int32_t* __restrict__ flag) {
  const int n1 = p + 1, m1 = q + 1;
  const int64_t nlc = (int64_t)m1 * m1 * m1, nlf = (int64_t)n1 * n1 * n1;
  GRID_STRIDE(t, (int64_t)n_elem * nlc) {
    const int64_t e = t / nlc;
    const int b = (int)(t % nlc);
    const int i = b / (m1 * m1), j = (b / m1) % m1, k = b % m1;
    flag[coarse_anchor(l2g + e * nlf, p, q, modal, i, j, k)] = 1;
  }
}
__global__ void coarse_map(int32_t n_elem, int p, int q, int modal, const int32_t* __restrict__ l2g,
                           const int64_t* __restrict__ rank, int32_t* __restrict__ l2g_c) {
  const int n1 = p + 1, m1 = q + 1;
  const int64_t nlc = (int64_t)m1 * m1 * m1, nlf = (int64_t)n1 * n1 * n1;
  GRID_STRIDE(t, (int64_t)n_elem * nlc) {
    const int64_t e = t / nlc;
    const int b = (int)(t % nlc);
    const int i = b / (m1 * m1), j = (b / m1) % m1, k = b % m1;
    l2g_c[t] = (int32_t)rank[coarse_anchor(l2g + e * nlf, p, q, modal, i, j, k)];
  }
}
__global__ void owner_min(int64_t slots, int nlf, const int32_t* __restrict__ l2g, int32_t* __restrict__ owner) {
  GRID_STRIDE(t, slots) atomicMin(&owner[l2g[t]], (int32_t)(t / nlf));
}
__global__ void owner_mask(int64_t slots, int nlf, const int32_t* __restrict__ l2g, const int32_t* __restrict__ owner,
                           uint8_t* __restrict__ own) {
  GRID_STRIDE(t, slots) own[t] = owner[l2g[t]] == (int32_t)(t / nlf) ? 1 : 0;
}

struct P1DConst {
  double t[(GIAMG_MAX_ORDER + 1) * (GIAMG_MAX_ORDER + 1)];
  int nz[GIAMG_MAX_ORDER + 1];  // non-zeros per row of the table
};

__global__ void p_row_counts(int64_t slots, int p, int q, const uint8_t* __restrict__ own, const int32_t* __restrict__ l2g,
                             P1DConst tab, int32_t* __restrict__ cnt) {
  const int n1 = p + 1, nlf = n1 * n1 * n1;
  GRID_STRIDE(t, slots) {
    if (!own[t]) continue;
    const int a = (int)(t % nlf);
    const int a1 = a / (n1 * n1), a2 = (a / n1) % n1, a3 = a % n1;
    cnt[l2g[t]] = tab.nz[a1] * tab.nz[a2] * tab.nz[a3];
  }
}

__global__ void p_row_fill(int64_t slots, int p, int q, const uint8_t* __restrict__ own, const int32_t* __restrict__ l2g,
                           const int32_t* __restrict__ l2g_c, P1DConst tab, const int64_t* __restrict__ prp,
                           int32_t* __restrict__ pci, double* __restrict__ pv) {
  const int n1 = p + 1, m1 = q + 1, nlf = n1 * n1 * n1, nlc = m1 * m1 * m1;
  GRID_STRIDE(t, slots) {
    if (!own[t]) continue;
    const int64_t e = t / nlf;
    const int a = (int)(t % nlf);
    const int a1 = a / (n1 * n1), a2 = (a / n1) % n1, a3 = a % n1;
    const int32_t row = l2g[t];
    const int64_t base = prp[row];
    int c = 0;
    for (int b = 0; b < nlc; ++b) {
      const int b1 = b / (m1 * m1), b2 = (b / m1) % m1, b3 = b % m1;
      const double f1 = tab.t[a1 * m1 + b1], f2 = tab.t[a2 * m1 + b2], f3 = tab.t[a3 * m1 + b3];
      if (f1 == 0.0 || f2 == 0.0 || f3 == 0.0) continue;
      const double v = __dmul_rn(__dmul_rn(f1, f2), f3);
      const int32_t col = l2g_c[e * nlc + b];
      // insertion into the sorted row
      int k = c;
      while (k > 0 && pci[base + k - 1] > col) {
        pci[base + k] = pci[base + k - 1];
        pv[base + k] = pv[base + k - 1];
        --k;
      }
      pci[base + k] = col;
      pv[base + k] = v;
      ++c;
    }
  }
}

__global__ void count_inc(int64_t slots, const int32_t* __restrict__ l2g_c, int32_t* __restrict__ cnt) {
  GRID_STRIDE(t, slots) atomicAdd(&cnt[l2g_c[t]], 1);
}
__global__ void fill_inc(int64_t slots, const int32_t* __restrict__ l2g_c, const int64_t* __restrict__ ptr,
                         int32_t* __restrict__ fillc, int32_t* __restrict__ inc) {
  GRID_STRIDE(t, slots) {
    const int32_t c = l2g_c[t];
    inc[ptr[c] + atomicAdd(&fillc[c], 1)] = (int32_t)t;
  }
}
__global__ void sort_segments(int64_t nseg, const int64_t* __restrict__ ptr, int32_t* __restrict__ v) {
  GRID_STRIDE(c, nseg) {
    const int64_t s = ptr[c], e = ptr[c + 1];
    for (int64_t i = s + 1; i < e; ++i) {
      const int32_t x = v[i];
      int64_t j = i - 1;
      while (j >= s && v[j] > x) {
        v[j + 1] = v[j];
        --j;
      }
      v[j + 1] = x;
    }
  }
}

// ================================================================== h-level construction
// MIS-2 keys: (state, hash, index) packed so that unsigned comparison is lexicographic.
constexpr uint64_t kOut = 0, kUnd = 1, kIn = 2;
__device__ __forceinline__ uint64_t mis_key(uint64_t st, uint32_t h, int64_t i) {
  return (st << 62) | ((uint64_t)h << 30) | (uint64_t)i;
}

__global__ void mis_pass1(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const uint8_t* __restrict__ strong, const uint8_t* __restrict__ st, int kind,
                          uint64_t* __restrict__ m1) {
  GRID_STRIDE(i, n) {
    uint64_t best = mis_key(st[i], dev_hash(kind, i), i);
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
      const int32_t j = ci[t];
      if (j == i || (strong && !strong[t])) continue;
      const uint64_t k = mis_key(st[j], dev_hash(kind, j), j);
      best = k > best ? k : best;
    }
    m1[i] = best;
  }
}
__global__ void mis_pass2(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const uint8_t* __restrict__ strong, const uint8_t* __restrict__ st, int kind,
                          const uint64_t* __restrict__ m1, uint8_t* __restrict__ st2, int32_t* __restrict__ und) {
  GRID_STRIDE(i, n) {
    uint64_t best = m1[i];
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
      const int32_t j = ci[t];
      if (j == i || (strong && !strong[t])) continue;
      best = m1[j] > best ? m1[j] : best;
    }
    uint8_t s = st[i];
    if (s == kUnd) {
      if (best == mis_key(kUnd, dev_hash(kind, i), i)) s = kIn;
      else if ((best >> 62) == kIn) s = kOut;
    }
    st2[i] = s;
    if (s == kUnd) atomicAdd(und, 1);
  }
}
__global__ void mis_init(int64_t n, uint8_t* st) { GRID_STRIDE(i, n) st[i] = kUnd; }
__global__ void is_root(int64_t n, const uint8_t* __restrict__ st, int32_t* __restrict__ f) {
  GRID_STRIDE(i, n) f[i] = st[i] == kIn ? 1 : 0;
}
__global__ void agg_phase1(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const uint8_t* __restrict__ strong, const uint8_t* __restrict__ st,
                           const int64_t* __restrict__ rank, int32_t* __restrict__ a1) {
  GRID_STRIDE(i, n) {
    int32_t g = -1;
    if (st[i] == kIn) g = (int32_t)rank[i];
    else
      for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
        const int32_t j = ci[t];
        if (j == i || (strong && !strong[t])) continue;
        if (st[j] == kIn) g = (int32_t)rank[j];
      }
    a1[i] = g;
  }
}
__global__ void agg_phase2(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const uint8_t* __restrict__ strong, const int32_t* __restrict__ a1, int32_t* __restrict__ agg,
                           int32_t* __restrict__ bad) {
  GRID_STRIDE(i, n) {
    int32_t g = a1[i];
    if (g < 0) {
      for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
        const int32_t j = ci[t];
        if (j == i || (strong && !strong[t])) continue;
        const int32_t c = a1[j];
        if (c >= 0 && (g < 0 || c < g)) g = c;
      }
      if (g < 0) atomicAdd(bad, 1);
    }
    agg[i] = g;
  }
}
__global__ void strength_mask(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ v, const double* __restrict__ dinv, double theta,
                              uint8_t* __restrict__ strong) {
  GRID_STRIDE(i, n) {
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
      const int32_t j = ci[t];
      const double aii = 1.0 / dinv[i], ajj = 1.0 / dinv[j];
      strong[t] = (j != i && fabs(v[t]) >= theta * sqrt(aii * ajj)) ? 1 : 0;
    }
  }
}
__global__ void tentative(int64_t n, const int32_t* __restrict__ agg, int64_t* __restrict__ trp, int32_t* __restrict__ tci,
                          double* __restrict__ tv) {
  GRID_STRIDE(i, n + 1) {
    trp[i] = i;
    if (i < n) {
      tci[i] = agg[i];
      tv[i] = 1.0;
    }
  }
}
// P = T - M (A T), M = diag(a_ii / sum_j a_ij^2), on the pattern of A T (which contains T).  Rows
// with no off-diagonal entry (Dirichlet identity rows, isolated nodes forming their own
// aggregates) keep T: M_ii = 0, since SPAI-0's 1/a_ii would zero their column of P.
__global__ void sa_smooth(int64_t n, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                          const double* __restrict__ av, const int32_t* __restrict__ agg,
                          const int64_t* __restrict__ crp, const int32_t* __restrict__ cci, double* __restrict__ cv,
                          int32_t* __restrict__ bad) {
  GRID_STRIDE(i, n) {
    double diag = 0.0, ss = 0.0;
    bool coupled = false;
    for (int64_t t = arp[i]; t < arp[i + 1]; ++t) {
      ss = __dadd_rn(ss, __dmul_rn(av[t], av[t]));
      if (aci[t] == i) diag = av[t];
      else coupled = true;
    }
    const double mi = coupled ? diag / ss : 0.0;
    int found = 0;
    for (int64_t t = crp[i]; t < crp[i + 1]; ++t) {
      const bool own = cci[t] == agg[i];
      found |= own;
      cv[t] = __dsub_rn(own ? 1.0 : 0.0, __dmul_rn(mi, cv[t]));
    }
    if (!found) atomicAdd(bad, 1);
  }
}

// ================================================================== validation, dense copy
__device__ __forceinline__ bool dirichlet_row(const int64_t* rp, const int32_t* ci, int64_t g) {
  return rp[g + 1] - rp[g] == 1 && ci[rp[g]] == g;
}
// The element map against A's pattern: every pair of one element's nodes must be an entry of A,
// except where either node is a Dirichlet (identity) row.  A block per element: its valid,
// non-Dirichlet nodes sorted in shared memory (bitonic), then a warp per local row merges that
// list with the row's ascending columns, a lane per piece of the list (one binary search for the
// piece's first node, then a forward walk).  Counts the pairs missing from the pattern and the map
// entries out of range.
constexpr int kValThreads = 256;
__global__ void __launch_bounds__(kValThreads) validate_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                               const int32_t* __restrict__ ci,
                                                               const int32_t* __restrict__ l2g, int nloc, int np2,
                                                               unsigned long long* __restrict__ bad) {
  extern __shared__ int32_t vsm[];
  int32_t* sorted = vsm;       // np2 keys: the checked nodes, then INT32_MAX
  int32_t* rows = vsm + np2;   // nloc: the node if its row is checked, else -1
  const int64_t e = blockIdx.x;
  unsigned long long nbad = 0;
  for (int a = threadIdx.x; a < np2; a += kValThreads) {
    int32_t key = INT32_MAX;
    if (a < nloc) {
      const int32_t g = l2g[e * nloc + a];
      int32_t row = -1;
      if (g < 0 || g >= n) ++nbad;
      else if (!dirichlet_row(rp, ci, g)) key = row = g;
      rows[a] = row;
    }
    sorted[a] = key;
  }
  __syncthreads();
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < np2; i += kValThreads) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t x = sorted[i], y = sorted[ixj];
          if ((x > y) == ((i & k) == 0)) {
            sorted[i] = y;
            sorted[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  int m = 0;
  {
    int lo = 0, hi = np2;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sorted[mid] < INT32_MAX) lo = mid + 1;
      else hi = mid;
    }
    m = lo;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cs = (m + 31) / 32, b0 = lane * cs, b1 = min(m, b0 + cs);
  for (int a = w; a < nloc; a += kValThreads / 32) {
    const int32_t g = rows[a];
    if (g < 0 || b0 >= b1) continue;
    const int64_t r1 = rp[g + 1];
    int64_t lo = rp[g], hi = r1;
    const int32_t x0 = sorted[b0];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ci[mid] < x0) lo = mid + 1;
      else hi = mid;
    }
    int64_t q = lo;
    for (int b = b0; b < b1; ++b) {
      const int32_t x = sorted[b];
      while (q < r1 && ci[q] < x) ++q;
      if (q >= r1 || ci[q] != x) ++nbad;
    }
  }
  for (int o = 16; o > 0; o >>= 1) nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
  if (lane == 0 && nbad) atomicAdd(bad, nbad);
}
__global__ void dense_cm(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const double* __restrict__ v, double* __restrict__ D) {
  GRID_STRIDE(i, n) {
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) D[(int64_t)ci[t] * n + i] = v[t];
  }
}

}  // namespace

// ================================================================== host entry points
uint32_t host_hash(int kind, int64_t i) {
  if (kind == 1) return (uint32_t)i;
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ULL + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (uint32_t)(z >> 32);
}

void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) { scan_impl<int32_t>(in, out, n, s); }
void scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) { scan_impl<int64_t>(in, out, n, s); }

void radix_sort_pairs(uint32_t* keys, int64_t* idx, int64_t n, int key_bits, cudaStream_t s) {
  if (n <= 1) return;
  const int64_t nt = (n + kRadixTile - 1) / kRadixTile;
  DBuf<uint32_t> k2;
  DBuf<int64_t> i2, hist, offs;
  k2.alloc(n, s);
  i2.alloc(n, s);
  hist.alloc(16 * nt, s);
  offs.alloc(16 * nt + 1, s);
  uint32_t *ka = keys, *kb = k2.get();
  int64_t *ia = idx, *ib = i2.get();
  int passes = std::max(1, (key_bits + 3) / 4);
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 4 * ps;
    { radix_hist<<<(unsigned)nt, kRadixThreads, 0, s>>>(ka, n, shift, nt, hist.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
    scan_i64(hist.get(), offs.get(), 16 * nt, s);
    { radix_scatter<<<(unsigned)nt, kRadixThreads, 0, s>>>(ka, ia, n, shift, nt, offs.get(), kb, ib); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(ia, ib);
  }
  if (ka != keys) {
    GIAMG_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    GIAMG_CUDA(cudaMemcpyAsync(idx, ia, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s));
  }
  GIAMG_CUDA(cudaStreamSynchronize(s));
}

static int bits_for(int64_t m) {
  int b = 1;
  while (b < 32 && ((int64_t)1 << b) < m) ++b;
  return b;
}

void csr_transpose(const DCSR& A, DCSR& T, cudaStream_t s) {
  T.n = A.m;
  T.m = A.n;
  T.nnz = A.nnz;
  T.rp.alloc(T.n + 1, s);
  T.ci.alloc(std::max<int64_t>(A.nnz, 1), s);
  T.v.alloc(std::max<int64_t>(A.nnz, 1), s);
  DBuf<int32_t> cnt, row_of;
  cnt.alloc(T.n + 1, s);
  cnt.zero(s);
  if (A.nnz > 0) {
    row_of.alloc(A.nnz, s);
    { expand_rows<<<blocks_for(A.n, 256, 65535), 256, 0, s>>>(A.rp.get(), A.n, row_of.get()); note_launch(); }
    { count_cols<<<blocks_for(A.nnz, 256, 65535), 256, 0, s>>>(A.ci.get(), A.nnz, cnt.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
  }
  scan_i32_to_i64(cnt.get(), T.rp.get(), T.n, s);
  if (A.nnz == 0) return;
  DBuf<uint32_t> keys;
  DBuf<int64_t> idx;
  keys.alloc(A.nnz, s);
  idx.alloc(A.nnz, s);
  { cols_as_keys<<<blocks_for(A.nnz, 256, 65535), 256, 0, s>>>(A.ci.get(), A.nnz, keys.get()); note_launch(); }
  { iota64<<<blocks_for(A.nnz, 256, 65535), 256, 0, s>>>(idx.get(), A.nnz); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  radix_sort_pairs(keys.get(), idx.get(), A.nnz, bits_for(A.m), s);
  { gather_transpose<<<blocks_for(A.nnz, 256, 65535), 256, 0, s>>>(idx.get(), A.nnz, row_of.get(), A.v.get(), T.ci.get(),
                                                                  T.v.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void spgemm(const DCSR& A, const DCSR& B, DCSR& C, cudaStream_t s) {
  GIAMG_CHECK(A.m == B.n, GIAMG_ERR_ARG, "spgemm: inner dimensions differ");
  static const bool log = getenv("GIAMG_SETUP_LOG") != nullptr;
  auto t0 = std::chrono::steady_clock::now();
  auto lap = [&](const char* what) {
    if (!log) return;
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    fprintf(stderr, "  spgemm %lld x %lld (A nnz %lld, B nnz %lld): %-10s %9.2f ms\n", (long long)A.n, (long long)B.m,
            (long long)A.nnz, (long long)B.nnz, what, std::chrono::duration<double, std::milli>(now - t0).count());
    t0 = now;
  };
  const int64_t n = A.n, m = B.m;
  C.n = n;
  C.m = m;
  C.rp.alloc(n + 1, s);
  DBuf<int32_t> cnt;
  cnt.alloc(std::max<int64_t>(n, 1), s);
  if (n > 0) {
    { spgemm_symbolic<<<blocks_for(n, kSymWarps), kSymWarps * 32, 0, s>>>(n, A.rp.get(), A.ci.get(), B.rp.get(),
                                                                        B.ci.get(), cnt.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
  }
  // rows that overflow the per-warp table
  DBuf<int32_t> ovf_rows, ovf_n;
  ovf_rows.alloc(std::max<int64_t>(n, 1), s);
  ovf_n.alloc(1, s);
  ovf_n.zero(s);
  if (n > 0) { list_overflow<<<blocks_for(n, 256, 65535), 256, 0, s>>>(cnt.get(), n, ovf_rows.get(), ovf_n.get()); note_launch(); }
  int32_t n_ovf = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&n_ovf, ovf_n.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  DBuf<int64_t> mark;
  DBuf<double> acc;
  int fb_blocks = 0;
  if (n_ovf > 0) {
    fb_blocks = (int)std::min<int64_t>(n_ovf, std::max<int64_t>(1, std::min<int64_t>(64, ((int64_t)1 << 30) / (m * 16 + 1))));
    mark.alloc((size_t)fb_blocks * m, s);
    acc.alloc((size_t)fb_blocks * m, s);
    GIAMG_CUDA(cudaMemsetAsync(mark.get(), 0xff, sizeof(int64_t) * fb_blocks * m, s));
    { spgemm_fallback<<<fb_blocks, 256, 0, s>>>(ovf_rows.get(), n_ovf, m, A.rp.get(), A.ci.get(), A.v.get(), B.rp.get(),
                                              B.ci.get(), B.v.get(), 0, cnt.get(), nullptr, nullptr, nullptr, mark.get(),
                                              acc.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
  }
  lap("symbolic");
  scan_i32_to_i64(cnt.get(), C.rp.get(), n, s);
  GIAMG_CUDA(cudaMemcpyAsync(&C.nnz, C.rp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  C.ci.alloc(std::max<int64_t>(C.nnz, 1), s);
  C.v.alloc(std::max<int64_t>(C.nnz, 1), s);
  if (n > 0) {
    const size_t sm = sizeof(NumSmem) * kNumWarps;
    static PerDevice attr;
    attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(spgemm_numeric, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); });
    { spgemm_numeric<<<blocks_for(n, kNumWarps), kNumWarps * 32, sm, s>>>(n, A.rp.get(), A.ci.get(), A.v.get(), B.rp.get(),
                                                                        B.ci.get(), B.v.get(), cnt.get(), C.rp.get(),
                                                                        C.ci.get(), C.v.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
  }
  lap("numeric");
  if (n_ovf > 0) {
    { spgemm_fallback<<<fb_blocks, 256, 0, s>>>(ovf_rows.get(), n_ovf, m, A.rp.get(), A.ci.get(), A.v.get(), B.rp.get(),
                                              B.ci.get(), B.v.get(), 1, cnt.get(), C.rp.get(), C.ci.get(), C.v.get(),
                                              mark.get(), acc.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
  }
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (log) fprintf(stderr, "  spgemm: C nnz %lld, %d rows on the fallback path\n", (long long)C.nnz, n_ovf);
  lap("fallback");
}

// ------------------------------------------------------------------ SpGEMM over row groups
// C = A B where the rows of A come in groups with identical column sets (Groups, pattern.cu): the
// rows of a group have identical rows in C's pattern (the union of B's rows over the group's
// columns), so the pattern -- a hash count, then the sorted distinct columns -- is found once per
// group instead of once per row, and the numeric pass only accumulates: each output position is
// found by a binary search in the group's sorted list held in shared memory, and the sums run in
// ascending inner index with separately rounded products, as in spgemm_numeric.
__global__ void __launch_bounds__(kSymWarps * 32) gsym_count(int64_t G, const int64_t* __restrict__ gptr,
                                                             const int32_t* __restrict__ gcol,
                                                             const int64_t* __restrict__ brp,
                                                             const int32_t* __restrict__ bci, int32_t* __restrict__ cnt) {
  __shared__ int32_t table[kSymWarps][kHashCap];
  __shared__ int32_t uc[kSymWarps];
  __shared__ int32_t ovf[kSymWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kSymWarps + w;
  if (g >= G) return;
  int32_t* tab = table[w];
  for (int i = lane; i < kHashCap; i += 32) tab[i] = -1;
  if (lane == 0) { uc[w] = 0; ovf[w] = 0; }
  __syncwarp();
  for (int64_t t = gptr[g]; t < gptr[g + 1]; ++t) {
    const int32_t k = gcol[t];
    for (int64_t u = brp[k] + lane; u < brp[k + 1]; u += 32) {
      const int r = hinsert(tab, bci[u]);
      if (r == 1) atomicAdd(&uc[w], 1);
      if (r < 0) ovf[w] = 1;
    }
    __syncwarp();
    if (uc[w] > kMaxUnique || ovf[w]) break;
  }
  __syncwarp();
  if (lane == 0) cnt[g] = (uc[w] > kMaxUnique || ovf[w]) ? -1 : uc[w];
}

// the group's distinct columns, ascending, at uoff[g] (the table again, then a bitonic sort)
__global__ void __launch_bounds__(kNumWarps * 32) gsym_fill(int64_t G, const int64_t* __restrict__ gptr,
                                                            const int32_t* __restrict__ gcol,
                                                            const int64_t* __restrict__ brp,
                                                            const int32_t* __restrict__ bci,
                                                            const int64_t* __restrict__ uoff, int32_t* __restrict__ ulist) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FillSmem* all = reinterpret_cast<FillSmem*>(smem_raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kNumWarps + w;
  if (g >= G) return;
  FillSmem& S = all[w];
  for (int i = lane; i < kHashCap; i += 32) S.tab[i] = -1;
  if (lane == 0) S.count = 0;
  __syncwarp();
  for (int64_t t = gptr[g]; t < gptr[g + 1]; ++t) {
    const int32_t k = gcol[t];
    for (int64_t u = brp[k] + lane; u < brp[k + 1]; u += 32) hinsert(S.tab, bci[u]);
  }
  __syncwarp();
  for (int i = lane; i < kHashCap; i += 32) {
    const int32_t key = S.tab[i];
    if (key >= 0) S.sorted[atomicAdd(&S.count, 1)] = key;
  }
  __syncwarp();
  const int u = S.count;
  int np2 = 1;
  while (np2 < u) np2 <<= 1;
  for (int i = u + lane; i < np2; i += 32) S.sorted[i] = INT32_MAX;
  __syncwarp();
  for (int kk = 2; kk <= np2; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < np2; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = S.sorted[i], b = S.sorted[ixj];
          const bool up = (i & kk) == 0;
          if ((a > b) == up) {
            S.sorted[i] = b;
            S.sorted[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
  }
  int32_t* out = ulist + uoff[g];
  for (int i = lane; i < u; i += 32) out[i] = S.sorted[i];
}

__global__ void group_row_counts(int64_t G, const int64_t* __restrict__ rptr, const int32_t* __restrict__ grow,
                                 const int32_t* __restrict__ ucnt, int32_t* __restrict__ gid, int32_t* __restrict__ cnt) {
  GRID_STRIDE(g, G) {
    for (int64_t t = rptr[g]; t < rptr[g + 1]; ++t) {
      gid[grow[t]] = (int32_t)g;
      cnt[grow[t]] = ucnt[g];
    }
  }
}

// numeric, per row: a warp per row; smem per warp: the group's sorted list (umax int32) and the
// sums (umax doubles); the lanes take the entries of B's row k, each finding its position by a
// binary search
__global__ void __launch_bounds__(kNumWarps * 32) gnum_rows(int64_t n, int umax, const int64_t* __restrict__ arp,
                                                            const int32_t* __restrict__ aci,
                                                            const double* __restrict__ av,
                                                            const int64_t* __restrict__ brp,
                                                            const int32_t* __restrict__ bci,
                                                            const double* __restrict__ bv,
                                                            const int32_t* __restrict__ gid,
                                                            const int64_t* __restrict__ uoff,
                                                            const int32_t* __restrict__ ulist,
                                                            const int64_t* __restrict__ crp, int32_t* __restrict__ cci,
                                                            double* __restrict__ cv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* acc = reinterpret_cast<double*>(smem_raw) + (size_t)w * umax;
  int32_t* cols = reinterpret_cast<int32_t*>(reinterpret_cast<double*>(smem_raw) + (size_t)kNumWarps * umax) +
                  (size_t)w * umax;
  const int64_t row = (int64_t)blockIdx.x * kNumWarps + w;
  if (row >= n) return;
  const int32_t g = gid[row];
  const int32_t* __restrict__ ul = ulist + uoff[g];
  const int u = (int)(uoff[g + 1] - uoff[g]);
  for (int i = lane; i < u; i += 32) {
    cols[i] = ul[i];
    acc[i] = 0.0;
  }
  __syncwarp();
  for (int64_t t = arp[row]; t < arp[row + 1]; ++t) {
    const int32_t k = aci[t];
    const double a = av[t];
    for (int64_t q = brp[k] + lane; q < brp[k + 1]; q += 32) {
      const int32_t c = bci[q];
      int lo = 0, hi = u - 1;  // c is in the list by construction
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cols[mid] < c) lo = mid + 1;
        else hi = mid;
      }
      acc[lo] = __dadd_rn(acc[lo], __dmul_rn(a, bv[q]));
    }
    __syncwarp();
  }
  const int64_t base = crp[row];
  for (int i = lane; i < u; i += 32) {
    cci[base + i] = cols[i];
    cv[base + i] = acc[i];
  }
}

// numeric, by warp work items (groups of many rows): a warp takes `nr` rows of one group with `ns`
// lanes per row (ns = 32 / nr rounded down, so pieces of few rows still fill the warp), the
// group's sorted output columns and the rows' sums ([position][row]) in shared memory.  For each
// inner index k of the group (ascending) the lanes find the positions of B's row k in the column
// list once for all of the warp's rows; the lanes of one row then split that row's entries
// (distinct positions), so every sum still runs in ascending k with separately rounded products, as
// in the per-row pass; a warp barrier between two k orders the updates of one sum made by
// different lanes.  Two entries are applied per step (their positions differ), which halves the
// dependent shared-memory chain; the next k's row bounds are loaded two steps ahead and its first
// 32 entries of B one step ahead.
struct GnumItem {
  int32_t g, r0, nr, ns;  // group, first row (offset in the group's row list), rows, lanes per row
};
constexpr int kGnumCap = 2048;    // target sums per warp item (doubles; 16 KB of shared memory)

__global__ void __launch_bounds__(32) gnum_warp(const GnumItem* __restrict__ items, int cap,
                                                const int64_t* __restrict__ arp, const double* __restrict__ av,
                                                const int64_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                                const double* __restrict__ bv, const int64_t* __restrict__ gptr,
                                                const int32_t* __restrict__ gcol, const int64_t* __restrict__ rptr,
                                                const int32_t* __restrict__ grow, const int64_t* __restrict__ uoff,
                                                const int32_t* __restrict__ ulist, const int64_t* __restrict__ crp,
                                                int32_t* __restrict__ cci, double* __restrict__ cv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr unsigned kFull = 0xffffffffu;
  const GnumItem it = items[blockIdx.x];
  const int lane = threadIdx.x;
  const int R = it.nr, S = it.ns;
  const int64_t g = it.g;
  const int u = (int)(uoff[g + 1] - uoff[g]);
  double* acc = reinterpret_cast<double*>(smem_raw);  // u * R <= cap sums, position-major
  int32_t* cols = reinterpret_cast<int32_t*>(acc + cap);
  const int32_t* __restrict__ ul = ulist + uoff[g];
  for (int i = lane; i < u; i += 32) cols[i] = ul[i];
  for (int i = lane; i < u * R; i += 32) acc[i] = 0.0;
  const int r = lane % R, sl = lane / R;
  const bool active = sl < S;
  const int64_t rbase = rptr[g] + it.r0;
  const double* __restrict__ arow = av + arp[grow[rbase + r]];
  double* accr = acc + r;
  const int64_t k0 = gptr[g], nk = gptr[g + 1] - k0;
  // pipeline registers: (q0, q1, a) and the first entries (cb, pvb) of the step to come, and the
  // bounds (nq0, nq1, na) of the one after it
  int64_t q0 = 0, q1 = 0, nq0 = 0, nq1 = 0;
  double a = 0.0, na = 0.0, pvb = 0.0;
  int32_t cb = 0;
  if (nk > 0) {
    const int32_t k = gcol[k0];
    q0 = brp[k];
    q1 = brp[k + 1];
    a = arow[0];
    if (lane < q1 - q0) {
      cb = bci[q0 + lane];
      pvb = bv[q0 + lane];
    }
    if (nk > 1) {
      const int32_t k2 = gcol[k0 + 1];
      nq0 = brp[k2];
      nq1 = brp[k2 + 1];
      na = arow[1];
    }
  }
  __syncwarp();
  for (int64_t t = 0; t < nk; ++t) {
    const int64_t tq0 = q0, tq1 = q1;
    const double ta = a;
    int32_t c = cb;
    double pv = pvb;
    q0 = nq0;
    q1 = nq1;
    a = na;
    if (t + 2 < nk) {
      const int32_t k2 = gcol[k0 + t + 2];
      nq0 = brp[k2];
      nq1 = brp[k2 + 1];
      na = arow[t + 2];
    }
    if (tq0 >= tq1 && t + 1 < nk) {  // B's row k is empty: the next step's entries now
      cb = 0;
      pvb = 0.0;
      if (lane < q1 - q0) {
        cb = bci[q0 + lane];
        pvb = bv[q0 + lane];
      }
    }
    for (int64_t qb = tq0; qb < tq1; qb += 32) {
      const int nb = tq1 - qb < 32 ? (int)(tq1 - qb) : 32;
      if (qb != tq0) {
        c = 0;
        pv = 0.0;
        if (lane < nb) {
          c = bci[qb + lane];
          pv = bv[qb + lane];
        }
      }
      if (qb + 32 >= tq1 && t + 1 < nk) {  // this step's last entries: load the next step's first
        cb = 0;
        pvb = 0.0;
        if (lane < q1 - q0) {
          cb = bci[q0 + lane];
          pvb = bv[q0 + lane];
        }
      }
      int pos = 0;
      if (lane < nb) {
        int lo = 0, hi = u - 1;  // c is in the list by construction
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (cols[mid] < c) lo = mid + 1;
          else hi = mid;
        }
        pos = lo;
      }
      for (int j0 = 0; j0 < nb; j0 += 2 * S) {  // uniform trip count: every lane joins the shuffles
        const int ja = j0 + sl, jb = ja + S;      // this lane's row: entries ja and jb
        const int p0 = __shfl_sync(kFull, pos, ja & 31), p1 = __shfl_sync(kFull, pos, jb & 31);
        const double v0 = __shfl_sync(kFull, pv, ja & 31), v1 = __shfl_sync(kFull, pv, jb & 31);
        if (active && jb < nb) {
          double x0 = accr[p0 * R], x1 = accr[p1 * R];
          x0 = __dadd_rn(x0, __dmul_rn(ta, v0));
          x1 = __dadd_rn(x1, __dmul_rn(ta, v1));
          accr[p0 * R] = x0;
          accr[p1 * R] = x1;
        } else if (active && ja < nb) {
          accr[p0 * R] = __dadd_rn(accr[p0 * R], __dmul_rn(ta, v0));
        }
      }
    }
    __syncwarp();
  }
  for (int rr = 0; rr < R; ++rr) {
    const int64_t base = crp[grow[rbase + rr]];
    for (int i = lane; i < u; i += 32) {
      cci[base + i] = cols[i];
      cv[base + i] = acc[i * R + rr];
    }
  }
}

bool spgemm_grouped(const DCSR& A, const DCSR& B, DCSR& C, cudaStream_t s) {
  const Groups& R = A.grp;
  if (!R.on || A.m != B.n) return false;
  static const bool log = getenv("GIAMG_SETUP_LOG") != nullptr;
  auto t0 = std::chrono::steady_clock::now();
  auto lap = [&](const char* what) {
    if (!log) return;
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    fprintf(stderr, "  spgemm by row groups %lld x %lld (%lld groups): %-10s %9.2f ms\n", (long long)A.n,
            (long long)B.m, (long long)R.n_groups, what, std::chrono::duration<double, std::milli>(now - t0).count());
    t0 = now;
  };
  const int64_t n = A.n, G = R.n_groups;
  DBuf<int32_t> ucnt;
  ucnt.alloc(std::max<int64_t>(G, 1), s);
  { gsym_count<<<blocks_for(G, kSymWarps), kSymWarps * 32, 0, s>>>(G, R.gptr.get(), R.gcol.get(), B.rp.get(), B.ci.get(),
                                                                  ucnt.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  std::vector<int32_t> uc(G);
  GIAMG_CUDA(cudaMemcpyAsync(uc.data(), ucnt.get(), sizeof(int32_t) * G, cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  int umax = 1;
  for (int32_t v : uc) {
    if (v < 0) return false;  // a group's pattern does not fit the table: the per-row product
    umax = std::max(umax, (int)v);
  }
  DBuf<int64_t> uoff;
  uoff.alloc(G + 1, s);
  scan_i32_to_i64(ucnt.get(), uoff.get(), G, s);
  int64_t utot = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&utot, uoff.get() + G, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  DBuf<int32_t> ulist, gid, cnt;
  ulist.alloc(std::max<int64_t>(utot, 1), s);
  {
    static PerDevice attr;
    const int fsm = (int)(sizeof(FillSmem) * kNumWarps);
    attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(gsym_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm)); });
    gsym_fill<<<blocks_for(G, kNumWarps), kNumWarps * 32, fsm, s>>>(G, R.gptr.get(), R.gcol.get(), B.rp.get(),
                                                                   B.ci.get(), uoff.get(), ulist.get());
    note_launch();
  }
  gid.alloc(n, s);
  cnt.alloc(n, s);
  { group_row_counts<<<blocks_for(G, 256, 65535), 256, 0, s>>>(G, R.rptr.get(), R.grow.get(), ucnt.get(), gid.get(),
                                                              cnt.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  lap("symbolic");
  C.n = n;
  C.m = B.m;
  C.rp.alloc(n + 1, s);
  scan_i32_to_i64(cnt.get(), C.rp.get(), n, s);
  GIAMG_CUDA(cudaMemcpyAsync(&C.nnz, C.rp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  C.ci.alloc(std::max<int64_t>(C.nnz, 1), s);
  C.v.alloc(std::max<int64_t>(C.nnz, 1), s);
  // the numeric pass: warp work items where the groups are large enough to share the position
  // searches among their rows, else a warp per row (environment GIAMG_SPGEMM_NUMERIC=1 / 2 forces
  // the per-row / warp-item pass, for measurements)
  static const int forced = [] {
    const char* e = getenv("GIAMG_SPGEMM_NUMERIC");
    return e ? atoi(e) : 0;
  }();
  const bool by_items = forced == 2 || (forced != 1 && 2 * n >= 3 * G);  // 1.5 rows a group or more
  if (by_items) {
    // each group in pieces of the largest power of two of rows (at most 32) whose sums fit
    // kGnumCap, the remainder last
    std::vector<int64_t> rp_h(G + 1);
    GIAMG_CUDA(cudaMemcpyAsync(rp_h.data(), R.rptr.get(), sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    std::vector<GnumItem> items;
    items.reserve((size_t)G * 2);
    int cap = 1;
    for (int64_t g = 0; g < G; ++g) {
      const int u = std::max(uc[g], 1);
      int rb = 32;
      while (rb > 1 && (int64_t)rb * u > kGnumCap) rb >>= 1;
      const int64_t nr = rp_h[g + 1] - rp_h[g];
      for (int64_t r0 = 0; r0 < nr; r0 += rb) {
        const int rows = (int)std::min<int64_t>(rb, nr - r0);
        items.push_back(GnumItem{(int32_t)g, (int32_t)r0, rows, 32 / rows});
        cap = std::max(cap, rows * u);
      }
    }
    cap = (cap + 1) & ~1;  // the column list starts on 16 bytes
    const size_t wsm = (size_t)cap * sizeof(double) + (size_t)umax * sizeof(int32_t);
    if (!items.empty()) {
      DBuf<GnumItem> items_d;
      items_d.alloc(items.size(), s);
      GIAMG_CUDA(cudaMemcpyAsync(items_d.get(), items.data(), sizeof(GnumItem) * items.size(), cudaMemcpyHostToDevice,
                                 s));
      static PerDevice attr;  // the largest request: cap <= max(kGnumCap, kMaxUnique) + 1, umax <= kMaxUnique
      attr.once([&] {
        GIAMG_CUDA(cudaFuncSetAttribute(gnum_warp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((kGnumCap + kMaxUnique + 2) * sizeof(double) +
                                              kMaxUnique * sizeof(int32_t))));
      });
      gnum_warp<<<(unsigned)items.size(), 32, wsm, s>>>(items_d.get(), cap, A.rp.get(), A.v.get(), B.rp.get(),
                                                        B.ci.get(), B.v.get(), R.gptr.get(), R.gcol.get(),
                                                        R.rptr.get(), R.grow.get(), uoff.get(), ulist.get(),
                                                        C.rp.get(), C.ci.get(), C.v.get());
      note_launch();
      GIAMG_CUDA(cudaGetLastError());
      GIAMG_CUDA(cudaStreamSynchronize(s));  // items_d is released at scope end
    }
  } else {
    const size_t sm = (size_t)kNumWarps * umax * (sizeof(double) + sizeof(int32_t));
    static PerDevice attr;
    attr.once([&] {
      GIAMG_CUDA(cudaFuncSetAttribute(gnum_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kNumWarps * kMaxUnique * (sizeof(double) + sizeof(int32_t)))));
    });
    gnum_rows<<<blocks_for(n, kNumWarps), kNumWarps * 32, sm, s>>>(n, umax, A.rp.get(), A.ci.get(), A.v.get(),
                                                                  B.rp.get(), B.ci.get(), B.v.get(), gid.get(),
                                                                  uoff.get(), ulist.get(), C.rp.get(), C.ci.get(),
                                                                  C.v.get());
    note_launch();
  }
  GIAMG_CUDA(cudaGetLastError());
  GIAMG_CUDA(cudaStreamSynchronize(s));
  lap("numeric");
  return true;
}

void csr_to32(DCSR& A, cudaStream_t s) {
  A.v32.alloc((size_t)A.nnz + 4, s);  // 16 bytes of tail room for L2 prefetches widened to 16 bytes
  if (A.nnz) { to32v<<<blocks_for(A.nnz, 256, 65535), 256, 0, s>>>(A.v.get(), A.v32.get(), A.nnz); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

bool diag_inverse(const DCSR& A, double* dinv, float* dinv32, cudaStream_t s) {
  DBuf<int> bad;
  bad.alloc(1, s);
  bad.zero(s);
  if (A.n) { diag_inv_kernel<<<blocks_for(A.n, 256, 65535), 256, 0, s>>>(A.n, A.rp.get(), A.ci.get(), A.v.get(), dinv,
                                                                         dinv32, nullptr, bad.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  int h = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&h, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  return h == 0;
}

// largest eigenvalue of a symmetric tridiagonal matrix by bisection on the Sturm count
static double tridiag_max(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double x = 0.5 * (lo + hi);
    if (x <= lo || x >= hi) break;
    int below = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++below;
    }
    if (below == m) hi = x;
    else lo = x;
  }
  return hi;
}

double lanczos_rho(const DCSR& A, int steps, int hash_kind, Hierarchy& H) {
  cudaStream_t s = H.stream;
  const int64_t n = A.n;
  DBuf<double> v, vp, w, t, dsq, diag, red;
  v.alloc(n, s); vp.alloc(n, s); w.alloc(n, s); t.alloc(n, s); dsq.alloc(n, s); diag.alloc(n, s);
  red.alloc(kRedBlocks + 4, s);
  vp.zero(s);
  {
    DBuf<int> bad;
    bad.alloc(1, s);
    bad.zero(s);
    { diag_inv_kernel<<<blocks_for(n, 256, 65535), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), A.v.get(), nullptr, nullptr,
                                                               diag.get(), bad.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
  }
  const unsigned g = blocks_for(n, 256, 152 * 16);
  { lanczos_start<<<g, 256, 0, s>>>(n, hash_kind, diag.get(), v.get(), dsq.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  double* scal = red.get() + kRedBlocks;  // [0] reduced value
  auto dot_dev = [&](const double* x, const double* y) {
    dot_partial(n, x, y, red.get(), s);
    reduce_to(red.get(), scal, s);
  };
  auto dot_host = [&](const double* x, const double* y) {
    dot_dev(x, y);
    double h = 0.0;
    GIAMG_CUDA(cudaMemcpyAsync(&h, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    return h;
  };
  const double nv = std::sqrt(dot_host(v.get(), v.get()));
  {
    DBuf<double> tmp;
    tmp.alloc(1, s);
    GIAMG_CUDA(cudaMemcpyAsync(tmp.get(), &nv, sizeof(double), cudaMemcpyHostToDevice, s));
    { vscale<<<g, 256, 0, s>>>(n, v.get(), tmp.get(), 1); note_launch(); }
    GIAMG_CUDA(cudaStreamSynchronize(s));
  }
  const int m = (int)std::min<int64_t>(steps, n);
  std::vector<double> al, be;
  double bprev = 0.0;
  const double avg = n ? (double)A.nnz / n : 0.0;
  for (int j = 0; j < m; ++j) {
    { vmul<<<g, 256, 0, s>>>(n, dsq.get(), v.get(), t.get()); note_launch(); }
    spmv(A, t.get(), w.get(), s, avg);
    { lanczos_w<<<g, 256, 0, s>>>(n, dsq.get(), w.get(), bprev, vp.get()); note_launch(); }
    dot_dev(w.get(), v.get());
    { lanczos_orth<<<g, 256, 0, s>>>(n, w.get(), v.get(), scal); note_launch(); }
    double a = 0.0;
    GIAMG_CUDA(cudaMemcpyAsync(&a, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    const double b = std::sqrt(dot_host(w.get(), w.get()));
    al.push_back(a);
    be.push_back(b);
    if (j == m - 1 || b <= 1e-14 * std::fabs(a)) break;
    { lanczos_next<<<g, 256, 0, s>>>(n, v.get(), vp.get(), w.get(), b); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
    bprev = b;
  }
  return tridiag_max(al, be);
}

// 1D tables of the nodal p-transfer: GLL nodes of order p and q and the Lagrange values
// P1D[a][b] = l_b^(q)(x_a^(p)) (product formula, ascending m).
static void gll(int p, double* x) {
  // Newton iteration on f(t) = P_{p-1}(t) - t P_p(t) = (1 - t^2) P_p'(t) / p, whose zeros are
  // the interior GLL nodes; the Legendre equation gives f'(t) = -(p + 1) P_p(t).  Started
  // from the Chebyshev-Gauss-Lobatto points; the left half is mirrored.
  x[0] = -1.0;
  x[p] = 1.0;
  for (int j = 1; j <= p / 2; ++j) {
    double t = -std::cos(M_PI * (double)j / (double)p);
    for (int it = 0; it < 100; ++it) {
      double pm = 1.0, pc = t;  // P_{k-1}, P_k
      for (int k = 1; k < p; ++k) {
        const double pn = ((2.0 * k + 1.0) * t * pc - k * pm) / (k + 1.0);
        pm = pc;
        pc = pn;
      }
      const double dt = (pm - t * pc) / (-(p + 1.0) * pc);
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[j] = t;
    x[p - j] = -t;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
}

void p_level_build(Level& F, Level& C, int modal, cudaStream_t s) {
  const int p = F.p, q = F.q;
  const int n1 = p + 1, m1 = q + 1, nlf = n1 * n1 * n1, nlc = m1 * m1 * m1;
  const int64_t nf = F.A.n;
  const int64_t slots_f = (int64_t)F.n_elem * nlf, slots_c = (int64_t)F.n_elem * nlc;
  // Algorithms 2-3: retained fine dofs marked; Algorithm 4: coarse id = rank among them
  DBuf<int32_t> flag;
  DBuf<int64_t> rank;
  flag.alloc(nf, s);
  flag.zero(s);
  rank.alloc(nf + 1, s);
  { mark_anchors<<<blocks_for(slots_c, 256, 65535), 256, 0, s>>>(F.n_elem, p, q, modal, F.l2g.get(), flag.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  scan_i32_to_i64(flag.get(), rank.get(), nf, s);
  int64_t nc = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&nc, rank.get() + nf, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  F.n_next = nc;
  F.l2g_c.alloc(slots_c, s);
  { coarse_map<<<blocks_for(slots_c, 256, 65535), 256, 0, s>>>(F.n_elem, p, q, modal, F.l2g.get(), rank.get(), F.l2g_c.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  // the coarse level's element map is the same array
  C.l2g.alloc(slots_c, s);
  GIAMG_CUDA(cudaMemcpyAsync(C.l2g.get(), F.l2g_c.get(), sizeof(int32_t) * slots_c, cudaMemcpyDeviceToDevice, s));
  C.n_elem = F.n_elem;
  // owners: the first element containing each fine dof
  DBuf<int32_t> owner;
  owner.alloc(nf, s);
  GIAMG_CUDA(cudaMemsetAsync(owner.get(), 0x7f, sizeof(int32_t) * nf, s));
  { owner_min<<<blocks_for(slots_f, 256, 65535), 256, 0, s>>>(slots_f, nlf, F.l2g.get(), owner.get()); note_launch(); }
  F.own.alloc(slots_f, s);
  { owner_mask<<<blocks_for(slots_f, 256, 65535), 256, 0, s>>>(slots_f, nlf, F.l2g.get(), owner.get(), F.own.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  // 1D table
  double xp[GIAMG_MAX_ORDER + 1], xq[GIAMG_MAX_ORDER + 1];
  gll(p, xp);
  gll(q, xq);
  P1DConst tab{};
  std::vector<float> t32(n1 * m1);
  for (int a = 0; a <= p; ++a) {
    int nz = 0;
    for (int b = 0; b <= q; ++b) {
      double v = 1.0;
      if (modal)  // injection (Algorithm 7 with values 1): fine mode a is coarse mode b
        v = a == (b == q ? p : b) ? 1.0 : 0.0;
      else
        for (int mm = 0; mm <= q; ++mm)
          if (mm != b) v = v * ((xp[a] - xq[mm]) / (xq[b] - xq[mm]));
      tab.t[a * m1 + b] = v;
      t32[a * m1 + b] = (float)v;
      nz += v != 0.0;
    }
    tab.nz[a] = nz;
  }
  F.p1d.alloc(n1 * m1, s);
  F.p1d32.alloc(n1 * m1, s);
  GIAMG_CUDA(cudaMemcpyAsync(F.p1d.get(), tab.t, sizeof(double) * n1 * m1, cudaMemcpyHostToDevice, s));
  GIAMG_CUDA(cudaMemcpyAsync(F.p1d32.get(), t32.data(), sizeof(float) * n1 * m1, cudaMemcpyHostToDevice, s));
  // Algorithm 7, nodal: assembled P, each row from its owning element, columns ascending
  DBuf<int32_t> cnt;
  cnt.alloc(nf, s);
  cnt.zero(s);
  { p_row_counts<<<blocks_for(slots_f, 256, 65535), 256, 0, s>>>(slots_f, p, q, F.own.get(), F.l2g.get(), tab, cnt.get()); note_launch(); }
  F.P.n = nf;
  F.P.m = nc;
  F.P.rp.alloc(nf + 1, s);
  scan_i32_to_i64(cnt.get(), F.P.rp.get(), nf, s);
  GIAMG_CUDA(cudaMemcpyAsync(&F.P.nnz, F.P.rp.get() + nf, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  F.P.ci.alloc(std::max<int64_t>(F.P.nnz, 1), s);
  F.P.v.alloc(std::max<int64_t>(F.P.nnz, 1), s);
  { p_row_fill<<<blocks_for(slots_f, 128, 65535), 128, 0, s>>>(slots_f, p, q, F.own.get(), F.l2g.get(), F.l2g_c.get(), tab,
                                                              F.P.rp.get(), F.P.ci.get(), F.P.v.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  // coarse incidence for the element-form restriction
  DBuf<int32_t> ccnt, cfill;
  ccnt.alloc(nc, s);
  ccnt.zero(s);
  cfill.alloc(nc, s);
  cfill.zero(s);
  { count_inc<<<blocks_for(slots_c, 256, 65535), 256, 0, s>>>(slots_c, F.l2g_c.get(), ccnt.get()); note_launch(); }
  F.cinc_ptr.alloc(nc + 1, s);
  scan_i32_to_i64(ccnt.get(), F.cinc_ptr.get(), nc, s);
  F.cinc.alloc(slots_c, s);
  { fill_inc<<<blocks_for(slots_c, 256, 65535), 256, 0, s>>>(slots_c, F.l2g_c.get(), F.cinc_ptr.get(), cfill.get(),
                                                            F.cinc.get()); note_launch(); }
  { sort_segments<<<blocks_for(nc, 256, 65535), 256, 0, s>>>(nc, F.cinc_ptr.get(), F.cinc.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  F.part.alloc(slots_c, s);
  F.part32.alloc(slots_c, s);
  csr_to32(F.P, s);
  GIAMG_CUDA(cudaStreamSynchronize(s));
}

int64_t h_level_aggregate(Level& F, double theta, int hash_kind, cudaStream_t s) {
  const int64_t n = F.A.n;
  GIAMG_CHECK(n < ((int64_t)1 << 30), GIAMG_ERR_ARG, "aggregation level too large for MIS-2 keys");
  DBuf<uint8_t> strong, st, st2;
  DBuf<uint64_t> m1;
  DBuf<int32_t> und, flag, a1, bad;
  DBuf<int64_t> rank;
  const uint8_t* sp = nullptr;
  if (theta > 0.0) {
    strong.alloc(std::max<int64_t>(F.A.nnz, 1), s);
    { strength_mask<<<blocks_for(n, 256, 65535), 256, 0, s>>>(n, F.A.rp.get(), F.A.ci.get(), F.A.v.get(), F.dinv.get(),
                                                             theta, strong.get()); note_launch(); }
    sp = strong.get();
  }
  st.alloc(n, s);
  st2.alloc(n, s);
  m1.alloc(n, s);
  und.alloc(1, s);
  const unsigned g = blocks_for(n, 256, 65535);
  { mis_init<<<g, 256, 0, s>>>(n, st.get()); note_launch(); }
  for (int round = 0; round < 100000; ++round) {
    und.zero(s);
    { mis_pass1<<<g, 256, 0, s>>>(n, F.A.rp.get(), F.A.ci.get(), sp, st.get(), hash_kind, m1.get()); note_launch(); }
    { mis_pass2<<<g, 256, 0, s>>>(n, F.A.rp.get(), F.A.ci.get(), sp, st.get(), hash_kind, m1.get(), st2.get(), und.get()); note_launch(); }
    GIAMG_CUDA(cudaGetLastError());
    st.swap(st2);
    int32_t h = 0;
    GIAMG_CUDA(cudaMemcpyAsync(&h, und.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    if (h == 0) break;
  }
  flag.alloc(n, s);
  rank.alloc(n + 1, s);
  { is_root<<<g, 256, 0, s>>>(n, st.get(), flag.get()); note_launch(); }
  scan_i32_to_i64(flag.get(), rank.get(), n, s);
  int64_t n_agg = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&n_agg, rank.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  a1.alloc(n, s);
  { agg_phase1<<<g, 256, 0, s>>>(n, F.A.rp.get(), F.A.ci.get(), sp, st.get(), rank.get(), a1.get()); note_launch(); }
  F.agg.alloc(n, s);
  bad.alloc(1, s);
  bad.zero(s);
  { agg_phase2<<<g, 256, 0, s>>>(n, F.A.rp.get(), F.A.ci.get(), sp, a1.get(), F.agg.get(), bad.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  int32_t hb = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&hb, bad.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  GIAMG_CHECK(hb == 0, GIAMG_ERR_ARG, "aggregation left a node without a phase-1 neighbour");
  F.n_next = n_agg;
  return n_agg;
}

void h_level_prolongation(Level& F, cudaStream_t s) {
  const int64_t n = F.A.n;
  DCSR T;
  T.n = n;
  T.m = F.n_next;
  T.nnz = n;
  T.rp.alloc(n + 1, s);
  T.ci.alloc(std::max<int64_t>(n, 1), s);
  T.v.alloc(std::max<int64_t>(n, 1), s);
  { tentative<<<blocks_for(n + 1, 256, 65535), 256, 0, s>>>(n, F.agg.get(), T.rp.get(), T.ci.get(), T.v.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  spgemm(F.A, T, F.P, s);  // A T
  DBuf<int32_t> bad;
  bad.alloc(1, s);
  bad.zero(s);
  { sa_smooth<<<blocks_for(n, 256, 65535), 256, 0, s>>>(n, F.A.rp.get(), F.A.ci.get(), F.A.v.get(), F.agg.get(),
                                                       F.P.rp.get(), F.P.ci.get(), F.P.v.get(), bad.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  int32_t hb = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&hb, bad.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  GIAMG_CHECK(hb == 0, GIAMG_ERR_NOT_SPD, "smoothed prolongation: a row of A T misses its own aggregate");
  csr_to32(F.P, s);
}

int64_t validate_map(const DCSR& A, const int32_t* l2g, int32_t n_elem, int nloc, cudaStream_t s) {
  DBuf<unsigned long long> bad;
  bad.alloc(1, s);
  bad.zero(s);
  int np2 = 1;
  while (np2 < nloc) np2 <<= 1;
  const size_t sm = (size_t)(np2 + nloc) * sizeof(int32_t);
  static PerDevice attr;  // the largest element: (GIAMG_MAX_ORDER + 1)^3 nodes
  attr.once([&] {
    GIAMG_CUDA(cudaFuncSetAttribute(validate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)((4096 + 13 * 13 * 13) * sizeof(int32_t))));
  });
  if (n_elem > 0) {
    validate_kernel<<<n_elem, kValThreads, sm, s>>>(A.n, A.rp.get(), A.ci.get(), l2g, nloc, np2, bad.get());
    note_launch();
  }
  GIAMG_CUDA(cudaGetLastError());
  unsigned long long h = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&h, bad.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  return (int64_t)h;
}

void csr_to_dense_cm(const DCSR& A, double* D, cudaStream_t s) {
  GIAMG_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * A.n * A.n, s));
  { dense_cm<<<blocks_for(A.n, 256, 65535), 256, 0, s>>>(A.n, A.rp.get(), A.ci.get(), A.v.get(), D); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

}  // namespace giamg
