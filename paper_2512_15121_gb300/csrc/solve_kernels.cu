// solve_kernels.cu -- kernels of one GIAMG-PCG iteration (Sec. 2, Algorithm 1):
//   CSR SpMV / residual / fused Jacobi-Chebyshev step on every level,
//   p-level restriction and prolongation as element contractions (Algorithms 2-4, 7 in
//   element form: one 1D interpolation table applied along the three directions),
//   h-level transfers as CSR products, the coarsest-level Cholesky solves, and the
//   deterministic reductions and vector updates of the outer conjugate gradients.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace giamg {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  return (unsigned)std::max<int64_t>(g, 1);
}

// ------------------------------------------------------------------ CSR row kernels
// TPR threads cooperate on one row; the group's partial sums are combined with shuffles.

template <int TPR, typename V, int MODE>
__global__ void __launch_bounds__(kThreads) csr_rows(int64_t n, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ ci, const V* __restrict__ val,
                                                     const V* __restrict__ x, const V* __restrict__ b,
                                                     V* __restrict__ y, V* __restrict__ d,
                                                     const V* __restrict__ dinv, V c1, V c2) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = gt / TPR;
  const int lane = threadIdx.x % TPR;
  const bool valid = row < n;
  V acc0 = 0, acc1 = 0;
  if (valid) {
    const int64_t s = rp[row], e = rp[row + 1];
    int64_t t = s + lane;
    for (; t + TPR < e; t += 2 * TPR) {
      acc0 = fma(__ldcs(val + t), x[__ldcs(ci + t)], acc0);
      acc1 = fma(__ldcs(val + t + TPR), x[__ldcs(ci + t + TPR)], acc1);
    }
    if (t < e) acc0 = fma(__ldcs(val + t), x[__ldcs(ci + t)], acc0);
  }
  V acc = acc0 + acc1;
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, TPR);
  if (!valid || lane != 0) return;
  if (MODE == kSpmv) {
    y[row] = acc;
  } else if (MODE == kAddSpmv) {
    y[row] += acc;
  } else if (MODE == kResidual) {
    y[row] = b[row] - acc;
  } else {  // Chebyshev step
    const V r = b[row] - acc;
    const V dn = (c1 == V(0) ? V(0) : c1 * d[row]) + c2 * dinv[row] * r;
    d[row] = dn;
    y[row] = x[row] + dn;
  }
}

// Prefetch the bytes [lo, hi) of an array into L2 with one bulk request: lo and hi are widened to
// 16-byte boundaries, hi clipped to `end` (the array's size rounded down to 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void* base, int64_t lo, int64_t hi, int64_t end) {
  lo &= ~(int64_t)15;
  hi = min((hi + 15) & ~(int64_t)15, end);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const char*>(base) + lo),
                 "r"((uint32_t)(hi - lo))
                 : "memory");
}

// Row kernels on a pattern-compressed matrix: the columns of row i are i + off[k] for the
// offsets of the row's template, which stay in L1/L2 while the values stream from HBM.
// TPR threads per row; consecutive threads take consecutive entries, so the x gathers of one
// instruction fall in a few runs of neighbouring columns.
//
// Blocks start roughly in row order, so with pf > 0 the first thread of every block prefetches
// into L2 (one bulk request) the values of the block pf rows ahead: by the time that block runs,
// its value loads wait on L2 instead of HBM.
template <int TPR, int U, typename V, int MODE, bool LIST = false>
__device__ __forceinline__ void pat_body(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ obase,
                                         const int32_t* __restrict__ toff,
                                         const V* __restrict__ val, const V* __restrict__ x, const V* __restrict__ b,
                                         V* __restrict__ y, V* __restrict__ d, const V* __restrict__ dinv, V c1, V c2,
                                         int64_t pf, int64_t vend, const int32_t* __restrict__ list = nullptr,
                                         int64_t block0 = 0) {
  // LIST: the group of threads t takes row list[t] of the n listed rows; block0: blocks before
  // this one that do other work in the same launch
  const int64_t gt = ((int64_t)blockIdx.x - block0) * blockDim.x + threadIdx.x;
  const int64_t idx = gt / TPR;
  const int lane = threadIdx.x % TPR;
  const bool valid = idx < n;
  const int64_t row = LIST ? (valid ? (int64_t)list[idx] : 0) : idx;
  if (pf > 0 && threadIdx.x == 0) {
    const int64_t rows = blockDim.x / TPR;
    const int64_t r0 = (int64_t)blockIdx.x * rows + pf;
    if (r0 < n) prefetch_l2(val, rp[r0] * (int64_t)sizeof(V), rp[min(r0 + rows, n)] * (int64_t)sizeof(V), vend);
  }
  V acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = 0;
  if (valid) {
    const int64_t s = rp[row];
    const int len = (int)(rp[row + 1] - s);
    const int32_t* __restrict__ off = toff + obase[row];
    const V* __restrict__ vr = val + s;
    const V* __restrict__ xr = x + row;
    int k = lane;
    if constexpr (U == 2) {
      for (; k + TPR < len; k += 2 * TPR) {
        acc[0] = fma(__ldcs(vr + k), xr[__ldg(off + k)], acc[0]);
        acc[1] = fma(__ldcs(vr + k + TPR), xr[__ldg(off + k + TPR)], acc[1]);
      }
      if (k < len) acc[0] = fma(__ldcs(vr + k), xr[__ldg(off + k)], acc[0]);
    } else {
      // U independent (offset -> gather -> fma) chains per step, the last step predicated: all
      // U offsets and values are requested before the gathers, so U latencies overlap
      for (; k < len; k += U * TPR) {
        int o[U];
        V v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool in = k + u * TPR < len;
          o[u] = in ? __ldg(off + k + u * TPR) : 0;
          v[u] = in ? __ldcs(vr + k + u * TPR) : V(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = fma(v[u], xr[o[u]], acc[u]);
      }
    }
  }
#pragma unroll
  for (int u = 1; u < U; ++u) acc[0] += acc[u];
  V a = acc[0];
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o, TPR);
  if (!valid || lane != 0) return;
  if (MODE == kSpmv) {
    y[row] = a;
  } else if (MODE == kAddSpmv) {
    y[row] += a;
  } else if (MODE == kResidual) {
    y[row] = b[row] - a;
  } else {
    const V r = b[row] - a;
    const V dn = (c1 == V(0) ? V(0) : c1 * d[row]) + c2 * dinv[row] * r;
    d[row] = dn;
    y[row] = x[row] + dn;
  }
}

#define PAT_KERNEL(NAME, V, MODE)                                                                              \
  template <int TPR, int U>                                                                                   \
  __global__ void __launch_bounds__(kThreads)                                                                 \
      NAME(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ obase,                      \
           const int32_t* __restrict__ toff, const V* __restrict__ val,     \
           const V* __restrict__ x, const V* __restrict__ b, V* __restrict__ y, V* __restrict__ d,            \
           const V* __restrict__ dinv, V c1, V c2, int64_t pf, int64_t vend) {                                \
    pat_body<TPR, U, V, MODE>(n, rp, obase, toff, val, x, b, y, d, dinv, c1, c2, pf, vend);              \
  }
PAT_KERNEL(pat_spmv_f64, double, kSpmv)
PAT_KERNEL(pat_spmv_f32, float, kSpmv)
PAT_KERNEL(pat_resid_f64, double, kResidual)
PAT_KERNEL(pat_resid_f32, float, kResidual)
PAT_KERNEL(pat_cheb_f64, double, kCheb)
PAT_KERNEL(pat_cheb_f32, float, kCheb)
PAT_KERNEL(pat_add_f64, double, kAddSpmv)
PAT_KERNEL(pat_add_f32, float, kAddSpmv)

template <typename V, int MODE>
struct PatKernel;
#define PAT_SELECT(V, MODE, NAME)                                                  \
  template <>                                                                     \
  struct PatKernel<V, MODE> {                                                     \
    template <int TPR, int U>                                                     \
    static constexpr decltype(&NAME<TPR, U>) get() { return &NAME<TPR, U>; }     \
  };
PAT_SELECT(double, kSpmv, pat_spmv_f64)
PAT_SELECT(float, kSpmv, pat_spmv_f32)
PAT_SELECT(double, kResidual, pat_resid_f64)
PAT_SELECT(float, kResidual, pat_resid_f32)
PAT_SELECT(double, kCheb, pat_cheb_f64)
PAT_SELECT(float, kCheb, pat_cheb_f32)
PAT_SELECT(double, kAddSpmv, pat_add_f64)
PAT_SELECT(float, kAddSpmv, pat_add_f32)

// The hybrid form in one launch.  Blocks 0 .. n_big-1 take the big row groups: one CTA per group
// gathers the group's x values into shared memory once; every warp then takes rows of the group,
// and each lane issues the loads of 8 of the row's values (stride 32) before their products, so
// a warp keeps 8 x 128 bytes of the value stream in flight with no dependent load in between.
// The later blocks run the row-pattern kernel over the list of the other rows; they start after
// the group blocks and fill the tail of the launch.
template <typename V, int MODE>
__device__ __forceinline__ void hyb_body(const int32_t* __restrict__ big, const int64_t* __restrict__ gptr,
                                         const int32_t* __restrict__ gcol, const int64_t* __restrict__ rptr,
                                         const int32_t* __restrict__ grow, const int64_t* __restrict__ rp,
                                         const V* __restrict__ val, const V* __restrict__ x, const V* __restrict__ b,
                                         V* __restrict__ y, V* __restrict__ d, const V* __restrict__ dinv, V c1, V c2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xs = reinterpret_cast<V*>(smem_raw);
  const int64_t g = big[blockIdx.x];
  const int64_t c0 = gptr[g];
  const int c = (int)(gptr[g + 1] - c0);
  for (int k = threadIdx.x; k < c; k += blockDim.x) xs[k] = x[__ldg(gcol + c0 + k)];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t t_end = rptr[g + 1];
  for (int64_t t = rptr[g] + warp; t < t_end; t += nw) {
    const int64_t row = grow[t];
    const V* __restrict__ vr = val + rp[row];
    V a[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < c; k0 += 256) {
      V v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int kk = k0 + lane + 32 * u;
        v[u] = kk < c ? __ldcs(vr + kk) : V(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int kk = k0 + lane + 32 * u;
        a[u & 3] = fma(v[u], xs[kk < c ? kk : 0], a[u & 3]);
      }
    }
    V acc = (a[0] + a[1]) + (a[2] + a[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane != 0) continue;
    if (MODE == kSpmv) {
      y[row] = acc;
    } else if (MODE == kAddSpmv) {
      y[row] += acc;
    } else if (MODE == kResidual) {
      y[row] = b[row] - acc;
    } else {
      const V r = b[row] - acc;
      const V dn = (c1 == V(0) ? V(0) : c1 * d[row]) + c2 * dinv[row] * r;
      d[row] = dn;
      y[row] = x[row] + dn;
    }
  }
}

#define HYB_KERNEL(NAME, V, MODE)                                                                              \
  __global__ void __launch_bounds__(kThreads)                                                                 \
      NAME(int64_t n_big, const int32_t* __restrict__ big, const int64_t* __restrict__ gptr,                  \
           const int32_t* __restrict__ gcol, const int64_t* __restrict__ rptr, const int32_t* __restrict__ grow, \
           int64_t n_rest, const int32_t* __restrict__ rest, const int32_t* __restrict__ obase,               \
           const int32_t* __restrict__ toff, const int64_t* __restrict__ rp, const V* __restrict__ val,       \
           const V* __restrict__ x, const V* __restrict__ b, V* __restrict__ y, V* __restrict__ d,            \
           const V* __restrict__ dinv, V c1, V c2) {                                                          \
    if ((int64_t)blockIdx.x < n_big)                                                                          \
      hyb_body<V, MODE>(big, gptr, gcol, rptr, grow, rp, val, x, b, y, d, dinv, c1, c2);                     \
    else                                                                                                      \
      pat_body<32, 2, V, MODE, true>(n_rest, rp, obase, toff, val, x, b, y, d, dinv, c1, c2, 0, 0, rest, n_big); \
  }
HYB_KERNEL(hyb_spmv_f64, double, kSpmv)
HYB_KERNEL(hyb_spmv_f32, float, kSpmv)
HYB_KERNEL(hyb_resid_f64, double, kResidual)
HYB_KERNEL(hyb_resid_f32, float, kResidual)
HYB_KERNEL(hyb_cheb_f64, double, kCheb)
HYB_KERNEL(hyb_cheb_f32, float, kCheb)
HYB_KERNEL(hyb_add_f64, double, kAddSpmv)
HYB_KERNEL(hyb_add_f32, float, kAddSpmv)

template <typename V, int MODE>
struct HybKernel;
#define HYB_SELECT(V, MODE, H)                           \
  template <>                                           \
  struct HybKernel<V, MODE> {                           \
    static constexpr decltype(&H) get() { return &H; }  \
  };
HYB_SELECT(double, kSpmv, hyb_spmv_f64)
HYB_SELECT(float, kSpmv, hyb_spmv_f32)
HYB_SELECT(double, kResidual, hyb_resid_f64)
HYB_SELECT(float, kResidual, hyb_resid_f32)
HYB_SELECT(double, kCheb, hyb_cheb_f64)
HYB_SELECT(float, kCheb, hyb_cheb_f32)
HYB_SELECT(double, kAddSpmv, hyb_add_f64)
HYB_SELECT(float, kAddSpmv, hyb_add_f32)

// ------------------------------------------------------------------ vector hybrid form (FP32)
// The hybrid form with the big groups read from a group-major copy of the FP32 values (hv): a
// group is one contiguous block and every row starts on 16 bytes (rows padded with zeros to a
// multiple of 4 values), so the warp of a row loads it with float4 loads, 4 per lane at once,
// from a sequential stream: one step covers a row of 344 padded values (86 float4 of 128
// slots), two a row of 640.  Against hyb_body's 4-byte loads from rows scattered over the value
// array this doubles the bytes a warp has in flight with the same 32 registers.  A warp leaves
// each row's sum in shared memory and goes on to its next row; after a barrier the block's
// threads finish all rows of the group at once (the step's reads of b, d, D^-1 and x and its
// writes), so the group pays that dependent latency once instead of once per row (4% per launch
// on 16^3 p = 6).  The other rows run the row-pattern kernel in the same launch, as in
// hyb_body's kernel.
template <typename V>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int kU = 4;
  static __device__ __forceinline__ T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void fma4(const T& v, const T& x, float* a) {
    a[0] = fmaf(v.x, x.x, a[0]);
    a[1] = fmaf(v.y, x.y, a[1]);
    a[2] = fmaf(v.z, x.z, a[2]);
    a[3] = fmaf(v.w, x.w, a[3]);
  }
};
template <>
struct Vec16<double> {
  using T = double2;
  static __device__ __forceinline__ T zero() { return make_double2(0.0, 0.0); }
  // alternate accumulator pairs between consecutive vectors: four FMA chains per lane
  static __device__ __forceinline__ void fma4(const T& v, const T& x, double* a, int u) {
    a[2 * (u & 1)] = fma(v.x, x.x, a[2 * (u & 1)]);
    a[2 * (u & 1) + 1] = fma(v.y, x.y, a[2 * (u & 1) + 1]);
  }
};
template <typename V, int MODE>
__device__ __forceinline__ void hyv_body(const int32_t* __restrict__ big, const int64_t* __restrict__ gptr,
                                         const int32_t* __restrict__ gcol, const int64_t* __restrict__ rptr,
                                         const int32_t* __restrict__ grow, const int64_t* __restrict__ hoff,
                                         const V* __restrict__ hv, const V* __restrict__ x,
                                         const V* __restrict__ b, V* __restrict__ y, V* __restrict__ d,
                                         const V* __restrict__ dinv, V c1, V c2, int cpmax) {
  using VT = typename Vec16<V>::T;
  constexpr int EV = 16 / sizeof(V), U = Vec16<V>::kU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xs = reinterpret_cast<V*>(smem_raw);
  V* sums = xs + cpmax;  // after the widest padded x list: one sum per row of the group
  const int64_t j = blockIdx.x;
  const int64_t g = big[j];
  const int64_t c0 = gptr[g];
  const int c = (int)(gptr[g + 1] - c0);
  const int cp = (c + 3) & ~3, nq = cp / EV;
  const int64_t t0 = rptr[g];
  const int rows = (int)(rptr[g + 1] - t0);
  const V* src = hv + hoff[j];
  for (int k = threadIdx.x; k < cp; k += blockDim.x) xs[k] = k < c ? x[__ldg(gcol + c0 + k)] : V(0);
  __syncthreads();
  const VT* xq = reinterpret_cast<const VT*>(xs);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = warp; t < rows; t += nw) {
    const VT* vr = reinterpret_cast<const VT*>(src + (int64_t)t * cp);
    V a[4] = {V(0), V(0), V(0), V(0)};
    for (int q0 = 0; q0 < nq; q0 += 32 * U) {
      VT v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + lane + 32 * u;
        v[u] = q < nq ? __ldcs(vr + q) : Vec16<V>::zero();
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + lane + 32 * u;
        Vec16<V>::fma4(v[u], xq[q < nq ? q : 0], a);  // a padded slot multiplies zeros
      }
    }
    V acc = (a[0] + a[1]) + (a[2] + a[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sums[t] = acc;
  }
  // the rows' epilogues together: one latency for the group instead of one per row
  __syncthreads();
  for (int t = threadIdx.x; t < rows; t += blockDim.x) {
    const V acc = sums[t];
    const int64_t row = grow[t0 + t];
    if (MODE == kSpmv) {
      y[row] = acc;
    } else if (MODE == kAddSpmv) {
      y[row] += acc;
    } else if (MODE == kResidual) {
      y[row] = b[row] - acc;
    } else {
      const V rr = b[row] - acc;
      const V dn = (c1 == V(0) ? V(0) : c1 * d[row]) + c2 * dinv[row] * rr;
      d[row] = dn;
      y[row] = x[row] + dn;
    }
  }
}

#define HYV_KERNEL(NAME, V, MODE)                                                                               \
  __global__ void __launch_bounds__(kThreads)                                                                 \
      NAME(int64_t n_big, const int32_t* __restrict__ big, const int64_t* __restrict__ gptr,                  \
           const int32_t* __restrict__ gcol, const int64_t* __restrict__ rptr, const int32_t* __restrict__ grow, \
           const int64_t* __restrict__ hoff, const V* __restrict__ hv,                                       \
           int64_t n_rest, const int32_t* __restrict__ rest, const int32_t* __restrict__ obase,               \
           const int32_t* __restrict__ toff, const int64_t* __restrict__ rp, const V* __restrict__ val,       \
           const V* __restrict__ x, const V* __restrict__ b, V* __restrict__ y, V* __restrict__ d,            \
           const V* __restrict__ dinv, V c1, V c2, int cpmax) {                                               \
    if ((int64_t)blockIdx.x < n_big)                                                                          \
      hyv_body<V, MODE>(big, gptr, gcol, rptr, grow, hoff, hv, x, b, y, d, dinv, c1, c2, cpmax);             \
    else                                                                                                      \
      pat_body<32, 2, V, MODE, true>(n_rest, rp, obase, toff, val, x, b, y, d, dinv, c1, c2, 0, 0, rest, n_big); \
  }
HYV_KERNEL(hyv_spmv_f32, float, kSpmv)
HYV_KERNEL(hyv_resid_f32, float, kResidual)
HYV_KERNEL(hyv_cheb_f32, float, kCheb)
HYV_KERNEL(hyv_add_f32, float, kAddSpmv)

template <typename V, int MODE>
struct HyvKernel;
#define HYV_SELECT(V, MODE, H)                          \
  template <>                                           \
  struct HyvKernel<V, MODE> {                           \
    static constexpr decltype(&H) get() { return &H; }  \
  };
HYV_SELECT(float, kSpmv, hyv_spmv_f32)
HYV_SELECT(float, kResidual, hyv_resid_f32)
HYV_SELECT(float, kCheb, hyv_cheb_f32)
HYV_SELECT(float, kAddSpmv, hyv_add_f32)

// ------------------------------------------------------------------ vector hybrid form (FP64)
// FP64 rows are bound by the FP64 pipe, which also executes the adds of a shuffle reduction as
// full-warp instructions: with 16 or 32 lanes per row they cost 4 or 5 FP64 instructions per row
// on top of about 11-22 FMAs, and two rows of different lengths in one warp leave lanes idle.
// Here the big groups (from the group-major FP64 copy hv64) take 4 lanes per row and 8 rows of
// one group per warp: every row of a group has the same length, so no lane waits on another
// row; the reduction is 2 shuffle levels; each lane loads the row's values with 16-byte loads,
// U at once; and the 8 rows read the same x words from shared memory (broadcasts).
template <typename V, int MODE>
__device__ __forceinline__ void hy4_body(const int32_t* __restrict__ big, const int64_t* __restrict__ gptr,
                                         const int32_t* __restrict__ gcol, const int64_t* __restrict__ rptr,
                                         const int32_t* __restrict__ grow, const int64_t* __restrict__ hoff,
                                         const V* __restrict__ hv, const V* __restrict__ x,
                                         const V* __restrict__ b, V* __restrict__ y, V* __restrict__ d,
                                         const V* __restrict__ dinv, V c1, V c2) {
  using VT = typename Vec16<V>::T;
  constexpr int EV = 16 / sizeof(V), U = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xs = reinterpret_cast<V*>(smem_raw);
  const int64_t j = blockIdx.x;
  const int64_t g = big[j];
  const int64_t c0 = gptr[g];
  const int c = (int)(gptr[g + 1] - c0);
  const int cp = (c + 3) & ~3, nq = cp / EV;  // 16-byte vectors per padded row
  const int64_t t0 = rptr[g];
  const int rows = (int)(rptr[g + 1] - t0);
  const V* src = hv + hoff[j];
  for (int k = threadIdx.x; k < cp; k += blockDim.x) xs[k] = k < c ? x[__ldg(gcol + c0 + k)] : V(0);
  __syncthreads();
  const VT* xq = reinterpret_cast<const VT*>(xs);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int sub = lane & 3, rw = lane >> 2;
  for (int tb = warp * 8; tb < rows; tb += nw * 8) {
    const int t = tb + rw;
    const bool valid = t < rows;
    const VT* vr = reinterpret_cast<const VT*>(src + (int64_t)(valid ? t : tb) * cp);
    V a[4] = {V(0), V(0), V(0), V(0)};
    for (int q0 = sub; q0 < nq; q0 += 4 * U) {
      VT v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + 4 * u;
        v[u] = q < nq ? __ldcs(vr + q) : Vec16<V>::zero();
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + 4 * u;
        Vec16<V>::fma4(v[u], xq[q < nq ? q : 0], a, u);  // a padded slot multiplies zeros
      }
    }
    V acc = (a[0] + a[1]) + (a[2] + a[3]);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (!valid || sub != 0) continue;
    const int64_t row = grow[t0 + t];
    if (MODE == kSpmv) {
      y[row] = acc;
    } else if (MODE == kAddSpmv) {
      y[row] += acc;
    } else if (MODE == kResidual) {
      y[row] = b[row] - acc;
    } else {
      const V rr = b[row] - acc;
      const V dn = (c1 == V(0) ? V(0) : c1 * d[row]) + c2 * dinv[row] * rr;
      d[row] = dn;
      y[row] = x[row] + dn;
    }
  }
}

#define HY4_KERNEL(NAME, V, MODE, REST)                                                                        \
  __global__ void __launch_bounds__(kThreads)                                                                 \
      NAME(int64_t n_big, const int32_t* __restrict__ big, const int64_t* __restrict__ gptr,                  \
           const int32_t* __restrict__ gcol, const int64_t* __restrict__ rptr, const int32_t* __restrict__ grow, \
           const int64_t* __restrict__ hoff, const V* __restrict__ hv, int64_t n_rest,                        \
           const int32_t* __restrict__ rest, const int32_t* __restrict__ obase, const int32_t* __restrict__ toff, \
           const int64_t* __restrict__ rp, const V* __restrict__ val, const V* __restrict__ x,                \
           const V* __restrict__ b, V* __restrict__ y, V* __restrict__ d, const V* __restrict__ dinv, V c1,    \
           V c2) {                                                                                            \
    if ((int64_t)blockIdx.x < n_big)                                                                          \
      hy4_body<V, MODE>(big, gptr, gcol, rptr, grow, hoff, hv, x, b, y, d, dinv, c1, c2);                    \
    else                                                                                                      \
      pat_body<REST, 2, V, MODE, true>(n_rest, rp, obase, toff, val, x, b, y, d, dinv, c1, c2, 0, 0, rest, n_big); \
  }
HY4_KERNEL(hy4_spmv_f64, double, kSpmv, 16)
HY4_KERNEL(hy4_resid_f64, double, kResidual, 16)
HY4_KERNEL(hy4_cheb_f64, double, kCheb, 16)
HY4_KERNEL(hy4_add_f64, double, kAddSpmv, 16)

// ------------------------------------------------------------------ sliced form (one lane per row)
// Every row of the level, in slices of 32 rows of (nearly) equal length (rows ordered by length,
// then group): a warp takes a slice and each lane one row, so the FP64 pipe executes one useful
// FMA per lane per instruction -- no shuffle reduction, no half-empty warp at the end of a
// 25-row face group (the slices mix the rows of several groups), and the per-row work after the
// sum is one instruction for 32 rows.  A lane reads W consecutive values of its row with one
// 16-byte load (the warp: 512 contiguous bytes); its column indices come from its group's list
// (shared with the group's other rows, so mostly one address per warp) and x from L1/L2.  The
// loop is software-pipelined: the next step's column indices and values are requested before
// this step's FMAs, so every lane keeps one dependent index -> x gather and two steps of value
// loads in flight (up to 64 registers, 4 CTAs per SM).  Measured per launch on the 16^3 p = 6
// operator against the vector hybrid: FP64 0.698 ms (1.18 TFLOP/s, 94% of the FP64 pipe's
// nominal rate) against 0.931, FP32 0.314 against 0.317; without the pipelining 1.32 / 0.54.
template <typename V>
struct SelVec;
template <>
struct SelVec<double> {
  using T = double2;
  static constexpr int W = 2;
  static __device__ __forceinline__ double at(const T& v, int i) { return i == 0 ? v.x : v.y; }
};
template <>
struct SelVec<float> {
  using T = float4;
  static constexpr int W = 4;
  static __device__ __forceinline__ float at(const T& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
};

template <typename V, int MODE, int K>
__device__ __forceinline__ void sel_body(int64_t n_slices, const int32_t* __restrict__ srow,
                                              const int32_t* __restrict__ sob, const int32_t* __restrict__ sclen,
                                              const int32_t* __restrict__ slen, const int64_t* __restrict__ sbase,
                                              const V* __restrict__ sv, const int32_t* __restrict__ gcol,
                                              const V* __restrict__ x, const V* __restrict__ b, V* __restrict__ y,
                                              V* __restrict__ d, const V* __restrict__ dinv, V c1, V c2) {
  using VT = typename SelVec<V>::T;
  constexpr int W = SelVec<V>::W, NV = K / W;
  const int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (sl >= n_slices) return;
  const int lane = threadIdx.x & 31;
  const int64_t li = sl * 32 + lane;
  const int row = srow[li];
  const int32_t* __restrict__ cl = gcol + sob[li];
  const int last = sclen[li] - 1;
  const int L = slen[sl];
  const VT* __restrict__ vp = reinterpret_cast<const VT*>(sv + sbase[sl]) + lane;
  V a[4] = {V(0), V(0), V(0), V(0)};
  int c[K];
  VT v[NV];
#pragma unroll
  for (int j = 0; j < K; ++j) c[j] = __ldg(cl + min(j, last));
#pragma unroll
  for (int u = 0; u < NV; ++u) v[u] = __ldcs(vp + (int64_t)u * 32);
  for (int k0 = 0; k0 < L; k0 += K) {
    V xv[K];
#pragma unroll
    for (int j = 0; j < K; ++j) xv[j] = __ldg(x + c[j]);
    VT vn[NV];
    const int kn = k0 + K < L ? k0 + K : k0;  // the last step reloads its own (unused) operands
#pragma unroll
    for (int j = 0; j < K; ++j) c[j] = __ldg(cl + min(kn + j, last));
#pragma unroll
    for (int u = 0; u < NV; ++u) vn[u] = __ldcs(vp + (int64_t)(kn / W + u) * 32);
#pragma unroll
    for (int j = 0; j < K; ++j) a[j & 3] = fma(SelVec<V>::at(v[j / W], j % W), xv[j], a[j & 3]);
#pragma unroll
    for (int u = 0; u < NV; ++u) v[u] = vn[u];
  }
  if (row < 0) return;
  const V acc = (a[0] + a[1]) + (a[2] + a[3]);
  if (MODE == kSpmv) {
    y[row] = acc;
  } else if (MODE == kAddSpmv) {
    y[row] += acc;
  } else if (MODE == kResidual) {
    y[row] = b[row] - acc;
  } else {
    const V rr = b[row] - acc;
    const V dn = (c1 == V(0) ? V(0) : c1 * d[row]) + c2 * dinv[row] * rr;
    d[row] = dn;
    y[row] = x[row] + dn;
  }
}

#define SEL_KERNEL(NAME, V, MODE)                                                                               \
  __global__ void __launch_bounds__(kThreads, 4)                                                              \
      NAME(int64_t n_slices, const int32_t* __restrict__ srow, const int32_t* __restrict__ sob,               \
           const int32_t* __restrict__ sclen, const int32_t* __restrict__ slen, const int64_t* __restrict__ sbase, \
           const V* __restrict__ sv, const int32_t* __restrict__ gcol, const V* __restrict__ x,              \
           const V* __restrict__ b, V* __restrict__ y, V* __restrict__ d, const V* __restrict__ dinv, V c1,    \
           V c2) {                                                                                            \
    sel_body<V, MODE, kSliceStep>(n_slices, srow, sob, sclen, slen, sbase, sv, gcol, x, b, y, d, dinv, c1, c2); \
  }
SEL_KERNEL(sel_spmv_f64, double, kSpmv)
SEL_KERNEL(sel_resid_f64, double, kResidual)
SEL_KERNEL(sel_cheb_f64, double, kCheb)
SEL_KERNEL(sel_add_f64, double, kAddSpmv)
SEL_KERNEL(sel_spmv_f32, float, kSpmv)
SEL_KERNEL(sel_resid_f32, float, kResidual)
SEL_KERNEL(sel_cheb_f32, float, kCheb)
SEL_KERNEL(sel_add_f32, float, kAddSpmv)

template <typename V, int MODE>
struct SelKernel;
#define SEL_SELECT(V, MODE, H)                          \
  template <>                                           \
  struct SelKernel<V, MODE> {                           \
    static constexpr decltype(&H) get() { return &H; }  \
  };
SEL_SELECT(double, kSpmv, sel_spmv_f64)
SEL_SELECT(double, kResidual, sel_resid_f64)
SEL_SELECT(double, kCheb, sel_cheb_f64)
SEL_SELECT(double, kAddSpmv, sel_add_f64)
SEL_SELECT(float, kSpmv, sel_spmv_f32)
SEL_SELECT(float, kResidual, sel_resid_f32)
SEL_SELECT(float, kCheb, sel_cheb_f32)
SEL_SELECT(float, kAddSpmv, sel_add_f32)

template <typename V, int MODE>
struct Hy4Kernel;
#define HY4_SELECT(V, MODE, H)                          \
  template <>                                           \
  struct Hy4Kernel<V, MODE> {                           \
    static constexpr decltype(&H) get() { return &H; }  \
  };
HY4_SELECT(double, kSpmv, hy4_spmv_f64)
HY4_SELECT(double, kResidual, hy4_resid_f64)
HY4_SELECT(double, kCheb, hy4_cheb_f64)
HY4_SELECT(double, kAddSpmv, hy4_add_f64)

// Row-group kernels: one CTA per group of rows with identical column sets; the group's x values
// are gathered once into shared memory, then every warp streams one row's values from HBM
// against them (consecutive lanes read consecutive shared words: no bank conflicts).
template <typename V, int MODE>
__device__ __forceinline__ void grp_body(const int64_t* __restrict__ gptr, const int32_t* __restrict__ gcol,
                                         const int64_t* __restrict__ rptr, const int32_t* __restrict__ grow,
                                         const int64_t* __restrict__ rp, const V* __restrict__ val,
                                         const V* __restrict__ x, const V* __restrict__ b, V* __restrict__ y,
                                         V* __restrict__ d, const V* __restrict__ dinv, V c1, V c2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xs = reinterpret_cast<V*>(smem_raw);
  const int64_t g = blockIdx.x;
  const int64_t c0 = gptr[g];
  const int c = (int)(gptr[g + 1] - c0);
  for (int k = threadIdx.x; k < c; k += blockDim.x) xs[k] = x[__ldg(gcol + c0 + k)];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t t = rptr[g] + warp; t < rptr[g + 1]; t += nw) {
    const int64_t row = grow[t];
    const V* __restrict__ vr = val + rp[row];
    V a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int k = lane;
    for (; k + 96 < c; k += 128) {
      a0 = fma(__ldcs(vr + k), xs[k], a0);
      a1 = fma(__ldcs(vr + k + 32), xs[k + 32], a1);
      a2 = fma(__ldcs(vr + k + 64), xs[k + 64], a2);
      a3 = fma(__ldcs(vr + k + 96), xs[k + 96], a3);
    }
    for (; k < c; k += 32) a0 = fma(__ldcs(vr + k), xs[k], a0);
    V a = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane != 0) continue;
    if (MODE == kSpmv) {
      y[row] = a;
    } else if (MODE == kAddSpmv) {
      y[row] += a;
    } else if (MODE == kResidual) {
      y[row] = b[row] - a;
    } else {
      const V r = b[row] - a;
      const V dn = (c1 == V(0) ? V(0) : c1 * d[row]) + c2 * dinv[row] * r;
      d[row] = dn;
      y[row] = x[row] + dn;
    }
  }
}

#define GRP_KERNEL(NAME, V, MODE)                                                                          \
  __global__ void __launch_bounds__(kThreads)                                                             \
      NAME(const int64_t* __restrict__ gptr, const int32_t* __restrict__ gcol, const int64_t* __restrict__ rptr, \
           const int32_t* __restrict__ grow, const int64_t* __restrict__ rp, const V* __restrict__ val,   \
           const V* __restrict__ x, const V* __restrict__ b, V* __restrict__ y, V* __restrict__ d,        \
           const V* __restrict__ dinv, V c1, V c2) {                                                      \
    grp_body<V, MODE>(gptr, gcol, rptr, grow, rp, val, x, b, y, d, dinv, c1, c2);                        \
  }
GRP_KERNEL(grp_spmv_f64, double, kSpmv)
GRP_KERNEL(grp_spmv_f32, float, kSpmv)
GRP_KERNEL(grp_resid_f64, double, kResidual)
GRP_KERNEL(grp_resid_f32, float, kResidual)
GRP_KERNEL(grp_cheb_f64, double, kCheb)
GRP_KERNEL(grp_cheb_f32, float, kCheb)
GRP_KERNEL(grp_add_f64, double, kAddSpmv)
GRP_KERNEL(grp_add_f32, float, kAddSpmv)

template <typename V, int MODE>
struct GrpKernel;
#define GRP_SELECT(V, MODE, NAME)                                      \
  template <>                                                         \
  struct GrpKernel<V, MODE> {                                         \
    static constexpr decltype(&NAME) get() { return &NAME; }         \
  };
GRP_SELECT(double, kSpmv, grp_spmv_f64)
GRP_SELECT(float, kSpmv, grp_spmv_f32)
GRP_SELECT(double, kResidual, grp_resid_f64)
GRP_SELECT(float, kResidual, grp_resid_f32)
GRP_SELECT(double, kCheb, grp_cheb_f64)
GRP_SELECT(float, kCheb, grp_cheb_f32)
GRP_SELECT(double, kAddSpmv, grp_add_f64)
GRP_SELECT(float, kAddSpmv, grp_add_f32)

template <typename V, int MODE>
void launch_grp(const DCSR& A, const V* val, const V* x, const V* b, V* y, V* d, const V* dinv, V c1, V c2,
                cudaStream_t s) {
  auto k = GrpKernel<V, MODE>::get();
  const size_t sm = sizeof(V) * (size_t)A.grp.cmax;
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)); });
  k<<<(unsigned)A.grp.n_groups, kThreads, sm, s>>>(A.grp.gptr.get(), A.grp.gcol.get(), A.grp.rptr.get(),
                                                   A.grp.grow.get(), A.rp.get(), val, x, b, y, d, dinv, c1, c2);
  note_launch();
}

template <typename V, int MODE>
void launch_hyb(const DCSR& A, const V* val, const V* x, const V* b, V* y, V* d, const V* dinv, V c1, V c2,
                cudaStream_t s) {
  auto k = HybKernel<V, MODE>::get();
  const size_t sm = sizeof(V) * (size_t)A.grp.cmax;
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)); });
  const int64_t rest_blocks = (A.grp.n_rest * 32 + kThreads - 1) / kThreads;
  k<<<(unsigned)(A.grp.n_big + rest_blocks), kThreads, sm, s>>>(
      A.grp.n_big, A.grp.big.get(), A.grp.gptr.get(), A.grp.gcol.get(), A.grp.rptr.get(), A.grp.grow.get(),
      A.grp.n_rest, A.grp.rest.get(), A.pat.obase.get(), A.pat.toff.get(), A.rp.get(), val, x, b, y, d, dinv, c1, c2);
  note_launch();
}

template <typename V, int MODE>
void launch_hyv(const DCSR& A, const V* val, const V* x, const V* b, V* y, V* d, const V* dinv, V c1, V c2,
                cudaStream_t s) {
  auto k = HyvKernel<V, MODE>::get();
  const size_t sm = (size_t)(A.grp.cpmax + A.grp.rmax) * sizeof(V);
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)); });
  const V* hv = A.grp.hv.get();
  // the listed rows' blocks (pat_body: 32 lanes per row) take rows at the block size used here
  const int threads = 32 * A.grp.hwarps;
  const int64_t rest_blocks = (A.grp.n_rest * 32 + threads - 1) / threads;
  k<<<(unsigned)(A.grp.n_big + rest_blocks), threads, sm, s>>>(
      A.grp.n_big, A.grp.big.get(), A.grp.gptr.get(), A.grp.gcol.get(), A.grp.rptr.get(), A.grp.grow.get(),
      A.grp.hoff.get(), hv, A.grp.n_rest, A.grp.rest.get(), A.pat.obase.get(), A.pat.toff.get(), A.rp.get(), val, x,
      b, y, d, dinv, c1, c2, A.grp.cpmax);
  note_launch();
}

template <typename V, int MODE>
void launch_sel(const DCSR& A, const V* sv, const V* x, const V* b, V* y, V* d, const V* dinv, V c1, V c2,
                cudaStream_t s) {
  auto k = SelKernel<V, MODE>::get();
  const Groups& R = A.grp;
  k<<<grid_for(R.n_slices * 32, kThreads), kThreads, 0, s>>>(R.n_slices, R.srow.get(), R.sob.get(), R.sclen.get(),
                                                            R.slen.get(), R.sbase.get(), sv, R.gcol.get(), x, b, y,
                                                            d, dinv, c1, c2);
  note_launch();
}

template <typename V, int MODE>  // V = double
void launch_hy4(const DCSR& A, const V* val, const V* x, const V* b, V* y, V* d, const V* dinv, V c1, V c2,
                cudaStream_t s) {
  auto k = Hy4Kernel<V, MODE>::get();
  const size_t sm = (size_t)A.grp.cpmax * sizeof(V);
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)); });
  const V* hv = A.grp.hv64.get();
  const int64_t rest_blocks = (A.grp.n_rest * 16 + kThreads - 1) / kThreads;
  k<<<(unsigned)(A.grp.n_big + rest_blocks), kThreads, sm, s>>>(
      A.grp.n_big, A.grp.big.get(), A.grp.gptr.get(), A.grp.gcol.get(), A.grp.rptr.get(), A.grp.grow.get(),
      A.grp.hoff.get(), hv, A.grp.n_rest, A.grp.rest.get(), A.pat.obase.get(), A.pat.toff.get(), A.rp.get(), val, x,
      b, y, d, dinv, c1, c2);
  note_launch();
}

template <int TPR, int U, typename V, int MODE>
void launch_pat(const DCSR& A, const V* val, const V* x, const V* b, V* y, V* d, const V* dinv, V c1, V c2,
                int64_t pf, cudaStream_t s) {
  const int64_t n = A.n;
  // L2 prefetches stay inside the level's own value arrays (other arrays: no prefetch)
  int64_t vend = 0;
  if ((const void*)val == (const void*)A.v32.get()) vend = (int64_t)(A.v32.n * sizeof(float)) & ~(int64_t)15;
  if ((const void*)val == (const void*)A.v.get()) vend = (int64_t)(A.v.n * sizeof(double)) & ~(int64_t)15;
  if (!vend) pf = 0;
  auto k = PatKernel<V, MODE>::template get<TPR, U>();
  k<<<grid_for(n * TPR, kThreads), kThreads, 0, s>>>(n, A.rp.get(), A.pat.obase.get(), A.pat.toff.get(), val, x, b, y,
                                                     d, dinv, c1, c2, pf, vend);
  note_launch();
}

template <int TPR, typename V, int MODE>
void launch_csr(const DCSR& A, const V* val, const V* x, const V* b, V* y, V* d, const V* dinv, V c1, V c2,
                cudaStream_t s) {
  const int64_t n = A.n;
  csr_rows<TPR, V, MODE><<<grid_for(n * TPR, kThreads), kThreads, 0, s>>>(n, A.rp.get(), A.ci.get(), val, x, b, y,
                                                                         d, dinv, c1, c2);
  note_launch();
}

// default threads per row from the average row length (before or without tuning)
inline int default_tpr(double avg) { return avg >= 48 ? 32 : avg >= 20 ? 16 : avg >= 8 ? 8 : 4; }

// threads per row for the automatic choice: about `per_lane` values per lane (fewer lanes per row
// mean fewer shuffle-reduction levels per row, which cost FP64 rows pipe time); a level whose
// rows then give fewer than 2^18 threads (under one wave of the GPU's 311,296) is latency-bound
// and keeps at least the lanes of the length rule default_tpr.  Measured in the solve: the 24^3
// p = 4 finest level (191 values per row) is fastest with 8 lanes per row in FP32 (16% faster
// solve than 32) and 4 in FP64; the 12^3 p = 8 p = 4-level (205) with 16; levels of a few
// thousand rows with the length rule.
inline int auto_tpr(int64_t n, double avg, double per_lane) {
  int t = 4;
  while (t < 32 && avg / t > per_lane) t *= 2;
  if ((double)n * t < (double)(1 << 18)) t = std::max(t, default_tpr(avg));
  return t;
}

template <typename V, int MODE>
void launch_variant(const DCSR& A, const RowVariant& var, double avg, const V* val, const V* x, const V* b, V* y, V* d,
                    const V* dinv, V c1, V c2, cudaStream_t s) {
  const int tpr = var.tpr ? var.tpr : default_tpr(avg);
  const bool pat = var.tpr ? var.pat : A.pat.on;
  if (var.sliced && A.grp.son) {
    if constexpr (std::is_same<V, float>::value) {
      if (A.grp.sv32on && val == A.v32.get()) {
        launch_sel<V, MODE>(A, A.grp.sv32.get(), x, b, y, d, dinv, c1, c2, s);
        GIAMG_CUDA(cudaGetLastError());
        return;
      }
    } else {
      if (A.grp.sv64on && val == A.v.get()) {
        launch_sel<V, MODE>(A, A.grp.sv64.get(), x, b, y, d, dinv, c1, c2, s);
        GIAMG_CUDA(cudaGetLastError());
        return;
      }
    }
  }
  bool vector = var.hybrid && var.vector && A.grp.hyb && A.pat.on;
  if constexpr (std::is_same<V, float>::value) vector = vector && A.grp.hvon && val == A.v32.get();
  else vector = vector && A.grp.hv64on && val == A.v.get();
  if (vector) {
    if constexpr (std::is_same<V, float>::value) launch_hyv<V, MODE>(A, val, x, b, y, d, dinv, c1, c2, s);
    else launch_hy4<V, MODE>(A, val, x, b, y, d, dinv, c1, c2, s);
  } else if (var.hybrid && A.grp.hyb && A.pat.on) {
    launch_hyb<V, MODE>(A, val, x, b, y, d, dinv, c1, c2, s);
  } else if (var.group && A.grp.on) {
    launch_grp<V, MODE>(A, val, x, b, y, d, dinv, c1, c2, s);
  } else if (pat && var.unroll == 8) {
    switch (tpr) {
      case 32: launch_pat<32, 8, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      case 16: launch_pat<16, 8, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      case 8: launch_pat<8, 8, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      default: launch_pat<4, 8, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
    }
  } else if (pat && var.unroll == 4) {
    switch (tpr) {
      case 32: launch_pat<32, 4, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      case 16: launch_pat<16, 4, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      case 8: launch_pat<8, 4, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      default: launch_pat<4, 4, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
    }
  } else if (pat) {
    switch (tpr) {
      case 32: launch_pat<32, 2, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      case 16: launch_pat<16, 2, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      case 8: launch_pat<8, 2, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
      default: launch_pat<4, 2, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, var.prefetch, s); break;
    }
  } else {
    switch (tpr) {
      case 32: launch_csr<32, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, s); break;
      case 16: launch_csr<16, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, s); break;
      case 8: launch_csr<8, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, s); break;
      default: launch_csr<4, V, MODE>(A, val, x, b, y, d, dinv, c1, c2, s); break;
    }
  }
  GIAMG_CUDA(cudaGetLastError());
}

template <typename V, int MODE>
void launch_rows(const DCSR& A, const V* val, const V* x, const V* b, V* y, V* d, const V* dinv, V c1, V c2,
                 cudaStream_t s, double avg) {
  if (A.n == 0) return;
  // the level's own values use its tuned variant; other matrices (P, R) take the default
  const bool own = val == (sizeof(V) == 8 ? (const V*)A.v.get() : (const V*)A.v32.get());
  RowVariant none;
  const RowVariant& var = own ? (sizeof(V) == 8 ? A.var64 : A.var32) : none;
  launch_variant<V, MODE>(A, var, avg, val, x, b, y, d, dinv, c1, c2, s);
}

// ------------------------------------------------------------------ element transfers
// Prolongation x_f += P e_c on a p-level: per element, gather the (q+1)^3 coarse values,
// interpolate to the (p+1)^3 fine nodes by three 1D passes with the table P1D[a][b]
// (Algorithm 7's nodal interpolation, sum-factorised), and write the fine dofs this element
// owns (the first element containing a dof owns it, as in the assembled P).
template <typename V>
__global__ void p_prolong_kernel(int32_t n_elem, int p, int q, const int32_t* __restrict__ l2g,
                                 const uint8_t* __restrict__ own, const int32_t* __restrict__ l2g_c,
                                 const V* __restrict__ p1d, const V* __restrict__ ec, V* __restrict__ xf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int n1 = p + 1, m1 = q + 1;
  const int nlf = n1 * n1 * n1, nlc = m1 * m1 * m1;
  V* T = sm;                  // n1 * m1
  V* u = T + n1 * m1;         // nlc
  V* t1 = u + nlc;            // m1 * m1 * n1
  V* t2 = t1 + m1 * m1 * n1;  // m1 * n1 * n1
  const int e = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n1 * m1; i += nt) T[i] = p1d[i];
  for (int b = tid; b < nlc; b += nt) u[b] = ec[l2g_c[(int64_t)e * nlc + b]];
  __syncthreads();
  for (int i = tid; i < m1 * m1 * n1; i += nt) {  // t1[b1][b2][a3]
    const int a3 = i % n1, b12 = i / n1;
    V s = 0;
    for (int b3 = 0; b3 < m1; ++b3) s += T[a3 * m1 + b3] * u[b12 * m1 + b3];
    t1[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < m1 * n1 * n1; i += nt) {  // t2[b1][a2][a3]
    const int a3 = i % n1, a2 = (i / n1) % n1, b1 = i / (n1 * n1);
    V s = 0;
    for (int b2 = 0; b2 < m1; ++b2) s += T[a2 * m1 + b2] * t1[(b1 * m1 + b2) * n1 + a3];
    t2[i] = s;
  }
  __syncthreads();
  for (int a = tid; a < nlf; a += nt) {
    const int64_t slot = (int64_t)e * nlf + a;
    if (!own[slot]) continue;
    const int a23 = a % (n1 * n1), a1 = a / (n1 * n1);
    V s = 0;
    for (int b1 = 0; b1 < m1; ++b1) s += T[a1 * m1 + b1] * t2[b1 * n1 * n1 + a23];
    xf[l2g[slot]] += s;
  }
}

// Restriction r_c = P^T r_f on a p-level, step 1: per element, the partial sums
// part[e][b] = sum over the fine dofs a the element owns of P_e[a][b] r_f[a].
template <typename V>
__global__ void p_restrict_kernel(int32_t n_elem, int p, int q, const int32_t* __restrict__ l2g,
                                  const uint8_t* __restrict__ own, const V* __restrict__ p1d,
                                  const V* __restrict__ rf, V* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int n1 = p + 1, m1 = q + 1;
  const int nlf = n1 * n1 * n1, nlc = m1 * m1 * m1;
  V* T = sm;                  // n1 * m1
  V* v = T + n1 * m1;         // nlf
  V* t1 = v + nlf;            // n1 * n1 * m1
  V* t2 = t1 + n1 * n1 * m1;  // n1 * m1 * m1
  const int e = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n1 * m1; i += nt) T[i] = p1d[i];
  for (int a = tid; a < nlf; a += nt) {
    const int64_t slot = (int64_t)e * nlf + a;
    v[a] = own[slot] ? rf[l2g[slot]] : V(0);
  }
  __syncthreads();
  for (int i = tid; i < n1 * n1 * m1; i += nt) {  // t1[a1][a2][b3]
    const int b3 = i % m1, a12 = i / m1;
    V s = 0;
    for (int a3 = 0; a3 < n1; ++a3) s += T[a3 * m1 + b3] * v[a12 * n1 + a3];
    t1[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < n1 * m1 * m1; i += nt) {  // t2[a1][b2][b3]
    const int b3 = i % m1, b2 = (i / m1) % m1, a1 = i / (m1 * m1);
    V s = 0;
    for (int a2 = 0; a2 < n1; ++a2) s += T[a2 * m1 + b2] * t1[(a1 * n1 + a2) * m1 + b3];
    t2[i] = s;
  }
  __syncthreads();
  for (int b = tid; b < nlc; b += nt) {
    const int b23 = b % (m1 * m1), b1 = b / (m1 * m1);
    V s = 0;
    for (int a1 = 0; a1 < n1; ++a1) s += T[a1 * m1 + b1] * t2[a1 * m1 * m1 + b23];
    part[(int64_t)e * nlc + b] = s;
  }
}

// step 2: every coarse dof sums its element partials in ascending element order
template <typename V>
__global__ void p_gather_kernel(int64_t nc, const int64_t* __restrict__ ptr, const int32_t* __restrict__ slot,
                                const V* __restrict__ part, V* __restrict__ rc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  V s = 0;
  for (int64_t t = ptr[c]; t < ptr[c + 1]; ++t) s += part[slot[t]];
  rc[c] = s;
}

template <typename V>
size_t prolong_smem(int p, int q) {
  const int n1 = p + 1, m1 = q + 1;
  return sizeof(V) * (size_t)(n1 * m1 + m1 * m1 * m1 + m1 * m1 * n1 + m1 * n1 * n1);
}
template <typename V>
size_t restrict_smem(int p, int q) {
  const int n1 = p + 1, m1 = q + 1;
  return sizeof(V) * (size_t)(n1 * m1 + n1 * n1 * n1 + n1 * n1 * m1 + n1 * m1 * m1);
}

// ------------------------------------------------------------------ coarsest level
// Right-looking Cholesky, column-major: step k scales column k, then updates the trailing
// lower triangle.  One launch pair per column; the pivot test writes a status word.
__global__ void chol_scale_col(double* L, int64_t nc, int64_t k, int* status) {
  __shared__ double piv;
  if (threadIdx.x == 0) {
    double d = L[k * nc + k];
    if (!(d > 0.0)) {
      *status = 1;
      d = 1.0;
    }
    piv = sqrt(d);
    L[k * nc + k] = piv;
  }
  __syncthreads();
  for (int64_t i = k + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x)
    L[k * nc + i] /= piv;
}
__global__ void chol_update(double* L, int64_t nc, int64_t k) {
  // columns j > k, rows i >= j: L[i][j] -= L[i][k] L[j][k]
  const int64_t m = nc - k - 1;
  const int64_t total = m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t jj = t / m, ii = t % m;
    if (ii < jj) continue;
    const int64_t j = k + 1 + jj, i = k + 1 + ii;
    L[j * nc + i] -= L[k * nc + i] * L[k * nc + j];
  }
}
__global__ void zero_upper(double* L, int64_t nc) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nc * nc; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / nc, i = t % nc;
    if (i < j) L[t] = 0.0;
  }
}

// L L^T x = b by forward substitution on the columns of L and backward substitution on the
// rows of L (one CTA; every step updates the remaining entries in parallel).
template <typename V>
__global__ void chol_solve_kernel(const double* __restrict__ L, int64_t nc, const V* __restrict__ b, V* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* y = reinterpret_cast<double*>(smem_raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int64_t i = tid; i < nc; i += nt) y[i] = (double)b[i];
  __syncthreads();
  for (int64_t k = 0; k < nc; ++k) {
    const double yk = y[k] / L[k * nc + k];
    for (int64_t i = k + 1 + tid; i < nc; i += nt) y[i] -= L[k * nc + i] * yk;
    __syncthreads();
    if (tid == 0) y[k] = yk;
    __syncthreads();
  }
  for (int64_t k = nc - 1; k >= 0; --k) {
    const double xk = y[k] / L[k * nc + k];
    for (int64_t i = tid; i < k; i += nt) y[i] -= L[i * nc + k] * xk;
    __syncthreads();
    if (tid == 0) y[k] = xk;
    __syncthreads();
  }
  for (int64_t i = tid; i < nc; i += nt) x[i] = (V)y[i];
}

// A^-1 from the Cholesky factor: block j applies the forward and backward substitutions of
// chol_solve_kernel to the unit vector e_j and stores column j of the inverse (column-major).
__global__ void chol_inverse_kernel(const double* __restrict__ L, int64_t nc, double* __restrict__ Ainv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* y = reinterpret_cast<double*>(smem_raw);
  const int64_t j = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int64_t i = tid; i < nc; i += nt) y[i] = i == j ? 1.0 : 0.0;
  __syncthreads();
  for (int64_t k = j; k < nc; ++k) {  // entries above j stay zero in the forward sweep
    const double yk = y[k] / L[k * nc + k];
    for (int64_t i = k + 1 + tid; i < nc; i += nt) y[i] -= L[k * nc + i] * yk;
    __syncthreads();
    if (tid == 0) y[k] = yk;
    __syncthreads();
  }
  for (int64_t k = nc - 1; k >= 0; --k) {
    const double xk = y[k] / L[k * nc + k];
    for (int64_t i = tid; i < k; i += nt) y[i] -= L[i * nc + k] * xk;
    __syncthreads();
    if (tid == 0) y[k] = xk;
    __syncthreads();
  }
  for (int64_t i = tid; i < nc; i += nt) Ainv[j * nc + i] = y[i];
}

// x = A^-1 b with the explicit inverse (symmetric, so its columns are its rows): one warp per row
template <typename V>
__global__ void dense_inverse_apply(const double* __restrict__ Ainv, int64_t nc, const V* __restrict__ b,
                                    V* __restrict__ x) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  if (row < nc)
    for (int64_t k = lane; k < nc; k += 32) s += Ainv[row * nc + k] * (double)b[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (row < nc && lane == 0) x[row] = (V)s;
}

// ------------------------------------------------------------------ reductions and vectors
__device__ __forceinline__ double block_sum(double v, double* sh) {
  // fixed-shape tree: warp shuffles, then warp leaders through shared memory
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kRedThreads) dot_kernel(int64_t n, const double* __restrict__ x,
                                                          const double* __restrict__ y, double* partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// two dots in one pass: <r, z> and, for flexible CG, <z, r - rold>
__global__ void __launch_bounds__(kRedThreads) dot_rz_kernel(int64_t n, const double* __restrict__ r,
                                                             const double* __restrict__ z,
                                                             const double* __restrict__ rold, int flexible,
                                                             double* partial) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = z[i], ri = r[i];
    s0 += ri * zi;
    if (flexible) s1 += zi * (ri - rold[i]);
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s0;
    partial[kRedBlocks + blockIdx.x] = s1;
  }
}

// sum of kRedBlocks partials by one block in a fixed order
__device__ double sum_partials(const double* partial, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) v += partial[i];
  return block_sum(v, sh);
}

__global__ void reduce_kernel(const double* partial, double* out) {
  __shared__ double sh[32];
  const double v = sum_partials(partial, sh);
  if (threadIdx.x == 0) *out = v;
}

__global__ void finish_bb_kernel(Scalars* sc, const double* partial) {
  __shared__ double sh[32];
  const double v = sum_partials(partial, sh);
  if (threadIdx.x == 0) {
    sc->bb = v;
    sc->rr = v;
    sc->status = 0;
  }
}

__global__ void finish_rz_kernel(Scalars* sc, const double* partial, int first, int flexible) {
  __shared__ double sh[32];
  const double rz = sum_partials(partial, sh);
  const double zd = sum_partials(partial + kRedBlocks, sh);
  if (threadIdx.x == 0) {
    if (!(rz > 0.0) && sc->status == 0) sc->status = GIAMG_ERR_BREAKDOWN;
    if (first) {
      sc->beta = 0.0;
    } else {
      sc->beta = (flexible ? zd : rz) / sc->rho;
    }
    sc->rho_old = sc->rho;
    sc->rho = rz;
  }
}

__global__ void finish_pq_kernel(Scalars* sc, const double* partial) {
  __shared__ double sh[32];
  const double pq = sum_partials(partial, sh);
  if (threadIdx.x == 0) {
    sc->pq = pq;
    if (!(pq > 0.0) && sc->status == 0) sc->status = GIAMG_ERR_BREAKDOWN;
    sc->alpha = sc->rho / pq;
  }
}

__global__ void finish_rr_kernel(Scalars* sc, const double* partial) {
  __shared__ double sh[32];
  const double rr = sum_partials(partial, sh);
  if (threadIdx.x == 0) {
    sc->rr = rr;
    if (!(rr == rr) && sc->status == 0) sc->status = GIAMG_ERR_BREAKDOWN;
  }
}

__global__ void update_p_kernel(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                                const Scalars* __restrict__ sc, int first) {
  const double beta = first ? 0.0 : sc->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = first ? z[i] : z[i] + beta * p[i];
}

__global__ void __launch_bounds__(kRedThreads) update_xr_kernel(int64_t n, const double* __restrict__ p,
                                                                const double* __restrict__ q, double* __restrict__ x,
                                                                double* __restrict__ r, double* __restrict__ rold,
                                                                int flexible, const Scalars* __restrict__ sc,
                                                                double* partial) {
  __shared__ double sh[32];
  const double alpha = sc->alpha;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    if (flexible) rold[i] = ri;
    x[i] = x[i] + alpha * p[i];
    const double rn = ri - alpha * q[i];
    r[i] = rn;
    s += rn * rn;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void pcg_init_kernel(int64_t n, const double* __restrict__ b, double* __restrict__ x,
                                double* __restrict__ r, double* partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    s += bi * bi;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename V>
__global__ void cheb_first_kernel(int64_t n, const V* __restrict__ b, const V* __restrict__ dinv, V c2, V* __restrict__ x,
                                  V* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const V v = c2 * dinv[i] * b[i];
    d[i] = v;
    x[i] = v;
  }
}

__global__ void copy_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) y[i] = x[i];
}
__global__ void fill_kernel(int64_t n, double v, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) y[i] = v;
}
__global__ void axpy_kernel(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = y[i] + a * x[i];
}
__global__ void to32_kernel(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void to64_kernel(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
__global__ void add32_kernel(int64_t n, const float* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = y[i] + x[i];
}

inline unsigned vec_grid(int64_t n) { return (unsigned)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 16); }

}  // namespace

// ================================================================== launchers
__global__ void tune_fill(int64_t n, double* x64) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x64[i] = 1.0 + 1e-3 * (double)(i % 97);
}

void fill_tune_vector(int64_t n, double* x, cudaStream_t s) {
  if (n > 0) { tune_fill<<<vec_grid(n), 256, 0, s>>>(n, x); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

RowVariant variant_for(const DCSR& A, int prec, int form, int threads) {
  const double avg = A.n ? (double)A.nnz / A.n : 0.0;
  RowVariant v;
  if (form == 0) {
    // defaults: the vector hybrid form (big row groups from a group-major copy with x in
    // shared memory, the other rows on the pattern form) where there are enough big groups to
    // fill the GPU for many waves and their rows are long (measured faster from 12^3 elements
    // at p = 6 and on the 12^3, p = 8 operator; slower at 8^3 and at p = 4), in both
    // precisions; else FP32 rows on the pattern form (halved index traffic) and FP64 rows,
    // which are bound by the 1/64-rate FP64 pipe, on CSR, threads per row by auto_tpr
    const bool big = A.pat.on && A.grp.hyb && A.grp.n_big >= 4096 && A.grp.big_cols >= 192.0;
    // the sliced form (one lane per row, slices of 32 rows of equal length) on levels of at
    // least 2^18 rows (8192 slices: several waves of warps; below that a warp's long serial
    // slice leaves the GPU latency-bound): the FP64 rows there, since it gives the FP64 pipe
    // one useful FMA per lane and instruction (16^3 p = 6: 0.70 ms per product against 0.93 for
    // the vector hybrid, 12^3 p = 8: 1.34 against 1.59, 24^3 p = 4: 0.32 against 0.58 on CSR),
    // and the FP32 rows where the vector hybrid does not apply (24^3 p = 4: 0.16 against 0.23
    // on row patterns; on the hybrid's operators the FP32 vector hybrid is as fast at p = 6 and
    // faster at p = 8, 0.52 against 0.68)
    const bool large = A.grp.on && A.n >= (1 << 18);
    v.sliced = large && (prec == 0 || !big);
    v.pat = !v.sliced && (prec == 1 || big) && A.pat.on;
    v.hybrid = !v.sliced && big;
    v.vector = !v.sliced && big;
    v.tpr = v.sliced ? 1 : big ? 32 : auto_tpr(A.n, avg, prec == 1 ? 24.0 : 48.0);
  } else {
    v.pat = (form == 2 || form == 4 || form == 5) && A.pat.on;
    v.group = form == 3 && A.grp.on;
    v.hybrid = (form == 4 || form == 5) && A.grp.hyb && A.pat.on;
    v.vector = form == 5 && v.hybrid;
    v.sliced = form == 6 && A.grp.on;
    v.tpr = v.group || v.hybrid ? 32 : v.sliced ? 1 : default_tpr(avg);
  }
  if (threads && !v.group && !v.hybrid && !v.sliced) v.tpr = threads;
  return v;
}

void choose_rows(DCSR& A, int form, int threads) {
  A.var64 = variant_for(A, 0, form, threads);
  A.var32 = variant_for(A, 1, form, threads);
}

// Default L2 prefetch distance of the pattern kernels, about the rows of half the warps resident
// on the whole GPU at once (152 SMs x 64 warps), measured best among 0 to 4x that on the
// 16^3, p = 6 operator.
constexpr int64_t kPrefetchRows = 152 * 32;

void set_prefetch(DCSR& A, int prefetch_rows, int chains) {
  const int64_t pf = prefetch_rows < 0 ? (A.nnz >= (1 << 22) ? kPrefetchRows : 0) : prefetch_rows;
  A.var32.prefetch = pf;
  A.var64.prefetch = pf;
  if (chains) A.var32.unroll = A.var64.unroll = chains;
}

void spmv(const DCSR& A, const double* x, double* y, cudaStream_t s, double avg) {
  launch_rows<double, kSpmv>(A, A.v.get(), x, nullptr, y, nullptr, nullptr, 0.0, 0.0, s, avg);
}
void spmv32(const DCSR& A, const float* x, float* y, cudaStream_t s, double avg) {
  launch_rows<float, kSpmv>(A, A.v32.get(), x, nullptr, y, nullptr, nullptr, 0.f, 0.f, s, avg);
}
void residual(const DCSR& A, const double* b, const double* x, double* r, cudaStream_t s, double avg) {
  launch_rows<double, kResidual>(A, A.v.get(), x, b, r, nullptr, nullptr, 0.0, 0.0, s, avg);
}
void residual32(const DCSR& A, const float* b, const float* x, float* r, cudaStream_t s, double avg) {
  launch_rows<float, kResidual>(A, A.v32.get(), x, b, r, nullptr, nullptr, 0.f, 0.f, s, avg);
}
void cheb_step(const DCSR& A, const double* b, const double* x, double* xo, double* d, const double* dinv, double c1,
               double c2, cudaStream_t s, double avg) {
  launch_rows<double, kCheb>(A, A.v.get(), x, b, xo, d, dinv, c1, c2, s, avg);
}
void cheb_step32(const DCSR& A, const float* b, const float* x, float* xo, float* d, const float* dinv, float c1,
                 float c2, cudaStream_t s, double avg) {
  launch_rows<float, kCheb>(A, A.v32.get(), x, b, xo, d, dinv, c1, c2, s, avg);
}
void cheb_first(int64_t n, const double* b, const double* dinv, double c2, double* x, double* d, cudaStream_t s) {
  { cheb_first_kernel<double><<<vec_grid(n), 256, 0, s>>>(n, b, dinv, c2, x, d); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void cheb_first32(int64_t n, const float* b, const float* dinv, float c2, float* x, float* d, cudaStream_t s) {
  { cheb_first_kernel<float><<<vec_grid(n), 256, 0, s>>>(n, b, dinv, c2, x, d); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

template <typename V>
static void p_restrict_t(const Level& L, const V* rf, V* rc, const V* p1d, V* part, cudaStream_t s) {
  const size_t sm = restrict_smem<V>(L.p, L.q);
  { p_restrict_kernel<V><<<(unsigned)L.n_elem, 128, sm, s>>>(L.n_elem, L.p, L.q, L.l2g.get(), L.own.get(), p1d, rf, part); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  { p_gather_kernel<V><<<grid_for(L.n_next, 256), 256, 0, s>>>(L.n_next, L.cinc_ptr.get(), L.cinc.get(), part, rc); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
template <typename V>
static void p_prolong_t(const Level& L, const V* ec, V* xf, const V* p1d, cudaStream_t s) {
  const size_t sm = prolong_smem<V>(L.p, L.q);
  { p_prolong_kernel<V><<<(unsigned)L.n_elem, 128, sm, s>>>(L.n_elem, L.p, L.q, L.l2g.get(), L.own.get(), L.l2g_c.get(),
                                                           p1d, ec, xf); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void p_restrict(const Level& L, const double* rf, double* rc, cudaStream_t s) {
  p_restrict_t<double>(L, rf, rc, L.p1d.get(), L.part.get(), s);
}
void p_prolong(const Level& L, const double* ec, double* xf, cudaStream_t s) { p_prolong_t<double>(L, ec, xf, L.p1d.get(), s); }
void p_restrict32(const Level& L, const float* rf, float* rc, cudaStream_t s) {
  p_restrict_t<float>(L, rf, rc, L.p1d32.get(), L.part32.get(), s);
}
void p_prolong32(const Level& L, const float* ec, float* xf, cudaStream_t s) { p_prolong_t<float>(L, ec, xf, L.p1d32.get(), s); }

void h_restrict(const Level& L, const double* rf, double* rc, cudaStream_t s) {
  launch_rows<double, kSpmv>(L.R, L.R.v.get(), rf, nullptr, rc, nullptr, nullptr, 0.0, 0.0, s,
                             L.R.n ? (double)L.R.nnz / L.R.n : 0.0);
}
void h_prolong(const Level& L, const double* ec, double* xf, cudaStream_t s) {
  launch_rows<double, kAddSpmv>(L.P, L.P.v.get(), ec, nullptr, xf, nullptr, nullptr, 0.0, 0.0, s,
                                L.P.n ? (double)L.P.nnz / L.P.n : 0.0);
}
void h_restrict32(const Level& L, const float* rf, float* rc, cudaStream_t s) {
  launch_rows<float, kSpmv>(L.R, L.R.v32.get(), rf, nullptr, rc, nullptr, nullptr, 0.f, 0.f, s,
                            L.R.n ? (double)L.R.nnz / L.R.n : 0.0);
}
void h_prolong32(const Level& L, const float* ec, float* xf, cudaStream_t s) {
  launch_rows<float, kAddSpmv>(L.P, L.P.v32.get(), ec, nullptr, xf, nullptr, nullptr, 0.f, 0.f, s,
                               L.P.n ? (double)L.P.nnz / L.P.n : 0.0);
}

int cholesky_factor(double* L, int64_t nc, cudaStream_t s) {
  int* st = nullptr;
  GIAMG_CUDA(cudaMallocAsync((void**)&st, sizeof(int), s));
  GIAMG_CUDA(cudaMemsetAsync(st, 0, sizeof(int), s));
  for (int64_t k = 0; k < nc; ++k) {
    { chol_scale_col<<<1, 256, 0, s>>>(L, nc, k, st); note_launch(); }
    const int64_t m = nc - k - 1;
    if (m > 0) { chol_update<<<grid_for(m * m, 256), 256, 0, s>>>(L, nc, k); note_launch(); }
  }
  { zero_upper<<<grid_for(nc * nc, 256), 256, 0, s>>>(L, nc); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  int h = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(st, s);
  return h ? GIAMG_ERR_NOT_SPD : GIAMG_OK;
}
static void chol_smem_attr() {
  static PerDevice done;
  done.once([&] {
    GIAMG_CUDA(cudaFuncSetAttribute(chol_solve_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8));
    GIAMG_CUDA(cudaFuncSetAttribute(chol_solve_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8));
  });
}
void chol_inverse(const double* L, int64_t nc, double* Ainv, cudaStream_t s) {
  chol_smem_attr();
  static PerDevice attr;
  attr.once([&] { GIAMG_CUDA(cudaFuncSetAttribute(chol_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8)); });
  { chol_inverse_kernel<<<(unsigned)nc, 256, sizeof(double) * nc, s>>>(L, nc, Ainv); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void inverse_apply(const double* Ainv, int64_t nc, const double* b, double* x, cudaStream_t s) {
  { dense_inverse_apply<double><<<grid_for(nc * 32, 256), 256, 0, s>>>(Ainv, nc, b, x); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void inverse_apply32(const double* Ainv, int64_t nc, const float* b, float* x, cudaStream_t s) {
  { dense_inverse_apply<float><<<grid_for(nc * 32, 256), 256, 0, s>>>(Ainv, nc, b, x); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void chol_solve(const double* L, int64_t nc, const double* b, double* x, cudaStream_t s) {
  chol_smem_attr();
  { chol_solve_kernel<double><<<1, 512, sizeof(double) * nc, s>>>(L, nc, b, x); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void chol_solve32(const double* L, int64_t nc, const float* b, float* x, cudaStream_t s) {
  chol_smem_attr();
  { chol_solve_kernel<float><<<1, 512, sizeof(double) * nc, s>>>(L, nc, b, x); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void dot_partial(int64_t n, const double* x, const double* y, double* partial, cudaStream_t s) {
  { dot_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, x, y, partial); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void reduce_to(const double* partial, double* out, cudaStream_t s) {
  { reduce_kernel<<<1, 1024, 0, s>>>(partial, out); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void vec_copy(int64_t n, const double* x, double* y, cudaStream_t s) {
  { copy_kernel<<<vec_grid(n), 256, 0, s>>>(n, x, y); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void vec_fill(int64_t n, double v, double* y, cudaStream_t s) {
  { fill_kernel<<<vec_grid(n), 256, 0, s>>>(n, v, y); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void vec_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  { axpy_kernel<<<vec_grid(n), 256, 0, s>>>(n, a, x, y); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void vec_to32(int64_t n, const double* x, float* y, cudaStream_t s) {
  { to32_kernel<<<vec_grid(n), 256, 0, s>>>(n, x, y); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void vec_to64(int64_t n, const float* x, double* y, cudaStream_t s) {
  { to64_kernel<<<vec_grid(n), 256, 0, s>>>(n, x, y); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void vec_add32(int64_t n, const float* x, float* y, cudaStream_t s) {
  { add32_kernel<<<vec_grid(n), 256, 0, s>>>(n, x, y); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void pcg_init(int64_t n, const double* b, double* x, double* r, double* partial, cudaStream_t s) {
  { pcg_init_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, x, r, partial); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void pcg_finish_bb(Scalars* sc, const double* partial, cudaStream_t s) {
  { finish_bb_kernel<<<1, 1024, 0, s>>>(sc, partial); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void pcg_dot_rz(int64_t n, const double* r, const double* z, const double* rold, int flexible, double* partial,
                cudaStream_t s) {
  { dot_rz_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, r, z, rold, flexible, partial); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void pcg_finish_rz(Scalars* sc, const double* partial, int first, int flexible, cudaStream_t s) {
  { finish_rz_kernel<<<1, 1024, 0, s>>>(sc, partial, first, flexible); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void pcg_update_p(int64_t n, const double* z, double* p, const Scalars* sc, int first, cudaStream_t s) {
  { update_p_kernel<<<vec_grid(n), 256, 0, s>>>(n, z, p, sc, first); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void pcg_spmv_pq(const DCSR& A, const double* p, double* q, double* partial, cudaStream_t s, double avg) {
  spmv(A, p, q, s, avg);
  dot_partial(A.n, p, q, partial, s);
}
void pcg_finish_pq(Scalars* sc, const double* partial, cudaStream_t s) {
  { finish_pq_kernel<<<1, 1024, 0, s>>>(sc, partial); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void pcg_update_xr(int64_t n, const double* p, const double* q, double* x, double* r, double* rold, int flexible,
                   const Scalars* sc, double* partial, cudaStream_t s) {
  { update_xr_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, p, q, x, r, rold, flexible, sc, partial); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}
void pcg_finish_rr(Scalars* sc, const double* partial, cudaStream_t s) {
  { finish_rr_kernel<<<1, 1024, 0, s>>>(sc, partial); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

}  // namespace giamg
