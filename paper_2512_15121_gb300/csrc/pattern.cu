// pattern.cu -- detection of repeated row patterns in a CSR matrix ("pattern-compressed CSR").
//
// In an assembled high-order operator on a mesh with a regular numbering, row i's columns are
// i + o_1, ..., i + o_L for one of a few hundred offset lists (the position of the node inside
// its element decides the list).  Storing one template id per row instead of one column index
// per nonzero removes the index stream from the SpMV: for FP32 values that halves the bytes
// the kernel must read.  Detection is exact: every row is compared with its template's
// representative; any mismatch, or too many templates, keeps the plain CSR path.  Values, row
// pointers and columns stay as they are (the setup and export paths use them).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace giamg {

namespace {

constexpr uint64_t kEmpty = ~0ull;

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

inline unsigned blocks(int64_t work) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 65535));
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// hash of the row's length and columns, relative to the row index (patterns) or absolute
// (row groups with identical column sets)
__global__ void row_hash(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int absolute,
                         uint64_t* __restrict__ h) {
  GRID_STRIDE(i, n) {
    uint64_t z = mix64((uint64_t)(rp[i + 1] - rp[i]) + 0x9E3779B97F4A7C15ULL);
    const int64_t base = absolute ? 0 : i;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) z = mix64(z ^ (uint64_t)(uint32_t)((int64_t)ci[t] - base));
    h[i] = z == kEmpty ? z - 1 : z;
  }
}

// row groups: every row's columns equal its group representative's columns exactly
__global__ void verify_groups(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const int32_t* __restrict__ gid, const int64_t* __restrict__ gptr,
                              const int32_t* __restrict__ gcol, int* __restrict__ bad) {
  GRID_STRIDE(i, n) {
    const int32_t g = gid[i];
    if (g < 0) {
      atomicAdd(bad, 1);
      continue;
    }
    const int64_t len = rp[i + 1] - rp[i];
    if (len != gptr[g + 1] - gptr[g]) {
      atomicAdd(bad, 1);
      continue;
    }
    for (int64_t k = 0; k < len; ++k)
      if (ci[rp[i] + k] != gcol[gptr[g] + k]) {
        atomicAdd(bad, 1);
        break;
      }
  }
}

__global__ void group_fill_cols(int64_t G, const uint32_t* __restrict__ rep_sorted, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ ci, const int64_t* __restrict__ gptr,
                                int32_t* __restrict__ gcol) {
  GRID_STRIDE(g, G) {
    const int64_t r = rep_sorted[g];
    for (int64_t k = 0; k < gptr[g + 1] - gptr[g]; ++k) gcol[gptr[g] + k] = ci[rp[r] + k];
  }
}

__global__ void group_count_rows(int64_t n, const int32_t* __restrict__ gid, int32_t* __restrict__ cnt) {
  GRID_STRIDE(i, n) atomicAdd(&cnt[gid[i]], 1);
}
__global__ void group_fill_rows(int64_t n, const int32_t* __restrict__ gid, const int64_t* __restrict__ rptr,
                                int32_t* __restrict__ fill, int32_t* __restrict__ grow) {
  GRID_STRIDE(i, n) {
    const int32_t g = gid[i];
    grow[rptr[g] + atomicAdd(&fill[g], 1)] = (int32_t)i;
  }
}
__global__ void group_sort_rows(int64_t G, const int64_t* __restrict__ rptr, int32_t* __restrict__ grow) {
  GRID_STRIDE(g, G) {
    const int64_t s = rptr[g], e = rptr[g + 1];
    for (int64_t i = s + 1; i < e; ++i) {
      const int32_t v = grow[i];
      int64_t j = i - 1;
      while (j >= s && grow[j] > v) {
        grow[j + 1] = grow[j];
        --j;
      }
      grow[j + 1] = v;
    }
  }
}

// open-addressing table hash -> slot; rep[slot] = smallest row with that hash
// The table holds at most max_distinct keys (a quarter of its slots); once more distinct keys
// have been seen every later insert gives up, so a matrix without repetition costs one pass.
__global__ void table_insert(int64_t n, const uint64_t* __restrict__ h, unsigned long long* keys,
                             int* rep, int64_t cap, int64_t max_distinct, int* distinct, int* overflow) {
  GRID_STRIDE(i, n) {
    if (*(volatile int*)distinct > max_distinct) {
      *(volatile int*)overflow = 1;
      continue;
    }
    const uint64_t k = h[i];
    uint64_t s = mix64(k) & (uint64_t)(cap - 1);
    bool done = false;
    const int64_t limit = cap < 4096 ? cap : 4096;
    for (int64_t probe = 0; probe < limit && !done; ++probe) {
      const unsigned long long prev = atomicCAS(&keys[s], (unsigned long long)kEmpty, (unsigned long long)k);
      if (prev == kEmpty || prev == k) {
        if (prev == kEmpty) atomicAdd(distinct, 1);
        atomicMin(&rep[s], (int)i);
        done = true;
      } else {
        s = (s + 1) & (uint64_t)(cap - 1);
      }
    }
    if (!done) atomicAdd(overflow, 1);
  }
}

__global__ void table_find(int64_t n, const uint64_t* __restrict__ h, const unsigned long long* __restrict__ keys,
                           const int* __restrict__ slot_tid, int64_t cap, int32_t* __restrict__ tid) {
  GRID_STRIDE(i, n) {
    const uint64_t k = h[i];
    uint64_t s = mix64(k) & (uint64_t)(cap - 1);
    int32_t t = -1;
    for (int64_t probe = 0; probe < cap; ++probe) {
      if (keys[s] == k) {
        t = slot_tid[s];
        break;
      }
      s = (s + 1) & (uint64_t)(cap - 1);
    }
    tid[i] = t;
  }
}

__global__ void occupied(int64_t cap, const unsigned long long* __restrict__ keys, int32_t* __restrict__ flag) {
  GRID_STRIDE(s, cap) flag[s] = keys[s] != kEmpty ? 1 : 0;
}

// representatives of occupied slots, compacted; key for sorting by representative row
__global__ void compact_reps(int64_t cap, const int32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                             const int* __restrict__ rep, uint32_t* __restrict__ rep_key, int64_t* __restrict__ slot_of) {
  GRID_STRIDE(s, cap) {
    if (flag[s]) {
      rep_key[pos[s]] = (uint32_t)rep[s];
      slot_of[pos[s]] = s;
    }
  }
}

// Start of each row's template offsets, so the row kernels read one index per row instead of
// the dependent pair tid -> tptr.
__global__ void row_obase(int64_t n, const int32_t* __restrict__ tid, const int64_t* __restrict__ tptr,
                          int32_t* __restrict__ obase) {
  GRID_STRIDE(i, n) obase[i] = (int32_t)tptr[tid[i]];
}

__global__ void assign_tid(int64_t T, const int64_t* __restrict__ slot_sorted, int* __restrict__ slot_tid) {
  GRID_STRIDE(t, T) slot_tid[slot_sorted[t]] = (int)t;
}

__global__ void template_len(int64_t T, const uint32_t* __restrict__ rep_sorted, const int64_t* __restrict__ rp,
                             int32_t* __restrict__ len) {
  GRID_STRIDE(t, T) len[t] = (int32_t)(rp[rep_sorted[t] + 1] - rp[rep_sorted[t]]);
}

__global__ void template_fill(int64_t T, const uint32_t* __restrict__ rep_sorted, const int64_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, const int64_t* __restrict__ tptr,
                              int32_t* __restrict__ toff) {
  GRID_STRIDE(t, T) {
    const int64_t r = rep_sorted[t];
    for (int64_t k = 0; k < tptr[t + 1] - tptr[t]; ++k) toff[tptr[t] + k] = (int32_t)((int64_t)ci[rp[r] + k] - r);
  }
}

// every row must equal its template exactly
__global__ void verify(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const int32_t* __restrict__ tid, const int64_t* __restrict__ tptr,
                       const int32_t* __restrict__ toff, int* __restrict__ bad) {
  GRID_STRIDE(i, n) {
    const int32_t t = tid[i];
    if (t < 0) {
      atomicAdd(bad, 1);
      continue;
    }
    const int64_t len = rp[i + 1] - rp[i];
    if (len != tptr[t + 1] - tptr[t]) {
      atomicAdd(bad, 1);
      continue;
    }
    for (int64_t k = 0; k < len; ++k)
      if ((int64_t)ci[rp[i] + k] - i != toff[tptr[t] + k]) {
        atomicAdd(bad, 1);
        break;
      }
  }
}

}  // namespace

bool pattern_build(DCSR& A, cudaStream_t s, int64_t max_templates, int64_t max_offsets) {
  Pattern& P = A.pat;
  P.on = false;
  const int64_t n = A.n;
  if (n < 1024 || A.nnz == 0) return false;  // small levels gain nothing
  int64_t cap = 1;
  while (cap < 4 * std::min<int64_t>(n, max_templates + 1)) cap <<= 1;
  DBuf<uint64_t> h;
  DBuf<unsigned long long> keys;
  DBuf<int> rep, ovf, slot_tid, bad, distinct;
  h.alloc(n, s);
  keys.alloc(cap, s);
  rep.alloc(cap, s);
  ovf.alloc(1, s);
  GIAMG_CUDA(cudaMemsetAsync(keys.get(), 0xff, sizeof(unsigned long long) * cap, s));
  GIAMG_CUDA(cudaMemsetAsync(rep.get(), 0x7f, sizeof(int) * cap, s));
  ovf.zero(s);
  distinct.alloc(1, s);
  distinct.zero(s);
  { row_hash<<<blocks(n), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), 0, h.get()); note_launch(); }
  { table_insert<<<blocks(n), 256, 0, s>>>(n, h.get(), keys.get(), rep.get(), cap, max_templates, distinct.get(), ovf.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  int hovf = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&hovf, ovf.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (hovf) return false;  // more distinct patterns than the table holds: keep CSR
  DBuf<int32_t> flag;
  DBuf<int64_t> pos;
  flag.alloc(cap, s);
  pos.alloc(cap + 1, s);
  { occupied<<<blocks(cap), 256, 0, s>>>(cap, keys.get(), flag.get()); note_launch(); }
  scan_i32_to_i64(flag.get(), pos.get(), cap, s);
  int64_t T = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&T, pos.get() + cap, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (T > max_templates || T * 4 > n) return false;  // fewer than 4 rows per pattern: no gain
  // template ids in order of first occurrence (smallest representative row)
  DBuf<uint32_t> rep_key;
  DBuf<int64_t> slot_of;
  rep_key.alloc(T, s);
  slot_of.alloc(T, s);
  { compact_reps<<<blocks(cap), 256, 0, s>>>(cap, flag.get(), pos.get(), rep.get(), rep_key.get(), slot_of.get()); note_launch(); }
  int bits = 1;
  while (bits < 32 && ((int64_t)1 << bits) < n) ++bits;
  radix_sort_pairs(rep_key.get(), slot_of.get(), T, bits, s);
  slot_tid.alloc(cap, s);
  { assign_tid<<<blocks(T), 256, 0, s>>>(T, slot_of.get(), slot_tid.get()); note_launch(); }
  DBuf<int32_t> len;
  len.alloc(T, s);
  { template_len<<<blocks(T), 256, 0, s>>>(T, rep_key.get(), A.rp.get(), len.get()); note_launch(); }
  P.tptr.alloc(T + 1, s);
  scan_i32_to_i64(len.get(), P.tptr.get(), T, s);
  int64_t total = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&total, P.tptr.get() + T, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (total > max_offsets) {
    P.tptr.release();
    return false;
  }
  P.toff.alloc(std::max<int64_t>(total, 1), s);
  { template_fill<<<blocks(T), 256, 0, s>>>(T, rep_key.get(), A.rp.get(), A.ci.get(), P.tptr.get(), P.toff.get()); note_launch(); }
  P.tid.alloc(n, s);
  { table_find<<<blocks(n), 256, 0, s>>>(n, h.get(), keys.get(), slot_tid.get(), cap, P.tid.get()); note_launch(); }
  bad.alloc(1, s);
  bad.zero(s);
  { verify<<<blocks(n), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), P.tid.get(), P.tptr.get(), P.toff.get(), bad.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  int hbad = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&hbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (hbad) {  // a hash collision between different patterns: keep CSR
    P.tid.release();
    P.tptr.release();
    P.toff.release();
    return false;
  }
  P.obase.alloc(n, s);
  { row_obase<<<blocks(n), 256, 0, s>>>(n, P.tid.get(), P.tptr.get(), P.obase.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  P.n_templates = T;
  P.n_offsets = total;
  P.on = true;
  return true;
}

// Row groups: rows with identical (absolute) column sets -- in a nodal high-order operator, the
// interior nodes of one element, the interior nodes of one shared face or edge.  A group's rows
// form a dense block over its columns, so the row kernels gather x once per group.
bool groups_build(DCSR& A, cudaStream_t s, int64_t max_groups, bool any_sharing) {
  Groups& R = A.grp;
  R.on = false;
  const int64_t n = A.n;
  if (n < 1024 || A.nnz == 0) return false;
  int64_t cap = 1;
  while (cap < 4 * std::min<int64_t>(n, max_groups + 1)) cap <<= 1;
  DBuf<uint64_t> h;
  DBuf<unsigned long long> keys;
  DBuf<int> rep, ovf, slot_gid, bad, distinct;
  h.alloc(n, s);
  keys.alloc(cap, s);
  rep.alloc(cap, s);
  ovf.alloc(1, s);
  distinct.alloc(1, s);
  GIAMG_CUDA(cudaMemsetAsync(keys.get(), 0xff, sizeof(unsigned long long) * cap, s));
  GIAMG_CUDA(cudaMemsetAsync(rep.get(), 0x7f, sizeof(int) * cap, s));
  ovf.zero(s);
  distinct.zero(s);
  { row_hash<<<blocks(n), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), 1, h.get()); note_launch(); }
  { table_insert<<<blocks(n), 256, 0, s>>>(n, h.get(), keys.get(), rep.get(), cap, max_groups, distinct.get(), ovf.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  int hovf = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&hovf, ovf.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (hovf) return false;
  DBuf<int32_t> flag;
  DBuf<int64_t> pos;
  flag.alloc(cap, s);
  pos.alloc(cap + 1, s);
  { occupied<<<blocks(cap), 256, 0, s>>>(cap, keys.get(), flag.get()); note_launch(); }
  scan_i32_to_i64(flag.get(), pos.get(), cap, s);
  int64_t G = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&G, pos.get() + cap, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (G > max_groups || (!any_sharing && G * 2 > n)) return false;  // groups of fewer than 2 rows on average
  DBuf<uint32_t> rep_key;
  DBuf<int64_t> slot_of;
  rep_key.alloc(G, s);
  slot_of.alloc(G, s);
  { compact_reps<<<blocks(cap), 256, 0, s>>>(cap, flag.get(), pos.get(), rep.get(), rep_key.get(), slot_of.get()); note_launch(); }
  int bits = 1;
  while (bits < 32 && ((int64_t)1 << bits) < n) ++bits;
  radix_sort_pairs(rep_key.get(), slot_of.get(), G, bits, s);
  slot_gid.alloc(cap, s);
  { assign_tid<<<blocks(G), 256, 0, s>>>(G, slot_of.get(), slot_gid.get()); note_launch(); }
  DBuf<int32_t> len, gid;
  len.alloc(G, s);
  { template_len<<<blocks(G), 256, 0, s>>>(G, rep_key.get(), A.rp.get(), len.get()); note_launch(); }
  R.gptr.alloc(G + 1, s);
  scan_i32_to_i64(len.get(), R.gptr.get(), G, s);
  int64_t total = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&total, R.gptr.get() + G, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (!any_sharing && total * 4 > A.nnz) {  // fewer than 4 rows share a column list on average: no gain
    R.gptr.release();
    return false;
  }
  R.gcol.alloc(std::max<int64_t>(total, 1), s);
  { group_fill_cols<<<blocks(G), 256, 0, s>>>(G, rep_key.get(), A.rp.get(), A.ci.get(), R.gptr.get(), R.gcol.get()); note_launch(); }
  gid.alloc(n, s);
  { table_find<<<blocks(n), 256, 0, s>>>(n, h.get(), keys.get(), slot_gid.get(), cap, gid.get()); note_launch(); }
  bad.alloc(1, s);
  bad.zero(s);
  { verify_groups<<<blocks(n), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), gid.get(), R.gptr.get(), R.gcol.get(), bad.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  int hbad = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&hbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (hbad) {
    R.gptr.release();
    R.gcol.release();
    return false;
  }
  DBuf<int32_t> cnt, fill;
  cnt.alloc(G, s);
  fill.alloc(G, s);
  cnt.zero(s);
  fill.zero(s);
  { group_count_rows<<<blocks(n), 256, 0, s>>>(n, gid.get(), cnt.get()); note_launch(); }
  R.rptr.alloc(G + 1, s);
  scan_i32_to_i64(cnt.get(), R.rptr.get(), G, s);
  R.grow.alloc(n, s);
  { group_fill_rows<<<blocks(n), 256, 0, s>>>(n, gid.get(), R.rptr.get(), fill.get(), R.grow.get()); note_launch(); }
  { group_sort_rows<<<blocks(G), 256, 0, s>>>(G, R.rptr.get(), R.grow.get()); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
  // largest column list (shared-memory size of the kernel)
  std::vector<int64_t> gp(G + 1);
  GIAMG_CUDA(cudaMemcpyAsync(gp.data(), R.gptr.get(), sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  int64_t cmax = 0;
  for (int64_t g = 0; g < G; ++g) cmax = std::max(cmax, gp[g + 1] - gp[g]);
  if (!any_sharing && cmax * 8 > 96 * 1024) {  // the FP64 x block must fit in shared memory
    R.gptr.release(); R.gcol.release(); R.rptr.release(); R.grow.release();
    return false;
  }
  R.n_groups = G;
  R.n_cols = total;
  R.cmax = (int)cmax;
  R.on = true;
  // hybrid form: big groups (at least kHybridRows rows) and the rows of all other groups
  if (A.pat.on) {
    std::vector<int64_t> rp_h(G + 1);
    std::vector<int32_t> rows(n);
    GIAMG_CUDA(cudaMemcpyAsync(rp_h.data(), R.rptr.get(), sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaMemcpyAsync(rows.data(), R.grow.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> big, rest;
    double big_nnz = 0.0, big_rows = 0.0;
    for (int64_t g = 0; g < G; ++g) {
      const int64_t r = rp_h[g + 1] - rp_h[g];
      if (r >= kHybridRows) {
        big.push_back((int32_t)g);
        big_rows += (double)r;
        big_nnz += (double)r * (double)(gp[g + 1] - gp[g]);
      } else {
        rest.insert(rest.end(), rows.begin() + rp_h[g], rows.begin() + rp_h[g + 1]);
      }
    }
    std::sort(rest.begin(), rest.end());
    if (!big.empty()) {
      R.big.alloc(big.size(), s);
      GIAMG_CUDA(cudaMemcpyAsync(R.big.get(), big.data(), sizeof(int32_t) * big.size(), cudaMemcpyHostToDevice, s));
      R.rest.alloc(std::max<size_t>(rest.size(), 1), s);
      if (!rest.empty())
        GIAMG_CUDA(cudaMemcpyAsync(R.rest.get(), rest.data(), sizeof(int32_t) * rest.size(), cudaMemcpyHostToDevice, s));
      GIAMG_CUDA(cudaStreamSynchronize(s));
      R.n_big = (int64_t)big.size();
      R.n_rest = (int64_t)rest.size();
      R.big_cols = big_rows > 0 ? big_nnz / big_rows : 0.0;
      R.hyb = true;
    }
  }
  return true;
}

namespace {
// One CTA per big group: the group's rows (in group order), each padded with zeros to a
// multiple of 4 values.
template <typename V>
__global__ void hv_gather(const int32_t* __restrict__ big, const int64_t* __restrict__ gptr,
                          const int64_t* __restrict__ rptr, const int32_t* __restrict__ grow,
                          const int64_t* __restrict__ rp, const V* __restrict__ val,
                          const int64_t* __restrict__ hoff, V* __restrict__ hv) {
  const int64_t j = blockIdx.x;
  const int64_t g = big[j];
  const int c = (int)(gptr[g + 1] - gptr[g]);
  const int cp = (c + 3) & ~3;
  const int64_t t0 = rptr[g], rows = rptr[g + 1] - t0;
  V* __restrict__ out = hv + hoff[j];
  for (int64_t e = threadIdx.x; e < rows * cp; e += blockDim.x) {
    const int64_t t = e / cp;
    const int k = (int)(e - t * cp);
    out[e] = k < c ? val[rp[grow[t0 + t]] + k] : V(0);
  }
}
}  // namespace

namespace {
// One CTA per slice: the values of its rows, interleaved by column in groups of W.
template <typename V, int W>
__global__ void slice_fill(const int32_t* __restrict__ srow, const int32_t* __restrict__ sclen,
                           const int32_t* __restrict__ slen, const int64_t* __restrict__ sbase,
                           const int64_t* __restrict__ rp, const V* __restrict__ val, V* __restrict__ sv) {
  const int64_t sl = blockIdx.x;
  const int64_t cnt = (int64_t)slen[sl] * 32;
  V* __restrict__ out = sv + sbase[sl];
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int64_t kw = e / (32 * W);
    const int rem = (int)(e - kw * 32 * W);
    const int lane = rem / W;
    const int k = (int)(kw * W + rem % W);
    const int row = srow[sl * 32 + lane];
    out[e] = row >= 0 && k < sclen[sl * 32 + lane] ? val[rp[row] + k] : V(0);
  }
}
}  // namespace

bool sliced_build(DCSR& A, int precision, cudaStream_t s) {
  Groups& R = A.grp;
  if (precision == 1 ? R.sv32on : R.sv64on) return true;
  if (!R.on || (precision == 1 ? !A.v32.get() : !A.v.get())) return false;
  const int64_t n = A.n, G = R.n_groups;
  if (!R.son) {  // the layout, shared by both precisions
    if (R.n_cols >= INT32_MAX) return false;
    std::vector<int64_t> gp(G + 1), rp_h(G + 1);
    std::vector<int32_t> rows(n);
    GIAMG_CUDA(cudaMemcpyAsync(gp.data(), R.gptr.get(), sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaMemcpyAsync(rp_h.data(), R.rptr.get(), sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaMemcpyAsync(rows.data(), R.grow.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> order(G);
    for (int64_t g = 0; g < G; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return gp[a + 1] - gp[a] > gp[b + 1] - gp[b]; });
    const int64_t ns = (n + 31) / 32;
    std::vector<int32_t> srow(ns * 32, -1), sob(ns * 32, 0), sclen(ns * 32, 1), slen(ns, kSliceStep);
    std::vector<int64_t> sbase(ns + 1, 0);
    int64_t li = 0;
    for (int64_t g : order) {
      const int32_t c = (int32_t)(gp[g + 1] - gp[g]);
      for (int64_t t = rp_h[g]; t < rp_h[g + 1]; ++t, ++li) {
        srow[li] = rows[t];
        sob[li] = (int32_t)gp[g];
        sclen[li] = std::max(c, 1);
      }
    }
    for (int64_t sl = 0; sl < ns; ++sl) {
      int32_t L = 1;
      for (int l = 0; l < 32; ++l) L = std::max(L, sclen[sl * 32 + l]);
      slen[sl] = (L + kSliceStep - 1) / kSliceStep * kSliceStep;
      sbase[sl + 1] = sbase[sl] + (int64_t)slen[sl] * 32;
    }
    R.srow.alloc(ns * 32, s);
    R.sob.alloc(ns * 32, s);
    R.sclen.alloc(ns * 32, s);
    R.slen.alloc(ns, s);
    R.sbase.alloc(ns + 1, s);
    GIAMG_CUDA(cudaMemcpyAsync(R.srow.get(), srow.data(), sizeof(int32_t) * ns * 32, cudaMemcpyHostToDevice, s));
    GIAMG_CUDA(cudaMemcpyAsync(R.sob.get(), sob.data(), sizeof(int32_t) * ns * 32, cudaMemcpyHostToDevice, s));
    GIAMG_CUDA(cudaMemcpyAsync(R.sclen.get(), sclen.data(), sizeof(int32_t) * ns * 32, cudaMemcpyHostToDevice, s));
    GIAMG_CUDA(cudaMemcpyAsync(R.slen.get(), slen.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
    GIAMG_CUDA(cudaMemcpyAsync(R.sbase.get(), sbase.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    R.n_slices = ns;
    R.son = true;
  }
  int64_t total = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&total, R.sbase.get() + R.n_slices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (precision == 1) {
    R.sv32.alloc((size_t)std::max<int64_t>(total, 4), s);
    { slice_fill<float, 4><<<(unsigned)R.n_slices, 256, 0, s>>>(R.srow.get(), R.sclen.get(), R.slen.get(), R.sbase.get(),
                                                                A.rp.get(), A.v32.get(), R.sv32.get()); note_launch(); }
    R.sv32on = true;
  } else {
    R.sv64.alloc((size_t)std::max<int64_t>(total, 2), s);
    { slice_fill<double, 2><<<(unsigned)R.n_slices, 256, 0, s>>>(R.srow.get(), R.sclen.get(), R.slen.get(), R.sbase.get(),
                                                                 A.rp.get(), A.v.get(), R.sv64.get()); note_launch(); }
    R.sv64on = true;
  }
  GIAMG_CUDA(cudaGetLastError());
  GIAMG_CUDA(cudaStreamSynchronize(s));
  return true;
}

bool batch_pairs_build(DCSR& A, cudaStream_t s) {
  Groups& R = A.grp;
  R.pon = false;
  if (!R.on) return false;
  const int64_t G = R.n_groups, n = A.n;
  std::vector<int64_t> rp_h(G + 1);
  std::vector<int32_t> rows(n);
  GIAMG_CUDA(cudaMemcpyAsync(rp_h.data(), R.rptr.get(), sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaMemcpyAsync(rows.data(), R.grow.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> ia, ib, ig;
  ia.reserve(n / 2 + G);
  for (int64_t g = 0; g < G; ++g) {
    for (int64_t t = rp_h[g]; t < rp_h[g + 1]; t += 2) {
      ia.push_back(rows[t]);
      ib.push_back(t + 1 < rp_h[g + 1] ? rows[t + 1] : -1);
      ig.push_back((int32_t)g);
    }
  }
  const size_t ni = ia.size();
  R.item_a.alloc(ni, s);
  R.item_b.alloc(ni, s);
  R.item_g.alloc(ni, s);
  GIAMG_CUDA(cudaMemcpyAsync(R.item_a.get(), ia.data(), sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s));
  GIAMG_CUDA(cudaMemcpyAsync(R.item_b.get(), ib.data(), sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s));
  GIAMG_CUDA(cudaMemcpyAsync(R.item_g.get(), ig.data(), sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  R.n_items = (int64_t)ni;
  R.pon = true;
  return true;
}

bool hybrid_vector_build(DCSR& A, int precision, cudaStream_t s) {
  Groups& R = A.grp;
  if (precision == 1 ? R.hvon : R.hv64on) return true;  // built already (by the setup-time tuner)
  if (!R.hyb || R.n_big == 0 || (precision == 1 ? !A.v32.get() : !A.v.get())) return false;
  const int64_t G = R.n_groups, nb = R.n_big;
  if (!R.hoff.get()) {  // the layout, shared by both precisions
    std::vector<int64_t> gp(G + 1), rp_h(G + 1);
    std::vector<int32_t> big(nb);
    GIAMG_CUDA(cudaMemcpyAsync(gp.data(), R.gptr.get(), sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaMemcpyAsync(rp_h.data(), R.rptr.get(), sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaMemcpyAsync(big.data(), R.big.get(), sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> hoff(nb + 1, 0);
    int cpmax = 0, rmax = 0;
    for (int64_t j = 0; j < nb; ++j) {
      const int64_t g = big[j];
      const int cp = (int)((gp[g + 1] - gp[g] + 3) & ~(int64_t)3);
      cpmax = std::max(cpmax, cp);
      rmax = std::max(rmax, (int)(rp_h[g + 1] - rp_h[g]));
      hoff[j + 1] = hoff[j] + (rp_h[g + 1] - rp_h[g]) * cp;
    }
    // x of a group in shared memory (FP64), and (FP32 form) the sums of its rows after it
    if ((size_t)cpmax * 8 > 96 * 1024 || (size_t)(cpmax + rmax) * 4 > 96 * 1024) return false;
    R.hoff.alloc(nb + 1, s);
    GIAMG_CUDA(cudaMemcpyAsync(R.hoff.get(), hoff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    R.cpmax = cpmax;
    R.rmax = rmax;
    // warps per block of the FP32 vector hybrid: 8, unless they leave more than 5% of the warp-rows
    // idle when each group's rows are dealt round-robin to the block's warps (measured in the
    // solve: 16^3 p = 6, groups of 125 and 25 rows, 10% idle with 8 warps, 2% faster with 5;
    // 12^3 p = 8, groups of 343 and 49 rows, 4.5% idle, 2% slower with 7); then the count from
    // 4 to 7 with the fewest idle warp-rows (ties: more warps)
    auto idle_of = [&](int w, int64_t& slots) {
      int64_t idle = 0;
      slots = 0;
      for (int64_t j = 0; j < nb; ++j) {
        const int64_t r = rp_h[big[j] + 1] - rp_h[big[j]];
        idle += (r + w - 1) / w * w - r;
        slots += (r + w - 1) / w * w;
      }
      return idle;
    };
    int64_t slots8 = 0;
    const int64_t idle8 = idle_of(8, slots8);
    R.hwarps = 8;
    if (idle8 * 20 > slots8) {
      int64_t best = idle8, slots = 0;
      for (int w = 7; w >= 4; --w) {
        const int64_t idle = idle_of(w, slots);
        if (idle < best) {
          best = idle;
          R.hwarps = w;
        }
      }
    }
  }
  int64_t total = 0;
  GIAMG_CUDA(cudaMemcpyAsync(&total, R.hoff.get() + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
  if (precision == 1) {
    R.hv.alloc((size_t)std::max<int64_t>(total, 4), s);
    { hv_gather<float><<<(unsigned)nb, 256, 0, s>>>(R.big.get(), R.gptr.get(), R.rptr.get(), R.grow.get(), A.rp.get(),
                                                    A.v32.get(), R.hoff.get(), R.hv.get()); note_launch(); }
    R.hvon = true;
  } else {
    R.hv64.alloc((size_t)std::max<int64_t>(total, 4), s);
    { hv_gather<double><<<(unsigned)nb, 256, 0, s>>>(R.big.get(), R.gptr.get(), R.rptr.get(), R.grow.get(),
                                                     A.rp.get(), A.v.get(), R.hoff.get(), R.hv64.get()); note_launch(); }
    R.hv64on = true;
  }
  GIAMG_CUDA(cudaGetLastError());
  GIAMG_CUDA(cudaStreamSynchronize(s));
  return true;
}

}  // namespace giamg
