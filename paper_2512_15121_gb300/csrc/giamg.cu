// giamg.cu -- the C ABI (include/giamg.h): hierarchy setup, the V-cycle of Algorithm 1 and
// the PCG / flexible CG loop of Sec. 2, orchestrated on the host with every step running in
// the library's own kernels on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace giamg {

static thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};

void set_error(int code, const std::string& msg) {
  (void)code;
  g_last_error = msg;
}

Hierarchy::~Hierarchy() {
  for (SolveGraph& G : graph)
    if (G.exec) cudaGraphExecDestroy(G.exec);
  for (auto* set : {&bgraph, &kgraph})
    for (auto& per_m : *set)
      for (SolveGraph& G : per_m)
        if (G.exec) cudaGraphExecDestroy(G.exec);
  if (capture_stream) cudaStreamDestroy(capture_stream);
  if (h_gst) cudaFreeHost(h_gst);
  if (h_bgst) cudaFreeHost(h_bgst);
  for (Level* L : lev) delete L;
  lev.clear();
  if (h_sc) cudaFreeHost(h_sc);
  if (h_bsc) cudaFreeHost(h_bsc);
  for (cudaEvent_t e : prof.ev) cudaEventDestroy(e);
}

namespace {

// p schedule: 0 halving (q = p/2; odd p: its largest proper divisor), 1 by one, 2 by two
int next_order(int p, int schedule) {
  if (p <= 1) return 1;
  if (schedule == 1) return p - 1;
  if (schedule == 2) return p > 2 ? p - 2 : 1;
  if (p % 2 == 0) return p / 2;
  for (int d = p / 2; d >= 1; --d)
    if (p % d == 0) return d;
  return 1;
}

// ------------------------------------------------------------------ profiling
int prof_begin(Hierarchy& H, int cat) {
  if (!H.prof.on) return -1;
  Prof& P = H.prof;
  if (P.used + 2 > P.ev.size()) {
    for (int k = 0; k < 256; ++k) {
      cudaEvent_t e;
      GIAMG_CUDA(cudaEventCreate(&e));
      P.ev.push_back(e);
    }
  }
  const int e0 = (int)P.used++;
  const int e1 = (int)P.used++;
  GIAMG_CUDA(cudaEventRecord(P.ev[e0], H.stream));
  P.recs.push_back({cat, e0, e1, 0.0});
  return (int)P.recs.size() - 1;
}
void prof_end(Hierarchy& H, int rec, double bytes) {
  if (rec < 0) return;
  Prof::Rec& R = H.prof.recs[rec];
  R.bytes = bytes;
  GIAMG_CUDA(cudaEventRecord(H.prof.ev[R.e1], H.stream));
}
// algorithmic bytes of one CSR row-kernel launch: matrix (values, column indices or one template
// id per row, row pointers), the gathered vector counted once, the output, and `vecs` further
// streamed vectors
double row_bytes(const DCSR& A, int vsize, int vecs) {
  const double index = A.pat.on ? 4.0 * A.n : 4.0 * A.nnz;
  return (double)A.nnz * vsize + index + 8.0 * (A.n + 1) + (double)vsize * A.n * (2 + vecs);
}

// copy count elements of a caller array (host or device) into a new device buffer
template <typename T>
void upload(DBuf<T>& dst, const T* src, size_t count, bool dev, cudaStream_t s) {
  dst.alloc(std::max<size_t>(count, 1), s);
  if (count)
    GIAMG_CUDA(cudaMemcpyAsync(dst.get(), src, count * sizeof(T), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

// Chebyshev coefficients of Saad's Algorithm 12.1 with the Jacobi preconditioner:
// step 0 uses c2 = 1/theta (and no previous direction), step s >= 1 uses
// c1 = rho_s rho_{s-1}, c2 = 2 rho_s / delta with rho_s = 1 / (2 sigma - rho_{s-1}).
struct Cheb {
  std::vector<double> c1, c2;
};
Cheb cheb_coeffs(double rho_hat, double lo, double hi, int k) {
  Cheb c;
  const double a = lo * rho_hat, b = hi * rho_hat;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  double rho = 1.0 / sigma;
  c.c1.push_back(0.0);
  c.c2.push_back(1.0 / theta);
  for (int s = 1; s < k; ++s) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c.c1.push_back(rn * rho);
    c.c2.push_back(2.0 * rn / delta);
    rho = rn;
  }
  return c;
}

struct LevelExtra {
  Cheb cheb;
};

struct Ctx {
  Hierarchy* H;
  std::vector<LevelExtra> ex;
};

// ------------------------------------------------------------------ V-cycle (Algorithm 1)
const double* vcycle64(Hierarchy& H, const std::vector<LevelExtra>& ex, int l, const double* b) {
  Level& L = *H.lev[l];
  cudaStream_t s = H.stream;
  if (L.kind == GIAMG_LEVEL_COARSEST) {  // direct solve of the coarsest matrix
    const int pr = prof_begin(H, kProfCoarsest);
    inverse_apply(L.Ainv.get(), L.nc, b, L.x.get(), s);
    prof_end(H, pr, 8.0 * L.nc * L.nc + 16.0 * L.nc);
    return L.x.get();
  }
  const Cheb& c = ex[l].cheb;
  const int k = (int)c.c1.size();
  double* x = L.x.get();
  double* x2 = L.x2.get();
  const int64_t n = L.A.n;
  const int rc = l == 0 ? kProfL0Rows : kProfCoarseRows;
  // presmooth (x enters as zero: the first step needs no product)
  cheb_first(n, b, L.dinv.get(), c.c2[0], x, L.d.get(), s);
  for (int j = 1; j < k; ++j) {
    const int pr = prof_begin(H, rc);
    cheb_step(L.A, b, x, x2, L.d.get(), L.dinv.get(), c.c1[j], c.c2[j], s, L.avg_row);
    prof_end(H, pr, row_bytes(L.A, 8, 4));
    std::swap(x, x2);
  }
  // residual, restriction (p- or h-), recursion, interpolation and correction
  int pr = prof_begin(H, rc);
  residual(L.A, b, x, L.r.get(), s, L.avg_row);
  prof_end(H, pr, row_bytes(L.A, 8, 1));
  Level& C = *H.lev[l + 1];
  pr = prof_begin(H, kProfTransfer);
  if (L.kind == GIAMG_LEVEL_P) p_restrict(L, L.r.get(), C.b.get(), s);
  else h_restrict(L, L.r.get(), C.b.get(), s);
  prof_end(H, pr, 8.0 * (L.A.n + L.n_next));
  const double* xc = vcycle64(H, ex, l + 1, C.b.get());
  pr = prof_begin(H, kProfTransfer);
  if (L.kind == GIAMG_LEVEL_P) p_prolong(L, xc, x, s);
  else h_prolong(L, xc, x, s);
  prof_end(H, pr, 8.0 * (2 * L.A.n + L.n_next));
  // postsmooth with the same polynomial
  for (int j = 0; j < k; ++j) {
    const int pq = prof_begin(H, rc);
    cheb_step(L.A, b, x, x2, L.d.get(), L.dinv.get(), c.c1[j], c.c2[j], s, L.avg_row);
    prof_end(H, pq, row_bytes(L.A, 8, j == 0 ? 3 : 4));
    std::swap(x, x2);
  }
  return x;
}

const float* vcycle32(Hierarchy& H, const std::vector<LevelExtra>& ex, int l, const float* b) {
  Level& L = *H.lev[l];
  cudaStream_t s = H.stream;
  if (L.kind == GIAMG_LEVEL_COARSEST) {
    const int pr = prof_begin(H, kProfCoarsest);
    inverse_apply32(L.Ainv.get(), L.nc, b, L.x32.get(), s);
    prof_end(H, pr, 8.0 * L.nc * L.nc + 8.0 * L.nc);
    return L.x32.get();
  }
  const Cheb& c = ex[l].cheb;
  const int k = (int)c.c1.size();
  float* x = L.x32.get();
  float* x2 = L.x232.get();
  const int64_t n = L.A.n;
  const int rc = l == 0 ? kProfL0Rows : kProfCoarseRows;
  cheb_first32(n, b, L.dinv32.get(), (float)c.c2[0], x, L.d32.get(), s);
  for (int j = 1; j < k; ++j) {
    const int pr = prof_begin(H, rc);
    cheb_step32(L.A, b, x, x2, L.d32.get(), L.dinv32.get(), (float)c.c1[j], (float)c.c2[j], s, L.avg_row);
    prof_end(H, pr, row_bytes(L.A, 4, 4));
    std::swap(x, x2);
  }
  int pr = prof_begin(H, rc);
  residual32(L.A, b, x, L.r32.get(), s, L.avg_row);
  prof_end(H, pr, row_bytes(L.A, 4, 1));
  Level& C = *H.lev[l + 1];
  pr = prof_begin(H, kProfTransfer);
  if (L.kind == GIAMG_LEVEL_P) p_restrict32(L, L.r32.get(), C.b32.get(), s);
  else h_restrict32(L, L.r32.get(), C.b32.get(), s);
  prof_end(H, pr, 4.0 * (L.A.n + L.n_next));
  const float* xc = vcycle32(H, ex, l + 1, C.b32.get());
  pr = prof_begin(H, kProfTransfer);
  if (L.kind == GIAMG_LEVEL_P) p_prolong32(L, xc, x, s);
  else h_prolong32(L, xc, x, s);
  prof_end(H, pr, 4.0 * (2 * L.A.n + L.n_next));
  for (int j = 0; j < k; ++j) {
    const int pq = prof_begin(H, rc);
    cheb_step32(L.A, b, x, x2, L.d32.get(), L.dinv32.get(), (float)c.c1[j], (float)c.c2[j], s, L.avg_row);
    prof_end(H, pq, row_bytes(L.A, 4, j == 0 ? 3 : 4));
    std::swap(x, x2);
  }
  return x;
}

// z = V(r) from the finest level; returns the device buffer holding z
const double* apply_vcycle(Ctx& C, int precision, const double* r) {
  Hierarchy& H = *C.H;
  Level& L0 = *H.lev[0];
  if (precision == 0) return vcycle64(H, C.ex, 0, r);
  vec_to32(L0.A.n, r, L0.b32.get(), H.stream);
  const float* z32 = vcycle32(H, C.ex, 0, L0.b32.get());
  vec_to64(L0.A.n, z32, H.z.get(), H.stream);
  return H.z.get();
}

void alloc_work(Level& L, cudaStream_t s) {
  const int64_t n = std::max<int64_t>(L.A.n, 1);
  L.x.alloc(n, s); L.x2.alloc(n, s); L.b.alloc(n, s); L.r.alloc(n, s); L.d.alloc(n, s);
  L.x32.alloc(n, s); L.x232.alloc(n, s); L.b32.alloc(n, s); L.r32.alloc(n, s); L.d32.alloc(n, s);
  L.x.zero(s); L.x2.zero(s); L.b.zero(s); L.r.zero(s); L.d.zero(s);
  L.x32.zero(s); L.x232.zero(s); L.b32.zero(s); L.r32.zero(s); L.d32.zero(s);
}

// Galerkin coarse operator A_c = R (A P), R = P^T (Sec. 2)
void galerkin(Level& F, DCSR& Ac, bool keep_R, cudaStream_t s) {
  DCSR R, AP;
  csr_transpose(F.P, R, s);
  // rows of A with identical column sets share A P's pattern: found once per row group
  if (!spgemm_grouped(F.A, F.P, AP, s)) spgemm(F.A, F.P, AP, s);
  // so do rows of R = P^T with identical fine supports (e.g. the coarse nodes inside one element)
  if (R.n >= 1024) groups_build(R, s, 1 << 22, true);
  if (!spgemm_grouped(R, AP, Ac, s)) spgemm(R, AP, Ac, s);
  if (R.grp.on) R.grp = Groups();  // R is kept (h-levels) for its CSR product only
  if (keep_R) {
    F.R = std::move(R);
    csr_to32(F.R, s);
  }
}

// the value copies the chosen row variants read (group-major for the vector hybrid, slices for the
// sliced form), built where missing; a variant whose copy cannot be built falls back to the
// default row kernel.  Copies no variant reads any more are released.
void build_variant_copies(DCSR& A, cudaStream_t s) {
  for (int prec = 0; prec < 2; ++prec) {
    RowVariant& v = prec == 0 ? A.var64 : A.var32;
    if (v.vector && !hybrid_vector_build(A, prec, s)) {
      v.vector = false;
    }
    if (v.sliced && !sliced_build(A, prec, s)) {
      v.sliced = false;
      v.tpr = 0;
    }
  }
  Groups& R = A.grp;
  if (R.hvon && !(A.var32.hybrid && A.var32.vector)) { R.hv.release(); R.hvon = false; }
  if (R.hv64on && !(A.var64.hybrid && A.var64.vector)) { R.hv64.release(); R.hv64on = false; }
  if (R.sv32on && !A.var32.sliced) { R.sv32.release(); R.sv32on = false; }
  if (R.sv64on && !A.var64.sliced) { R.sv64.release(); R.sv64on = false; }
}

void check_coords(const double* coords_h, const std::vector<int32_t>& l2g, int32_t n_elem, int p, int64_t n) {
  // nodes must be the trilinear image of the GLL tensor points of each element
  const int n1 = p + 1, nl = n1 * n1 * n1;
  std::vector<double> xi(n1);
  xi[0] = -1.0;
  xi[p] = 1.0;
  for (int j = 1; j <= p / 2; ++j) {  // Newton on P_{p-1} - x P_p (the GLL interior nodes)
    double t = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double pm = 1.0, pc = t;
      for (int k = 1; k < p; ++k) {
        const double pn = ((2.0 * k + 1.0) * t * pc - k * pm) / (k + 1.0);
        pm = pc;
        pc = pn;
      }
      const double dt = (pm - t * pc) / (-(p + 1.0) * pc);
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    xi[j] = t;
    xi[p - j] = -t;
  }
  if (p % 2 == 0) xi[p / 2] = 0.0;
  for (int32_t e = 0; e < n_elem; ++e) {
    const int32_t* m = &l2g[(size_t)e * nl];
    double v[8][3];
    double h = 0.0;
    for (int c = 0; c < 8; ++c) {
      const int i = (c >> 2) & 1, j = (c >> 1) & 1, k = c & 1;
      const int32_t g = m[(i * p) * n1 * n1 + (j * p) * n1 + k * p];
      GIAMG_CHECK(g >= 0 && g < n, GIAMG_ERR_MAP, "element map entry out of range");
      for (int d = 0; d < 3; ++d) v[c][d] = coords_h[3 * (int64_t)g + d];
    }
    for (int d = 0; d < 3; ++d) h = std::max(h, std::fabs(v[7][d] - v[0][d]));
    for (int a = 0; a < nl; ++a) {
      const int i = a / (n1 * n1), j = (a / n1) % n1, k = a % n1;
      const double s = xi[i], t = xi[j], u = xi[k];
      for (int d = 0; d < 3; ++d) {
        double x = 0.0;
        for (int c = 0; c < 8; ++c) {
          const int ci = (c >> 2) & 1, cj = (c >> 1) & 1, ck = c & 1;
          const double w = (ci ? 1 + s : 1 - s) * (cj ? 1 + t : 1 - t) * (ck ? 1 + u : 1 - u) / 8.0;
          x += w * v[c][d];
        }
        GIAMG_CHECK(std::fabs(x - coords_h[3 * (int64_t)m[a] + d]) <= 1e-8 * std::max(h, 1e-300), GIAMG_ERR_MAP,
                    "coordinates are not the trilinear image of the GLL points of element " + std::to_string(e));
      }
    }
  }
}

__global__ void csr_check_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 unsigned long long* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rp[i], e = rp[i + 1];
    if (e < s) {
      atomicAdd(bad, 1ull);
      continue;
    }
    for (int64_t t = s; t < e; ++t) {
      const int32_t c = ci[t];
      if (c < 0 || c >= n || (t > s && ci[t - 1] >= c)) atomicAdd(bad, 1ull);
    }
  }
}

// Host copy of a caller array.  Device arrays are read on the handle's stream, so an input the
// caller produced on that stream (and not yet finished) is read after it is written.
void read_host(void* dst, const void* src, size_t bytes, bool dev, cudaStream_t s) {
  if (!bytes) return;
  if (!dev) {
    std::memcpy(dst, src, bytes);
    return;
  }
  GIAMG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
  GIAMG_CUDA(cudaStreamSynchronize(s));
}

// Opt-in setup timing (environment GIAMG_SETUP_LOG set): wall time of each setup phase, taken
// after a synchronisation of the stream, printed to stderr.
struct SetupClock {
  bool on = getenv("GIAMG_SETUP_LOG") != nullptr;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  explicit SetupClock(cudaStream_t st) : s(st) {}
  void mark(const char* what, int level = -1) {
    if (!on) return;
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    fprintf(stderr, "setup %-22s level %2d %9.2f ms\n", what, level,
            std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

Ctx* setup_impl(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val, int32_t n_elem,
                const int32_t* elem_dof, const int32_t* elem_order, const double* coords, const giamg_options* optp,
                void* stream) {
  giamg_options opt;
  if (optp) opt = *optp;
  else giamg_default_options(&opt);
  GIAMG_CHECK(n > 0 && n < ((int64_t)1 << 31), GIAMG_ERR_ARG, "n must be in [1, 2^31)");
  GIAMG_CHECK(row_ptr && col_idx && val, GIAMG_ERR_ARG, "row_ptr, col_idx and val are required");
  GIAMG_CHECK(opt.cheb_degree >= 1 && opt.cheb_degree <= 64, GIAMG_ERR_ARG, "cheb_degree must be in [1, 64]");
  GIAMG_CHECK(opt.cheb_lo > 0 && opt.cheb_hi > opt.cheb_lo, GIAMG_ERR_ARG, "need 0 < cheb_lo < cheb_hi");
  GIAMG_CHECK(opt.max_levels >= 1 && opt.max_levels <= 64, GIAMG_ERR_ARG, "max_levels must be in [1, 64]");
  GIAMG_CHECK(opt.lanczos_steps >= 1, GIAMG_ERR_ARG, "lanczos_steps must be >= 1");
  GIAMG_CHECK(opt.precision == 0 || opt.precision == 1, GIAMG_ERR_ARG, "precision must be 0 or 1");
  GIAMG_CHECK(opt.row_form >= 0 && opt.row_form <= 6, GIAMG_ERR_ARG, "row_form must be in 0..6");
  GIAMG_CHECK(opt.row_threads == 0 || opt.row_threads == 4 || opt.row_threads == 8 || opt.row_threads == 16 ||
                  opt.row_threads == 32,
              GIAMG_ERR_ARG, "row_threads must be 0, 4, 8, 16 or 32");
  GIAMG_CHECK(opt.prefetch_rows >= -1, GIAMG_ERR_ARG, "prefetch_rows must be -1, 0 or positive");
  GIAMG_CHECK(opt.graphs >= 0 && opt.graphs <= 2, GIAMG_ERR_ARG, "graphs must be 0, 1 or 2");
  GIAMG_CHECK(opt.p_schedule >= 0 && opt.p_schedule <= 2, GIAMG_ERR_ARG, "p_schedule must be 0, 1 or 2");
  GIAMG_CHECK(opt.basis == 0 || opt.basis == 1, GIAMG_ERR_ARG, "basis must be 0 (nodal) or 1 (modal)");
  GIAMG_CHECK(!(coords && opt.basis == 1), GIAMG_ERR_ARG,
              "coordinates validate nodal elements only; pass NULL with the modal basis");
  GIAMG_CHECK(opt.row_chains == 0 || opt.row_chains == 2 || opt.row_chains == 4 || opt.row_chains == 8, GIAMG_ERR_ARG,
              "row_chains must be 0, 2, 4 or 8");
  const bool dev = opt.device_ptrs != 0;
  cudaStream_t s = (cudaStream_t)stream;

  // element orders: uniform p
  int p = 1;
  if (n_elem > 0) {
    GIAMG_CHECK(elem_order != nullptr, GIAMG_ERR_ARG, "elem_order is required when n_elem > 0");
    std::vector<int32_t> ord(n_elem);
    read_host(ord.data(), elem_order, sizeof(int32_t) * n_elem, dev, s);
    p = ord[0];
    for (int32_t e = 0; e < n_elem; ++e)
      GIAMG_CHECK(ord[e] == p, GIAMG_ERR_ORDER, "element orders are not uniform");
    GIAMG_CHECK(p >= 1 && p <= GIAMG_MAX_ORDER, GIAMG_ERR_ORDER, "element order outside 1..12");
    GIAMG_CHECK(p == 1 || elem_dof != nullptr, GIAMG_ERR_MAP, "elem_dof is required for p > 1");
  } else {
    GIAMG_CHECK(elem_dof == nullptr || n_elem == 0, GIAMG_ERR_ARG, "n_elem must be positive with elem_dof");
  }
  int64_t nnz = 0;
  read_host(&nnz, row_ptr + n, sizeof(int64_t), dev, s);
  GIAMG_CHECK(nnz >= n, GIAMG_ERR_ARG, "row_ptr[n] smaller than n (a diagonal is needed in every row)");

  Ctx* C = new Ctx();
  C->H = new Hierarchy();
  Hierarchy& H = *C->H;
  SetupClock clk(s);
  try {
    H.opt = opt;
    H.stream = s;
    GIAMG_CUDA(cudaGetDevice(&H.device));
    noalloc_prepare();  // the allocation-free residual check's static scratch, loaded while allocating is allowed
    H.n = n;
    Level* L0 = new Level();
    H.lev.push_back(L0);
    L0->order = p;
    L0->A.n = n;
    L0->A.m = n;
    L0->A.nnz = nnz;
    upload(L0->A.rp, row_ptr, (size_t)n + 1, dev, s);
    upload(L0->A.ci, col_idx, (size_t)nnz, dev, s);
    upload(L0->A.v, val, (size_t)nnz, dev, s);
    clk.mark("input copy");
    {
      DBuf<unsigned long long> bad;
      bad.alloc(1, s);
      bad.zero(s);
      { csr_check_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(n, L0->A.rp.get(),
                                                                                            L0->A.ci.get(), bad.get()); note_launch(); }
      GIAMG_CUDA(cudaGetLastError());
      unsigned long long hb = 0;
      GIAMG_CUDA(cudaMemcpyAsync(&hb, bad.get(), sizeof(hb), cudaMemcpyDeviceToHost, s));
      GIAMG_CUDA(cudaStreamSynchronize(s));
      GIAMG_CHECK(hb == 0, GIAMG_ERR_ARG, "CSR invalid: row pointers decrease, or columns out of range / not ascending");
    }
    clk.mark("CSR check");
    L0->avg_row = (double)nnz / n;
    const int nl0 = (p + 1) * (p + 1) * (p + 1);
    if (p > 1) {
      upload(L0->l2g, elem_dof, (size_t)n_elem * nl0, dev, s);
      const int64_t bad = validate_map(L0->A, L0->l2g.get(), n_elem, nl0, s);
      GIAMG_CHECK(bad == 0, GIAMG_ERR_MAP,
                  "element map inconsistent with A: " + std::to_string(bad) + " entries out of range or missing from the pattern");
      L0->n_elem = n_elem;
      clk.mark("element map check");
    }
    if (coords && p >= 1 && n_elem > 0 && elem_dof) {
      std::vector<double> ch((size_t)n * 3);
      std::vector<int32_t> mh((size_t)n_elem * nl0);
      read_host(ch.data(), coords, sizeof(double) * 3 * n, dev, s);
      read_host(mh.data(), elem_dof, sizeof(int32_t) * mh.size(), dev, s);
      check_coords(ch.data(), mh, n_elem, p, n);
    }
    L0->dinv.alloc(n, s);
    L0->dinv32.alloc(n, s);
    GIAMG_CHECK(diag_inverse(L0->A, L0->dinv.get(), L0->dinv32.get(), s), GIAMG_ERR_NOT_SPD,
                "A has a non-positive or missing diagonal entry");

    clk.mark("coordinates, diagonal");
    // p-coarsening (Algorithms 2-4, 7) down to order 1
    while (H.lev.back()->order > 1 && (int)H.lev.size() < opt.max_levels) {
      Level& F = *H.lev.back();
      Level* Cl = new Level();
      F.p = F.order;
      F.q = next_order(F.order, opt.p_schedule);
      F.n_elem = n_elem;
      p_level_build(F, *Cl, opt.basis, s);
      clk.mark("p-level map and P", (int)H.lev.size() - 1);
      if (opt.compress_patterns && !F.A.grp.on) {  // the row groups serve A P below and the row kernels later
        pattern_build(F.A, s, 1 << 16, 1 << 24);
        groups_build(F.A, s, 1 << 22);
        clk.mark("row patterns and groups", (int)H.lev.size() - 1);
      }
      Cl->order = F.q;
      galerkin(F, Cl->A, false, s);
      clk.mark("p-level RAP", (int)H.lev.size() - 1);
      F.kind = GIAMG_LEVEL_P;
      Cl->avg_row = Cl->A.n ? (double)Cl->A.nnz / Cl->A.n : 0.0;
      Cl->dinv.alloc(std::max<int64_t>(Cl->A.n, 1), s);
      Cl->dinv32.alloc(std::max<int64_t>(Cl->A.n, 1), s);
      GIAMG_CHECK(diag_inverse(Cl->A, Cl->dinv.get(), Cl->dinv32.get(), s), GIAMG_ERR_NOT_SPD,
                  "coarse operator has a non-positive diagonal entry");
      H.lev.push_back(Cl);
    }
    // h-coarsening by smoothed aggregation (Sec. 2.5)
    while (H.lev.back()->A.n > opt.coarse_max && (int)H.lev.size() < opt.max_levels) {
      Level& F = *H.lev.back();
      const int64_t n_agg = h_level_aggregate(F, opt.strength_theta, opt.hash_kind, s);
      clk.mark("MIS-2, aggregates", (int)H.lev.size() - 1);
      if ((double)n_agg > 0.9 * (double)F.A.n) {
        F.agg.release();
        F.n_next = 0;
        break;
      }
      h_level_prolongation(F, s);
      Level* Cl = new Level();
      galerkin(F, Cl->A, true, s);
      clk.mark("SA-P and RAP", (int)H.lev.size() - 1);
      F.kind = GIAMG_LEVEL_H;
      Cl->order = 0;
      Cl->avg_row = Cl->A.n ? (double)Cl->A.nnz / Cl->A.n : 0.0;
      Cl->dinv.alloc(std::max<int64_t>(Cl->A.n, 1), s);
      Cl->dinv32.alloc(std::max<int64_t>(Cl->A.n, 1), s);
      GIAMG_CHECK(diag_inverse(Cl->A, Cl->dinv.get(), Cl->dinv32.get(), s), GIAMG_ERR_NOT_SPD,
                  "coarse operator has a non-positive diagonal entry");
      H.lev.push_back(Cl);
    }
    // coarsest level: dense Cholesky
    Level& Lc = *H.lev.back();
    Lc.kind = GIAMG_LEVEL_COARSEST;
    Lc.nc = Lc.A.n;
    GIAMG_CHECK(Lc.nc <= 8192, GIAMG_ERR_ARG,
                "coarsest level has " + std::to_string(Lc.nc) + " rows (> 8192); aggregation stalled");
    Lc.L.alloc((size_t)Lc.nc * Lc.nc, s);
    csr_to_dense_cm(Lc.A, Lc.L.get(), s);
    GIAMG_CHECK(cholesky_factor(Lc.L.get(), Lc.nc, s) == GIAMG_OK, GIAMG_ERR_NOT_SPD,
                "coarsest matrix is not positive definite");
    Lc.Ainv.alloc((size_t)Lc.nc * Lc.nc, s);
    chol_inverse(Lc.L.get(), Lc.nc, Lc.Ainv.get(), s);
    clk.mark("coarsest Cholesky");
    // smoother bounds, FP32 copies, work vectors
    C->ex.resize(H.lev.size());
    for (size_t l = 0; l < H.lev.size(); ++l) {
      Level& L = *H.lev[l];
      csr_to32(L.A, s);
      clk.mark("FP32 copy", (int)l);
      if (opt.compress_patterns) {
        if (!L.A.pat.on && !L.A.grp.on) {  // p-levels with groups have them from the Galerkin product
          pattern_build(L.A, s, 1 << 16, 1 << 24);
          clk.mark("row patterns", (int)l);
          groups_build(L.A, s, 1 << 22);
        }
        batch_pairs_build(L.A, s);
        clk.mark("row groups, hybrid", (int)l);
      }
      choose_rows(L.A, opt.row_form, opt.row_threads);
      build_variant_copies(L.A, s);
      clk.mark("row-form copies", (int)l);
      set_prefetch(L.A, opt.prefetch_rows, opt.row_chains);
      alloc_work(L, s);
      if (L.kind != GIAMG_LEVEL_COARSEST) {
        L.rho = lanczos_rho(L.A, opt.lanczos_steps, opt.hash_kind, H);
        clk.mark("Lanczos", (int)l);
        GIAMG_CHECK(L.rho > 0.0 && std::isfinite(L.rho), GIAMG_ERR_NOT_SPD, "Lanczos bound is not positive");
        C->ex[l].cheb = cheb_coeffs(L.rho, opt.cheb_lo, opt.cheb_hi, opt.cheb_degree);
      }
    }
    // PCG work
    H.r.alloc(n, s); H.z.alloc(n, s); H.p.alloc(n, s); H.q.alloc(n, s);
    H.xw.alloc(n, s); H.rold.alloc(n, s); H.tmp.alloc(n, s);
    H.partial.alloc(2 * kRedBlocks, s);
    H.sc.alloc(1, s);
    H.sc.zero(s);
    GIAMG_CUDA(cudaMallocHost((void**)&H.h_sc, sizeof(Scalars)));
    GIAMG_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    delete C->H;
    delete C;
    throw;
  }
  return C;
}

// staging of caller vectors in host mode
template <typename T>
struct InVecT {
  const T* d = nullptr;
  DBuf<T> buf;
  InVecT(const T* p, int64_t n, bool dev, cudaStream_t s) {
    if (dev) d = p;
    else {
      buf.alloc(std::max<int64_t>(n, 1), s);
      GIAMG_CUDA(cudaMemcpyAsync(buf.get(), p, sizeof(T) * n, cudaMemcpyHostToDevice, s));
      d = buf.get();
    }
  }
};
template <typename T>
struct OutVecT {
  T* d = nullptr;
  T* host = nullptr;
  int64_t n;
  cudaStream_t s;
  DBuf<T> buf;
  OutVecT(T* p, int64_t n_, bool dev, cudaStream_t s_, bool load) : n(n_), s(s_) {
    if (dev) d = p;
    else {
      host = p;
      buf.alloc(std::max<int64_t>(n, 1), s);
      d = buf.get();
      if (load) GIAMG_CUDA(cudaMemcpyAsync(d, p, sizeof(T) * n, cudaMemcpyHostToDevice, s));
    }
  }
  void finish() {
    if (host) GIAMG_CUDA(cudaMemcpyAsync(host, d, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
  }
};
using InVec = InVecT<double>;
using OutVec = OutVecT<double>;

// The two halves of a PCG iteration (Sec. 2: one product with A and one V-cycle per iteration),
// shared by the host-driven loop and the loop captured as a CUDA graph.
// precondition: z = V(r); rho = <z, r> (flexible: <z, r - r_old>); p = z + beta p (p = z first)
void pcg_precondition(Ctx& C, int precision, int first) {
  Hierarchy& H = *C.H;
  const int flexible = precision ? 1 : 0;
  const double* z = apply_vcycle(C, precision, H.r.get());
  pcg_dot_rz(H.n, H.r.get(), z, H.rold.get(), flexible, H.partial.get(), H.stream);
  pcg_finish_rz(H.sc.get(), H.partial.get(), first, flexible, H.stream);
  pcg_update_p(H.n, z, H.p.get(), H.sc.get(), first, H.stream);
}
// step: q = A p; alpha = rho / <p, q>; x += alpha p; r -= alpha q; ||r||^2
void pcg_step(Ctx& C, int precision, double* x) {
  Hierarchy& H = *C.H;
  Level& L0 = *H.lev[0];
  cudaStream_t s = H.stream;
  const int pr = prof_begin(H, kProfOuterSpmv);
  spmv(L0.A, H.p.get(), H.q.get(), s, L0.avg_row);
  prof_end(H, pr, row_bytes(L0.A, 8, 0));
  dot_partial(H.n, H.p.get(), H.q.get(), H.partial.get(), s);
  pcg_finish_pq(H.sc.get(), H.partial.get(), s);
  pcg_update_xr(H.n, H.p.get(), H.q.get(), x, H.r.get(), H.rold.get(), precision ? 1 : 0, H.sc.get(), H.partial.get(), s);
  pcg_finish_rr(H.sc.get(), H.partial.get(), s);
}

// Append a conditional node to the graph being captured on `cs` (after the work captured so far,
// and before what is captured next); returns its body graph.
cudaGraph_t add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  GIAMG_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, &deps, &edges, &nd));
  GIAMG_CHECK(st == cudaStreamCaptureStatusActive, GIAMG_ERR_CUDA, "stream capture is not active");
  cudaGraphNodeParams prm{};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  GIAMG_CUDA(cudaGraphAddNode(&node, g, deps, edges, nd, &prm));
  GIAMG_CUDA(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return prm.conditional.phGraph_out[0];
}

// Capture the whole PCG solve for one V-cycle precision as a CUDA graph:
//   init (r = b, x = 0, ||b||^2); start (relres_0, go = b != 0);
//   IF go: precondition (first);
//   WHILE cont: step; check (relres, stopping rule -> cont); IF cont: precondition.
// The graph reads b from H.gb and writes x to H.gx; rtol and the limit are read from H.gst.
void capture_solve(Ctx& C, int precision) {
  Hierarchy& H = *C.H;
  SolveGraph& G = H.graph[precision];
  if (!H.capture_stream) GIAMG_CUDA(cudaStreamCreateWithFlags(&H.capture_stream, cudaStreamNonBlocking));
  const int64_t cap = (int64_t)H.opt.max_iter + 1;
  if (!H.gb.get()) {
    H.gb.alloc(H.n, H.stream);
    H.gx.alloc(H.n, H.stream);
    H.ghist.alloc(cap, H.stream);
    H.gst.alloc(1, H.stream);
    GIAMG_CUDA(cudaMallocHost((void**)&H.h_gst, sizeof(GraphState)));
  }
  GIAMG_CUDA(cudaStreamSynchronize(H.stream));  // buffers ready before the capture stream uses them
  cudaStream_t user = H.stream;
  cudaStream_t cs = H.capture_stream;
  cudaGraph_t g = nullptr;
  struct Restore {  // the launchers use H.stream: point it at the capture stream meanwhile
    Hierarchy& H;
    cudaStream_t user;
    cudaGraph_t& g;
    ~Restore() {
      H.stream = user;
      cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(H.capture_stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
        cudaGraph_t partial = nullptr;  // a capture that failed part way: end and drop it
        cudaStreamEndCapture(H.capture_stream, &partial);
        if (partial && partial != g) cudaGraphDestroy(partial);
      }
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
    }
  } restore{H, user, g};
  H.stream = cs;
  GIAMG_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h_first, h_loop, h_more;
  GIAMG_CUDA(cudaGraphConditionalHandleCreate(&h_first, g, 0, cudaGraphCondAssignDefault));
  GIAMG_CUDA(cudaGraphConditionalHandleCreate(&h_loop, g, 0, cudaGraphCondAssignDefault));
  const long long c0 = g_launches.load();
  GIAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  pcg_init(H.n, H.gb.get(), H.gx.get(), H.r.get(), H.partial.get(), cs);
  pcg_finish_bb(H.sc.get(), H.partial.get(), cs);
  pcg_graph_start(H.sc.get(), H.gst.get(), H.ghist.get(), h_first, h_loop, cs);
  cudaGraph_t body_first = add_conditional(cs, h_first, cudaGraphCondTypeIf);
  cudaGraph_t body_loop = add_conditional(cs, h_loop, cudaGraphCondTypeWhile);
  GIAMG_CUDA(cudaStreamEndCapture(cs, &g));
  const long long c1 = g_launches.load();
  GIAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, body_first, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  pcg_precondition(C, precision, 1);
  GIAMG_CUDA(cudaStreamEndCapture(cs, &body_first));
  const long long c2 = g_launches.load();
  GIAMG_CUDA(cudaGraphConditionalHandleCreate(&h_more, body_loop, 0, cudaGraphCondAssignDefault));
  GIAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, body_loop, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  pcg_step(C, precision, H.gx.get());
  pcg_graph_check(H.sc.get(), H.gst.get(), H.ghist.get(), h_loop, h_more, cs);
  cudaGraph_t body_more = add_conditional(cs, h_more, cudaGraphCondTypeIf);
  GIAMG_CUDA(cudaStreamEndCapture(cs, &body_loop));
  const long long c3 = g_launches.load();
  GIAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, body_more, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  pcg_precondition(C, precision, 0);
  GIAMG_CUDA(cudaStreamEndCapture(cs, &body_more));
  const long long c4 = g_launches.load();
  GIAMG_CUDA(cudaGraphInstantiate(&G.exec, g, 0));
  G.n_init = c1 - c0;
  G.n_first = c2 - c1;
  G.n_loop = c3 - c2;
  G.n_more = c4 - c3;
  g_launches.fetch_sub(c4 - c0);  // captured, not executed
}

int solve_impl(Ctx& C, int precision, int force_iters, const double* b_in, double* x_out, double rtol, int* iters,
               double* relres) {
  Hierarchy& H = *C.H;
  cudaStream_t s = H.stream;
  const int64_t n = H.n;
  const bool dev = H.opt.device_ptrs != 0;
  GIAMG_CHECK(b_in && x_out, GIAMG_ERR_ARG, "b and x are required");
  GIAMG_CHECK(precision == 0 || precision == 1, GIAMG_ERR_ARG, "precision must be 0 or 1");
  GIAMG_CHECK(rtol >= 0.0, GIAMG_ERR_ARG, "rtol must be non-negative");
  const int limit = force_iters > 0 ? force_iters : H.opt.max_iter;
  int it = 0;
  double rr = 1.0;
  int status = GIAMG_OK;
  // the graph path: profiling off (its events are host-recorded) and the limit within the
  // capacity of the captured history
  SolveGraph& SG = H.graph[precision];
  const bool graph = H.opt.graphs && !H.prof.on && limit <= H.opt.max_iter && (SG.exec || ++SG.uses >= (H.opt.graphs == 2 ? 1 : 2));
  if (graph) {
    if (!SG.exec) capture_solve(C, precision);
    const SolveGraph& G = H.graph[precision];
    GIAMG_CUDA(cudaMemcpyAsync(H.gb.get(), b_in, sizeof(double) * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    GraphState& hs = *H.h_gst;
    hs = GraphState{rtol, 1.0, limit, force_iters > 0 ? 1 : 0, 0, 0};
    GIAMG_CUDA(cudaMemcpyAsync(H.gst.get(), &hs, sizeof(GraphState), cudaMemcpyHostToDevice, s));
    GIAMG_CUDA(cudaGraphLaunch(G.exec, s));
    GIAMG_CUDA(cudaMemcpyAsync(&hs, H.gst.get(), sizeof(GraphState), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaMemcpyAsync(x_out, H.gx.get(), sizeof(double) * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    vec_copy(n, H.gb.get(), H.tmp.get(), s);  // b and x for the true residual of giamg_solve_stats
    vec_copy(n, H.gx.get(), H.xw.get(), s);
    GIAMG_CUDA(cudaStreamSynchronize(s));
    it = hs.it;
    rr = hs.relres;
    status = hs.status;
    H.hist.assign((size_t)it + 1, 0.0);
    GIAMG_CUDA(cudaMemcpyAsync(H.hist.data(), H.ghist.get(), sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    if (status) H.hist.resize(it);  // breakdown: the last iteration recorded no residual
    const long long run = G.n_init + (H.hist[0] != 0.0 && limit > 0 ? G.n_first + it * G.n_loop + std::max(it - 1, 0) * G.n_more : 0);
    g_launches.fetch_add(run);
    if (status == GIAMG_OK && H.hist[0] != 0.0 && force_iters <= 0 && !(rr <= rtol)) status = GIAMG_ERR_MAXITER;
    if (H.hist[0] == 0.0) rr = 0.0;
  } else {
    InVec b(b_in, n, dev, s);
    OutVec x(x_out, n, dev, s, false);
    Scalars* sc = H.sc.get();
    H.hist.clear();
    pcg_init(n, b.d, x.d, H.r.get(), H.partial.get(), s);
    pcg_finish_bb(sc, H.partial.get(), s);
    GIAMG_CUDA(cudaMemcpyAsync(H.h_sc, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    const double bb = H.h_sc->bb;
    if (bb == 0.0) {
      H.hist.push_back(0.0);
      rr = 0.0;
    } else {
      H.hist.push_back(1.0);
      if (limit > 0) pcg_precondition(C, precision, 1);
      while (it < limit) {
        pcg_step(C, precision, x.d);
        GIAMG_CUDA(cudaMemcpyAsync(H.h_sc, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
        GIAMG_CUDA(cudaStreamSynchronize(s));
        ++it;
        if (H.h_sc->status != 0) {
          status = GIAMG_ERR_BREAKDOWN;
          break;
        }
        rr = std::sqrt(H.h_sc->rr / bb);
        H.hist.push_back(rr);
        if (force_iters <= 0 && rr <= rtol) break;
        if (it == limit) break;
        pcg_precondition(C, precision, 0);
      }
      if (status == GIAMG_OK && force_iters <= 0 && !(rr <= rtol)) status = GIAMG_ERR_MAXITER;
    }
    // keep b and x for the true residual of giamg_solve_stats
    vec_copy(n, b.d, H.tmp.get(), s);
    vec_copy(n, x.d, H.xw.get(), s);
    x.finish();
  }
  H.last_iters = it;
  H.last_true_relres = -1.0;
  if (iters) *iters = it;
  if (relres) *relres = rr;
  if (status == GIAMG_ERR_BREAKDOWN) throw Error{status, "CG breakdown (p^T A p <= 0, r^T z <= 0 or NaN)"};
  if (status == GIAMG_ERR_MAXITER) throw Error{status, "max_iter reached before rtol"};
  return GIAMG_OK;
}

// ------------------------------------------------------------------ multi-right-hand-side solve
void drop_batch_graphs(Hierarchy& H) {
  for (auto* set : {&H.bgraph, &H.kgraph})
    for (auto& per_m : *set)
      for (SolveGraph& G : per_m)
        if (G.exec) {
          GIAMG_CUDA(cudaGraphExecDestroy(G.exec));
          G = SolveGraph{};
        }
}

void alloc_batch(Hierarchy& H, int m) {
  if (H.bm >= m) return;
  cudaStream_t s = H.stream;
  drop_batch_graphs(H);  // captured graphs hold the old buffers
  for (Level* Lp : H.lev) {
    Level& L = *Lp;
    const size_t nm = (size_t)std::max<int64_t>(L.A.n, 1) * m;
    L.bx.alloc(nm, s); L.bx2.alloc(nm, s); L.bb.alloc(nm, s); L.br.alloc(nm, s); L.bd.alloc(nm, s);
    L.bx32.alloc(nm, s); L.bx232.alloc(nm, s); L.bb32.alloc(nm, s); L.br32.alloc(nm, s); L.bd32.alloc(nm, s);
    if (L.kind == GIAMG_LEVEL_P) {
      const size_t pm = (size_t)L.n_elem * (L.q + 1) * (L.q + 1) * (L.q + 1) * m;
      L.bpart.alloc(pm, s);
      L.bpart32.alloc(pm, s);
    }
    L.bm = m;
  }
  const size_t nm = (size_t)H.n * m;
  H.bR.alloc(nm, s); H.bZ.alloc(nm, s); H.bP.alloc(nm, s); H.bQ.alloc(nm, s); H.bRold.alloc(nm, s);
  H.bX.alloc(nm, s); H.bB.alloc(nm, s);
  H.bpartial.alloc((size_t)2 * batch_reduction_blocks() * 32, s);
  H.bsc.alloc(batch_scalars_bytes(), s);
  H.kpartial.alloc((size_t)block_gram_blocks() * 2 * 1024, s);
  H.kst.alloc(1, s);
  if (!H.h_bsc) GIAMG_CUDA(cudaMallocHost(&H.h_bsc, batch_scalars_bytes()));
  H.bm = m;
}

// Algorithm 1 on m columns at once (same smoother polynomial and transfers as vcycle64)
const double* bvcycle64(Hierarchy& H, const std::vector<LevelExtra>& ex, int l, int m, const double* b) {
  Level& L = *H.lev[l];
  cudaStream_t s = H.stream;
  if (L.kind == GIAMG_LEVEL_COARSEST) {
    bat_inverse(L.Ainv.get(), L.nc, m, b, L.bx.get(), s);
    return L.bx.get();
  }
  const Cheb& c = ex[l].cheb;
  const int k = (int)c.c1.size();
  double* x = L.bx.get();
  double* x2 = L.bx2.get();
  const int64_t n = L.A.n;
  bat_cheb_first64(n, m, b, L.dinv.get(), c.c2[0], x, L.bd.get(), s);
  for (int j = 1; j < k; ++j) {
    bat_rows_launch64(L.A, m, 2, L.A.v.get(), x, b, x2, L.bd.get(), L.dinv.get(), c.c1[j], c.c2[j], s);
    std::swap(x, x2);
  }
  bat_rows_launch64(L.A, m, 1, L.A.v.get(), x, b, L.br.get(), nullptr, nullptr, 0.0, 0.0, s);
  Level& C = *H.lev[l + 1];
  if (L.kind == GIAMG_LEVEL_P) bat_p_restrict(L, m, L.br.get(), C.bb.get(), L.bpart.get(), s);
  else bat_rows_launch64(L.R, m, 0, L.R.v.get(), L.br.get(), nullptr, C.bb.get(), nullptr, nullptr, 0.0, 0.0, s);
  const double* xc = bvcycle64(H, ex, l + 1, m, C.bb.get());
  if (L.kind == GIAMG_LEVEL_P) bat_p_prolong(L, m, xc, x, s);
  else bat_rows_launch64(L.P, m, 3, L.P.v.get(), xc, nullptr, x, nullptr, nullptr, 0.0, 0.0, s);
  for (int j = 0; j < k; ++j) {
    bat_rows_launch64(L.A, m, 2, L.A.v.get(), x, b, x2, L.bd.get(), L.dinv.get(), c.c1[j], c.c2[j], s);
    std::swap(x, x2);
  }
  return x;
}

const float* bvcycle32(Hierarchy& H, const std::vector<LevelExtra>& ex, int l, int m, const float* b) {
  Level& L = *H.lev[l];
  cudaStream_t s = H.stream;
  if (L.kind == GIAMG_LEVEL_COARSEST) {
    bat_inverse32(L.Ainv.get(), L.nc, m, b, L.bx32.get(), s);
    return L.bx32.get();
  }
  const Cheb& c = ex[l].cheb;
  const int k = (int)c.c1.size();
  float* x = L.bx32.get();
  float* x2 = L.bx232.get();
  const int64_t n = L.A.n;
  bat_cheb_first32(n, m, b, L.dinv32.get(), (float)c.c2[0], x, L.bd32.get(), s);
  for (int j = 1; j < k; ++j) {
    bat_rows_launch32(L.A, m, 2, L.A.v32.get(), x, b, x2, L.bd32.get(), L.dinv32.get(), (float)c.c1[j], (float)c.c2[j], s);
    std::swap(x, x2);
  }
  bat_rows_launch32(L.A, m, 1, L.A.v32.get(), x, b, L.br32.get(), nullptr, nullptr, 0.f, 0.f, s);
  Level& C = *H.lev[l + 1];
  if (L.kind == GIAMG_LEVEL_P) bat_p_restrict32(L, m, L.br32.get(), C.bb32.get(), L.bpart32.get(), s);
  else bat_rows_launch32(L.R, m, 0, L.R.v32.get(), L.br32.get(), nullptr, C.bb32.get(), nullptr, nullptr, 0.f, 0.f, s);
  const float* xc = bvcycle32(H, ex, l + 1, m, C.bb32.get());
  if (L.kind == GIAMG_LEVEL_P) bat_p_prolong32(L, m, xc, x, s);
  else bat_rows_launch32(L.P, m, 3, L.P.v32.get(), xc, nullptr, x, nullptr, nullptr, 0.f, 0.f, s);
  for (int j = 0; j < k; ++j) {
    bat_rows_launch32(L.A, m, 2, L.A.v32.get(), x, b, x2, L.bd32.get(), L.dinv32.get(), (float)c.c1[j], (float)c.c2[j], s);
    std::swap(x, x2);
  }
  return x;
}

const double* apply_bvcycle(Ctx& C, int precision, int m, const double* r) {
  Hierarchy& H = *C.H;
  Level& L0 = *H.lev[0];
  if (precision == 0) return bvcycle64(H, C.ex, 0, m, r);
  bat_to32(L0.A.n * m, r, L0.bb32.get(), H.stream);
  const float* z32 = bvcycle32(H, C.ex, 0, m, L0.bb32.get());
  bat_to64(L0.A.n * m, z32, H.bZ.get(), H.stream);
  return H.bZ.get();
}

// The halves of a multi-right-hand-side iteration, shared by the host loop and the graph.
void bat_precondition(Ctx& C, int precision, int m, int first) {
  Hierarchy& H = *C.H;
  const double* Z = apply_bvcycle(C, precision, m, H.bR.get());
  bat_pcg_rz(H.n, m, H.bR.get(), Z, H.bRold.get(), precision ? 1 : 0, first, H.bpartial.get(), H.bsc.get(), H.stream);
  bat_pcg_update_p(H.n, m, Z, H.bP.get(), H.bsc.get(), first, H.stream);
}
void bat_step(Ctx& C, int precision, int m, double* X) {
  Hierarchy& H = *C.H;
  Level& L0 = *H.lev[0];
  cudaStream_t s = H.stream;
  bat_rows_launch64(L0.A, m, 0, L0.A.v.get(), H.bP.get(), nullptr, H.bQ.get(), nullptr, nullptr, 0.0, 0.0, s);
  bat_pcg_pq(H.n, m, H.bP.get(), H.bQ.get(), H.bpartial.get(), H.bsc.get(), s);
  bat_pcg_update_xr(H.n, m, H.bP.get(), H.bQ.get(), X, H.bR.get(), H.bRold.get(), precision ? 1 : 0, H.bpartial.get(),
                    H.bsc.get(), s);
}

// The halves of a block CG iteration (O'Leary 1980, A-conjugate directions): after the
// V-cycle, beta = -G^+ Q^T Z and P = Z + P beta; the step Q = A P, G = P^T Q, C = P^T R,
// alpha = G^+ C, X += P alpha, R -= Q alpha.
// With the FP32 V-cycle (precision 1) the Gram products and P beta take FP32 arithmetic.
void blk_precondition(Ctx& C, int precision, int m, int first) {
  Hierarchy& H = *C.H;
  const double* Z = apply_bvcycle(C, precision, m, H.bR.get());
  if (!first) {
    blk_gram(H.n, m, H.bQ.get(), Z, nullptr, precision, H.kpartial.get(), H.kst.get(), H.stream);
    blk_coef(m, 1, precision ? kBlockDropTol32 : kBlockDropTol, H.kst.get(), H.stream);
  }
  blk_update_p(H.n, m, Z, H.bP.get(), H.kst.get(), first, precision, H.stream);
}
void blk_step(Ctx& C, int precision, int m, double* X) {
  Hierarchy& H = *C.H;
  Level& L0 = *H.lev[0];
  cudaStream_t s = H.stream;
  bat_rows_launch64(L0.A, m, 0, L0.A.v.get(), H.bP.get(), nullptr, H.bQ.get(), nullptr, nullptr, 0.0, 0.0, s);
  blk_gram(H.n, m, H.bP.get(), H.bQ.get(), H.bR.get(), precision, H.kpartial.get(), H.kst.get(), s);
  blk_coef(m, 0, precision ? kBlockDropTol32 : kBlockDropTol, H.kst.get(), s);
  blk_update_xr(H.n, m, H.bP.get(), H.bQ.get(), X, H.bR.get(), H.kst.get(), H.bpartial.get(), H.bsc.get(), s);
}

// Capture the multi-right-hand-side solve for (precision, m) as one CUDA graph, shaped like the
// single-vector one: init; start; IF go: precondition (first); WHILE cont: step; check;
// IF cont: precondition.  It reads B from H.bB and writes X to H.bX.  block: block CG instead
// of independent columns.
void capture_batch(Ctx& C, int precision, int m, bool block) {
  Hierarchy& H = *C.H;
  SolveGraph& G = (block ? H.kgraph : H.bgraph)[precision][m];
  auto precondition = block ? blk_precondition : bat_precondition;
  auto step = block ? blk_step : bat_step;
  if (!H.capture_stream) GIAMG_CUDA(cudaStreamCreateWithFlags(&H.capture_stream, cudaStreamNonBlocking));
  if (!H.bgst.get()) {
    H.bgst.alloc(1, H.stream);
    GIAMG_CUDA(cudaMallocHost((void**)&H.h_bgst, sizeof(BatchGraphState)));
  }
  GIAMG_CUDA(cudaStreamSynchronize(H.stream));
  cudaStream_t user = H.stream;
  cudaStream_t cs = H.capture_stream;
  cudaGraph_t g = nullptr;
  struct Restore {
    Hierarchy& H;
    cudaStream_t user;
    cudaGraph_t& g;
    ~Restore() {
      H.stream = user;
      cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(H.capture_stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
        cudaGraph_t partial = nullptr;
        cudaStreamEndCapture(H.capture_stream, &partial);
        if (partial && partial != g) cudaGraphDestroy(partial);
      }
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
    }
  } restore{H, user, g};
  H.stream = cs;
  GIAMG_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h_first, h_loop, h_more;
  GIAMG_CUDA(cudaGraphConditionalHandleCreate(&h_first, g, 0, cudaGraphCondAssignDefault));
  GIAMG_CUDA(cudaGraphConditionalHandleCreate(&h_loop, g, 0, cudaGraphCondAssignDefault));
  const long long c0 = g_launches.load();
  GIAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  bat_pcg_init(H.n, m, H.bB.get(), H.bX.get(), H.bR.get(), H.bpartial.get(), H.bsc.get(), cs);
  bat_graph_start_launch(H.bsc.get(), m, H.bgst.get(), h_first, h_loop, cs);
  cudaGraph_t body_first = add_conditional(cs, h_first, cudaGraphCondTypeIf);
  cudaGraph_t body_loop = add_conditional(cs, h_loop, cudaGraphCondTypeWhile);
  GIAMG_CUDA(cudaStreamEndCapture(cs, &g));
  const long long c1 = g_launches.load();
  GIAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, body_first, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  precondition(C, precision, m, 1);
  GIAMG_CUDA(cudaStreamEndCapture(cs, &body_first));
  const long long c2 = g_launches.load();
  GIAMG_CUDA(cudaGraphConditionalHandleCreate(&h_more, body_loop, 0, cudaGraphCondAssignDefault));
  GIAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, body_loop, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  step(C, precision, m, H.bX.get());
  bat_graph_check_launch(H.bsc.get(), m, H.bgst.get(), h_loop, h_more, cs);
  cudaGraph_t body_more = add_conditional(cs, h_more, cudaGraphCondTypeIf);
  GIAMG_CUDA(cudaStreamEndCapture(cs, &body_loop));
  const long long c3 = g_launches.load();
  GIAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, body_more, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  precondition(C, precision, m, 0);
  GIAMG_CUDA(cudaStreamEndCapture(cs, &body_more));
  const long long c4 = g_launches.load();
  GIAMG_CUDA(cudaGraphInstantiate(&G.exec, g, 0));
  G.n_init = c1 - c0;
  G.n_first = c2 - c1;
  G.n_loop = c3 - c2;
  G.n_more = c4 - c3;
  g_launches.fetch_sub(c4 - c0);
}

int solve_batch_impl(Ctx& C, int precision, int force_iters, int m, const double* B_in, double* X_out, double rtol,
                     int* iters, double* relres, bool block) {
  Hierarchy& H = *C.H;
  cudaStream_t s = H.stream;
  const int64_t n = H.n;
  GIAMG_CHECK(m >= 1 && m <= 32, GIAMG_ERR_ARG, "m must be in [1, 32]");
  GIAMG_CHECK(B_in && X_out, GIAMG_ERR_ARG, "B and X are required");
  GIAMG_CHECK(precision == 0 || precision == 1, GIAMG_ERR_ARG, "precision must be 0 or 1");
  GIAMG_CHECK(rtol >= 0.0, GIAMG_ERR_ARG, "rtol must be non-negative");
  alloc_batch(H, m);
  const bool dev = H.opt.device_ptrs != 0;
  BatchScalarsHost* hs = (BatchScalarsHost*)H.h_bsc;
  void* sc = H.bsc.get();
  const int force = force_iters > 0 ? 1 : 0;
  const int limit = force ? force_iters : H.opt.max_iter;
  // the stopping rule's parameters live on the device (both paths read them there)
  hs->tol2 = rtol * rtol;
  hs->force = force;
  GIAMG_CUDA(cudaMemcpyAsync((char*)sc + offsetof(BatchScalarsHost, tol2), &hs->tol2, sizeof(double) + 2 * sizeof(int),
                             cudaMemcpyHostToDevice, s));
  std::vector<int> its(m, 0);
  int it = 0;
  bool breakdown = false;
  SolveGraph& BG = (block ? H.kgraph : H.bgraph)[precision][m];
  if (H.opt.graphs && !H.prof.on && (BG.exec || ++BG.uses >= (H.opt.graphs == 2 ? 1 : 2))) {
    if (!BG.exec) capture_batch(C, precision, m, block);
    const SolveGraph& G = BG;
    GIAMG_CUDA(cudaMemcpyAsync(H.bB.get(), B_in, sizeof(double) * n * m, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    BatchGraphState& gs = *H.h_bgst;
    gs.limit = limit;
    GIAMG_CUDA(cudaMemcpyAsync(&H.bgst.get()->limit, &gs.limit, sizeof(int), cudaMemcpyHostToDevice, s));
    GIAMG_CUDA(cudaGraphLaunch(G.exec, s));
    GIAMG_CUDA(cudaMemcpyAsync(&gs, H.bgst.get(), sizeof(BatchGraphState), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaMemcpyAsync(hs, sc, sizeof(BatchScalarsHost), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaMemcpyAsync(X_out, H.bX.get(), sizeof(double) * n * m, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    it = gs.it;
    breakdown = gs.breakdown != 0;
    for (int j = 0; j < m; ++j) its[j] = block ? it : gs.its[j];
    const bool ran = it > 0;
    g_launches.fetch_add(G.n_init + (ran ? G.n_first + it * G.n_loop + (it - 1) * G.n_more : 0));
  } else {
    const double* Bd = B_in;
    double* Xd = X_out;
    if (!dev) {
      GIAMG_CUDA(cudaMemcpyAsync(H.bB.get(), B_in, sizeof(double) * n * m, cudaMemcpyHostToDevice, s));
      Bd = H.bB.get();
      Xd = H.bX.get();
    }
    bat_pcg_init(n, m, Bd, Xd, H.bR.get(), H.bpartial.get(), sc, s);
    GIAMG_CUDA(cudaMemcpyAsync(hs, sc, sizeof(BatchScalarsHost), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    int active = 0;
    for (int j = 0; j < m; ++j) active += hs->active[j];
    auto precondition = block ? blk_precondition : bat_precondition;
    auto step = block ? blk_step : bat_step;
    if (active > 0 && limit > 0) precondition(C, precision, m, 1);
    while (active > 0 && it < limit) {
      step(C, precision, m, Xd);
      const std::vector<int> was(hs->active, hs->active + m);
      GIAMG_CUDA(cudaMemcpyAsync(hs, sc, sizeof(BatchScalarsHost), cudaMemcpyDeviceToHost, s));
      GIAMG_CUDA(cudaStreamSynchronize(s));
      ++it;
      active = 0;
      for (int j = 0; j < m; ++j) {
        if (was[j] || block) its[j] = it;
        if (hs->status[j] != 0) breakdown = true;
        active += hs->active[j];
      }
      if (breakdown || active == 0 || it == limit) break;
      precondition(C, precision, m, 0);
    }
    if (!dev) GIAMG_CUDA(cudaMemcpyAsync(X_out, Xd, sizeof(double) * n * m, cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
  }
  bool unconverged = false;
  for (int j = 0; j < m; ++j) {
    const double rr = hs->bb[j] > 0.0 ? std::sqrt(hs->rr[j] / hs->bb[j]) : 0.0;
    if (iters) iters[j] = its[j];
    if (relres) relres[j] = rr;
    if (!force && !(rr <= rtol)) unconverged = true;
  }
  if (breakdown) throw Error{GIAMG_ERR_BREAKDOWN, block ? "block CG breakdown" : "CG breakdown in at least one column"};
  if (unconverged) throw Error{GIAMG_ERR_MAXITER, "max_iter reached before rtol in at least one column"};
  return GIAMG_OK;
}

// ------------------------------------------------------------------ grouped solves
// The multi-right-hand-side solves of several hierarchies at once (FP32 V-cycle in FP64 flexible
// CG): every phase of an iteration is one launch for all hierarchies that take part in it, and
// each hierarchy runs exactly the kernel sequence of its own solve_batch_impl host loop, with the
// same per-block arithmetic (the grouped kernels give each hierarchy its standalone grid), so its
// results are bit for bit those of giamg_solve_batch.  The V-cycle is aligned by level index:
// hierarchies with fewer levels reach their coarsest solve earlier and wait for the ascent.
struct GroupMember {
  Ctx* C;
  int m;
  const double* B;
  double* X;
  int it = 0;
  bool running = false, breakdown = false;
  std::vector<int> its;
  std::vector<float*> x, x2;  // per level: the V-cycle iterate and its spare
};

GrpVecArgs gv(int64_t n, int m, const void* a = nullptr, const void* b = nullptr, void* c = nullptr, void* d = nullptr,
              const void* e = nullptr, double v = 0.0, void* sc = nullptr, double* partial = nullptr, int f1 = 0,
              int f2 = 0) {
  GrpVecArgs g{};
  g.n = n;
  g.m = m;
  g.a = a;
  g.b = b;
  g.c = c;
  g.d = d;
  g.e = e;
  g.v = v;
  g.sc = sc;
  g.partial = partial;
  g.flag1 = f1;
  g.flag2 = f2;
  return g;
}

void group_vcycle32(std::vector<GroupMember*>& ms, cudaStream_t s) {
  std::vector<GrpVecArgs> va;
  int maxL = 0, maxk = 0;
  for (GroupMember* g : ms) {
    Hierarchy& H = *g->C->H;
    va.push_back(gv(H.lev[0]->A.n * g->m, g->m, H.bR.get(), nullptr, H.lev[0]->bb32.get()));
    maxL = std::max(maxL, (int)H.lev.size());
    for (size_t l = 0; l < H.lev.size(); ++l)
      if (H.lev[l]->kind != GIAMG_LEVEL_COARSEST) maxk = std::max(maxk, (int)g->C->ex[l].cheb.c1.size());
    g->x.assign(H.lev.size(), nullptr);
    g->x2.assign(H.lev.size(), nullptr);
  }
  grp_vec(kGvTo32H, va, s);
  auto smoothing = [&](int l, int j0, std::vector<GroupMember*>& S) {
    for (int j = j0; j < maxk; ++j) {
      std::vector<GrpRowsArgs> ra;
      std::vector<GroupMember*> took;
      for (GroupMember* g : S) {
        const Cheb& c = g->C->ex[l].cheb;
        if (j >= (int)c.c1.size()) continue;
        Level& L = *g->C->H->lev[l];
        ra.push_back(grp_rows_args(L.A, g->m, L.A.v32.get(), g->x[l], L.bb32.get(), g->x2[l], L.bd32.get(),
                                   L.dinv32.get(), (float)c.c1[j], (float)c.c2[j], true));
        took.push_back(g);
      }
      if (ra.empty()) continue;
      grp_rows32(2, ra, s);
      for (GroupMember* g : took) std::swap(g->x[l], g->x2[l]);
    }
  };
  // descent: presmoothing, residual, restriction; coarsest solves where a hierarchy ends
  for (int l = 0; l < maxL; ++l) {
    std::vector<GroupMember*> S;
    std::vector<GrpVecArgs> inv, first;
    for (GroupMember* g : ms) {
      Hierarchy& H = *g->C->H;
      if (l >= (int)H.lev.size()) continue;
      Level& L = *H.lev[l];
      if (L.kind == GIAMG_LEVEL_COARSEST) {
        inv.push_back(gv(L.nc, g->m, L.Ainv.get(), L.bb32.get(), L.bx32.get()));
        g->x[l] = L.bx32.get();
        continue;
      }
      g->x[l] = L.bx32.get();
      g->x2[l] = L.bx232.get();
      first.push_back(gv(L.A.n, g->m, L.bb32.get(), L.dinv32.get(), g->x[l], L.bd32.get(), nullptr,
                         (double)(float)g->C->ex[l].cheb.c2[0]));
      S.push_back(g);
    }
    if (!inv.empty()) grp_vec(kGvInverse32H, inv, s);
    if (S.empty()) continue;
    grp_vec(kGvChebFirst32H, first, s);
    smoothing(l, 1, S);
    std::vector<GrpRowsArgs> res, hres;
    std::vector<GrpTransferArgs> pres;
    for (GroupMember* g : S) {
      Hierarchy& H = *g->C->H;
      Level& L = *H.lev[l];
      Level& Cn = *H.lev[l + 1];
      res.push_back(grp_rows_args(L.A, g->m, L.A.v32.get(), g->x[l], L.bb32.get(), L.br32.get(), nullptr, nullptr,
                                  0.0, 0.0, true));
      if (L.kind == GIAMG_LEVEL_P) pres.push_back(grp_transfer_args(L, g->m, L.br32.get(), Cn.bb32.get(), L.bpart32.get()));
      else hres.push_back(grp_rows_args(L.R, g->m, L.R.v32.get(), L.br32.get(), nullptr, Cn.bb32.get(), nullptr,
                                        nullptr, 0.0, 0.0, true));
    }
    grp_rows32(1, res, s);
    if (!pres.empty()) grp_p_restrict32(pres, s);
    if (!hres.empty()) grp_rows32(0, hres, s);
  }
  // ascent: interpolation and correction, postsmoothing
  for (int l = maxL - 2; l >= 0; --l) {
    std::vector<GroupMember*> S;
    std::vector<GrpRowsArgs> hpro;
    std::vector<GrpTransferArgs> ppro;
    for (GroupMember* g : ms) {
      Hierarchy& H = *g->C->H;
      if (l >= (int)H.lev.size() - 1) continue;
      Level& L = *H.lev[l];
      const float* xc = g->x[l + 1];
      if (L.kind == GIAMG_LEVEL_P) ppro.push_back(grp_transfer_args(L, g->m, xc, g->x[l], nullptr));
      else hpro.push_back(grp_rows_args(L.P, g->m, L.P.v32.get(), xc, nullptr, g->x[l], nullptr, nullptr, 0.0, 0.0,
                                        true));
      S.push_back(g);
    }
    if (S.empty()) continue;
    if (!ppro.empty()) grp_p_prolong32(ppro, s);
    if (!hpro.empty()) grp_rows32(3, hpro, s);
    smoothing(l, 0, S);
  }
  va.clear();
  for (GroupMember* g : ms) {
    Hierarchy& H = *g->C->H;
    va.push_back(gv(H.lev[0]->A.n * g->m, g->m, g->x[0], nullptr, H.bZ.get()));
  }
  grp_vec(kGvTo64H, va, s);
}

void group_precondition(std::vector<GroupMember*>& ms, int first, cudaStream_t s) {
  group_vcycle32(ms, s);
  std::vector<GrpVecArgs> rz, fin, up;
  for (GroupMember* g : ms) {
    Hierarchy& H = *g->C->H;
    rz.push_back(gv(H.n, g->m, H.bR.get(), H.bZ.get(), nullptr, nullptr, H.bRold.get(), 0.0, nullptr, H.bpartial.get(), 1));
    fin.push_back(gv(0, g->m, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, H.bsc.get(), H.bpartial.get(), first, 1));
    up.push_back(gv(H.n, g->m, H.bZ.get(), nullptr, H.bP.get(), nullptr, nullptr, 0.0, H.bsc.get(), nullptr, first));
  }
  grp_vec(kGvDotRzH, rz, s);
  grp_vec(kGvFinishRzH, fin, s);
  grp_vec(kGvUpdatePH, up, s);
}

void group_step(std::vector<GroupMember*>& ms, cudaStream_t s) {
  std::vector<GrpRowsArgs> q;
  std::vector<GrpVecArgs> dot, fpq, uxr, frr;
  for (GroupMember* g : ms) {
    Hierarchy& H = *g->C->H;
    Level& L0 = *H.lev[0];
    q.push_back(grp_rows_args(L0.A, g->m, L0.A.v.get(), H.bP.get(), nullptr, H.bQ.get(), nullptr, nullptr, 0.0, 0.0, false));
    dot.push_back(gv(H.n, g->m, H.bP.get(), H.bQ.get(), nullptr, nullptr, nullptr, 0.0, nullptr, H.bpartial.get()));
    fpq.push_back(gv(0, g->m, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, H.bsc.get(), H.bpartial.get()));
    uxr.push_back(gv(H.n, g->m, H.bP.get(), H.bQ.get(), g->X, H.bR.get(), H.bRold.get(), 0.0, H.bsc.get(),
                     H.bpartial.get(), 1));
    frr.push_back(gv(0, g->m, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, H.bsc.get(), H.bpartial.get()));
  }
  grp_rows64(0, q, s);
  grp_vec(kGvDotH, dot, s);
  grp_vec(kGvFinishPqH, fpq, s);
  grp_vec(kGvUpdateXrH, uxr, s);
  grp_vec(kGvFinishRrH, frr, s);
}

void solve_grouped_impl(std::vector<GroupMember>& mem, double rtol, int* iters, double* relres, int* status) {
  GIAMG_CHECK(!mem.empty(), GIAMG_ERR_ARG, "no hierarchies");
  GIAMG_CHECK(rtol >= 0.0, GIAMG_ERR_ARG, "rtol must be non-negative");
  Hierarchy& H0 = *mem[0].C->H;
  cudaStream_t s = H0.stream;
  for (size_t i = 0; i < mem.size(); ++i) {
    Hierarchy& H = *mem[i].C->H;
    GIAMG_CHECK(mem[i].m >= 1 && mem[i].m <= 32, GIAMG_ERR_ARG, "m must be in [1, 32]");
    GIAMG_CHECK(mem[i].B && mem[i].X, GIAMG_ERR_ARG, "B and X are required");
    GIAMG_CHECK(H.opt.device_ptrs != 0, GIAMG_ERR_ARG, "a grouped solve needs device pointers (device_ptrs = 1)");
    GIAMG_CHECK(H.device == H0.device, GIAMG_ERR_ARG, "the hierarchies of a grouped solve must share one device");
    for (size_t j = 0; j < i; ++j)
      GIAMG_CHECK(mem[j].C != mem[i].C, GIAMG_ERR_ARG, "a hierarchy appears twice in a grouped solve");
    GIAMG_CUDA(cudaStreamSynchronize(H.stream));  // its earlier work (and allocations) done
    alloc_batch(H, mem[i].m);
    GIAMG_CUDA(cudaStreamSynchronize(H.stream));
  }
  std::vector<GrpVecArgs> ini, fbb;
  for (GroupMember& g : mem) {
    Hierarchy& H = *g.C->H;
    BatchScalarsHost* hs = (BatchScalarsHost*)H.h_bsc;
    hs->tol2 = rtol * rtol;
    hs->force = 0;
    GIAMG_CUDA(cudaMemcpyAsync((char*)H.bsc.get() + offsetof(BatchScalarsHost, tol2), &hs->tol2,
                               sizeof(double) + 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    ini.push_back(gv(H.n, g.m, g.B, nullptr, g.X, H.bR.get(), nullptr, 0.0, nullptr, H.bpartial.get()));
    fbb.push_back(gv(0, g.m, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, H.bsc.get(), H.bpartial.get()));
  }
  grp_vec(kGvInitH, ini, s);
  grp_vec(kGvFinishBbH, fbb, s);
  auto read_scalars = [&]() {
    for (GroupMember& g : mem) {
      Hierarchy& H = *g.C->H;
      GIAMG_CUDA(cudaMemcpyAsync(H.h_bsc, H.bsc.get(), sizeof(BatchScalarsHost), cudaMemcpyDeviceToHost, s));
    }
    GIAMG_CUDA(cudaStreamSynchronize(s));
  };
  read_scalars();
  std::vector<GroupMember*> run;
  for (GroupMember& g : mem) {
    BatchScalarsHost* hs = (BatchScalarsHost*)g.C->H->h_bsc;
    g.its.assign(g.m, 0);
    int active = 0;
    for (int j = 0; j < g.m; ++j) active += hs->active[j];
    g.running = active > 0 && g.C->H->opt.max_iter > 0;
    if (g.running) run.push_back(&g);
  }
  if (!run.empty()) group_precondition(run, 1, s);
  while (!run.empty()) {
    group_step(run, s);
    std::vector<std::vector<int>> was;
    for (GroupMember* g : run) {
      BatchScalarsHost* hs = (BatchScalarsHost*)g->C->H->h_bsc;
      was.emplace_back(hs->active, hs->active + g->m);
    }
    read_scalars();
    std::vector<GroupMember*> next;
    for (size_t i = 0; i < run.size(); ++i) {
      GroupMember* g = run[i];
      BatchScalarsHost* hs = (BatchScalarsHost*)g->C->H->h_bsc;
      ++g->it;
      int active = 0;
      for (int j = 0; j < g->m; ++j) {
        if (was[i][j]) g->its[j] = g->it;
        if (hs->status[j] != 0) g->breakdown = true;
        active += hs->active[j];
      }
      if (!(g->breakdown || active == 0 || g->it == g->C->H->opt.max_iter)) next.push_back(g);
    }
    run.swap(next);
    if (!run.empty()) group_precondition(run, 0, s);
  }
  GIAMG_CUDA(cudaStreamSynchronize(s));
  int64_t k = 0;
  for (size_t i = 0; i < mem.size(); ++i) {
    GroupMember& g = mem[i];
    BatchScalarsHost* hs = (BatchScalarsHost*)g.C->H->h_bsc;
    bool unconverged = false;
    for (int j = 0; j < g.m; ++j, ++k) {
      const double rr = hs->bb[j] > 0.0 ? std::sqrt(hs->rr[j] / hs->bb[j]) : 0.0;
      if (iters) iters[k] = g.its[j];
      if (relres) relres[k] = rr;
      if (!(rr <= rtol)) unconverged = true;
    }
    if (status) status[i] = g.breakdown ? GIAMG_ERR_BREAKDOWN : unconverged ? GIAMG_ERR_MAXITER : GIAMG_OK;
  }
}

// The solve enqueued on the handle's stream with no host synchronisation: the captured graph
// (captured here on first use, which synchronises once), parameters passed as kernel arguments,
// results written to device memory by a kernel after the graph.  b, x and the results are
// device pointers (device_ptrs mode).
int solve_async_impl(Ctx& C, int precision, const double* b, double* x, double rtol, int* iters, double* relres,
                     int* status) {
  Hierarchy& H = *C.H;
  cudaStream_t s = H.stream;
  const int64_t n = H.n;
  GIAMG_CHECK(b && x, GIAMG_ERR_ARG, "b and x are required");
  GIAMG_CHECK(precision == 0 || precision == 1, GIAMG_ERR_ARG, "precision must be 0 or 1");
  GIAMG_CHECK(rtol >= 0.0, GIAMG_ERR_ARG, "rtol must be non-negative");
  GIAMG_CHECK(H.opt.device_ptrs != 0, GIAMG_ERR_ARG, "an asynchronous solve needs device pointers (device_ptrs = 1)");
  GIAMG_CHECK(H.opt.graphs != 0, GIAMG_ERR_ARG, "an asynchronous solve runs the captured graph (graphs != 0)");
  GIAMG_CHECK(!H.prof.on, GIAMG_ERR_ARG, "an asynchronous solve cannot run with profiling enabled");
  const int force = H.opt.force_iters;
  const int limit = force > 0 ? force : H.opt.max_iter;
  GIAMG_CHECK(limit <= H.opt.max_iter, GIAMG_ERR_ARG, "force_iters beyond max_iter needs the synchronous solve");
  SolveGraph& SG = H.graph[precision];
  if (!SG.exec) capture_solve(C, precision);
  GIAMG_CUDA(cudaMemcpyAsync(H.gb.get(), b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  pcg_graph_params(H.gst.get(), rtol, limit, force > 0 ? 1 : 0, s);
  GIAMG_CUDA(cudaGraphLaunch(SG.exec, s));
  pcg_graph_results(H.gst.get(), H.ghist.get(), iters, relres, status, s);
  GIAMG_CUDA(cudaMemcpyAsync(x, H.gx.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  vec_copy(n, H.gb.get(), H.tmp.get(), s);  // b and x for the true residual of giamg_solve_stats
  vec_copy(n, H.gx.get(), H.xw.get(), s);
  H.hist.clear();  // the history of an asynchronous solve stays on the device
  g_launches.fetch_add(SG.n_init);  // the iterations' kernels are not known on the host
  return GIAMG_OK;
}

// The captured solve graphs hold kernels, their arguments and launch shapes: any change of a
// level's row kernel or polynomial makes them stale.
void drop_solve_graphs(Hierarchy& H) {
  for (SolveGraph& G : H.graph)
    if (G.exec) {
      GIAMG_CUDA(cudaGraphExecDestroy(G.exec));
      G = SolveGraph{};
    }
  drop_batch_graphs(H);
}

// Row-kernel choice on the finest level by time to solution: each candidate variant runs
// kTuneIters forced CG iterations (the whole solve loop: every level's V-cycle kernels and the
// outer product) twice on a fixed right-hand side, and the faster of the two CUDA-event times
// counts; per precision the fastest candidate is kept.  Isolated products mispredict the
// solve (caches, the coarse levels' kernels and the vector passes between them), so the
// candidates are timed where they run.  GIAMG_TUNE_LOG=1 prints the timings.
constexpr int kTuneIters = 3;
struct TuneCandidate {
  int form, threads;
};
void autotune_in_solve(Ctx& C) {
  Hierarchy& H = *C.H;
  Level& L0 = *H.lev[0];
  if (L0.A.nnz < (1 << 20)) return;  // small operators: the defaults
  const bool log = getenv("GIAMG_TUNE_LOG") != nullptr;
  cudaStream_t s = H.stream;
  const int64_t n = H.n;
  DBuf<double> b, x;
  b.alloc(n, s);
  x.alloc(n, s);
  fill_tune_vector(n, b.get(), s);
  cudaEvent_t e0, e1;
  GIAMG_CUDA(cudaEventCreate(&e0));
  GIAMG_CUDA(cudaEventCreate(&e1));
  const giamg_options saved = H.opt;
  H.opt.device_ptrs = 1;
  H.opt.graphs = 0;  // every candidate on the host loop (the same kernels as the captured graph)
  const std::vector<TuneCandidate> cands[2] = {
      {{0, 0}, {1, 16}, {1, 32}, {2, 16}, {5, 0}, {6, 0}},            // FP64
      {{0, 0}, {2, 8}, {2, 32}, {4, 0}, {5, 0}, {6, 0}}};             // FP32
  try {
    for (int prec = 0; prec < 2; ++prec) {
      RowVariant best = prec == 0 ? L0.A.var64 : L0.A.var32;
      float best_ms = 1e30f;
      for (const TuneCandidate& c : cands[prec]) {
        RowVariant& v = prec == 0 ? L0.A.var64 : L0.A.var32;
        const RowVariant keep = v;
        v = variant_for(L0.A, prec, c.form, c.threads);
        const RowVariant want = v;
        build_variant_copies(L0.A, s);
        if (v.vector != want.vector || v.sliced != want.sliced) {  // the form does not apply here
          v = keep;
          build_variant_copies(L0.A, s);
          continue;
        }
        float t = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          int it = 0;
          double rr = 0.0;
          GIAMG_CUDA(cudaEventRecord(e0, s));
          solve_impl(C, prec, kTuneIters, b.get(), x.get(), 0.0, &it, &rr);
          GIAMG_CUDA(cudaEventRecord(e1, s));
          GIAMG_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          GIAMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          t = std::min(t, ms);
        }
        if (log)
          fprintf(stderr, "tune %s form=%d threads=%d (%s, %d lanes): %.3f ms for %d iterations\n",
                  prec ? "fp32" : "fp64", c.form, c.threads,
                  v.sliced ? "sliced" : v.vector ? "vector" : v.hybrid ? "hybrid" : v.group ? "groups" : v.pat ? "pattern" : "csr",
                  v.tpr, t, kTuneIters);
        if (t < best_ms) {
          best_ms = t;
          best = v;
        }
      }
      (prec == 0 ? L0.A.var64 : L0.A.var32) = best;
      build_variant_copies(L0.A, s);
    }
  } catch (...) {
    H.opt = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  H.opt = saved;
  H.hist.clear();
  H.last_iters = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_solve_graphs(H);
  GIAMG_CUDA(cudaStreamSynchronize(s));
}

Ctx* ctx_of(giamg_handle h) {
  GIAMG_CHECK(h != nullptr, GIAMG_ERR_ARG, "NULL handle");
  return reinterpret_cast<Ctx*>(h);
}
Level& level_of(Ctx& C, int l) {
  GIAMG_CHECK(l >= 0 && l < (int)C.H->lev.size(), GIAMG_ERR_ARG, "level index out of range");
  return *C.H->lev[l];
}

template <typename F>
int guarded(F&& f) {
  try {
    g_last_error.clear();
    return f();
  } catch (const Error& e) {
    set_error(e.code, e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error(GIAMG_ERR_OOM, "host allocation failed");
    return GIAMG_ERR_OOM;
  } catch (...) {
    set_error(GIAMG_ERR_ARG, "unexpected error");
    return GIAMG_ERR_ARG;
  }
}

template <typename T>
void copy_out(T* dst, const T* src, size_t count, bool dev, cudaStream_t s) {
  if (!dst || count == 0) return;
  GIAMG_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * count, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

}  // namespace

Hierarchy* hierarchy_of(giamg_handle h) { return ctx_of(h)->H; }

}  // namespace giamg

using namespace giamg;

extern "C" {

void giamg_default_options(giamg_options* o) {
  if (!o) return;
  o->cheb_degree = 3;
  o->cheb_lo = 0.1;
  o->cheb_hi = 1.1;
  o->lanczos_steps = 20;
  o->coarse_max = 500;
  o->max_levels = 16;
  o->strength_theta = 0.0;
  o->precision = 0;
  o->max_iter = 1000;
  o->force_iters = 0;
  o->device_ptrs = 0;
  o->hash_kind = 0;
  o->compress_patterns = 1;
  o->autotune = 0;
  o->row_form = 0;
  o->row_threads = 0;
  o->prefetch_rows = -1;
  o->graphs = 1;
  o->p_schedule = 0;
  o->basis = 0;
  o->row_chains = 0;
}

int giamg_setup(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val, int32_t n_elem,
                const int32_t* elem_dof, const int32_t* elem_order, const double* coords, const giamg_options* opt,
                void* cuda_stream, giamg_handle* out) {
  return guarded([&] {
    GIAMG_CHECK(out != nullptr, GIAMG_ERR_ARG, "out is NULL");
    *out = nullptr;
    Ctx* C = setup_impl(n, row_ptr, col_idx, val, n_elem, elem_dof, elem_order, coords, opt, cuda_stream);
    if (C->H->opt.autotune) {
      try {
        autotune_in_solve(*C);
      } catch (...) {
        cudaStream_t st = C->H->stream;
        delete C->H;
        delete C;
        cudaStreamSynchronize(st);
        throw;
      }
    }
    *out = reinterpret_cast<giamg_handle>(C);
    return GIAMG_OK;
  });
}

int giamg_solve(giamg_handle h, const double* b, double* x, double rtol, int* iters, double* relres) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    return solve_impl(C, C.H->opt.precision, C.H->opt.force_iters, b, x, rtol, iters, relres);
  });
}

int giamg_solve_ex(giamg_handle h, int precision, int force_iters, const double* b, double* x, double rtol, int* iters,
                   double* relres) {
  return guarded([&] { return solve_impl(*ctx_of(h), precision, force_iters, b, x, rtol, iters, relres); });
}

int giamg_solve_async(giamg_handle h, int precision, const double* b, double* x, double rtol, int* iters,
                      double* relres, int* status) {
  return guarded([&] { return solve_async_impl(*ctx_of(h), precision, b, x, rtol, iters, relres, status); });
}

int giamg_solve_batch(giamg_handle h, int m, const double* B, double* X, double rtol, int* iters, double* relres) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    return solve_batch_impl(C, C.H->opt.precision, C.H->opt.force_iters, m, B, X, rtol, iters, relres, false);
  });
}

int giamg_solve_batch_ex(giamg_handle h, int precision, int force_iters, int m, const double* B, double* X, double rtol,
                         int* iters, double* relres) {
  return guarded([&] { return solve_batch_impl(*ctx_of(h), precision, force_iters, m, B, X, rtol, iters, relres, false); });
}

int giamg_solve_block(giamg_handle h, int precision, int force_iters, int m, const double* B, double* X, double rtol,
                      int* iters, double* relres) {
  return guarded([&] { return solve_batch_impl(*ctx_of(h), precision, force_iters, m, B, X, rtol, iters, relres, true); });
}

int giamg_solve_stats(giamg_handle h, double* hist, int len, double* true_relres) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Hierarchy& H = *C.H;
    if (hist)
      for (int i = 0; i < len && i < (int)H.hist.size(); ++i) hist[i] = H.hist[i];
    if (true_relres) {
      cudaStream_t s = H.stream;
      Level& L0 = *H.lev[0];
      residual(L0.A, H.tmp.get(), H.xw.get(), H.q.get(), s, L0.avg_row);
      DBuf<double> out;
      out.alloc(2, s);
      dot_partial(H.n, H.q.get(), H.q.get(), H.partial.get(), s);
      reduce_to(H.partial.get(), out.get(), s);
      dot_partial(H.n, H.tmp.get(), H.tmp.get(), H.partial.get(), s);
      reduce_to(H.partial.get(), out.get() + 1, s);
      double hv[2];
      GIAMG_CUDA(cudaMemcpyAsync(hv, out.get(), sizeof(hv), cudaMemcpyDeviceToHost, s));
      GIAMG_CUDA(cudaStreamSynchronize(s));
      *true_relres = hv[1] > 0 ? std::sqrt(hv[0] / hv[1]) : 0.0;
    }
    return GIAMG_OK;
  });
}

int giamg_num_levels(giamg_handle h, int* n_levels) {
  return guarded([&] {
    GIAMG_CHECK(n_levels, GIAMG_ERR_ARG, "n_levels is NULL");
    *n_levels = (int)ctx_of(h)->H->lev.size();
    return GIAMG_OK;
  });
}

int giamg_level_info(giamg_handle h, int level, int* kind, int64_t* n, int64_t* nnz, int* order, int64_t* p_nnz,
                     int64_t* n_next) {
  return guarded([&] {
    Level& L = level_of(*ctx_of(h), level);
    if (kind) *kind = L.kind;
    if (n) *n = L.A.n;
    if (nnz) *nnz = L.A.nnz;
    if (order) *order = L.order;
    if (p_nnz) *p_nnz = L.kind == GIAMG_LEVEL_COARSEST ? 0 : L.P.nnz;
    if (n_next) *n_next = L.kind == GIAMG_LEVEL_COARSEST ? 0 : L.n_next;
    return GIAMG_OK;
  });
}

int giamg_export_level(giamg_handle h, int level, int64_t* row_ptr, int32_t* col_idx, double* val, int32_t* aggregates) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    const bool dev = C.H->opt.device_ptrs != 0;
    cudaStream_t s = C.H->stream;
    copy_out(row_ptr, L.A.rp.get(), (size_t)L.A.n + 1, dev, s);
    copy_out(col_idx, L.A.ci.get(), (size_t)L.A.nnz, dev, s);
    copy_out(val, L.A.v.get(), (size_t)L.A.nnz, dev, s);
    if (aggregates && L.kind == GIAMG_LEVEL_H) copy_out(aggregates, L.agg.get(), (size_t)L.A.n, dev, s);
    GIAMG_CUDA(cudaStreamSynchronize(s));
    return GIAMG_OK;
  });
}

int giamg_export_prolongation(giamg_handle h, int level, int64_t* row_ptr, int32_t* col_idx, double* val) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(L.kind != GIAMG_LEVEL_COARSEST, GIAMG_ERR_ARG, "the coarsest level has no prolongation");
    const bool dev = C.H->opt.device_ptrs != 0;
    cudaStream_t s = C.H->stream;
    copy_out(row_ptr, L.P.rp.get(), (size_t)L.P.n + 1, dev, s);
    copy_out(col_idx, L.P.ci.get(), (size_t)L.P.nnz, dev, s);
    copy_out(val, L.P.v.get(), (size_t)L.P.nnz, dev, s);
    GIAMG_CUDA(cudaStreamSynchronize(s));
    return GIAMG_OK;
  });
}

int giamg_level_templates(giamg_handle h, int level, int64_t* n_templates, int64_t* n_offsets) {
  return guarded([&] {
    Level& L = level_of(*ctx_of(h), level);
    if (n_templates) *n_templates = L.A.pat.on ? L.A.pat.n_templates : 0;
    if (n_offsets) *n_offsets = L.A.pat.on ? L.A.pat.n_offsets : 0;
    return GIAMG_OK;
  });
}

int giamg_level_kernel(giamg_handle h, int level, int precision, int* threads_per_row, int* pattern) {
  return guarded([&] {
    Level& L = level_of(*ctx_of(h), level);
    GIAMG_CHECK(precision == 0 || precision == 1, GIAMG_ERR_ARG, "precision must be 0 or 1");
    const RowVariant& v = precision == 0 ? L.A.var64 : L.A.var32;
    const double avg = L.A.n ? (double)L.A.nnz / L.A.n : 0.0;
    const bool vec = v.hybrid && v.vector && (precision == 1 ? L.A.grp.hvon : L.A.grp.hv64on);
    const bool sel = v.sliced && L.A.grp.son && (precision == 1 ? L.A.grp.sv32on : L.A.grp.sv64on);
    if (threads_per_row)  // the FP64 vector hybrid takes 4 lanes per row of a big group, the sliced form 1
      *threads_per_row = sel ? 1 : vec && precision == 0 ? 4 : v.tpr ? v.tpr : (avg >= 48 ? 32 : avg >= 20 ? 16 : avg >= 8 ? 8 : 4);
    if (pattern)
      *pattern = sel ? 5 : v.hybrid ? (vec ? 4 : 3) : v.group ? 2 : v.tpr ? (v.pat ? 1 : 0) : (L.A.pat.on ? 1 : 0);
    return GIAMG_OK;
  });
}

int giamg_set_cheb_degree(giamg_handle h, int degree) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Hierarchy& H = *C.H;
    GIAMG_CHECK(degree >= 1 && degree <= 64, GIAMG_ERR_ARG, "cheb_degree must be in [1, 64]");
    GIAMG_CUDA(cudaStreamSynchronize(H.stream));  // no solve of the old polynomial in flight
    H.opt.cheb_degree = degree;
    for (size_t l = 0; l < H.lev.size(); ++l)
      if (H.lev[l]->kind != GIAMG_LEVEL_COARSEST)
        C.ex[l].cheb = cheb_coeffs(H.lev[l]->rho, H.opt.cheb_lo, H.opt.cheb_hi, degree);
    // the captured solve graphs hold the old coefficients as kernel arguments
    drop_solve_graphs(H);
    return GIAMG_OK;
  });
}

int giamg_solve_grouped(int count, const giamg_handle* handles, const int* m, const double* const* B,
                        double* const* X, double rtol, int* iters, double* relres, int* status) {
  return guarded([&] {
    GIAMG_CHECK(count >= 1 && handles && m && B && X, GIAMG_ERR_ARG, "count >= 1 and handles, m, B, X are required");
    std::vector<GroupMember> mem((size_t)count);
    for (int i = 0; i < count; ++i) {
      mem[i].C = ctx_of(handles[i]);
      mem[i].m = m[i];
      mem[i].B = B[i];
      mem[i].X = X[i];
    }
    solve_grouped_impl(mem, rtol, iters, relres, status);
    return GIAMG_OK;
  });
}

int giamg_set_row_kernel(giamg_handle h, int level, int precision, int form, int threads) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Hierarchy& H = *C.H;
    Level& L = level_of(C, level);
    GIAMG_CHECK(precision == 0 || precision == 1, GIAMG_ERR_ARG, "precision must be 0 or 1");
    GIAMG_CHECK(form >= 0 && form <= 6, GIAMG_ERR_ARG, "form must be in 0..6");
    GIAMG_CHECK(threads == 0 || threads == 4 || threads == 8 || threads == 16 || threads == 32, GIAMG_ERR_ARG,
                "threads must be 0, 4, 8, 16 or 32");
    GIAMG_CUDA(cudaStreamSynchronize(H.stream));  // no solve of the old kernels in flight
    (precision == 0 ? L.A.var64 : L.A.var32) = variant_for(L.A, precision, form, threads);
    build_variant_copies(L.A, H.stream);
    drop_solve_graphs(H);
    return GIAMG_OK;
  });
}

int giamg_set_batch_rows(giamg_handle h, int level, int rows_per_item) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Hierarchy& H = *C.H;
    Level& L = level_of(C, level);
    GIAMG_CHECK(rows_per_item >= 0 && rows_per_item <= 2, GIAMG_ERR_ARG, "rows_per_item must be 0, 1 or 2");
    GIAMG_CUDA(cudaStreamSynchronize(H.stream));
    L.A.batch_rows = rows_per_item;
    drop_batch_graphs(H);
    return GIAMG_OK;
  });
}

int giamg_level_rho(giamg_handle h, int level, double* rho_hat) {
  return guarded([&] {
    GIAMG_CHECK(rho_hat, GIAMG_ERR_ARG, "rho_hat is NULL");
    *rho_hat = level_of(*ctx_of(h), level).rho;
    return GIAMG_OK;
  });
}

int giamg_apply_vcycle(giamg_handle h, int precision, const double* r, double* z) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Hierarchy& H = *C.H;
    GIAMG_CHECK(r && z, GIAMG_ERR_ARG, "r and z are required");
    GIAMG_CHECK(precision == 0 || precision == 1, GIAMG_ERR_ARG, "precision must be 0 or 1");
    const bool dev = H.opt.device_ptrs != 0;
    InVec ri(r, H.n, dev, H.stream);
    OutVec zo(z, H.n, dev, H.stream, false);
    const double* zz = apply_vcycle(C, precision, ri.d);
    vec_copy(H.n, zz, zo.d, H.stream);
    zo.finish();
    return GIAMG_OK;
  });
}

int giamg_level_spmv(giamg_handle h, int level, const double* x, double* y) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(x && y, GIAMG_ERR_ARG, "x and y are required");
    const bool dev = C.H->opt.device_ptrs != 0;
    InVec xi(x, L.A.n, dev, C.H->stream);
    OutVec yo(y, L.A.n, dev, C.H->stream, false);
    spmv(L.A, xi.d, yo.d, C.H->stream, L.avg_row);
    yo.finish();
    return GIAMG_OK;
  });
}

int giamg_level_spmv32(giamg_handle h, int level, const float* x, float* y) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(x && y, GIAMG_ERR_ARG, "x and y are required");
    const bool dev = C.H->opt.device_ptrs != 0;
    InVecT<float> xi(x, L.A.n, dev, C.H->stream);
    OutVecT<float> yo(y, L.A.n, dev, C.H->stream, false);
    spmv32(L.A, xi.d, yo.d, C.H->stream, L.avg_row);
    yo.finish();
    return GIAMG_OK;
  });
}

int giamg_level_smooth(giamg_handle h, int level, const double* b, double* x, int x_is_zero) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(L.kind != GIAMG_LEVEL_COARSEST, GIAMG_ERR_ARG, "the coarsest level is solved, not smoothed");
    GIAMG_CHECK(b && x, GIAMG_ERR_ARG, "b and x are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVec bi(b, L.A.n, dev, s);
    OutVec xo(x, L.A.n, dev, s, !x_is_zero);
    const Cheb& c = C.ex[level].cheb;
    double* xa = L.x.get();
    double* xb = L.x2.get();
    int j0 = 0;
    if (x_is_zero) {
      cheb_first(L.A.n, bi.d, L.dinv.get(), c.c2[0], xa, L.d.get(), s);
      j0 = 1;
    } else {
      vec_copy(L.A.n, xo.d, xa, s);
    }
    for (int j = j0; j < (int)c.c1.size(); ++j) {
      cheb_step(L.A, bi.d, xa, xb, L.d.get(), L.dinv.get(), c.c1[j], c.c2[j], s, L.avg_row);
      std::swap(xa, xb);
    }
    vec_copy(L.A.n, xa, xo.d, s);
    xo.finish();
    return GIAMG_OK;
  });
}

int giamg_level_restrict(giamg_handle h, int level, const double* r_f, double* r_c) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(L.kind != GIAMG_LEVEL_COARSEST, GIAMG_ERR_ARG, "the coarsest level has no restriction");
    GIAMG_CHECK(r_f && r_c, GIAMG_ERR_ARG, "r_f and r_c are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVec ri(r_f, L.A.n, dev, s);
    OutVec ro(r_c, L.n_next, dev, s, false);
    if (L.kind == GIAMG_LEVEL_P) p_restrict(L, ri.d, ro.d, s);
    else h_restrict(L, ri.d, ro.d, s);
    ro.finish();
    return GIAMG_OK;
  });
}

int giamg_level_prolong(giamg_handle h, int level, const double* e_c, double* x_f) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(L.kind != GIAMG_LEVEL_COARSEST, GIAMG_ERR_ARG, "the coarsest level has no prolongation");
    GIAMG_CHECK(e_c && x_f, GIAMG_ERR_ARG, "e_c and x_f are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVec ei(e_c, L.n_next, dev, s);
    OutVec xo(x_f, L.A.n, dev, s, true);
    if (L.kind == GIAMG_LEVEL_P) p_prolong(L, ei.d, xo.d, s);
    else h_prolong(L, ei.d, xo.d, s);
    xo.finish();
    return GIAMG_OK;
  });
}

int giamg_coarse_solve(giamg_handle h, const double* r, double* x) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = *C.H->lev.back();
    GIAMG_CHECK(r && x, GIAMG_ERR_ARG, "r and x are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVec ri(r, L.nc, dev, s);
    OutVec xo(x, L.nc, dev, s, false);
    chol_solve(L.L.get(), L.nc, ri.d, xo.d, s);
    xo.finish();
    return GIAMG_OK;
  });
}

int giamg_level_residual(giamg_handle h, int level, const double* b, const double* x, double* r) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(b && x && r, GIAMG_ERR_ARG, "b, x and r are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVec bi(b, L.A.n, dev, s);
    InVec xi(x, L.A.n, dev, s);
    OutVec ro(r, L.A.n, dev, s, false);
    residual(L.A, bi.d, xi.d, ro.d, s, L.avg_row);
    ro.finish();
    return GIAMG_OK;
  });
}

// ---- single steps of the FP32 V-cycle: the launchers vcycle32 uses, on FP32 vectors
int giamg_level_residual32(giamg_handle h, int level, const float* b, const float* x, float* r) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(b && x && r, GIAMG_ERR_ARG, "b, x and r are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVecT<float> bi(b, L.A.n, dev, s);
    InVecT<float> xi(x, L.A.n, dev, s);
    OutVecT<float> ro(r, L.A.n, dev, s, false);
    residual32(L.A, bi.d, xi.d, ro.d, s, L.avg_row);
    ro.finish();
    return GIAMG_OK;
  });
}

int giamg_level_smooth32(giamg_handle h, int level, const float* b, float* x, int x_is_zero) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(L.kind != GIAMG_LEVEL_COARSEST, GIAMG_ERR_ARG, "the coarsest level is solved, not smoothed");
    GIAMG_CHECK(b && x, GIAMG_ERR_ARG, "b and x are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    const int64_t n = L.A.n;
    InVecT<float> bi(b, n, dev, s);
    OutVecT<float> xo(x, n, dev, s, !x_is_zero);
    const Cheb& c = C.ex[level].cheb;
    float* xa = L.x32.get();
    float* xb = L.x232.get();
    int j0 = 0;
    if (x_is_zero) {
      cheb_first32(n, bi.d, L.dinv32.get(), (float)c.c2[0], xa, L.d32.get(), s);
      j0 = 1;
    } else if (n > 0) {
      GIAMG_CUDA(cudaMemcpyAsync(xa, xo.d, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    }
    for (int j = j0; j < (int)c.c1.size(); ++j) {
      cheb_step32(L.A, bi.d, xa, xb, L.d32.get(), L.dinv32.get(), (float)c.c1[j], (float)c.c2[j], s, L.avg_row);
      std::swap(xa, xb);
    }
    if (n > 0) GIAMG_CUDA(cudaMemcpyAsync(xo.d, xa, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    xo.finish();
    return GIAMG_OK;
  });
}

int giamg_level_restrict32(giamg_handle h, int level, const float* r_f, float* r_c) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(L.kind != GIAMG_LEVEL_COARSEST, GIAMG_ERR_ARG, "the coarsest level has no restriction");
    GIAMG_CHECK(r_f && r_c, GIAMG_ERR_ARG, "r_f and r_c are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVecT<float> ri(r_f, L.A.n, dev, s);
    OutVecT<float> ro(r_c, L.n_next, dev, s, false);
    if (L.kind == GIAMG_LEVEL_P) p_restrict32(L, ri.d, ro.d, s);
    else h_restrict32(L, ri.d, ro.d, s);
    ro.finish();
    return GIAMG_OK;
  });
}

int giamg_level_prolong32(giamg_handle h, int level, const float* e_c, float* x_f) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = level_of(C, level);
    GIAMG_CHECK(L.kind != GIAMG_LEVEL_COARSEST, GIAMG_ERR_ARG, "the coarsest level has no prolongation");
    GIAMG_CHECK(e_c && x_f, GIAMG_ERR_ARG, "e_c and x_f are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVecT<float> ei(e_c, L.n_next, dev, s);
    OutVecT<float> xo(x_f, L.A.n, dev, s, true);
    if (L.kind == GIAMG_LEVEL_P) p_prolong32(L, ei.d, xo.d, s);
    else h_prolong32(L, ei.d, xo.d, s);
    xo.finish();
    return GIAMG_OK;
  });
}

int giamg_coarse_solve32(giamg_handle h, const float* r, float* x) {
  return guarded([&] {
    Ctx& C = *ctx_of(h);
    Level& L = *C.H->lev.back();
    GIAMG_CHECK(r && x, GIAMG_ERR_ARG, "r and x are required");
    cudaStream_t s = C.H->stream;
    const bool dev = C.H->opt.device_ptrs != 0;
    InVecT<float> ri(r, L.nc, dev, s);
    OutVecT<float> xo(x, L.nc, dev, s, false);
    inverse_apply32(L.Ainv.get(), L.nc, ri.d, xo.d, s);
    xo.finish();
    return GIAMG_OK;
  });
}

int giamg_free(giamg_handle h) {
  if (!h) return GIAMG_OK;
  return guarded([&] {
    Ctx* C = reinterpret_cast<Ctx*>(h);
    cudaStream_t s = C->H->stream;
    delete C->H;
    delete C;
    GIAMG_CUDA(cudaStreamSynchronize(s));
    return GIAMG_OK;
  });
}

const char* giamg_last_error(void) { return g_last_error.c_str(); }

int giamg_set_device_ptrs(giamg_handle h, int device_ptrs) {
  return guarded([&] {
    GIAMG_CHECK(device_ptrs == 0 || device_ptrs == 1, GIAMG_ERR_ARG, "device_ptrs must be 0 or 1");
    ctx_of(h)->H->opt.device_ptrs = device_ptrs;
    return GIAMG_OK;
  });
}

int giamg_profile_enable(giamg_handle h, int enable) {
  return guarded([&] {
    Hierarchy& H = *ctx_of(h)->H;
    GIAMG_CUDA(cudaStreamSynchronize(H.stream));
    H.prof.on = enable != 0;
    H.prof.recs.clear();
    H.prof.used = 0;
    return GIAMG_OK;
  });
}

int giamg_profile_read(giamg_handle h, int category, double* total_ms, int64_t* launches, double* bytes) {
  return guarded([&] {
    Hierarchy& H = *ctx_of(h)->H;
    GIAMG_CHECK(category >= 0 && category < kProfCats, GIAMG_ERR_ARG, "profile category out of range");
    GIAMG_CUDA(cudaStreamSynchronize(H.stream));
    double ms = 0.0, by = 0.0;
    int64_t cnt = 0;
    for (const Prof::Rec& R : H.prof.recs) {
      if (R.cat != category) continue;
      float t = 0.f;
      GIAMG_CUDA(cudaEventElapsedTime(&t, H.prof.ev[R.e0], H.prof.ev[R.e1]));
      ms += t;
      by += R.bytes;
      ++cnt;
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = cnt;
    if (bytes) *bytes = by;
    return GIAMG_OK;
  });
}

int giamg_launch_count(int64_t* count) {
  if (!count) return GIAMG_ERR_ARG;
  *count = (int64_t)g_launches.load();
  return GIAMG_OK;
}

}  // extern "C"
