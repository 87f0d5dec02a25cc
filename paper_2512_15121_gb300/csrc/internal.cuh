// internal.cuh -- data structures and kernel launchers shared by the library's translation
// units.  Nothing here is part of the C ABI (see include/giamg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "giamg.h"

namespace giamg {

// ------------------------------------------------------------------ launch counter
extern std::atomic<long long> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ------------------------------------------------------------------ errors
struct Error {
  int code;
  std::string msg;
};
void set_error(int code, const std::string& msg);

#define GIAMG_CUDA(call)                                                                      \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      throw ::giamg::Error{GIAMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define GIAMG_CHECK(cond, code, msg) \
  do {                               \
    if (!(cond)) throw ::giamg::Error{(code), (msg)}; \
  } while (0)

// A per-function setting that belongs to one device (cudaFuncSetAttribute applies to the device
// current at the call): once(f) runs f the first time it is reached with a given device current.
// Two threads may both run f for the same device; every f here sets the same value, so that
// is harmless.
class PerDevice {
  std::atomic<unsigned long long> done_{0};

 public:
  template <typename F>
  void once(F&& f) {
    int d = 0;
    GIAMG_CUDA(cudaGetDevice(&d));
    const unsigned long long bit = d >= 0 && d < 64 ? 1ull << d : 0ull;
    if (bit && (done_.load(std::memory_order_acquire) & bit)) return;
    f();
    if (bit) done_.fetch_or(bit, std::memory_order_acq_rel);
  }
};

// ------------------------------------------------------------------ device memory
// Owning device buffer (stream-ordered allocation on the handle's stream).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { swap(o); }
  DBuf& operator=(DBuf&& o) noexcept { release(); swap(o); return *this; }
  ~DBuf() { release(); }
  void swap(DBuf& o) { std::swap(p, o.p); std::swap(n, o.n); std::swap(s, o.s); }
  void alloc(size_t count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    if (count == 0) return;
    cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), stream);
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      (void)cudaGetLastError();
      throw Error{GIAMG_ERR_OOM, std::string("device allocation of ") + std::to_string(count * sizeof(T)) +
                                     " bytes failed: " + cudaGetErrorString(e)};
    }
  }
  void zero(cudaStream_t stream) {
    if (n) GIAMG_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), stream));
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  T* get() const { return p; }
};

// Repeated row patterns: row i's columns are i + toff[tptr[t] + k], k < len(row i), t = tid[i].
struct Pattern {
  bool on = false;
  int64_t n_templates = 0, n_offsets = 0;
  DBuf<int32_t> tid;
  DBuf<int64_t> tptr;
  DBuf<int32_t> toff;
  DBuf<int32_t> obase;  // obase[i] = tptr[tid[i]]: where row i's offsets start in toff
};

// Row groups: rows with identical column sets; group g holds rows grow[rptr[g] .. rptr[g+1]) and
// columns gcol[gptr[g] .. gptr[g+1]).
struct Groups {
  bool on = false;
  int64_t n_groups = 0, n_cols = 0;
  int cmax = 0;
  DBuf<int64_t> gptr, rptr;
  DBuf<int32_t> gcol, grow;
  // hybrid form: the groups of at least kHybridRows rows (big) and every other row (rest,
  // ascending); needs the row-pattern form for the rest
  bool hyb = false;
  int64_t n_big = 0, n_rest = 0;
  double big_cols = 0.0;  // average column count of the rows in big groups
  DBuf<int32_t> big, rest;
  // vector hybrid forms: the big groups' values copied group by group (in the order of `big`),
  // each row padded with zeros to a multiple of 4 values, so every row starts on 16 bytes and a
  // group is one contiguous block; hv from the FP32 values, hv64 from the FP64 values
  bool hvon = false, hv64on = false;
  int cpmax = 0;                // widest padded row of a big group
  int rmax = 0;                 // most rows of a big group
  int hwarps = 8;               // FP32 vector hybrid: warps per block (rows of a group split evenly)
  DBuf<int64_t> hoff;           // start of big group j's block (values), n_big + 1 entries
  DBuf<float> hv;
  DBuf<double> hv64;
  // sliced form: every row of the level in slices of 32 rows, one lane per row, the rows ordered
  // by length (longest first), then by group, so one slice mixes rows of a few groups of equal
  // length; a slice is padded with zeros to its longest row rounded up to a multiple of 8, and
  // its values are interleaved by column: element ((k / W) * 32 + lane) * W + k % W of the
  // slice's block, W = 2 (FP64) or 4 (FP32), so a lane's W columns are one 16-byte load and the
  // warp's load is 512 contiguous bytes.  A lane reads its row's columns from its group's list in
  // gcol (positions past its row's length repeat its last column against a zero value).
  bool son = false, sv64on = false, sv32on = false;
  int64_t n_slices = 0;
  DBuf<int32_t> srow;   // per lane: the row (-1: padding)
  DBuf<int32_t> sob;    // per lane: start of the row's column list in gcol
  DBuf<int32_t> sclen;  // per lane: the row's length (1 for padding)
  DBuf<int32_t> slen;   // per slice: padded length
  DBuf<int64_t> sbase;  // per slice: first value of its block (n_slices + 1 entries)
  DBuf<double> sv64;
  DBuf<float> sv32;
  // multi-right-hand-side FP32 products: work items of two rows of one group (or one row), so a
  // warp applies each gathered row of X to both; a group's rows are paired in list order
  bool pon = false;
  int64_t n_items = 0;
  DBuf<int32_t> item_a, item_b, item_g;  // rows (item_b = -1 for a single row) and their group
};
constexpr int kHybridRows = 16;

// Row-kernel variant chosen for a matrix: threads per row and whether the pattern form is used
// (one choice per value precision; set by the setup-time tuner, or from the row length).
struct RowVariant {
  int tpr = 0;       // 0: not tuned, choose from the average row length
  bool pat = false;
  int unroll = 2;    // independent load chains per thread and step (pattern form: 2, 4 or 8)
  bool group = false;  // row-group form (one CTA per group, x gathered once into shared memory)
  bool hybrid = false;  // big row groups by the group kernel, the other rows by the pattern kernel
  int64_t prefetch = 0;  // pattern form: L2 prefetch distance in rows (0: none)
  bool vector = false;   // hybrid form: big groups read with 16-byte loads from the group-major copy
  bool sliced = false;   // sliced form: one lane per row, 32 rows of equal length per warp
};

struct DCSR {
  int64_t n = 0, m = 0, nnz = 0;
  DBuf<int64_t> rp;
  DBuf<int32_t> ci;
  DBuf<double> v;
  DBuf<float> v32;
  Pattern pat;  // optional compressed column structure for the row kernels
  Groups grp;   // optional row groups with identical column sets
  RowVariant var64, var32;
  int batch_rows = 0;  // multi-right-hand-side FP32 products: 0 automatic (two rows of a group per
                       // warp when m > 16), 1 one row per warp, 2 two rows of a group per warp
};

// ------------------------------------------------------------------ hierarchy
struct Level {
  int kind = GIAMG_LEVEL_COARSEST;
  int order = 0;  // p of a p-level, 0 for aggregated levels
  DCSR A;
  double avg_row = 0.0;
  DBuf<double> dinv;
  DBuf<float> dinv32;
  double rho = 0.0;  // Lanczos estimate of lambda_max(D^-1 A)

  // transfer to the next level
  DCSR P;  // assembled prolongation n x n_next (built in setup; used by h-levels and export)
  DCSR R;  // R = P^T (h-levels)
  int64_t n_next = 0;
  // p-level element form
  int p = 0, q = 0;
  int32_t n_elem = 0;
  DBuf<int32_t> l2g;      // [n_elem][(p+1)^3] this level's element map
  DBuf<uint8_t> own;      // [n_elem][(p+1)^3] 1 if the element is the fine dof's first element
  DBuf<int32_t> l2g_c;    // [n_elem][(q+1)^3] next level's element map
  DBuf<double> p1d;       // [(p+1)][(q+1)]
  DBuf<float> p1d32;
  DBuf<int64_t> cinc_ptr; // coarse dof -> element slots e*(q+1)^3+b, ascending
  DBuf<int32_t> cinc;
  DBuf<double> part;      // [n_elem][(q+1)^3] restriction partial sums
  DBuf<float> part32;
  // h-level
  DBuf<int32_t> agg;

  // coarsest level
  int64_t nc = 0;
  DBuf<double> L;     // dense Cholesky factor, column-major lower triangle, nc x nc
  DBuf<double> Ainv;  // A^-1 formed from the factor at setup, nc x nc

  // work vectors (FP64 and FP32 copies)
  DBuf<double> x, x2, b, r, d;
  DBuf<float> x32, x232, b32, r32, d32;
  // multi-right-hand-side work blocks (n x bm, row-major), allocated on first use
  int bm = 0;
  DBuf<double> bx, bx2, bb, br, bd, bpart;
  DBuf<float> bx32, bx232, bb32, br32, bd32, bpart32;
};

struct Scalars {  // PCG scalars kept on the device
  double rho, rho_old, pq, alpha, beta, rr, bb, zr_old;
  int status;
  int pad;
};

// Device-side state of the solve captured as a CUDA graph: the stopping rule's inputs (rtol, the
// iteration limit, whether the count is forced) and outputs (iterations, last relres, status).
struct GraphState {
  double rtol;
  double relres;
  int limit;
  int force;
  int it;
  int status;
};

// Block CG (O'Leary) on m <= 32 columns: the m x m matrices of one iteration, row-major 32 x 32
// with entry [a * 32 + c] = direction a, column c.
struct BlockState {
  double gram[2][1024];  // last reduced block products: G = P^T Q and C = P^T R, or E = Q^T Z in [0]
  double L[1024];        // Cholesky factor of diag(G)^-1/2 G diag(G)^-1/2 on the kept directions
  double alpha[1024];    // G^+ C
  double beta[1024];     // -G^+ E
  double s[32];          // diag(G)^-1/2, 0 for a dropped direction
  int keep[32];
  int rank, pad;
};
// Device-side state of the multi-right-hand-side solve captured as a CUDA graph.
struct BatchGraphState {
  int it, limit, breakdown, pad;
  int its[32], was[32];
};

// One instantiated solve graph (per V-cycle precision) and the kernel launches of its parts, so
// the launch counter can be advanced by what a run executed.
struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  int uses = 0;  // solves of this shape so far (graphs = 1 captures from the second one)
  long long n_init = 0, n_first = 0, n_loop = 0, n_more = 0;
};

// Opt-in CUDA-event timers by category (they add event records to the stream)
enum ProfCat {
  kProfL0Rows = 0,
  kProfCoarseRows = 1,
  kProfTransfer = 2,
  kProfCoarsest = 3,
  kProfVector = 4,
  kProfOuterSpmv = 5,
  kProfCats = 6
};
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  struct Rec {
    int cat;
    int e0, e1;
    double bytes;
  };
  std::vector<Rec> recs;
  size_t used = 0;
};

struct Hierarchy {
  giamg_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<Level*> lev;
  int64_t n = 0;
  // PCG work
  DBuf<double> r, z, p, q, xw, rold, tmp;
  DBuf<double> partial;  // reduction partial sums
  DBuf<Scalars> sc;
  Scalars* h_sc = nullptr;  // pinned host copy
  std::vector<double> hist;
  int last_iters = 0;
  double last_true_relres = -1.0;
  Prof prof;
  // multi-right-hand-side PCG work (n x bm)
  int bm = 0;
  DBuf<double> bR, bZ, bP, bQ, bRold, bX, bB, bpartial;
  DBuf<unsigned char> bsc;
  void* h_bsc = nullptr;
  // the solve as a CUDA graph (internal right-hand side, solution and relres history)
  SolveGraph graph[2];
  cudaStream_t capture_stream = nullptr;
  DBuf<double> gb, gx, ghist;
  DBuf<GraphState> gst;
  GraphState* h_gst = nullptr;  // pinned host copy
  SolveGraph bgraph[2][33];       // multi-right-hand-side solve graphs by precision and m
  SolveGraph kgraph[2][33];       // block CG solve graphs by precision and m
  DBuf<double> kpartial;          // block CG: per-block partial Gram products
  DBuf<BlockState> kst;           // block CG: the m x m matrices of the current iteration
  DBuf<BatchGraphState> bgst;
  BatchGraphState* h_bgst = nullptr;
  ~Hierarchy();
};

// the hierarchy behind a C handle (throws GIAMG_ERR_ARG for NULL)
Hierarchy* hierarchy_of(giamg_handle h);
// giamg_true_relres_noalloc's static scratch: load its module on the current device and look
// up the array's address there (called by giamg_setup, while the caller can still allocate)
void noalloc_prepare();

// ------------------------------------------------------------------ kernels (launchers)
// reductions: fixed-size grid, partial sums reduced in a fixed order (bitwise reproducible)
constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

// SpMV family on a CSR level (FP64 and FP32 values)
// row-kernel modes
enum RowMode { kSpmv = 0, kResidual = 1, kCheb = 2, kAddSpmv = 3 };

void spmv(const DCSR& A, const double* x, double* y, cudaStream_t s, double avg_row);
void spmv32(const DCSR& A, const float* x, float* y, cudaStream_t s, double avg_row);
// y = b - A x
void residual(const DCSR& A, const double* b, const double* x, double* r, cudaStream_t s, double avg_row);
void residual32(const DCSR& A, const float* b, const float* x, float* r, cudaStream_t s, double avg_row);
// Chebyshev step: r = b - A x; d = c1 d + c2 dinv r (c1 == 0: d is not read); xo = x + d
void cheb_step(const DCSR& A, const double* b, const double* x, double* xo, double* d, const double* dinv,
               double c1, double c2, cudaStream_t s, double avg_row);
void cheb_step32(const DCSR& A, const float* b, const float* x, float* xo, float* d, const float* dinv,
                 float c1, float c2, cudaStream_t s, double avg_row);
// first step from x = 0: d = dinv b * c2; x = d
void cheb_first(int64_t n, const double* b, const double* dinv, double c2, double* x, double* d, cudaStream_t s);
void cheb_first32(int64_t n, const float* b, const float* dinv, float c2, float* x, float* d, cudaStream_t s);

// p-level transfers in element form
void p_restrict(const Level& L, const double* rf, double* rc, cudaStream_t s);
void p_prolong(const Level& L, const double* ec, double* xf, cudaStream_t s);
void p_restrict32(const Level& L, const float* rf, float* rc, cudaStream_t s);
void p_prolong32(const Level& L, const float* ec, float* xf, cudaStream_t s);
// h-level transfers: rc = R rf ; xf += P ec
void h_restrict(const Level& L, const double* rf, double* rc, cudaStream_t s);
void h_prolong(const Level& L, const double* ec, double* xf, cudaStream_t s);
void h_restrict32(const Level& L, const float* rf, float* rc, cudaStream_t s);
void h_prolong32(const Level& L, const float* ec, float* xf, cudaStream_t s);

// coarsest level
int cholesky_factor(double* Lcm, int64_t nc, cudaStream_t s);  // returns GIAMG_OK or NOT_SPD
void chol_solve(const double* Lcm, int64_t nc, const double* b, double* x, cudaStream_t s);
void chol_solve32(const double* Lcm, int64_t nc, const float* b, float* x, cudaStream_t s);
// A^-1 = L^-T L^-1 by the same substitutions applied to the unit vectors (setup), and its use
void chol_inverse(const double* Lcm, int64_t nc, double* Ainv, cudaStream_t s);
void inverse_apply(const double* Ainv, int64_t nc, const double* b, double* x, cudaStream_t s);
void inverse_apply32(const double* Ainv, int64_t nc, const float* b, float* x, cudaStream_t s);

// vectors
void dot_partial(int64_t n, const double* x, const double* y, double* partial, cudaStream_t s);
void vec_copy(int64_t n, const double* x, double* y, cudaStream_t s);
void vec_fill(int64_t n, double v, double* y, cudaStream_t s);
void vec_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s);
void vec_to32(int64_t n, const double* x, float* y, cudaStream_t s);
void vec_to64(int64_t n, const float* x, double* y, cudaStream_t s);
void vec_add32(int64_t n, const float* x, float* y, cudaStream_t s);

// PCG kernels working on device scalars
void pcg_init(int64_t n, const double* b, double* x, double* r, double* partial, cudaStream_t s);
void pcg_finish_bb(Scalars* sc, const double* partial, cudaStream_t s);
void pcg_dot_rz(int64_t n, const double* r, const double* z, const double* rold, int flexible, double* partial,
                cudaStream_t s);
void pcg_finish_rz(Scalars* sc, const double* partial, int first, int flexible, cudaStream_t s);
void pcg_update_p(int64_t n, const double* z, double* p, const Scalars* sc, int first, cudaStream_t s);
void pcg_spmv_pq(const DCSR& A, const double* p, double* q, double* partial, cudaStream_t s, double avg_row);
void pcg_finish_pq(Scalars* sc, const double* partial, cudaStream_t s);
void pcg_update_xr(int64_t n, const double* p, const double* q, double* x, double* r, double* rold, int flexible,
                   const Scalars* sc, double* partial, cudaStream_t s);
void pcg_finish_rr(Scalars* sc, const double* partial, cudaStream_t s);
// control of the graph-captured loop (graph_kernels.cu)
// asynchronous solve: parameters into the graph state; results (device pointers, each may be NULL)
void pcg_graph_params(GraphState* st, double rtol, int limit, int force, cudaStream_t s);
void pcg_graph_results(const GraphState* st, const double* hist, int* iters, double* relres, int* status,
                       cudaStream_t s);
void pcg_graph_start(const Scalars* sc, GraphState* st, double* hist, cudaGraphConditionalHandle first,
                     cudaGraphConditionalHandle loop, cudaStream_t s);
void pcg_graph_check(const Scalars* sc, GraphState* st, double* hist, cudaGraphConditionalHandle loop,
                     cudaGraphConditionalHandle more, cudaStream_t s);
void reduce_to(const double* partial, double* out, cudaStream_t s);

// multi-right-hand-side kernels (batch_kernels.cu); modes: 0 SpMM, 1 residual, 2 Chebyshev, 3 add
void bat_rows_launch64(const DCSR& A, int m, int mode, const double* val, const double* X, const double* B, double* Y,
                       double* D, const double* dinv, double c1, double c2, cudaStream_t s);
void bat_rows_launch32(const DCSR& A, int m, int mode, const float* val, const float* X, const float* B, float* Y,
                       float* D, const float* dinv, float c1, float c2, cudaStream_t s);
void bat_p_restrict(const Level& L, int m, const double* rf, double* rc, double* part, cudaStream_t s);
void bat_p_restrict32(const Level& L, int m, const float* rf, float* rc, float* part, cudaStream_t s);
void bat_p_prolong(const Level& L, int m, const double* ec, double* xf, cudaStream_t s);
void bat_p_prolong32(const Level& L, int m, const float* ec, float* xf, cudaStream_t s);
void bat_inverse(const double* Ainv, int64_t nc, int m, const double* B, double* X, cudaStream_t s);
void bat_inverse32(const double* Ainv, int64_t nc, int m, const float* B, float* X, cudaStream_t s);
void bat_cheb_first64(int64_t n, int m, const double* B, const double* dinv, double c2, double* X, double* D, cudaStream_t s);
void bat_cheb_first32(int64_t n, int m, const float* B, const float* dinv, float c2, float* X, float* D, cudaStream_t s);
void bat_to32(int64_t count, const double* x, float* y, cudaStream_t s);
void bat_to64(int64_t count, const float* x, double* y, cudaStream_t s);
size_t batch_scalars_bytes();
int batch_reduction_blocks();
void bat_pcg_init(int64_t n, int m, const double* B, double* X, double* R, double* partial, void* sc, cudaStream_t s);
void bat_pcg_rz(int64_t n, int m, const double* R, const double* Z, const double* Rold, int flexible, int first,
                double* partial, void* sc, cudaStream_t s);
void bat_pcg_update_p(int64_t n, int m, const double* Z, double* P, const void* sc, int first, cudaStream_t s);
void bat_pcg_pq(int64_t n, int m, const double* P, const double* Q, double* partial, void* sc, cudaStream_t s);
void bat_pcg_update_xr(int64_t n, int m, const double* P, const double* Q, double* X, double* R, double* Rold,
                       int flexible, double* partial, void* sc, cudaStream_t s);
void bat_graph_start_launch(const void* sc, int m, BatchGraphState* st, cudaGraphConditionalHandle first,
                            cudaGraphConditionalHandle loop, cudaStream_t s);
void bat_graph_check_launch(const void* sc, int m, BatchGraphState* st, cudaGraphConditionalHandle loop,
                            cudaGraphConditionalHandle more, cudaStream_t s);
// grouped multi-right-hand-side phases: several hierarchies' work of one phase in one launch,
// each hierarchy computing exactly what its standalone launch computes (batch_kernels.cu)
constexpr int kGroupMax = 16;  // hierarchies per launch (more are split into several launches)
struct GrpRowsArgs {           // a multi-RHS row kernel on one matrix (bat_rows / bat_pairs)
  int64_t n, n_items;
  int m, G, pat, pairs;
  const int64_t* rp;
  const int32_t *ci, *obase, *toff, *ia, *ib, *ig;
  const int64_t* gptr;
  const int32_t* gcol;
  const void *val, *X, *B;
  void *Y, *D;
  const void* dinv;
  double c1, c2;
};
struct GrpTransferArgs {       // an FP32 element transfer of one p-level
  int p, q, m;
  int32_t n_elem;
  int64_t n_next;
  const int32_t *l2g, *l2g_c, *cinc;
  const uint8_t* own;
  const float* p1d;
  const int64_t* cptr;
  const float* in;
  float *out, *part;
};
struct GrpVecArgs {            // a vector phase (GrpVecOp in batch_kernels.cu)
  int64_t n;
  int m, flag1, flag2;
  const void *a, *b, *e;
  void *c, *d;
  double v;
  void* sc;
  double* partial;
};
enum GrpVecOpHost { kGvInverse32H = 0, kGvChebFirst32H, kGvTo32H, kGvTo64H, kGvInitH, kGvDotRzH, kGvDotH,
                    kGvUpdateXrH, kGvUpdatePH, kGvFinishBbH, kGvFinishRzH, kGvFinishPqH, kGvFinishRrH };
// mode: 0 SpMM, 1 residual, 2 Chebyshev step, 3 add (as bat_rows_launch64/32); fp32: val is A.v32
GrpRowsArgs grp_rows_args(const DCSR& A, int m, const void* val, const void* X, const void* B, void* Y, void* D,
                          const void* dinv, double c1, double c2, bool fp32);
void grp_rows64(int mode, const std::vector<GrpRowsArgs>& ops, cudaStream_t s);
void grp_rows32(int mode, const std::vector<GrpRowsArgs>& ops, cudaStream_t s);
GrpTransferArgs grp_transfer_args(const Level& L, int m, const float* in, float* out, float* part);
void grp_p_restrict32(const std::vector<GrpTransferArgs>& ops, cudaStream_t s);
void grp_p_prolong32(const std::vector<GrpTransferArgs>& ops, cudaStream_t s);
void grp_vec(int op, const std::vector<GrpVecArgs>& ops, cudaStream_t s);

// host view of the batched CG scalars (layout shared with batch_kernels.cu)
struct BatchScalarsHost {
  double rho[32], pq[32], alpha[32], beta[32], rr[32], bb[32];
  int status[32], active[32];
  double tol2;
  int force;
  int pad;
};

// per-column partial sums over a fixed partition of the rows: block b handles rows
// [b*chunk, (b+1)*chunk); lane j of each warp accumulates column j (m <= 32)
__device__ __forceinline__ void column_block_sum(double v, int m, double* sh, double* out) {
  // v: this thread's partial for column (threadIdx.x & 31); reduce over the block's warps
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  sh[w * 32 + l] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sh[k * 32 + threadIdx.x];
    if (threadIdx.x < m) out[threadIdx.x] = s;
  }
  __syncthreads();
}

// pivot of the unit-diagonal Gram matrix below which a direction is dropped: FP64 products,
// and FP32 products (whose entries carry ~1e-7 relative rounding)
constexpr double kBlockDropTol = 1e-10;
constexpr double kBlockDropTol32 = 1e-5;
int block_gram_blocks();
// O = Lf^T R1 (and Lf^T R2), reduced into st->gram[0] (and [1]); Lf, R1, R2 are n x m row-major;
// fp32: products in FP32 arithmetic, FP64 accumulation across chunks
void blk_gram(int64_t n, int m, const double* Lf, const double* R1, const double* R2, int fp32, double* partial,
              BlockState* st, cudaStream_t s);
// factor G = st->gram[0] and alpha = G^+ st->gram[1] (mode 0); beta = -G^+ st->gram[0] (mode 1)
void blk_coef(int m, int mode, double tau, BlockState* st, cudaStream_t s);
// X += P alpha; R -= Q alpha; per-column ||r||^2, convergence and breakdown into the batch scalars
void blk_update_xr(int64_t n, int m, const double* P, const double* Q, double* X, double* R, const BlockState* st,
                   double* partial, void* sc, cudaStream_t s);
// P = Z + P beta (first: P = Z); fp32: P beta in FP32 arithmetic
void blk_update_p(int64_t n, int m, const double* Z, double* P, const BlockState* st, int first, int fp32,
                  cudaStream_t s);

// ------------------------------------------------------------------ setup kernels
uint32_t host_hash(int kind, int64_t i);
// exclusive scan of int32 flags/counts into int64 offsets (out has n+1 entries)
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
void scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// stable LSD radix sort of (key, idx) pairs by key (keys < 2^key_bits)
void radix_sort_pairs(uint32_t* keys, int64_t* idx, int64_t n, int key_bits, cudaStream_t s);
// transpose of a CSR matrix, rows of the result in ascending order
void csr_transpose(const DCSR& A, DCSR& T, cudaStream_t s);
// C = A B: symbolic union, no dropping, columns ascending, entries summed in ascending inner
// index with separately rounded products (matches a sequential Gustavson product bit for bit)
void spgemm(const DCSR& A, const DCSR& B, DCSR& C, cudaStream_t s);
// the same product when A has row groups (A.grp.on): the pattern once per group; false (C
// untouched) when the groups' patterns do not fit its tables
bool spgemm_grouped(const DCSR& A, const DCSR& B, DCSR& C, cudaStream_t s);
void csr_to32(DCSR& A, cudaStream_t s);
// the group-major copy of the big groups' values for the vector hybrid form from the FP32
// (precision 1, A.v32) or FP64 (precision 0, A.v) values; needs the hybrid lists; false if the
// form does not apply
bool hybrid_vector_build(DCSR& A, int precision, cudaStream_t s);
// the row-pair work items of the multi-right-hand-side FP32 products (needs the row groups)
bool batch_pairs_build(DCSR& A, cudaStream_t s);
// the sliced form's layout (once) and its copy of the FP64 (precision 0) or FP32 (1) values; needs
// the row groups; false if the form does not apply
bool sliced_build(DCSR& A, int precision, cudaStream_t s);
constexpr int kSliceStep = 8;  // columns per step of the sliced kernels (slice lengths are multiples)
// the row-kernel variant of A for precision prec (0 FP64, 1 FP32): form 0 the defaults measured
// best inside the solve, 1..6 forced (CSR, row patterns, row groups, hybrid, vector hybrid,
// sliced); threads forces threads per row where the form has a choice
RowVariant variant_for(const DCSR& A, int prec, int form, int threads);
// set A.var64 / A.var32 from forced options or the defaults measured best inside the solve
void choose_rows(DCSR& A, int form, int threads);
// a deterministic, nonzero test vector (the tuner's right-hand side)
void fill_tune_vector(int64_t n, double* x, cudaStream_t s);
// prefetch_rows -1: automatic, 0: off, > 0: distance in rows; chains 0: keep, else 2, 4 or 8
void set_prefetch(DCSR& A, int prefetch_rows, int chains);
// detect row groups with identical column sets (exact; leaves A.grp off if not worthwhile for the
// row kernels, unless any_sharing: then kept whenever the detection succeeds, for SpGEMM)
bool groups_build(DCSR& A, cudaStream_t s, int64_t max_groups, bool any_sharing = false);
// detect repeated row patterns (exact; returns false and leaves A.pat off if not worthwhile)
bool pattern_build(DCSR& A, cudaStream_t s, int64_t max_templates, int64_t max_offsets);
// diagonal inverse (checks positivity; returns false if a diagonal entry is <= 0 or missing)
bool diag_inverse(const DCSR& A, double* dinv, float* dinv32, cudaStream_t s);
// Lanczos estimate of lambda_max(D^-1/2 A D^-1/2)
double lanczos_rho(const DCSR& A, int steps, int hash_kind, Hierarchy& H);
// p-level construction: next map, owners, assembled P
// modal: hierarchical basis (prefix of modes, injection P); else nodal GLL (interpolation P)
void p_level_build(Level& F, Level& C, int modal, cudaStream_t s);
// h-level construction: MIS-2, aggregates, smoothed prolongation
int64_t h_level_aggregate(Level& F, double theta, int hash_kind, cudaStream_t s);
void h_level_prolongation(Level& F, cudaStream_t s);
// validation of the element map against A's pattern; returns number of violations
int64_t validate_map(const DCSR& A, const int32_t* l2g, int32_t n_elem, int nloc, cudaStream_t s);
// dense copy of a small CSR into column-major storage
void csr_to_dense_cm(const DCSR& A, double* D, cudaStream_t s);

}  // namespace giamg
