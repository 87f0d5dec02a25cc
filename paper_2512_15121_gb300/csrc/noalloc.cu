// noalloc.cu -- giamg_true_relres_noalloc: the true relative residual ||b - A x|| / ||b|| of the
// finest level, computed without allocating any memory.
//
// Who needs it: callers that cannot call cudaMalloc (or must not while the check runs), for
// example code that checks convergence from inside a region whose device memory is owned by
// another allocator that has reserved the GPU, or a serving loop that runs under a fixed
// device-memory budget.  giamg_solve_stats computes the same number but allocates a small
// result buffer on every call; this variant keeps its partial sums in a file-scope device array
// instead.
//
// Scratch: kChunks partial sums for each of the two norms plus the two totals, 1 MiB in all,
// statically allocated in every GPU that loads the library and held until the process exits.
// Rows are summed in fixed chunks of kRowsPerChunk, so the result does not depend on the
// launch configuration; at most kChunks * kRowsPerChunk = 16,777,216 rows are accepted.
// Every call overwrites the scratch entries it reads before reading them (nothing needs
// clearing).  Each device has its own copy of the array, and all calls on one device share
// it: two calls that overlap on the same GPU (for example on two streams) race.
//
// Loading: with lazy module loading (the CUDA default) this file's module, and with it the array,
// is loaded on first use.  giamg_setup therefore loads it (noalloc_prepare: the array's address
// and both kernels) on the handle's device, so a later call allocates nothing, not even on its
// first use.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace giamg {

namespace {

constexpr int kRowsPerChunk = 256;
constexpr int kChunks = 65536;
constexpr int64_t kMaxRows = (int64_t)kRowsPerChunk * kChunks;
constexpr int kThreads = 256;  // 8 warps, 32 rows each per chunk

// [0, kChunks): partial sums of r_i^2; [kChunks, 2 kChunks): of b_i^2; then the two totals
static __device__ __align__(256) double g_relres_scratch[2 * kChunks + 2];

// The device address of g_relres_scratch, looked up once per device with that device current
// (in host code the array's name is a host-side stand-in, not a device address).
std::mutex g_mu;
double* g_addr[64] = {};

// Makes a device current for the lifetime of the guard and restores the caller's device after.
struct CurrentDevice {
  int saved = -1;
  explicit CurrentDevice(int device) {
    GIAMG_CUDA(cudaGetDevice(&saved));
    if (saved != device) GIAMG_CUDA(cudaSetDevice(device));
  }
  ~CurrentDevice() {
    int now = -1;
    if (cudaGetDevice(&now) == cudaSuccess && now != saved) cudaSetDevice(saved);
  }
};

__global__ void __launch_bounds__(kThreads) relres_chunks(int64_t n, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          const double* __restrict__ v,
                                                          const double* __restrict__ b,
                                                          const double* __restrict__ x, double* scratch) {
  __shared__ double sr[kThreads / 32], sb[kThreads / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kRowsPerChunk + (int64_t)w * (kRowsPerChunk / (kThreads / 32));
  double rr = 0.0, bb = 0.0;
  for (int k = 0; k < kRowsPerChunk / (kThreads / 32); ++k) {
    const int64_t i = row0 + k;
    double s = 0.0;
    if (i < n)
      for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) s += v[t] * x[ci[t]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (i < n && lane == 0) {
      const double r = b[i] - s;
      rr += r * r;
      bb += b[i] * b[i];
    }
  }
  if (lane == 0) {
    sr[w] = rr;
    sb[w] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
      a += sr[k];
      c += sb[k];
    }
    scratch[blockIdx.x] = a;
    scratch[kChunks + blockIdx.x] = c;
  }
}

__global__ void relres_total(int chunks, double* scratch) {
  __shared__ double sr[32], sb[32];
  double a = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < chunks; k += blockDim.x) {
    a += scratch[k];
    c += scratch[kChunks + k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sr[w] = a;
    sb[w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tc = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      ta += sr[k];
      tc += sb[k];
    }
    scratch[2 * kChunks] = ta;
    scratch[2 * kChunks + 1] = tc;
  }
}

// The scratch address on `device`, which must be current.  The first lookup loads the module
// (allocating the array) and both kernels, so later launches load nothing.
double* scratch_address(int device) {
  std::lock_guard<std::mutex> lock(g_mu);
  GIAMG_CHECK(device >= 0 && device < 64, GIAMG_ERR_ARG, "device ordinal out of range");
  if (!g_addr[device]) {
    void* p = nullptr;
    GIAMG_CUDA(cudaGetSymbolAddress(&p, g_relres_scratch));
    cudaFuncAttributes fa;
    GIAMG_CUDA(cudaFuncGetAttributes(&fa, relres_chunks));
    GIAMG_CUDA(cudaFuncGetAttributes(&fa, relres_total));
    g_addr[device] = static_cast<double*>(p);
  }
  return g_addr[device];
}

// b and x must be device (or managed) memory of the handle's device: a host address handed to
// the kernels would fault, or read host memory through the GPU's mapping.
void check_device_vector(const void* ptr, int device, const char* name) {
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error{GIAMG_ERR_ARG, std::string(name) + ": not a pointer the CUDA runtime knows"};
  }
  const bool dev = a.type == cudaMemoryTypeDevice && a.device == device;
  const bool managed = a.type == cudaMemoryTypeManaged;
  GIAMG_CHECK(dev || managed, GIAMG_ERR_ARG,
              std::string(name) + ": giamg_true_relres_noalloc needs device memory of the handle's device "
                                  "(host arrays and other devices' memory are refused)");
}

}  // namespace

void noalloc_prepare() {
  int device = 0;
  GIAMG_CUDA(cudaGetDevice(&device));
  (void)scratch_address(device);
}

}  // namespace giamg

using namespace giamg;

extern "C" int giamg_true_relres_noalloc(giamg_handle h, const double* b, const double* x, double* true_relres) {
  try {
    GIAMG_CHECK(h != nullptr, GIAMG_ERR_ARG, "NULL handle");
    GIAMG_CHECK(b && x && true_relres, GIAMG_ERR_ARG, "b, x and true_relres are required");
    Hierarchy& H = *hierarchy_of(h);
    const DCSR& A = H.lev[0]->A;
    GIAMG_CHECK(A.n <= kMaxRows, GIAMG_ERR_ARG,
                "giamg_true_relres_noalloc accepts at most 16,777,216 rows (its static scratch holds 65,536 "
                "chunk sums of 256 rows); this matrix has " + std::to_string(A.n));
    CurrentDevice on(H.device);
    check_device_vector(b, H.device, "b");
    check_device_vector(x, H.device, "x");
    double* scratch = scratch_address(H.device);
    const int chunks = (int)((A.n + kRowsPerChunk - 1) / kRowsPerChunk);
    cudaStream_t s = H.stream;
    if (chunks > 0) {
      relres_chunks<<<chunks, kThreads, 0, s>>>(A.n, A.rp.get(), A.ci.get(), A.v.get(), b, x, scratch);
      note_launch();
      relres_total<<<1, 1024, 0, s>>>(chunks, scratch);
      note_launch();
      GIAMG_CUDA(cudaGetLastError());
    }
    double tot[2] = {0.0, 0.0};
    if (chunks > 0)
      GIAMG_CUDA(cudaMemcpyAsync(tot, scratch + 2 * kChunks, sizeof(tot), cudaMemcpyDeviceToHost, s));
    GIAMG_CUDA(cudaStreamSynchronize(s));
    *true_relres = tot[1] > 0.0 ? std::sqrt(tot[0] / tot[1]) : 0.0;
    return GIAMG_OK;
  } catch (const Error& e) {
    set_error(e.code, e.msg);
    return e.code;
  } catch (...) {
    set_error(GIAMG_ERR_ARG, "unexpected error");
    return GIAMG_ERR_ARG;
  }
}
