// graph_kernels.cu -- the outer conjugate-gradient loop's control on the device, for the solve
// captured as one CUDA graph: a start kernel after the initial residual norm, and a check kernel
// after every iteration's residual update.  They record the relative residual history, apply the
// stopping rule of the host loop (relres <= rtol, the iteration limit, breakdown) and set the
// graph's conditional handles, so the loop runs with no host round trip per iteration.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.cuh"

namespace giamg {

namespace {

// x0 = 0: relres_0 = 1 (0 for b = 0, which needs no iteration)
__global__ void graph_start_kernel(const Scalars* __restrict__ sc, GraphState* __restrict__ st, double* hist,
                                   cudaGraphConditionalHandle first, cudaGraphConditionalHandle loop) {
  const double bb = sc->bb;
  st->it = 0;
  st->status = 0;
  st->relres = bb == 0.0 ? 0.0 : 1.0;
  hist[0] = st->relres;
  const unsigned go = (bb != 0.0 && st->limit > 0) ? 1u : 0u;
  cudaGraphSetConditional(first, go);
  cudaGraphSetConditional(loop, go);
}

// after iteration it: relres_it = sqrt(||r||^2 / ||b||^2); continue while the limit is not reached
// and, unless the iteration count is forced, relres > rtol
__global__ void graph_check_kernel(const Scalars* __restrict__ sc, GraphState* __restrict__ st, double* hist,
                                   cudaGraphConditionalHandle loop, cudaGraphConditionalHandle more) {
  const int it = st->it + 1;
  st->it = it;
  unsigned cont = 0;
  if (sc->status != 0) {
    st->status = GIAMG_ERR_BREAKDOWN;
  } else {
    const double rr = sqrt(sc->rr / sc->bb);
    st->relres = rr;
    hist[it] = rr;
    cont = (it < st->limit && (st->force || !(rr <= st->rtol))) ? 1u : 0u;
  }
  cudaGraphSetConditional(loop, cont);
  cudaGraphSetConditional(more, cont);
}

// an asynchronous solve's parameters, from kernel arguments (a host buffer could be overwritten
// by the next call before the copy ran)
__global__ void graph_params_kernel(GraphState* __restrict__ st, double rtol, int limit, int force) {
  st->rtol = rtol;
  st->limit = limit;
  st->force = force;
  st->it = 0;
  st->status = 0;
}

// an asynchronous solve's results, with the synchronous call's rules: b = 0 gives relres 0 and
// no iteration; the limit reached above rtol (iteration count not forced) is GIAMG_ERR_MAXITER
__global__ void graph_results_kernel(const GraphState* __restrict__ st, const double* __restrict__ hist,
                                     int* iters, double* relres, int* status) {
  const bool zero = hist[0] == 0.0;
  int code = st->status;
  if (code == GIAMG_OK && !zero && !st->force && !(st->relres <= st->rtol)) code = GIAMG_ERR_MAXITER;
  if (iters) *iters = st->it;
  if (relres) *relres = zero ? 0.0 : st->relres;
  if (status) *status = code;
}

}  // namespace

void pcg_graph_params(GraphState* st, double rtol, int limit, int force, cudaStream_t s) {
  { graph_params_kernel<<<1, 1, 0, s>>>(st, rtol, limit, force); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void pcg_graph_results(const GraphState* st, const double* hist, int* iters, double* relres, int* status,
                       cudaStream_t s) {
  { graph_results_kernel<<<1, 1, 0, s>>>(st, hist, iters, relres, status); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void pcg_graph_start(const Scalars* sc, GraphState* st, double* hist, cudaGraphConditionalHandle first,
                     cudaGraphConditionalHandle loop, cudaStream_t s) {
  { graph_start_kernel<<<1, 1, 0, s>>>(sc, st, hist, first, loop); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

void pcg_graph_check(const Scalars* sc, GraphState* st, double* hist, cudaGraphConditionalHandle loop,
                     cudaGraphConditionalHandle more, cudaStream_t s) {
  { graph_check_kernel<<<1, 1, 0, s>>>(sc, st, hist, loop, more); note_launch(); }
  GIAMG_CUDA(cudaGetLastError());
}

}  // namespace giamg
