// Mixed-precision iterative refinement with an inner conjugate-gradient
// solver (the paper's motivation for a fast SpMV is iterative solvers,
// Section 1).  FP64 is used only where it decides the final accuracy:
//   outer loop (FP64):  r = b - A64 x;  stop when ||r|| <= tol ||b||;
//                       solve A d = r / ||r|| approximately (inner CG);
//                       x += ||r|| d
//   inner CG (FP32 vectors, FP32/BF16/FP64 matrix values, FP32 products,
//   dot products accumulated in FP64): plain CG on the scaled residual,
//   stopped at a relative residual inner_tol or max_inner iterations.
// One inner iteration is a fixed sequence of kernels whose scalars (alpha,
// beta, r.r) live in device memory; it is captured once as a CUDA graph and
// replayed, and the host reads r.r only every few iterations.  Reductions
// are two-level (per-block partials, then one block sums them in fixed
// order), so the solver is deterministic for a deterministic SpMV.  In the
// inner iteration the second level runs in the last block of the first to
// finish (a ticket counter) and computes alpha or beta right there, so an
// iteration is the SpMV plus three launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "spc5_internal.h"

namespace spc5 {
namespace {

constexpr int kT = 256;
constexpr int kRedBlocks = 1024;  // partials of a dot product

struct Scal {
  double rr, rr_new, pq, alpha, beta, rr0;
};

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = (threadIdx.x < kT / 32) ? sh[threadIdx.x] : 0.0;
  if (threadIdx.x < 32)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kT) k_dot_partial(int64_t n, const T *a, const T *b,
                                                    double *part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    s += (double)a[i] * (double)b[i];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Sums the partials into *out (one block, fixed order).
__global__ void __launch_bounds__(kT) k_dot_final(const double *part, int nparts, double *out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kT) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// The last of the grid's blocks to finish (ticket) sums the partials in
// block order, as k_dot_final does, and its thread 0 stores the sum in
// *out; returns true in that block only.  The ticket is reset for the next
// launch.  Each block publishes its partial with a fence before taking its
// ticket, and the last block reads the partials through L2.
__device__ __forceinline__ bool last_block_sum(double s, double *part, unsigned *ticket,
                                               double *out) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kT) t += __ldcg(part + i);
  t = block_sum(t);
  if (threadIdx.x == 0) {
    *out = t;
    *ticket = 0u;
  }
  return true;
}

// p.q, then alpha = rr / p.q (one launch of the inner iteration)
template <typename T>
__global__ void __launch_bounds__(kT) k_dot_alpha(int64_t n, const T *p, const T *q,
                                                  double *part, unsigned *ticket, Scal *sc) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    s += (double)p[i] * (double)q[i];
  s = block_sum(s);
  double pq;
  if (last_block_sum(s, part, ticket, &pq) && threadIdx.x == 0) {
    sc->pq = pq;
    sc->alpha = (pq != 0.0) ? sc->rr / pq : 0.0;
  }
}

// p = r, rr = rr_new (start of the inner solve), d = 0.
template <typename T>
__global__ void k_cg_start(int64_t n, const T *r, T *p, T *d) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    p[i] = r[i];
    d[i] = (T)0;
  }
}

__global__ void k_scalars_init(Scal *s) {
  s->rr = s->rr_new;
  s->rr0 = s->rr_new;
}

// d += alpha p; r -= alpha q; r.r, then beta = r.r / rr and rr = r.r
template <typename T>
__global__ void __launch_bounds__(kT) k_cg_update(int64_t n, Scal *sc, const T *p, const T *q,
                                                  T *d, T *r, double *part, unsigned *ticket) {
  const T a = (T)sc->alpha;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    d[i] = fma(a, p[i], d[i]);
    const T ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    s += (double)ri * (double)ri;
  }
  s = block_sum(s);
  double rr_new;
  if (last_block_sum(s, part, ticket, &rr_new) && threadIdx.x == 0) {
    sc->rr_new = rr_new;
    sc->beta = (sc->rr != 0.0) ? rr_new / sc->rr : 0.0;
    sc->rr = rr_new;
  }
}

// p = r + beta p
template <typename T>
__global__ void k_cg_dir(int64_t n, const Scal *sc, const T *r, T *p) {
  const T b = (T)sc->beta;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    p[i] = fma(b, p[i], r[i]);
}

// r_lo = r / nrm ; (FP64 -> inner precision)
template <typename T>
__global__ void k_scale_down(int64_t n, const double *r, double inv, T *out) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    out[i] = (T)(r[i] * inv);
}

// x += nrm * d
template <typename T>
__global__ void k_update_x(int64_t n, const T *d, double nrm, double *x) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    x[i] = fma(nrm, (double)d[i], x[i]);
}

template <typename T>
struct Buf {
  T *p = nullptr;
  cudaError_t alloc(int64_t n) { return cudaMalloc((void **)&p, sizeof(T) * std::max<int64_t>(n, 1)); }
  ~Buf() {
    if (p) cudaFree(p);
  }
};

unsigned grid_n(int64_t n) {
  return (unsigned)std::min<int64_t>(std::max<int64_t>((n + kT - 1) / kT, 1), kRedBlocks);
}

template <typename T>
spc5_status dot(int64_t n, const T *a, const T *b, double *part, double *out, cudaStream_t s) {
  k_dot_partial<T><<<kRedBlocks, kT, 0, s>>>(n, a, b, part);
  k_dot_final<<<1, kT, 0, s>>>(part, kRedBlocks, out);
  return cuda_check(cudaGetLastError(), "dot");
}

#define CK(call, what)                            \
  do {                                            \
    spc5_status _st = cuda_check((call), (what)); \
    if (_st != SPC5_OK) return _st;               \
  } while (0)
#define CS(expr)                      \
  do {                                \
    spc5_status _st = (expr);         \
    if (_st != SPC5_OK) return _st;   \
  } while (0)

template <typename T>
spc5_status ircg(const spc5_matrix *A64, const spc5_matrix *Alo, const double *b, double *x,
                 double tol, int max_outer, double inner_tol, int max_inner, cudaStream_t s,
                 spc5_cg_report *rep) {
  const int64_t n = A64->nrows;
  Buf<double> r64, part, dev_nrm;
  Buf<T> rlo, p, q, d;
  Buf<Scal> sc;
  Buf<unsigned> ticket;
  CK(r64.alloc(n), "alloc");
  CK(ticket.alloc(1), "alloc");
  CK(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned), s), "zero ticket");
  CK(part.alloc(kRedBlocks), "alloc");
  CK(dev_nrm.alloc(2), "alloc");
  CK(rlo.alloc(n), "alloc");
  CK(p.alloc(n), "alloc");
  CK(q.alloc(n), "alloc");
  CK(d.alloc(n), "alloc");
  CK(sc.alloc(1), "alloc");
  const unsigned g = grid_n(n);

  // ||b||
  CS(dot<double>(n, b, b, part.p, dev_nrm.p, s));
  double bb = 0.0;
  CK(cudaMemcpyAsync(&bb, dev_nrm.p, sizeof(double), cudaMemcpyDeviceToHost, s), "read");
  CK(cudaStreamSynchronize(s), "sync");
  const double nb = sqrt(bb);
  rep->outer_iters = 0;
  rep->inner_iters = 0;
  rep->relres = 0.0;
  if (nb == 0.0) {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s), "zero x");
    CK(cudaStreamSynchronize(s), "sync");
    return SPC5_OK;
  }

  // One inner iteration, captured as a graph on a private stream.
  cudaStream_t cs = nullptr;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  spc5_status st = cuda_check(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal),
                              "begin capture");
  if (st == SPC5_OK) {
    spc5_status sst = spmv_device(Alo, p.p, q.p, 1.0, 0.0, cs);
    k_dot_alpha<T><<<kRedBlocks, kT, 0, cs>>>(n, p.p, q.p, part.p, ticket.p, sc.p);
    k_cg_update<T><<<kRedBlocks, kT, 0, cs>>>(n, sc.p, p.p, q.p, d.p, rlo.p, part.p, ticket.p);
    k_cg_dir<T><<<g, kT, 0, cs>>>(n, sc.p, rlo.p, p.p);
    st = cuda_check(cudaStreamEndCapture(cs, &graph), "end capture");
    if (st == SPC5_OK && sst != SPC5_OK) st = sst;
  }
  if (st == SPC5_OK) st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "instantiate");

  const int check_every = 8;
  for (int outer = 0; st == SPC5_OK && outer < max_outer; ++outer) {
    // r = b - A64 x  (FP64)
    st = cuda_check(cudaMemcpyAsync(r64.p, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s),
                    "copy b");
    if (st != SPC5_OK) break;
    st = spmv_device(A64, x, r64.p, -1.0, 1.0, s);
    if (st != SPC5_OK) break;
    st = dot<double>(n, r64.p, r64.p, part.p, dev_nrm.p, s);
    if (st != SPC5_OK) break;
    double rr = 0.0;
    st = cuda_check(cudaMemcpyAsync(&rr, dev_nrm.p, sizeof(double), cudaMemcpyDeviceToHost, s),
                    "read");
    if (st == SPC5_OK) st = cuda_check(cudaStreamSynchronize(s), "sync");
    if (st != SPC5_OK) break;
    const double nr = sqrt(rr);
    rep->relres = nr / nb;
    if (nr <= tol * nb) break;
    rep->outer_iters = outer + 1;
    // inner solve of A d = r / ||r||
    k_scale_down<T><<<g, kT, 0, s>>>(n, r64.p, 1.0 / nr, rlo.p);
    k_cg_start<T><<<g, kT, 0, s>>>(n, rlo.p, p.p, d.p);
    k_dot_partial<T><<<kRedBlocks, kT, 0, s>>>(n, rlo.p, rlo.p, part.p);
    k_dot_final<<<1, kT, 0, s>>>(part.p, kRedBlocks, &sc.p->rr_new);
    k_scalars_init<<<1, 1, 0, s>>>(sc.p);
    st = cuda_check(cudaGetLastError(), "inner start");
    int it = 0;
    while (st == SPC5_OK && it < max_inner) {
      const int burst = std::min(check_every, max_inner - it);
      for (int i = 0; i < burst && st == SPC5_OK; ++i)
        st = cuda_check(cudaGraphLaunch(exec, s), "graph launch");
      it += burst;
      Scal hs;
      if (st == SPC5_OK)
        st = cuda_check(cudaMemcpyAsync(&hs, sc.p, sizeof(Scal), cudaMemcpyDeviceToHost, s),
                        "read scalars");
      if (st == SPC5_OK) st = cuda_check(cudaStreamSynchronize(s), "sync");
      if (st != SPC5_OK) break;
      if (!(hs.rr > 0.0) || sqrt(hs.rr / hs.rr0) <= inner_tol) break;
    }
    rep->inner_iters += it;
    if (st != SPC5_OK) break;
    k_update_x<T><<<g, kT, 0, s>>>(n, d.p, nr, x);
    st = cuda_check(cudaGetLastError(), "update x");
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (st == SPC5_OK) st = cuda_check(cudaStreamSynchronize(s), "sync");
  return st;
}

}  // namespace
}  // namespace spc5

using namespace spc5;

extern "C" spc5_status spc5_ircg(const spc5_matrix *A64, const spc5_matrix *Alo, const double *b,
                                 double *x, double tol, int max_outer, double inner_tol,
                                 int max_inner, void *stream, spc5_cg_report *report) {
  if (!A64 || !Alo || !b || !x || !report || tol <= 0.0 || max_outer < 1 || max_inner < 1 ||
      !(inner_tol > 0.0 && inner_tol < 1.0)) {
    set_error("invalid argument");
    return SPC5_EINVAL;
  }
  if (A64->value_dtype != SPC5_F64 || A64->nrows != A64->ncols || Alo->nrows != A64->nrows ||
      Alo->ncols != A64->ncols) {
    set_error("A64 must be a square FP64 matrix and Alo the same matrix in any precision");
    return SPC5_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (Alo->value_dtype == SPC5_F64)
    return ircg<double>(A64, Alo, b, x, tol, max_outer, inner_tol, max_inner, s, report);
  return ircg<float>(A64, Alo, b, x, tol, max_outer, inner_tol, max_inner, s, report);
}
