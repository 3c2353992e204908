// Autotuner.  The paper reports that the best block shape depends on the
// machine and the matrix (Section 4.3: beta(4,VS) best on A64FX, beta(8,VS)
// on Cascade Lake) and that cost grows with the number of blocks.  On the
// GPU there is a second knob, the number of lanes sharing one row (G): more
// lanes per row shorten each warp's serial block loop, fewer lanes keep the
// x accesses of neighbouring rows together.  Rather than a model, the tuner
// times the candidates on the caller's vectors:
//   spc5_tune           G in {1, 2, 4, 8} (those that fit 32 / r), the
//                       one-lane-per-row bodies, the two block-balanced
//                       plans and the expanded plan for one converted
//                       matrix, keeping the fastest plan;
//   spc5_convert_tuned  every requested beta(r,c), each tuned, keeping the
//                       fastest matrix (spc5_convert_tuned_ex: optionally
//                       ranked by the row-group plan the batched kernel runs).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "spc5_internal.h"

namespace spc5 {
namespace {

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  Events() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Median time of `iters` products, in microseconds (negative on error).
double time_spmv(const spc5_matrix *A, const void *x, void *y, int iters, cudaStream_t s) {
  Events ev;
  std::vector<double> t;
  for (int i = 0; i < 2; ++i)
    if (spmv_device(A, x, y, 1.0, 0.0, s) != SPC5_OK) return -1.0;
  for (int i = 0; i < iters; ++i) {
    cudaEventRecord(ev.a, s);
    if (spmv_device(A, x, y, 1.0, 0.0, s) != SPC5_OK) return -1.0;
    cudaEventRecord(ev.b, s);
    if (cudaEventSynchronize(ev.b) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    t.push_back(ms * 1e3);
  }
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

spc5_status tune(spc5_matrix *A, const void *x, void *y, int iters, cudaStream_t s) {
  int log2r = 0;
  while ((1 << log2r) < A->r) ++log2r;
  const int max_log2g = std::min(3, 5 - log2r);
  struct Cand {
    int log2g, body, flat;
  };
  // the block-balanced (two kernels) and expanded plans, and row-group plans (lanes per
  // row; bodies 2 to 4 need one lane per row)
  std::vector<Cand> cands;
  cands.push_back({0, 0, 1});
  cands.push_back({0, 0, 2});
  cands.push_back({0, 0, 3});
  cands.push_back({0, 2, 0});
  cands.push_back({0, 3, 0});
  cands.push_back({0, 4, 0});
  cands.push_back({0, 5, 0});
  cands.push_back({0, 6, 0});
  cands.push_back({0, 7, 0});
  for (int lg = 0; lg <= max_log2g; ++lg) cands.push_back({lg, 0, 0});
  // the predicated loop over the c bits spends an FMA on every bit: cheap
  // with FP32 arithmetic (64 FMAs per cycle per SM), not with FP64 (2)
  if (A->value_dtype != SPC5_F64)
    for (int lg = 0; lg <= max_log2g; ++lg) cands.push_back({lg, 1, 0});
  double best = -1.0, best_rows = -1.0;
  size_t best_i = 0, best_rows_i = 1;
  for (size_t i = 0; i < cands.size(); ++i) {
    PlanOptions o;
    o.kernel = 0;
    o.log2g = cands[i].log2g;
    o.body = cands[i].body;
    o.flat = cands[i].flat;
    spc5_status st = replan(A, s, o);
    if (st != SPC5_OK) return st;
    double us = time_spmv(A, x, y, iters, s);
    if (us < 0) {
      set_error("timing a candidate plan failed");
      return SPC5_ECUDA;
    }
    if (best < 0 || us < best) {
      best = us;
      best_i = i;
    }
    if (!cands[i].flat && (best_rows < 0 || us < best_rows)) {
      best_rows = us;
      best_rows_i = i;
    }
  }
  // The row-group plan is kept at its own best (the transposed product, the
  // gradient and the batched kernel use it even when the SpMV is flat).
  if (best_i != cands.size() - 1 || best_rows_i != cands.size() - 1) {
    PlanOptions o;
    o.kernel = 0;
    o.log2g = cands[best_rows_i].log2g;
    o.body = cands[best_rows_i].body;
    o.flat = cands[best_i].flat;
    spc5_status st = replan(A, s, o);
    if (st != SPC5_OK) return st;
  }
  // When row groups win, also try taking their tiles from a counter instead
  // of dealing them grid-stride (uneven tiles: a few percent either way).
  if (!cands[best_i].flat) {
    PlanOptions o;
    o.kernel = 0;
    o.log2g = cands[best_rows_i].log2g;
    o.body = cands[best_rows_i].body;
    o.flat = 0;
    o.dynamic = 1;
    spc5_status st = replan(A, s, o);
    if (st != SPC5_OK) return st;
    const double us = time_spmv(A, x, y, iters, s);
    if (us < 0) {
      set_error("timing a candidate plan failed");
      return SPC5_ECUDA;
    }
    if (us < best) {
      best = best_rows = us;
    } else {
      o.dynamic = 0;
      st = replan(A, s, o);
      if (st != SPC5_OK) return st;
    }
    // and cutting the groups of the last round of tiles in halves
    o.halves = 1;
    st = replan(A, s, o);
    if (st != SPC5_OK) return st;
    const double uh = time_spmv(A, x, y, iters, s);
    if (uh < 0) {
      set_error("timing a candidate plan failed");
      return SPC5_ECUDA;
    }
    if (uh < best) {
      best = best_rows = uh;
    } else {
      o.halves = 0;
      st = replan(A, s, o);
      if (st != SPC5_OK) return st;
    }
  }
  A->tuned_us = best;
  A->tuned_rows_us = best_rows;
  return SPC5_OK;
}

}  // namespace
}  // namespace spc5

using namespace spc5;

extern "C" spc5_status spc5_tune(spc5_matrix *A, const void *x, void *y, int iters,
                                 void *stream) {
  if (!A || (A->ncols > 0 && !x) || (A->nrows > 0 && !y) || iters < 1) {
    set_error("invalid argument");
    return SPC5_EINVAL;
  }
  if (A->nrows == 0) return SPC5_OK;
  return tune(A, x, y, iters, (cudaStream_t)stream);
}

extern "C" spc5_status spc5_convert_tuned(int64_t nrows, int64_t ncols, int64_t nnz,
                                          const int32_t *rowptr, const int32_t *colidx,
                                          const void *vals, spc5_dtype vals_dtype,
                                          spc5_dtype store_dtype, const int *shapes, int nshapes,
                                          int iters, void *stream, spc5_matrix **out) {
  return spc5_convert_tuned_ex(nrows, ncols, nnz, rowptr, colidx, vals, vals_dtype, store_dtype,
                               shapes, nshapes, iters, 0, stream, out);
}

extern "C" spc5_status spc5_convert_tuned_ex(int64_t nrows, int64_t ncols, int64_t nnz,
                                             const int32_t *rowptr, const int32_t *colidx,
                                             const void *vals, spc5_dtype vals_dtype,
                                             spc5_dtype store_dtype, const int *shapes,
                                             int nshapes, int iters, int rows_plan, void *stream,
                                             spc5_matrix **out) {
  static const int kAll[12] = {1, 8, 2, 4, 2, 8, 4, 4, 4, 8, 8, 4};
  if (!out || iters < 1 || (shapes && nshapes < 1)) {
    set_error("invalid argument");
    return SPC5_EINVAL;
  }
  if (!shapes) {
    shapes = kAll;
    nshapes = 6;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t es = store_dtype == SPC5_F64 ? 8 : 4;
  void *x = nullptr, *y = nullptr;
  spc5_status st = cuda_check(cudaMallocAsync(&x, (size_t)std::max<int64_t>(ncols, 1) * es, s),
                              "alloc tuning x");
  if (st != SPC5_OK) return st;
  st = cuda_check(cudaMallocAsync(&y, (size_t)std::max<int64_t>(nrows, 1) * es, s),
                  "alloc tuning y");
  if (st == SPC5_OK)
    st = cuda_check(cudaMemsetAsync(x, 0, (size_t)std::max<int64_t>(ncols, 1) * es, s),
                    "zero tuning x");
  spc5_matrix *best = nullptr;
  for (int i = 0; st == SPC5_OK && i < nshapes; ++i) {
    spc5_matrix *A = nullptr;
    st = spc5_convert_csr(nrows, ncols, nnz, rowptr, colidx, vals, vals_dtype, store_dtype,
                          shapes[2 * i], shapes[2 * i + 1], stream, &A);
    if (st != SPC5_OK) break;
    st = tune(A, x, y, iters, s);
    if (st != SPC5_OK) {
      spc5_destroy(A);
      break;
    }
    const double t = rows_plan ? A->tuned_rows_us : A->tuned_us;
    if (!best || t < (rows_plan ? best->tuned_rows_us : best->tuned_us)) {
      if (best) spc5_destroy(best);
      best = A;
    } else {
      spc5_destroy(A);
    }
  }
  cudaFreeAsync(x, s);
  cudaFreeAsync(y, s);
  cudaStreamSynchronize(s);
  if (st != SPC5_OK) {
    if (best) spc5_destroy(best);
    return st;
  }
  *out = best;
  return SPC5_OK;
}
