// Products needed to differentiate y = A(vals) x:
//   spc5_spmv_t      dx = alpha * A^T g + beta * dx
//   spc5_values_grad dvals[e] = alpha * g[row(e)] * x[col(e)] for every stored
//                    entry e, returned in CSR order
//   spc5_set_values  store new CSR-ordered values into the converted matrix
//
// The first two walk the same work tiles and lane mapping as the SpMV (lane
// (j, q, g) = row q of panel j, G lanes sharing a row's blocks, value offsets
// from the panel offset plus popcount scans), so long panels are split into
// bounded pieces here too; they need no row reduction.  The transpose
// scatters with atomic adds (results are exact up to the order of the
// additions).  The values gradient writes a row's entries from the row's
// CSR start (kept by the converter), since a lane walks its row's entries
// in column order, which is CSR order; pieces of long panels, which do not
// see their rows' earlier entries, address them through value_src, the CSR
// index of every stored value.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "spc5_internal.h"

namespace spc5 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;


// Calls f(row, col, mq, off, rc) for every block of the lane's row in the
// tile: row = global row, col = block start column, mq = the row's c-bit
// mask, off = index of the row's first value of the block, rc (COUNT only)
// = the row's values in the tile's earlier blocks (a group scan of the row
// bits over the G lanes of the row).
template <int R, int C, bool COUNT = false, typename F>
__device__ __forceinline__ void walk_tile(const Tile &cur, int lane,
                                          const int32_t *__restrict__ brp,
                                          const int32_t *__restrict__ vptr,
                                          const int32_t *__restrict__ bcol,
                                          const typename MaskType<R, C>::T *__restrict__ masks,
                                          int64_t nrows, F &&f) {
  const bool segment = (cur.mode & kSegment) != 0;
  const int log2G = cur.mode & 15;
  const int G = 1 << log2G;
  const int shift_j = Log2<R>::v + log2G;
  const int g = lane & (G - 1);
  const int q = (lane >> log2G) & (R - 1);
  const int j = lane >> shift_j;
  const uint32_t row_low = (q == 0) ? 0u : ((1u << (q * C)) - 1u);
  const uint32_t cmask = (1u << C) - 1u;
  bool pvalid;
  int32_t bl, nbp, v;
  int64_t p;
  if (segment) {
    p = cur.p0;
    pvalid = (j == 0);
    bl = cur.b0;
    nbp = cur.b1 - cur.b0;
    v = cur.v0;
  } else {
    p = (int64_t)cur.p0 + j;
    // a heavy panel (kSkip) has tiles of its own
    pvalid = p < cur.p1 && !((cur.mode & kSkip) && (((uint32_t)cur.slot >> j) & 1u));
    bl = pvalid ? brp[p] : 0;
    nbp = pvalid ? brp[p + 1] - bl : 0;
    v = pvalid ? vptr[p] : 0;
  }
  const int64_t row = p * R + q;
  const bool rvalid = pvalid && row < nrows;
  const int32_t maxnb = __reduce_max_sync(kFull, nbp);
  int32_t rc = 0;
  for (int32_t it = 0; it < maxnb; it += G) {
    const int32_t idx = it + g;
    const bool valid = idx < nbp;
    const uint32_t m = valid ? (uint32_t)masks[bl + idx] : 0u;
    const int32_t col = valid ? bcol[bl + idx] : 0;
    const uint32_t mq = (m >> (q * C)) & cmask;
    const int pc = __popc(m);
    int incl = pc;
    for (int o = 1; o < G; o <<= 1) {
      int t = __shfl_up_sync(kFull, incl, o, G);
      if (g >= o) incl += t;
    }
    const int total = (G > 1) ? __shfl_sync(kFull, incl, G - 1, G) : pc;
    const int32_t off = v + (incl - pc) + __popc(m & row_low);
    int32_t rq = 0;
    if (COUNT) {  // the row's values in the earlier blocks of this round
      const int pq = __popc(mq);
      int iq = pq;
      for (int o = 1; o < G; o <<= 1) {
        int t = __shfl_up_sync(kFull, iq, o, G);
        if (g >= o) iq += t;
      }
      rq = rc + iq - pq;
      rc += (G > 1) ? __shfl_sync(kFull, iq, G - 1, G) : pq;
    }
    if (rvalid) f(row, col, mq, off, rq);
    v += total;
  }
}

template <int R, int C, typename VT, typename AT>
__global__ void __launch_bounds__(kThreads)
    k_spmv_t(const Tile *__restrict__ tiles, int64_t ntiles, const int32_t *__restrict__ brp,
             const int32_t *__restrict__ vptr, const int32_t *__restrict__ bcol,
             const typename MaskType<R, C>::T *__restrict__ masks, const VT *__restrict__ vals,
             const AT *__restrict__ g, AT *__restrict__ dx, AT alpha, int64_t nrows) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles;
       t += nwarps) {
    const Tile cur = tiles[t];
    walk_tile<R, C>(cur, lane, brp, vptr, bcol, masks, nrows,
                    [&](int64_t row, int32_t col, uint32_t mq, int32_t off, int32_t) {
                      const AT gr = alpha * g[row];
                      while (mq) {
                        const int k = __ffs(mq) - 1;
                        mq &= mq - 1u;
                        atomicAdd(dx + col + k, (AT)widen(vals[off++]) * gr);
                      }
                    });
  }
}

template <int R, int C, typename AT>
__global__ void __launch_bounds__(kThreads)
    k_values_grad(const Tile *__restrict__ tiles, int64_t ntiles,
                  const int32_t *__restrict__ brp, const int32_t *__restrict__ vptr,
                  const int32_t *__restrict__ bcol,
                  const typename MaskType<R, C>::T *__restrict__ masks,
                  const int32_t *__restrict__ value_src, const int32_t *__restrict__ csr_rowptr,
                  const AT *__restrict__ g, const AT *__restrict__ x, AT *__restrict__ dvals,
                  AT alpha, int64_t nrows, bool pieces_only) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles;
       t += nwarps) {
    const Tile cur = tiles[t];
    if (pieces_only && !(cur.mode & kPartial)) continue;
    if ((cur.mode & kPartial) || !csr_rowptr) {  // a piece of a long panel: its rows'
                                                 // earlier values are in other tiles, so
                                                 // the positions come from value_src
      walk_tile<R, C>(cur, lane, brp, vptr, bcol, masks, nrows,
                      [&](int64_t row, int32_t col, uint32_t mq, int32_t off, int32_t) {
                        const AT gr = alpha * g[row];
                        while (mq) {
                          const int k = __ffs(mq) - 1;
                          mq &= mq - 1u;
                          dvals[value_src[off++]] = gr * x[col + k];
                        }
                      });
    } else {  // whole panels: a row's entries in column order are its CSR entries, written
              // from the row's CSR start on (value_src is not read)
      walk_tile<R, C, true>(cur, lane, brp, vptr, bcol, masks, nrows,
                            [&](int64_t row, int32_t col, uint32_t mq, int32_t, int32_t rc) {
                              const AT gr = alpha * g[row];
                              AT *dst = dvals + csr_rowptr[row] + rc;
                              while (mq) {
                                const int k = __ffs(mq) - 1;
                                mq &= mq - 1u;
                                *dst++ = gr * x[col + k];
                              }
                            });
    }
  }
}

// Values gradient by panels: one warp per panel, 32 / r lanes per row (a
// segment tile of the whole panel), so a row's lanes take consecutive
// blocks and write a contiguous run of the row's CSR entries per round,
// where the row-group tiles (one lane per row) write 32 scattered rows.
// Panels cut into pieces (listed, ascending, in long_panels) are left to
// the piece tiles of k_values_grad.
template <int R, int C, typename AT>
__global__ void __launch_bounds__(kThreads)
    k_values_grad_panels(int64_t npanels, const int32_t *__restrict__ brp,
                         const int32_t *__restrict__ vptr, const int32_t *__restrict__ bcol,
                         const typename MaskType<R, C>::T *__restrict__ masks,
                         const int32_t *__restrict__ long_panels, int64_t nlong,
                         const int32_t *__restrict__ csr_rowptr, const AT *__restrict__ g,
                         const AT *__restrict__ x, AT *__restrict__ dvals, AT alpha,
                         int64_t nrows) {
  constexpr int kLog2G = 5 - Log2<R>::v;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npanels;
       p += nwarps) {
    if (nlong > 0) {  // is p cut into pieces?
      int64_t lo = 0, hi = nlong;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (long_panels[mid] < p)
          lo = mid + 1;
        else
          hi = mid;
      }
      if (lo < nlong && long_panels[lo] == p) continue;
    }
    const Tile cur{(int32_t)p, (int32_t)p + 1, brp[p], brp[p + 1], vptr[p], vptr[p + 1], 0,
                   kSegment | kLog2G};
    walk_tile<R, C, true>(cur, lane, brp, vptr, bcol, masks, nrows,
                          [&](int64_t row, int32_t col, uint32_t mq, int32_t, int32_t rc) {
                            const AT gr = alpha * g[row];
                            AT *dst = dvals + csr_rowptr[row] + rc;
                            while (mq) {
                              const int k = __ffs(mq) - 1;
                              mq &= mq - 1u;
                              *dst++ = gr * x[col + k];
                            }
                          });
  }
}

template <typename AT>
__global__ void k_scale(int64_t n, AT *y, AT beta) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (beta == (AT)0) ? (AT)0 : beta * y[i];
}

// Storage conversions (round to nearest even), as in the converter.
__device__ __forceinline__ void store(double *dst, double d) { *dst = d; }
__device__ __forceinline__ void store(float *dst, double d) { *dst = __double2float_rn(d); }
__device__ __forceinline__ void store(uint16_t *dst, double d) {
  float f = __double2float_rz(d);  // round to odd into FP32, then to nearest even into BF16
  uint32_t b = __float_as_uint(f);
  if ((double)f != d) b |= 1u;
  b += 0x7FFFu + ((b >> 16) & 1u);
  *dst = (uint16_t)(b >> 16);
}

template <typename VT>
__global__ void k_set_values(int64_t nnz, const int32_t *__restrict__ value_src,
                             const double *__restrict__ vals_csr, VT *__restrict__ values) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x)
    store(values + i, vals_csr[value_src[i]]);
}

int sms() { return device_sm_count(); }

unsigned tile_grid(int64_t ntiles) {
  int64_t blocks = (ntiles + (kThreads / 32) - 1) / (kThreads / 32);
  blocks = std::min<int64_t>(std::max<int64_t>(blocks, 1), (int64_t)sms() * 8);
  return (unsigned)blocks;
}

unsigned flat_grid(int64_t n) {
  int64_t blocks = (n + kThreads - 1) / kThreads;
  blocks = std::min<int64_t>(std::max<int64_t>(blocks, 1), (int64_t)sms() * 16);
  return (unsigned)blocks;
}

template <int R, int C, typename VT, typename AT>
cudaError_t run_t(const spc5_matrix *A, const void *g, void *dx, double alpha, double beta,
                  cudaStream_t s) {
  using MT = typename MaskType<R, C>::T;
  k_scale<AT><<<flat_grid(A->ncols), kThreads, 0, s>>>(A->ncols, (AT *)dx, (AT)beta);
  if (A->ntiles > 0)
    k_spmv_t<R, C, VT, AT><<<tile_grid(A->ntiles), kThreads, 0, s>>>(
        A->tiles, A->ntiles, A->block_rowptr, A->panel_vptr, A->block_colidx,
        (const MT *)A->masks, (const VT *)A->values, (const AT *)g, (AT *)dx, (AT)alpha,
        A->nrows);
  return cudaGetLastError();
}

template <int R, int C, typename AT>
cudaError_t run_grad(const spc5_matrix *A, const void *g, const void *x, void *dvals,
                     double alpha, cudaStream_t s) {
  using MT = typename MaskType<R, C>::T;
  const bool by_panels = A->csr_rowptr != nullptr;
  if (by_panels && A->npanels > 0)
    k_values_grad_panels<R, C, AT><<<tile_grid(A->npanels), kThreads, 0, s>>>(
        A->npanels, A->block_rowptr, A->panel_vptr, A->block_colidx, (const MT *)A->masks,
        A->long_panels, A->nlong, A->csr_rowptr, (const AT *)g, (const AT *)x, (AT *)dvals,
        (AT)alpha, A->nrows);
  if (A->ntiles > 0 && (!by_panels || A->nlong > 0))
    k_values_grad<R, C, AT><<<tile_grid(A->ntiles), kThreads, 0, s>>>(
        A->tiles, A->ntiles, A->block_rowptr, A->panel_vptr, A->block_colidx,
        (const MT *)A->masks, A->value_src, A->csr_rowptr, (const AT *)g, (const AT *)x,
        (AT *)dvals, (AT)alpha, A->nrows, by_panels);
  return cudaGetLastError();
}

template <int R, int C>
cudaError_t dispatch_t(const spc5_matrix *A, const void *g, void *dx, double alpha,
                       double beta, cudaStream_t s) {
  if (A->value_dtype == SPC5_F64) return run_t<R, C, double, double>(A, g, dx, alpha, beta, s);
  if (A->value_dtype == SPC5_F32) return run_t<R, C, float, float>(A, g, dx, alpha, beta, s);
  return run_t<R, C, uint16_t, float>(A, g, dx, alpha, beta, s);
}

template <int R, int C>
cudaError_t dispatch_grad(const spc5_matrix *A, const void *g, const void *x, void *dvals,
                          double alpha, cudaStream_t s) {
  if (A->value_dtype == SPC5_F64) return run_grad<R, C, double>(A, g, x, dvals, alpha, s);
  return run_grad<R, C, float>(A, g, x, dvals, alpha, s);
}

bool device_readable(const void *p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace spc5

using namespace spc5;

extern "C" spc5_status spc5_spmv_t(const spc5_matrix *A, const void *g, void *dx, double alpha,
                                   double beta, void *stream) {
  if (!A || (A->nrows > 0 && !g) || (A->ncols > 0 && !dx)) {
    set_error("NULL argument");
    return SPC5_EINVAL;
  }
  if (A->hybrid) {
    set_error("spc5_spmv_t does not take hybrid matrices");
    return SPC5_EUNSUPPORTED;
  }
  if (A->ncols == 0) return SPC5_OK;
  if ((A->nrows > 0 && !device_readable(g)) || !device_readable(dx)) {
    set_error("spc5_spmv_t takes device vectors");
    return SPC5_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // with a transposed copy the product is an ordinary SpMV over A^T
  if (A->transpose) return spmv_device(A->transpose, g, dx, alpha, beta, s);
  cudaError_t e = cudaSuccess;
  switch (A->r * 100 + A->c) {
    case 108: e = dispatch_t<1, 8>(A, g, dx, alpha, beta, s); break;
    case 204: e = dispatch_t<2, 4>(A, g, dx, alpha, beta, s); break;
    case 208: e = dispatch_t<2, 8>(A, g, dx, alpha, beta, s); break;
    case 404: e = dispatch_t<4, 4>(A, g, dx, alpha, beta, s); break;
    case 408: e = dispatch_t<4, 8>(A, g, dx, alpha, beta, s); break;
    case 804: e = dispatch_t<8, 4>(A, g, dx, alpha, beta, s); break;
    default: set_error("unsupported block shape"); return SPC5_EUNSUPPORTED_RC;
  }
  return cuda_check(e, "spmv_t launch");
}

extern "C" spc5_status spc5_values_grad(const spc5_matrix *A, const void *g, const void *x,
                                        void *dvals, double alpha, void *stream) {
  if (!A || (A->nrows > 0 && !g) || (A->ncols > 0 && !x) || (A->nnz > 0 && !dvals)) {
    set_error("NULL argument");
    return SPC5_EINVAL;
  }
  if (A->hybrid) {
    set_error("spc5_values_grad does not take hybrid matrices");
    return SPC5_EUNSUPPORTED;
  }
  if (A->nnz == 0) return SPC5_OK;
  if (!device_readable(g) || !device_readable(x) || !device_readable(dvals)) {
    set_error("spc5_values_grad takes device arrays");
    return SPC5_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  switch (A->r * 100 + A->c) {
    case 108: e = dispatch_grad<1, 8>(A, g, x, dvals, alpha, s); break;
    case 204: e = dispatch_grad<2, 4>(A, g, x, dvals, alpha, s); break;
    case 208: e = dispatch_grad<2, 8>(A, g, x, dvals, alpha, s); break;
    case 404: e = dispatch_grad<4, 4>(A, g, x, dvals, alpha, s); break;
    case 408: e = dispatch_grad<4, 8>(A, g, x, dvals, alpha, s); break;
    case 804: e = dispatch_grad<8, 4>(A, g, x, dvals, alpha, s); break;
    default: set_error("unsupported block shape"); return SPC5_EUNSUPPORTED_RC;
  }
  return cuda_check(e, "values_grad launch");
}

extern "C" spc5_status spc5_set_values(spc5_matrix *A, const double *vals, void *stream) {
  if (!A || (A->nnz > 0 && !vals)) {
    set_error("NULL argument");
    return SPC5_EINVAL;
  }
  if (A->hybrid) {
    set_error("spc5_set_values does not take hybrid matrices");
    return SPC5_EUNSUPPORTED;
  }
  if (A->nnz == 0) return SPC5_OK;
  if (!device_readable(vals)) {
    set_error("spc5_set_values takes device values");
    return SPC5_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = flat_grid(A->nnz);
  if (A->value_dtype == SPC5_F64)
    k_set_values<double><<<grid, kThreads, 0, s>>>(A->nnz, A->value_src, vals,
                                                   (double *)A->values);
  else if (A->value_dtype == SPC5_F32)
    k_set_values<float><<<grid, kThreads, 0, s>>>(A->nnz, A->value_src, vals,
                                                  (float *)A->values);
  else
    k_set_values<uint16_t><<<grid, kThreads, 0, s>>>(A->nnz, A->value_src, vals,
                                                     (uint16_t *)A->values);
  spc5_status st = cuda_check(cudaGetLastError(), "set_values launch");
  // the transposed copy's value sources index the same CSR
  if (st == SPC5_OK && A->transpose) st = spc5_set_values(A->transpose, vals, stream);
  return st;
}
