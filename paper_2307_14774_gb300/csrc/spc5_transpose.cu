// The transposed matrix A^T in beta(r,c), attached to A so that the
// transposed product is an ordinary SpMV (deterministic, no atomics).
//
// spc5_build_transpose reads A's stored blocks, not the CSR it came from:
//   1. one thread per panel walks the panel's blocks and, in the stored
//      value order (block, row, column: Algorithm 1's idxVal), counts the
//      entries of every column;
//   2. a prefix sum of the counts gives the row pointer of A^T; a second
//      walk places every entry in its column (a slot taken with an atomic
//      cursor, so the order within a column is arbitrary at this point);
//   3. one warp per column ranks the column's entries by row in shared
//      memory (rows are distinct within a column) and writes them sorted:
//      the CSR of A^T, with the values widened from the storage type;
//   4. spc5_convert_csr converts that CSR with A's block shape and storage
//      type (rounding the widened values back is exact), and the new
//      matrix's value sources are composed with the entries' CSR indices in
//      A, so spc5_set_values(A, vals) refreshes A^T from the same vals.
// Columns of more than kColCap entries are ranked by one CTA each, reading
// the rows from global memory; a column of more than kLongCap entries is
// rejected (SPC5_EUNSUPPORTED): the transposed product then keeps its
// atomic scatter.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "spc5_internal.h"
#include "spc5_scan.cuh"

namespace spc5 {
namespace {

constexpr int kThreads = 256;
constexpr int kColCap = 1024;    // entries of a column ranked in shared memory by a warp
constexpr int kLongCap = 65536;  // entries of a column ranked by a CTA (more: rejected)
constexpr int kSortWarps = 4;

inline unsigned grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 1 << 20);
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

// PLACE = false: cnt[col] += 1 for every stored entry.  PLACE = true: the
// entry goes to slot colptr[col] + cursor[col]++ with its row, its value
// (widened) and its CSR index in A.
template <bool PLACE, typename MaskT, typename VT>
__global__ void k_walk_panels(int64_t np, int64_t nrows, int r, int c,
                              const int32_t *__restrict__ brp, const int32_t *__restrict__ vptr,
                              const int32_t *__restrict__ colidx, const MaskT *__restrict__ masks,
                              const VT *__restrict__ values, const int32_t *__restrict__ value_src,
                              int32_t *cnt, const int32_t *__restrict__ colptr, int32_t *cursor,
                              int32_t *prow, double *pval, int32_t *psrc) {
  GRID_STRIDE(p, np) {
    int32_t v = vptr[p];
    for (int32_t b = brp[p]; b < brp[p + 1]; ++b) {
      uint32_t m = (uint32_t)masks[b];
      const int32_t c0 = colidx[b];
      while (m) {  // bit q * c + k, ascending: the stored order of the block's values
        const int bit = __ffs(m) - 1;
        m &= m - 1u;
        const int q = bit / c;
        const int32_t col = c0 + (bit - q * c);
        if (!PLACE) {
          atomicAdd(&cnt[col], 1);
        } else {
          const int32_t pos = colptr[col] + atomicAdd(&cursor[col], 1);
          prow[pos] = (int32_t)(p * r + q);
          pval[pos] = (double)widen(values[v]);
          psrc[pos] = value_src[v];
        }
        ++v;
      }
    }
  }
}

// One warp per column: rank the column's entries by row (distinct rows, so
// the rank is the count of smaller rows) and write them in that order.
__global__ void __launch_bounds__(32 * kSortWarps)
    k_sort_columns(int64_t ncols, const int32_t *__restrict__ colptr,
                   const int32_t *__restrict__ prow, const double *__restrict__ pval,
                   const int32_t *__restrict__ psrc, int32_t *srow, double *sval, int32_t *ssrc,
                   uint32_t *nlong, int32_t *long_cols) {
  __shared__ int32_t s_row[kSortWarps][kColCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t *rows = s_row[warp];
  const int64_t nw = (int64_t)gridDim.x * kSortWarps;
  for (int64_t j = (int64_t)blockIdx.x * kSortWarps + warp; j < ncols; j += nw) {
    const int32_t a = colptr[j], len = colptr[j + 1] - a;
    if (len > kColCap) {  // ranked by k_sort_long_columns
      if (lane == 0) long_cols[atomicAdd(nlong, 1u)] = (int32_t)j;
      continue;
    }
    __syncwarp();
    for (int32_t t = lane; t < len; t += 32) rows[t] = prow[a + t];
    __syncwarp();
    for (int32_t t = lane; t < len; t += 32) {
      const int32_t key = rows[t];
      int32_t rank = 0;
      for (int32_t u = 0; u < len; ++u) rank += rows[u] < key ? 1 : 0;
      srow[a + rank] = key;
      sval[a + rank] = pval[a + t];
      ssrc[a + rank] = psrc[a + t];
    }
  }
}

// One CTA per column longer than kColCap: the same ranking, rows read from
// global memory (through L1).
__global__ void __launch_bounds__(kThreads)
    k_sort_long_columns(const int32_t *__restrict__ long_cols, const int32_t *__restrict__ colptr,
                        const int32_t *__restrict__ prow, const double *__restrict__ pval,
                        const int32_t *__restrict__ psrc, int32_t *srow, double *sval,
                        int32_t *ssrc, uint32_t *too_long) {
  const int32_t j = long_cols[blockIdx.x];
  const int32_t a = colptr[j], len = colptr[j + 1] - a;
  if (len > kLongCap) {
    if (threadIdx.x == 0) atomicOr(too_long, 1u);
    return;
  }
  for (int32_t t = threadIdx.x; t < len; t += blockDim.x) {
    const int32_t key = prow[a + t];
    int32_t rank = 0;
    for (int32_t u = 0; u < len; ++u) rank += __ldg(prow + a + u) < key ? 1 : 0;
    srow[a + rank] = key;
    sval[a + rank] = pval[a + t];
    ssrc[a + rank] = psrc[a + t];
  }
}

// value_src of A^T, from indices into the CSR built here to CSR indices of A.
__global__ void k_compose(int64_t nnz, int32_t *value_src, const int32_t *__restrict__ ssrc) {
  GRID_STRIDE(i, nnz) { value_src[i] = ssrc[value_src[i]]; }
}

struct ReadCnt {  // cnt[i] for i < n, 0 at i == n
  const int32_t *m;
  int64_t n;
  __device__ int32_t operator()(int64_t i) const { return i < n ? m[i] : 0; }
};
struct WritePtr {
  int32_t *o;
  __device__ void operator()(int64_t i, int32_t v) const { o[i] = v; }
};
struct AddPtr {
  __device__ int32_t operator()(int32_t a, int32_t b) const { return a + b; }
};

template <typename T>
struct Buf {
  T *p = nullptr;
  cudaStream_t s;
  explicit Buf(cudaStream_t st) : s(st) {}
  cudaError_t alloc(int64_t n) {
    return scratch_alloc((void **)&p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), s);
  }
  ~Buf() {
    if (p) cudaFreeAsync(p, s);
  }
};

#define CK(call, what)                            \
  do {                                            \
    spc5_status _st = cuda_check((call), (what)); \
    if (_st != SPC5_OK) return _st;               \
  } while (0)

template <typename MaskT, typename VT>
void walk(bool place, const spc5_matrix *A, int32_t *cnt, const int32_t *colptr,
          int32_t *cursor, int32_t *prow, double *pval, int32_t *psrc, cudaStream_t s) {
  if (A->npanels == 0) return;
  const unsigned grid = grid_for(A->npanels);
  if (place)
    k_walk_panels<true, MaskT, VT><<<grid, kThreads, 0, s>>>(
        A->npanels, A->nrows, A->r, A->c, A->block_rowptr, A->panel_vptr, A->block_colidx,
        (const MaskT *)A->masks, (const VT *)A->values, A->value_src, cnt, colptr, cursor, prow,
        pval, psrc);
  else
    k_walk_panels<false, MaskT, VT><<<grid, kThreads, 0, s>>>(
        A->npanels, A->nrows, A->r, A->c, A->block_rowptr, A->panel_vptr, A->block_colidx,
        (const MaskT *)A->masks, (const VT *)A->values, A->value_src, cnt, colptr, cursor, prow,
        pval, psrc);
}

template <typename MaskT>
void walk_mask(bool place, const spc5_matrix *A, int32_t *cnt, const int32_t *colptr,
               int32_t *cursor, int32_t *prow, double *pval, int32_t *psrc, cudaStream_t s) {
  if (A->value_dtype == SPC5_F64)
    walk<MaskT, double>(place, A, cnt, colptr, cursor, prow, pval, psrc, s);
  else if (A->value_dtype == SPC5_F32)
    walk<MaskT, float>(place, A, cnt, colptr, cursor, prow, pval, psrc, s);
  else
    walk<MaskT, uint16_t>(place, A, cnt, colptr, cursor, prow, pval, psrc, s);
}

void walk_any(bool place, const spc5_matrix *A, int32_t *cnt, const int32_t *colptr,
              int32_t *cursor, int32_t *prow, double *pval, int32_t *psrc, cudaStream_t s) {
  const int mb = A->r * A->c / 8;
  if (mb == 1)
    walk_mask<uint8_t>(place, A, cnt, colptr, cursor, prow, pval, psrc, s);
  else if (mb == 2)
    walk_mask<uint16_t>(place, A, cnt, colptr, cursor, prow, pval, psrc, s);
  else
    walk_mask<uint32_t>(place, A, cnt, colptr, cursor, prow, pval, psrc, s);
}

spc5_status build(spc5_matrix *A, cudaStream_t s, spc5_matrix **out) {
  const int64_t nnz = A->nnz, ncols = A->ncols;
  Buf<int32_t> cnt(s), colptr(s), cursor(s), prow(s), psrc(s), srow(s), ssrc(s), tmp(s);
  Buf<double> pval(s), sval(s);
  Buf<uint32_t> flag(s);
  Buf<int32_t> long_cols(s);
  CK(cnt.alloc(ncols), "alloc");
  CK(colptr.alloc(ncols + 1), "alloc");
  CK(cursor.alloc(ncols), "alloc");
  CK(prow.alloc(nnz), "alloc");
  CK(psrc.alloc(nnz), "alloc");
  CK(pval.alloc(nnz), "alloc");
  CK(srow.alloc(nnz), "alloc");
  CK(ssrc.alloc(nnz), "alloc");
  CK(sval.alloc(nnz), "alloc");
  CK(flag.alloc(2), "alloc");
  CK(long_cols.alloc(ncols), "alloc");
  CK(tmp.alloc(scan_tmp_elems(ncols + 1)), "alloc");
  CK(cudaMemsetAsync(cnt.p, 0, (size_t)std::max<int64_t>(ncols, 1) * 4, s), "memset");
  CK(cudaMemsetAsync(cursor.p, 0, (size_t)std::max<int64_t>(ncols, 1) * 4, s), "memset");
  CK(cudaMemsetAsync(flag.p, 0, 8, s), "memset");
  walk_any(false, A, cnt.p, nullptr, nullptr, nullptr, nullptr, nullptr, s);
  CK(device_scan<int32_t>(ncols + 1, ReadCnt{cnt.p, ncols}, WritePtr{colptr.p}, AddPtr{}, 0,
                          false, tmp.p, s),
     "scan column counts");
  walk_any(true, A, nullptr, colptr.p, cursor.p, prow.p, pval.p, psrc.p, s);
  if (ncols > 0) {
    const int64_t blocks =
        std::min<int64_t>((ncols + kSortWarps - 1) / kSortWarps, (int64_t)device_sm_count() * 16);
    k_sort_columns<<<(unsigned)blocks, 32 * kSortWarps, 0, s>>>(
        ncols, colptr.p, prow.p, pval.p, psrc.p, srow.p, sval.p, ssrc.p, flag.p, long_cols.p);
  }
  CK(cudaGetLastError(), "transpose kernels");
  uint32_t nlong = 0;
  CK(cudaMemcpyAsync(&nlong, flag.p, 4, cudaMemcpyDeviceToHost, s), "read long columns");
  CK(cudaStreamSynchronize(s), "sync transpose");
  if (nlong > 0) {
    k_sort_long_columns<<<nlong, kThreads, 0, s>>>(long_cols.p, colptr.p, prow.p, pval.p,
                                                  psrc.p, srow.p, sval.p, ssrc.p, flag.p + 1);
    uint32_t too_long = 0;
    CK(cudaGetLastError(), "long column sort");
    CK(cudaMemcpyAsync(&too_long, flag.p + 1, 4, cudaMemcpyDeviceToHost, s), "read flag");
    CK(cudaStreamSynchronize(s), "sync transpose");
    if (too_long) {
      set_error("a column holds more than 65536 entries: no transposed copy (spc5_spmv_t "
                "keeps its atomic scatter)");
      return SPC5_EUNSUPPORTED;
    }
  }
  spc5_matrix *T = nullptr;
  spc5_status st = spc5_convert_csr(ncols, A->nrows, nnz, colptr.p, srow.p, sval.p, SPC5_F64,
                                    A->value_dtype, A->r, A->c, s, &T);
  if (st != SPC5_OK) return st;
  if (nnz > 0) k_compose<<<grid_for(nnz), kThreads, 0, s>>>(nnz, T->value_src, ssrc.p);
  st = cuda_check(cudaGetLastError(), "compose value sources");
  if (st == SPC5_OK) st = cuda_check(cudaStreamSynchronize(s), "sync transpose");
  if (st != SPC5_OK) {
    spc5_destroy(T);
    return st;
  }
  *out = T;
  return SPC5_OK;
}

}  // namespace
}  // namespace spc5

using namespace spc5;

extern "C" spc5_status spc5_build_transpose(spc5_matrix *A, void *stream) {
  if (!A) {
    set_error("NULL argument");
    return SPC5_EINVAL;
  }
  if (A->hybrid) {
    set_error("spc5_build_transpose does not take hybrid matrices");
    return SPC5_EUNSUPPORTED;
  }
  int dev = 0;
  spc5_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != SPC5_OK) return st;
  if (dev != A->device) {
    set_error("the matrix lives on another device than the current one");
    return SPC5_EDEVICE;
  }
  spc5_matrix *T = nullptr;
  st = build(A, (cudaStream_t)stream, &T);
  if (st != SPC5_OK) return st;
  if (A->transpose) spc5_destroy(A->transpose);
  A->transpose = T;
  return SPC5_OK;
}
