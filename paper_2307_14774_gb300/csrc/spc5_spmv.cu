// y = alpha * A x + beta * y over beta(r,c) (Algorithm 1).
//
// GPU mapping.  Algorithm 1 walks a panel's blocks with one running value
// index idxVal, so a block's values cannot be located without the
// popcounts of all earlier blocks.  The converter stores every panel's first
// value offset (panel_vptr), which removes the dependency between panels;
// inside a panel the offsets come from popcounts:
//   - a warp holds PPW = 32 / (r * G) panels; lane (j, q, g) works on row q
//     of panel j, and the G lanes of a row take the panel's blocks G at a
//     time (G = 2^log2G, chosen per matrix),
//   - a round loads G blocks (start column, packed mask word), the G lanes
//     exclusive-scan the blocks' popcounts, and each lane finds its row's
//     values at  panel offset + scan + popc(mask bits of rows < q),
//   - each lane loops over its row's set bits (the scalar path of
//     Algorithm 1, one bit per iteration) with FP64 FMAs; x is read through
//     L1/L2 at column start + k,
//   - the G partial sums of a row are combined with shuffles and one lane
//     stores y (Section 3.2's single write of the reduced row results).
#include <cuda_runtime.h>
#include <stdint.h>

#include "spc5_internal.h"

namespace spc5 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSpmvThreads = 256;

template <int R, int C>
struct MaskType {
  using T = uint32_t;
};
template <>
struct MaskType<1, 8> {
  using T = uint8_t;
};
template <>
struct MaskType<2, 4> {
  using T = uint8_t;
};
template <>
struct MaskType<2, 8> {
  using T = uint16_t;
};
template <>
struct MaskType<4, 4> {
  using T = uint16_t;
};

template <int R, int C>
__global__ void __launch_bounds__(kSpmvThreads)
    k_spmv_rowlanes(int64_t npanels, int64_t nrows, const int32_t *__restrict__ block_rowptr,
                    const int32_t *__restrict__ panel_vptr,
                    const int32_t *__restrict__ block_colidx,
                    const typename MaskType<R, C>::T *__restrict__ masks,
                    const double *__restrict__ vals, const double *__restrict__ x,
                    double *__restrict__ y, double alpha, double beta, int log2G) {
  static_assert(R * C <= 32, "mask word must fit 32 bits");
  const int lane = threadIdx.x & 31;
  const int G = 1 << log2G;
  int log2R = 0;
  while ((1 << log2R) < R) ++log2R;
  const int shift_j = log2R + log2G;
  const int ppw = 32 >> shift_j;  // panels per warp
  const int g = lane & (G - 1);
  const int q = (lane >> log2G) & (R - 1);
  const int j = lane >> shift_j;
  const uint32_t row_low = (q == 0) ? 0u : ((1u << (q * C)) - 1u);
  const uint32_t cmask = (1u << C) - 1u;

  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp_id; w * ppw < npanels; w += nwarps) {
    const int64_t p = w * ppw + j;
    const bool pvalid = p < npanels;
    const int32_t b0 = pvalid ? block_rowptr[p] : 0;
    const int32_t nbp = pvalid ? block_rowptr[p + 1] - b0 : 0;
    int32_t v = pvalid ? panel_vptr[p] : 0;
    const int32_t maxnb = __reduce_max_sync(kFull, nbp);
    double acc = 0.0;
    for (int32_t it = 0; it < maxnb; it += G) {
      const bool valid = (it + g) < nbp;
      const int32_t b = b0 + it + g;
      const uint32_t m = valid ? (uint32_t)masks[b] : 0u;
      const int32_t col = valid ? block_colidx[b] : 0;
      const int pc = __popc(m);
      int incl = pc;
      for (int o = 1; o < G; o <<= 1) {
        int t = __shfl_up_sync(kFull, incl, o, G);
        if (g >= o) incl += t;
      }
      const int total = (G > 1) ? __shfl_sync(kFull, incl, G - 1, G) : pc;
      int32_t off = v + (incl - pc) + __popc(m & row_low);
      uint32_t mq = (m >> (q * C)) & cmask;
      while (mq) {
        const int k = __ffs(mq) - 1;
        mq &= mq - 1u;
        acc = fma(vals[off], x[col + k], acc);
        ++off;
      }
      v += total;
    }
    for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o, G);
    const int64_t row = p * R + q;
    if (pvalid && g == 0 && row < nrows) {
      double out = alpha * acc;
      if (beta != 0.0) out = fma(beta, y[row], out);
      y[row] = out;
    }
  }
}

template <int R, int C>
cudaError_t launch(const spc5_matrix *A, const double *x, double *y, double alpha, double beta,
                   cudaStream_t s) {
  using MaskT = typename MaskType<R, C>::T;
  int log2G = A->log2_lanes_per_row;
  int log2R = 0;
  while ((1 << log2R) < R) ++log2R;
  if (log2R + log2G > 5) log2G = 5 - log2R;
  const int ppw = 32 >> (log2R + log2G);
  int64_t warps = (A->npanels + ppw - 1) / ppw;
  int64_t blocks = (warps + (kSpmvThreads / 32) - 1) / (kSpmvThreads / 32);
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_spmv_rowlanes<R, C><<<(unsigned)blocks, kSpmvThreads, 0, s>>>(
      A->npanels, A->nrows, A->block_rowptr, A->panel_vptr, A->block_colidx,
      (const MaskT *)A->masks, (const double *)A->values, x, y, alpha, beta, log2G);
  return cudaGetLastError();
}

}  // namespace

spc5_status spmv_device(const spc5_matrix *A, const double *x, double *y, double alpha,
                        double beta, cudaStream_t s) {
  if (A->nrows == 0) return SPC5_OK;
  cudaError_t e;
  switch (A->r * 100 + A->c) {
    case 108: e = launch<1, 8>(A, x, y, alpha, beta, s); break;
    case 204: e = launch<2, 4>(A, x, y, alpha, beta, s); break;
    case 208: e = launch<2, 8>(A, x, y, alpha, beta, s); break;
    case 404: e = launch<4, 4>(A, x, y, alpha, beta, s); break;
    case 408: e = launch<4, 8>(A, x, y, alpha, beta, s); break;
    case 804: e = launch<8, 4>(A, x, y, alpha, beta, s); break;
    default:
      set_error("unsupported block shape");
      return SPC5_EUNSUPPORTED_RC;
  }
  return cuda_check(e, "spmv launch");
}

}  // namespace spc5
