// Hybrid form of beta(r,c): a block holding a single value costs a block's
// column index, mask and mask test for one product, and the paper finds SPC5
// slower than CSR below about two values per block; its closing remarks
// propose mixing the block format with a scalar one.  Here every block
// whose r masks hold exactly one set bit becomes a scalar entry (row, column,
// value) in a CSR of scalars, columns ascending in each row, and every other
// block stays a block (a beta(r,c) matrix of its own, values in Algorithm 1's
// order).  A single-value block's bit is always its block's first column
// (a block opens at an entry), so the scalar's column is the block's start.
//
// The split runs on the GPU after the conversion, with flat passes and
// prefix sums: popcounts give the single-value blocks; prefix sums of the
// kept blocks and of their values give the compacted block arrays; for
// each row-in-panel q, a prefix sum of the blocks holding a scalar of row q
// gives every scalar's rank in its row and the rows' counts (a CSR row
// pointer after one more prefix sum).  Integer work: the result equals any
// other implementation of the same rule (the CPU oracle checks it byte for
// byte).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "spc5_internal.h"
#include "spc5_scan.cuh"

namespace spc5 {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n) {
  int64_t blocks = (n + kThreads - 1) / kThreads;
  if (blocks < 1) blocks = 1;
  if (blocks > 1048576) blocks = 1048576;
  return (unsigned)blocks;
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

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

// a block's r*c-bit mask word, whatever its storage width
__device__ __forceinline__ uint32_t mask_at(const void *masks, int mb, int64_t b) {
  if (mb == 1) return ((const uint8_t *)masks)[b];
  if (mb == 2) return ((const uint16_t *)masks)[b];
  return ((const uint32_t *)masks)[b];
}

__global__ void k_popc(int64_t nb, const void *masks, int mb, int32_t *pc) {
  GRID_STRIDE(b, nb) { pc[b] = __popc(mask_at(masks, mb, b)); }
}

__global__ void k_mark_panel_starts(int64_t np, int64_t nb, const int32_t *brp, int32_t *mark) {
  GRID_STRIDE(p, np - 1) {
    const int32_t b = brp[p + 1];
    if (b < nb) atomicAdd(&mark[b], 1);
  }
}

struct ReadI32 {
  const int32_t *m;
  __device__ int32_t operator()(int64_t i) const { return m[i]; }
};
struct WriteI32 {
  int32_t *o;
  __device__ void operator()(int64_t i, int32_t v) const { o[i] = v; }
};
// flags over nb blocks, 0 at index nb (an exclusive scan of nb + 1 gives the total)
struct KeepFlag {  // block holds two or more values
  const int32_t *pc;
  int64_t nb;
  __device__ int32_t operator()(int64_t i) const { return i < nb && pc[i] != 1 ? 1 : 0; }
};
struct KeptValues {
  const int32_t *pc;
  int64_t nb;
  __device__ int32_t operator()(int64_t i) const { return i < nb && pc[i] != 1 ? pc[i] : 0; }
};
struct AllValues {
  const int32_t *pc;
  int64_t nb;
  __device__ int32_t operator()(int64_t i) const { return i < nb ? pc[i] : 0; }
};
struct ScalarOfRow {  // block is a single value in row q of its panel
  const int32_t *pc;
  const void *masks;
  int64_t nb;
  int mb, c, q;
  __device__ int32_t operator()(int64_t i) const {
    if (i >= nb || pc[i] != 1) return 0;
    return (__ffs(mask_at(masks, mb, i)) - 1) / c == q ? 1 : 0;
  }
};
struct ReadPad {
  const int32_t *m;
  int64_t n;
  __device__ int32_t operator()(int64_t i) const { return i < n ? m[i] : 0; }
};

// block part's panel pointers
__global__ void k_part_ptrs(int64_t np, const int32_t *brp, const int32_t *kscan,
                            const int32_t *vkscan, int32_t *brp_b, int32_t *vptr_b) {
  GRID_STRIDE(p, np + 1) {
    brp_b[p] = kscan[brp[p]];
    vptr_b[p] = vkscan[brp[p]];
  }
}

template <typename MT, typename VT>
__global__ void k_compact(int64_t nb, const int32_t *pc, const int32_t *kscan,
                          const int32_t *vkscan, const int32_t *boff, const int32_t *bcol,
                          const MT *masks, const VT *vals, const int32_t *vsrc, int32_t *bcol_b,
                          MT *masks_b, VT *vals_b, int32_t *vsrc_b) {
  GRID_STRIDE(b, nb) {
    if (pc[b] == 1) continue;
    const int32_t k = kscan[b];
    bcol_b[k] = bcol[b];
    masks_b[k] = masks[b];
    for (int i = 0; i < pc[b]; ++i) {
      vals_b[vkscan[b] + i] = vals[boff[b] + i];
      vsrc_b[vkscan[b] + i] = vsrc[boff[b] + i];
    }
  }
}

// scalars per row for row-in-panel q
__global__ void k_row_counts(int64_t np, int64_t nrows, int r, int q, const int32_t *brp,
                             const int32_t *sq, int32_t *cnt) {
  GRID_STRIDE(p, np) {
    const int64_t row = p * r + q;
    if (row < nrows) cnt[row] = sq[brp[p + 1]] - sq[brp[p]];
  }
}

template <typename VT>
__global__ void k_scatter_scalars(int64_t nb, int r, int c, int q, const int32_t *pc,
                                  const void *masks, int mb, const int32_t *bpanel,
                                  const int32_t *brp, const int32_t *sq,
                                  const int32_t *s_rowptr, const int32_t *boff,
                                  const int32_t *bcol, const VT *vals, int32_t *s_colidx,
                                  VT *s_vals) {
  GRID_STRIDE(b, nb) {
    if (pc[b] != 1) continue;
    const int bit = __ffs(mask_at(masks, mb, b)) - 1;
    if (bit / c != q) continue;
    const int32_t p = bpanel[b];
    const int64_t row = (int64_t)p * r + q;
    const int32_t pos = s_rowptr[row] + (sq[b] - sq[brp[p]]);
    s_colidx[pos] = bcol[b] + bit % c;
    s_vals[pos] = vals[boff[b]];
  }
}

__global__ void k_iota(int64_t n, int32_t *o) {
  GRID_STRIDE(i, n) { o[i] = (int32_t)i; }
}

#define CK(call, what)                            \
  do {                                            \
    spc5_status _st = cuda_check((call), (what)); \
    if (_st != SPC5_OK) return _st;               \
  } while (0)

template <typename MT, typename VT>
spc5_status split_typed(spc5_matrix *A, cudaStream_t s) {
  const int64_t nb = A->nblocks, np = A->npanels, nrows = A->nrows;
  const int r = A->r, c = A->c, mb = r * c / 8;
  Buf<int32_t> pc(s), kscan(s), vkscan(s), boff(s), bpanel(s), sq(s), cnt(s), tmp(s);
  CK(pc.alloc(nb), "alloc");
  CK(kscan.alloc(nb + 1), "alloc");
  CK(vkscan.alloc(nb + 1), "alloc");
  CK(boff.alloc(nb + 1), "alloc");
  CK(bpanel.alloc(nb), "alloc");
  CK(sq.alloc(nb + 1), "alloc");
  CK(cnt.alloc(nrows + 1), "alloc");
  CK(tmp.alloc(scan_tmp_elems(std::max<int64_t>(nb, nrows) + 1)), "alloc");
  if (nb > 0) k_popc<<<grid_for(nb), kThreads, 0, s>>>(nb, A->masks, mb, pc.p);
  CK(device_scan<int32_t>(nb + 1, KeepFlag{pc.p, nb}, WriteI32{kscan.p}, AddI32{}, 0, false,
                          tmp.p, s),
     "scan kept blocks");
  CK(device_scan<int32_t>(nb + 1, KeptValues{pc.p, nb}, WriteI32{vkscan.p}, AddI32{}, 0, false,
                          tmp.p, s),
     "scan kept values");
  CK(device_scan<int32_t>(nb + 1, AllValues{pc.p, nb}, WriteI32{boff.p}, AddI32{}, 0, false,
                          tmp.p, s),
     "scan values");
  if (nb > 0) {
    CK(cudaMemsetAsync(bpanel.p, 0, (size_t)nb * sizeof(int32_t), s), "memset");
    if (np > 1)
      k_mark_panel_starts<<<grid_for(np), kThreads, 0, s>>>(np, nb, A->block_rowptr, bpanel.p);
    CK(device_scan<int32_t>(nb, ReadI32{bpanel.p}, WriteI32{bpanel.p}, AddI32{}, 0, true, tmp.p,
                            s),
       "scan panels");
  }
  int32_t tot[2] = {0, 0};
  CK(cudaMemcpyAsync(&tot[0], kscan.p + nb, 4, cudaMemcpyDeviceToHost, s), "rd");
  CK(cudaMemcpyAsync(&tot[1], vkscan.p + nb, 4, cudaMemcpyDeviceToHost, s), "rd");
  CK(cudaStreamSynchronize(s), "sync hybrid counts");
  const int64_t nb_b = tot[0], nnz_b = tot[1], ns = A->nnz - nnz_b;

  // block part
  int32_t *brp_b = nullptr, *vptr_b = nullptr, *bcol_b = nullptr, *vsrc_b = nullptr;
  void *masks_b = nullptr, *vals_b = nullptr;
  CK(cudaMalloc((void **)&brp_b, (size_t)(np + 1) * sizeof(int32_t) + 16), "alloc");
  CK(cudaMalloc((void **)&vptr_b, (size_t)(np + 1) * sizeof(int32_t) + 16), "alloc");
  CK(cudaMalloc((void **)&bcol_b, (size_t)nb_b * sizeof(int32_t) + 16), "alloc");
  CK(cudaMalloc(&masks_b, (size_t)nb_b * mb + 16), "alloc");
  CK(cudaMalloc(&vals_b, (size_t)nnz_b * sizeof(VT) + 16), "alloc");
  CK(cudaMalloc((void **)&vsrc_b, (size_t)nnz_b * sizeof(int32_t) + 16), "alloc");
  k_part_ptrs<<<grid_for(np + 1), kThreads, 0, s>>>(np, A->block_rowptr, kscan.p, vkscan.p,
                                                     brp_b, vptr_b);
  if (nb > 0)
    k_compact<MT, VT><<<grid_for(nb), kThreads, 0, s>>>(
        nb, pc.p, kscan.p, vkscan.p, boff.p, A->block_colidx, (const MT *)A->masks,
        (const VT *)A->values, A->value_src, bcol_b, (MT *)masks_b, (VT *)vals_b, vsrc_b);

  // scalars: counts per row, CSR row pointer, then the scatter
  CK(cudaMalloc((void **)&A->s_rowptr, (size_t)(nrows + 1) * sizeof(int32_t) + 16), "alloc");
  CK(cudaMalloc((void **)&A->s_colidx, (size_t)ns * sizeof(int32_t) + 16), "alloc");
  CK(cudaMalloc(&A->s_vals, (size_t)ns * sizeof(VT) + 16), "alloc");
  CK(cudaMemsetAsync(cnt.p, 0, (size_t)(nrows + 1) * sizeof(int32_t), s), "memset");
  for (int q = 0; q < r; ++q) {
    CK(device_scan<int32_t>(nb + 1, ScalarOfRow{pc.p, A->masks, nb, mb, c, q}, WriteI32{sq.p},
                            AddI32{}, 0, false, tmp.p, s),
       "scan scalars of a row");
    if (np > 0)
      k_row_counts<<<grid_for(np), kThreads, 0, s>>>(np, nrows, r, q, A->block_rowptr, sq.p,
                                                     cnt.p);
  }
  CK(device_scan<int32_t>(nrows + 1, ReadPad{cnt.p, nrows}, WriteI32{A->s_rowptr}, AddI32{}, 0,
                          false, tmp.p, s),
     "scan scalar rows");
  for (int q = 0; q < r && nb > 0; ++q) {
    CK(device_scan<int32_t>(nb + 1, ScalarOfRow{pc.p, A->masks, nb, mb, c, q}, WriteI32{sq.p},
                            AddI32{}, 0, false, tmp.p, s),
       "scan scalars of a row");
    k_scatter_scalars<VT><<<grid_for(nb), kThreads, 0, s>>>(
        nb, r, c, q, pc.p, A->masks, mb, bpanel.p, A->block_rowptr, sq.p, A->s_rowptr, boff.p,
        A->block_colidx, (const VT *)A->values, A->s_colidx, (VT *)A->s_vals);
  }
  CK(cudaGetLastError(), "hybrid split kernels");
  CK(cudaStreamSynchronize(s), "sync hybrid split");

  // the block part replaces the handle's arrays
  cudaFree(A->block_rowptr);
  cudaFree(A->panel_vptr);
  cudaFree(A->block_colidx);
  cudaFree(A->masks);
  cudaFree(A->values);
  cudaFree(A->value_src);
  A->block_rowptr = brp_b;
  A->panel_vptr = vptr_b;
  A->block_colidx = bcol_b;
  A->masks = masks_b;
  A->values = vals_b;
  A->value_src = vsrc_b;
  A->device_bytes += (nb_b - nb) * (int64_t)(4 + mb) + (nnz_b - A->nnz) * (int64_t)(sizeof(VT) + 4) +
                     (nrows + 1) * 4 + ns * (int64_t)(4 + sizeof(VT)) + 48;
  A->nblocks = nb_b;
  A->nnz = nnz_b;
  A->nscalars = ns;
  A->hybrid = 1;
  return SPC5_OK;
}

spc5_status plan_scalars(spc5_matrix *A, cudaStream_t s) {
  const int64_t ns = A->nscalars;
  Buf<int32_t> iota(s);
  CK(iota.alloc(ns + 1), "alloc");
  if (ns > 0) k_iota<<<grid_for(ns), kThreads, 0, s>>>(ns, iota.p);
  ExpandedPlan ep;
  spc5_status st =
      build_expanded(A->nrows, ns, ns, 1, A->s_rowptr, A->s_rowptr, iota.p, s, &ep);
  if (st != SPC5_OK) return st;
  A->stiles = ep.tiles;
  A->sntiles = ep.ntiles;
  A->slong_rows = ep.long_panels;
  A->slong_slots = ep.long_slots;
  A->snlong = ep.nlong;
  A->snpieces = ep.npieces;
  CK(cudaMalloc((void **)&A->spartial, (size_t)std::max<int64_t>(ep.npieces, 1) * sizeof(double)),
     "alloc scalar partial sums");
  A->device_bytes += ep.ntiles * (int64_t)sizeof(Tile) + ep.nlong * 12 + ep.npieces * 8;
  CK(cudaStreamSynchronize(s), "sync scalar plan");
  return SPC5_OK;
}

}  // namespace

spc5_status hybrid_split(spc5_matrix *A, cudaStream_t s) {
  spc5_status st;
  const int mb = A->r * A->c / 8;
  if (mb == 1) {
    st = A->value_dtype == SPC5_F64   ? split_typed<uint8_t, double>(A, s)
         : A->value_dtype == SPC5_F32 ? split_typed<uint8_t, float>(A, s)
                                      : split_typed<uint8_t, uint16_t>(A, s);
  } else if (mb == 2) {
    st = A->value_dtype == SPC5_F64   ? split_typed<uint16_t, double>(A, s)
         : A->value_dtype == SPC5_F32 ? split_typed<uint16_t, float>(A, s)
                                      : split_typed<uint16_t, uint16_t>(A, s);
  } else {
    st = A->value_dtype == SPC5_F64   ? split_typed<uint32_t, double>(A, s)
         : A->value_dtype == SPC5_F32 ? split_typed<uint32_t, float>(A, s)
                                      : split_typed<uint32_t, uint16_t>(A, s);
  }
  if (st != SPC5_OK) return st;
  st = replan(A, s, PlanOptions());  // the block part's plans
  if (st != SPC5_OK) return st;
  return plan_scalars(A, s);
}

}  // namespace spc5
