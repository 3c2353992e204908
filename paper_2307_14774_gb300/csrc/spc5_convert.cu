// CSR -> beta(r,c) conversion on the GPU (Section 2.4).
//
// Block rule (for r > 1 the paper only says that a block "is mapped to
// several rows"): inside a panel of r rows, take the sorted union U of the
// rows' columns; the smallest column of U not covered yet opens a block that
// covers [start, start + c) in all r rows.  Blocks are ordered by start and
// values by (block, row, column), Algorithm 1's idxVal order.
//
// The greedy choice of block starts is a chain over U (each start is the
// first union column >= previous start + c), so a long panel looks
// sequential.  Here every step is a flat pass over all entries, whatever the
// row lengths:
//   1. row id of every entry (mark row starts, prefix sum),
//   2. merged rank of every entry inside its panel (binary searches in the
//      panel's other rows) -> union U of each panel, deduplicated,
//   3. U is cut into chunks of 32; each warp builds the map "first block
//      start in my chunk -> first block start in the next chunk" (at most c
//      possible entries, since starts are >= c apart), a prefix scan of these
//      maps under composition fixes every chunk's entry, then each warp
//      marks its chunk's block starts,
//   4. prefix sums turn marks into block indices; masks are built with
//      atomicOr, value offsets with a prefix sum of popcounts, and every
//      value is scattered to its packed position.
// All integer work, so the result is identical to any other implementation
// of the same rule (the CPU oracle checks it byte for byte).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "spc5_internal.h"
#include "spc5_scan.cuh"

namespace spc5 {
namespace {

constexpr int kThreads = 256;

enum : uint32_t {
  kErrRowptr = 1u,
  kErrRange = 2u,
  kErrUnsorted = 4u,
  kErrInternal = 8u,
};

inline unsigned grid_for(int64_t n, int per_thread = 1) {
  int64_t blocks = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  if (blocks < 1) blocks = 1;
  if (blocks > 1048576) blocks = 1048576;
  return (unsigned)blocks;
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- checks --

__global__ void k_check_rowptr(int64_t nrows, int64_t nnz, const int32_t *rowptr,
                               uint32_t *err) {
  GRID_STRIDE(i, nrows) {
    if (rowptr[i + 1] < rowptr[i]) atomicOr(err, kErrRowptr);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (rowptr[0] != 0 || (int64_t)rowptr[nrows] != nnz) atomicOr(err, kErrRowptr);
  }
}

// mark[e] = number of rows i in [1, nrows) with rowptr[i] == e; an inclusive
// prefix sum of mark is then the row of entry e.  Out-of-range pointers are
// skipped here and reported by k_check_rowptr.
__global__ void k_mark_rows(int64_t nrows, int64_t nnz, const int32_t *rowptr, int32_t *mark) {
  GRID_STRIDE(i, nrows - 1) {
    int32_t s = rowptr[i + 1];
    if (s >= 0 && s < nnz) atomicAdd(&mark[s], 1);
  }
}

__global__ void k_check_cols(int64_t nnz, int64_t ncols, int64_t nrows, const int32_t *rowptr,
                             const int32_t *colidx, const int32_t *rowid, uint32_t *err) {
  GRID_STRIDE(e, nnz) {
    int32_t row = rowid[e];
    int32_t col = colidx[e];
    if (row < 0 || row >= nrows) {
      atomicOr(err, kErrRowptr);
      continue;
    }
    if (col < 0 || col >= ncols) atomicOr(err, kErrRange);
    int32_t start = rowptr[row];
    if (e > start && e > 0 && colidx[e - 1] >= col) atomicOr(err, kErrUnsorted);
  }
}

// ---------------------------------------------------------- merged ranks --

__device__ __forceinline__ int32_t lower_bound_i32(const int32_t *a, int32_t lo, int32_t hi,
                                                   int32_t v) {
  while (lo < hi) {
    int32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// For entry e of row i = p*r + q: its rank in the panel's merged sequence
// ordered by (column, row) is its index inside its own row plus, for every
// other row q' of the panel, the number of entries with a smaller column
// (q' > q) or a column not larger (q' < q).  It is a duplicate of the union
// when an earlier row holds the same column.
// flags[pos]: bit 0 = first occurrence of the column in the panel,
//             bit 1 = first element of the panel.
__global__ void k_merge_rank(int64_t nnz, int64_t nrows, int r, const int32_t *rowptr,
                             const int32_t *colidx, const int32_t *rowid, int32_t *merged_col,
                             uint8_t *flags, int32_t *elem_pos) {
  GRID_STRIDE(e, nnz) {
    int32_t i = rowid[e];
    int32_t p = i / r, q = i - p * r;
    int32_t x = colidx[e];
    int32_t rank = (int32_t)e - rowptr[i];
    bool dup = false;
    for (int qq = 0; qq < r; ++qq) {
      int64_t row = (int64_t)p * r + qq;
      if (qq == q || row >= nrows) continue;
      int32_t lo = rowptr[row], hi = rowptr[row + 1];
      int32_t lb = lower_bound_i32(colidx, lo, hi, x);
      int32_t cnt = lb - lo;
      if (qq < q) {
        bool has = (lb < hi) && colidx[lb] == x;
        cnt += has ? 1 : 0;
        dup |= has;
      }
      rank += cnt;
    }
    int32_t pos = rowptr[(int64_t)p * r] + rank;
    merged_col[pos] = x;
    flags[pos] = (uint8_t)((dup ? 0 : 1) | (rank == 0 ? 2 : 0));
    elem_pos[e] = pos;
  }
}

struct FlagFirst {
  const uint8_t *f;
  __device__ int32_t operator()(int64_t i) const { return f[i] & 1; }
};
struct ReadI32 {
  const int32_t *m;
  __device__ int32_t operator()(int64_t i) const { return m[i]; }
};
struct WriteI32 {
  int32_t *o;
  __device__ void operator()(int64_t i, int32_t v) const { o[i] = v; }
};

// U[k] = column of the k-th first occurrence; ustart[k] = panel start flag.
__global__ void k_compact_union(int64_t nnz, const int32_t *merged_col, const uint8_t *flags,
                                const int32_t *uidx_incl, int32_t *U, uint8_t *ustart) {
  GRID_STRIDE(pos, nnz) {
    uint8_t f = flags[pos];
    if (f & 1) {
      int32_t k = uidx_incl[pos] - 1;
      U[k] = merged_col[pos];
      ustart[k] = (f >> 1) & 1;
    }
  }
}

// ------------------------------------------------------------ chain maps --

// A chunk map sends the entry state of a chunk (the lane, 0..c-1, of the
// first block start of the panel that continues from the previous chunk;
// kNone if there is none) to the entry state of the next chunk.
constexpr int kNone = 8;
struct ChainMap {
  uint8_t m[16];
};
struct ComposeMap {  // apply a, then b
  __device__ ChainMap operator()(const ChainMap &a, const ChainMap &b) const {
    ChainMap h;
#pragma unroll
    for (int e = 0; e < 16; ++e) h.m[e] = (e <= kNone) ? b.m[a.m[e]] : (uint8_t)kNone;
    return h;
  }
};
__host__ __device__ inline ChainMap identity_map() {
  ChainMap h;
  for (int e = 0; e < 16; ++e) h.m[e] = (uint8_t)(e <= kNone ? e : kNone);
  return h;
}

// Jump codes inside a chunk: 0..31 = a lane of this chunk; 32 + e = lane e of
// the next chunk (e < c); kEnd = the panel ends without another start.
constexpr int kEnd = 255;

// Per-lane "next block start if I start a block": the first later element
// of the same panel whose column is >= mine + c.  Needs the chunk's 32
// elements and the first c of the next chunk (staged in shared memory).
__device__ __forceinline__ int next_start(int lane, int c, const int32_t *su, const uint8_t *sst,
                                          int navail) {
  int32_t lim = su[lane] + c;
  for (int j = 1; j <= c; ++j) {
    int idx = lane + j;
    if (idx >= navail || sst[idx]) return kEnd;  // panel ends before a start qualifies
    if (su[idx] >= lim) return idx;              // idx < 32 + c
  }
  return kEnd;  // unreachable for strictly ascending U: U[lane + c] >= U[lane] + c
}

constexpr int kChunkWarps = 8;

// Builds one chunk's map.  One warp per chunk of 32 union elements.
__global__ void __launch_bounds__(32 * kChunkWarps)
    k_chain_maps(int64_t nu, int c, const int32_t *U, const uint8_t *ustart, ChainMap *maps) {
  __shared__ int32_t su_all[kChunkWarps][40];
  __shared__ uint8_t sst_all[kChunkWarps][40];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t chunk = (int64_t)blockIdx.x * kChunkWarps + warp;
  const int64_t nchunks = (nu + 31) / 32;
  if (chunk >= nchunks) return;
  int32_t *su = su_all[warp];
  uint8_t *sst = sst_all[warp];
  const int64_t base = chunk * 32;
  int navail = (int)((nu - base) < (int64_t)(32 + c) ? (nu - base) : (int64_t)(32 + c));
  for (int t = lane; t < 40; t += 32) {
    if (t < navail) {
      su[t] = U[base + t];
      sst[t] = ustart[base + t];
    } else {
      su[t] = 0;
      sst[t] = 1;
    }
  }
  __syncwarp();
  const bool valid = lane < navail;
  int jump = valid ? next_start(lane, c, su, sst, navail) : kEnd;
  // pointer doubling until every jump leaves the chunk
#pragma unroll
  for (int it = 0; it < 5; ++it) {
    int tgt = (jump < 32) ? jump : 0;
    int j2 = __shfl_sync(0xffffffffu, jump, tgt);
    if (jump < 32) jump = j2;
  }
  // last panel start inside the chunk (if any) decides a constant map
  unsigned starts = __ballot_sync(0xffffffffu, valid && sst[lane]);
  ChainMap mp;
  auto code_to_state = [&](int code) -> uint8_t {
    return (code >= 32 && code < 32 + 8) ? (uint8_t)(code - 32) : (uint8_t)kNone;
  };
  if (starts) {
    int s_last = 31 - __clz(starts);
    int code = __shfl_sync(0xffffffffu, jump, s_last);
    uint8_t st = code_to_state(code);
    for (int e = 0; e < 16; ++e) mp.m[e] = st;
  } else {
    for (int e = 0; e < 16; ++e) {
      int code = __shfl_sync(0xffffffffu, jump, e < 8 ? e : 0);
      mp.m[e] = (e < c) ? code_to_state(code) : (uint8_t)kNone;
    }
  }
  if (lane == 0) maps[chunk] = mp;
}

struct MapIn {
  const ChainMap *maps;
  __device__ ChainMap operator()(int64_t i) const { return maps[i]; }
};
struct MapOutEntry {  // exclusive prefix applied to the start state kNone
  uint8_t *entry;
  __device__ void operator()(int64_t i, const ChainMap &m) const { entry[i] = m.m[kNone]; }
};

// Marks the block starts of every chunk, given its entry state.
__global__ void __launch_bounds__(32 * kChunkWarps)
    k_chain_marks(int64_t nu, int c, const int32_t *U, const uint8_t *ustart,
                  const uint8_t *entry, int32_t *is_start) {
  __shared__ int32_t su_all[kChunkWarps][40];
  __shared__ uint8_t sst_all[kChunkWarps][40];
  __shared__ uint8_t hit_all[kChunkWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t chunk = (int64_t)blockIdx.x * kChunkWarps + warp;
  const int64_t nchunks = (nu + 31) / 32;
  if (chunk >= nchunks) return;
  int32_t *su = su_all[warp];
  uint8_t *sst = sst_all[warp];
  uint8_t *hit = hit_all[warp];
  const int64_t base = chunk * 32;
  int navail = (int)((nu - base) < (int64_t)(32 + c) ? (nu - base) : (int64_t)(32 + c));
  for (int t = lane; t < 40; t += 32) {
    if (t < navail) {
      su[t] = U[base + t];
      sst[t] = ustart[base + t];
    } else {
      su[t] = 0;
      sst[t] = 1;
    }
  }
  hit[lane] = 0;
  __syncwarp();
  const bool valid = lane < navail && lane < 32;
  int jump = valid ? next_start(lane, c, su, sst, navail) : kEnd;
  const int e = entry[chunk];
  bool marked = valid && (sst[lane] || (e != kNone && lane == e));
  // propagate marks along jumps: after round t, everything reachable in
  // fewer than 2^(t+1) jumps is marked
#pragma unroll
  for (int it = 0; it < 5; ++it) {
    if (marked && jump < 32) hit[jump] = 1;
    __syncwarp();
    marked = marked || (hit[lane] != 0);
    __syncwarp();
    int tgt = (jump < 32) ? jump : 0;
    int j2 = __shfl_sync(0xffffffffu, jump, tgt);
    if (jump < 32) jump = j2;
  }
  if (lane < navail && lane < 32 && base + lane < nu) is_start[base + lane] = marked ? 1 : 0;
}

// --------------------------------------------------------- block arrays --

__global__ void k_block_colidx(int64_t nu, const int32_t *U, const int32_t *is_start,
                               const int32_t *bidx_incl, int32_t *block_colidx) {
  GRID_STRIDE(k, nu) {
    if (is_start[k]) block_colidx[bidx_incl[k] - 1] = U[k];
  }
}

__global__ void k_panel_ptrs(int64_t npanels, int64_t nrows, int r, const int32_t *rowptr,
                             const int32_t *uidx_incl, const int32_t *bidx_incl,
                             int32_t *panel_vptr, int32_t *block_rowptr) {
  GRID_STRIDE(p, npanels + 1) {
    int64_t row = (p * r < nrows) ? p * r : nrows;
    int32_t v = rowptr[row];
    panel_vptr[p] = v;
    int32_t ustart = (v == 0) ? 0 : uidx_incl[v - 1];
    block_rowptr[p] = (ustart == 0) ? 0 : bidx_incl[ustart - 1];
  }
}

// Block of entry e and its bit inside the block's packed mask word.
__device__ __forceinline__ void entry_block(int64_t e, int r, int c, const int32_t *colidx,
                                            const int32_t *rowid, const int32_t *elem_pos,
                                            const int32_t *uidx_incl, const int32_t *bidx_incl,
                                            const int32_t *block_colidx, int32_t *blk,
                                            int *bit) {
  int32_t pos = elem_pos[e];
  int32_t k = uidx_incl[pos] - 1;
  int32_t b = bidx_incl[k] - 1;
  int32_t q = rowid[e] % r;
  *blk = b;
  *bit = q * c + (colidx[e] - block_colidx[b]);
}

__global__ void k_masks(int64_t nnz, int r, int c, const int32_t *colidx, const int32_t *rowid,
                        const int32_t *elem_pos, const int32_t *uidx_incl,
                        const int32_t *bidx_incl, const int32_t *block_colidx, uint32_t *mask32,
                        uint32_t *err) {
  GRID_STRIDE(e, nnz) {
    int32_t b;
    int bit;
    entry_block(e, r, c, colidx, rowid, elem_pos, uidx_incl, bidx_incl, block_colidx, &b, &bit);
    int k = bit - (rowid[e] % r) * c;
    if (k < 0 || k >= c) {
      atomicOr(err, kErrInternal);
      continue;
    }
    atomicOr(&mask32[b], 1u << bit);
  }
}

struct PopcIn {
  const uint32_t *m;
  __device__ int32_t operator()(int64_t i) const { return __popc(m[i]); }
};

// Storage conversions of the values (round to nearest, ties to even).
struct StoreF64 {
  using T = double;
  __device__ static double cvt(double d) { return d; }
};
struct StoreF32 {
  using T = float;
  __device__ static float cvt(double d) { return __double2float_rn(d); }
};
// FP64 -> BF16 with a single correct rounding: first round toward zero to
// FP32 and, if inexact, force the last FP32 bit to 1 (round to odd; Boldo
// and Melquiond, IEEE TC 2008), then round the FP32 bit pattern to the
// nearest BF16, ties to even.  FP32 carries 16 more significand bits than
// BF16, so the odd intermediate never creates a false tie.  Finite inputs
// inside the FP32 normal range.
struct StoreBF16 {
  using T = uint16_t;
  __device__ static uint16_t cvt(double d) {
    float f = __double2float_rz(d);
    uint32_t b = __float_as_uint(f);
    if ((double)f != d) b |= 1u;
    b += 0x7FFFu + ((b >> 16) & 1u);
    return (uint16_t)(b >> 16);
  }
};

template <typename Store>
__global__ void k_values(int64_t nnz, int r, int c, const int32_t *colidx, const int32_t *rowid,
                         const int32_t *elem_pos, const int32_t *uidx_incl,
                         const int32_t *bidx_incl, const int32_t *block_colidx,
                         const uint32_t *mask32, const int32_t *boff, const double *vals,
                         typename Store::T *values, int32_t *value_src) {
  GRID_STRIDE(e, nnz) {
    int32_t b;
    int bit;
    entry_block(e, r, c, colidx, rowid, elem_pos, uidx_incl, bidx_incl, block_colidx, &b, &bit);
    int k = bit - (rowid[e] % r) * c;
    if (k < 0 || k >= c) continue;  // reported by k_masks
    int32_t dst = boff[b] + __popc(mask32[b] & ((1u << bit) - 1u));
    if (dst < 0 || dst >= nnz) continue;
    values[dst] = Store::cvt(vals[e]);
    value_src[dst] = (int32_t)e;
  }
}

template <typename MaskT>
__global__ void k_pack_masks(int64_t nb, const uint32_t *mask32, MaskT *out) {
  GRID_STRIDE(b, nb) { out[b] = (MaskT)mask32[b]; }
}

// Consistency: the value offset of every panel's first block must be the
// panel's CSR offset.
__global__ void k_check_offsets(int64_t npanels, const int32_t *block_rowptr,
                                const int32_t *panel_vptr, const int32_t *boff, int64_t nb,
                                uint32_t *err) {
  GRID_STRIDE(p, npanels) {
    int32_t b = block_rowptr[p];
    if (b < block_rowptr[p + 1] && b < nb && boff[b] != panel_vptr[p]) atomicOr(err, kErrInternal);
  }
}

template <typename T>
struct DevBuf {
  T *p = nullptr;
  cudaStream_t s;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  cudaError_t alloc(int64_t n) { return cudaMallocAsync((void **)&p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), s); }
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
};

spc5_status err_to_status(uint32_t err) {
  if (err & kErrRowptr) {
    set_error("invalid row pointers (rowptr[0] != 0, decreasing, or rowptr[nrows] != nnz)");
    return SPC5_EROWPTR;
  }
  if (err & kErrRange) {
    set_error("a column index lies outside [0, ncols)");
    return SPC5_ERANGE;
  }
  if (err & kErrUnsorted) {
    set_error("column indices of a row are not strictly ascending");
    return SPC5_EUNSORTED;
  }
  if (err & kErrInternal) {
    set_error("internal inconsistency detected by a conversion kernel");
    return SPC5_EDEVICE;
  }
  return SPC5_OK;
}

}  // namespace

#define CK(call, what)                              \
  do {                                              \
    spc5_status _st = cuda_check((call), (what));   \
    if (_st != SPC5_OK) return _st;                 \
  } while (0)

spc5_status convert_device(spc5_matrix *A, const int32_t *rowptr, const int32_t *colidx,
                           const double *vals, cudaStream_t s) {
  const int64_t n = A->nrows, nnz = A->nnz, np = A->npanels;
  const int r = A->r, c = A->c;
  const int mask_bytes = r * c / 8;

  DevBuf<uint32_t> err(s);
  CK(err.alloc(1), "alloc err");
  CK(cudaMemsetAsync(err.p, 0, sizeof(uint32_t), s), "memset err");

  // 1. row ids and validation
  DevBuf<int32_t> rowid(s), scan_tmp(s);
  CK(rowid.alloc(nnz), "alloc rowid");
  CK(scan_tmp.alloc(scan_tmp_elems(std::max<int64_t>(nnz, 1))), "alloc scan tmp");
  k_check_rowptr<<<grid_for(std::max<int64_t>(n, 1)), kThreads, 0, s>>>(n, nnz, rowptr, err.p);
  if (nnz > 0) {
    CK(cudaMemsetAsync(rowid.p, 0, (size_t)nnz * sizeof(int32_t), s), "memset rowid");
    if (n > 1) k_mark_rows<<<grid_for(n), kThreads, 0, s>>>(n, nnz, rowptr, rowid.p);
    CK(device_scan<int32_t>(nnz, ReadI32{rowid.p}, WriteI32{rowid.p}, AddI32{}, 0, true, scan_tmp.p, s),
       "scan rows");
    k_check_cols<<<grid_for(nnz), kThreads, 0, s>>>(nnz, A->ncols, n, rowptr, colidx, rowid.p,
                                                   err.p);
  }
  uint32_t herr = 0;
  CK(cudaMemcpyAsync(&herr, err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read err");
  CK(cudaStreamSynchronize(s), "sync validation");
  if (herr) return err_to_status(herr);

  // outputs
  int64_t nb = 0;
  const size_t vsize = A->value_dtype == SPC5_F64 ? 8 : A->value_dtype == SPC5_F32 ? 4 : 2;
  // every array is padded by 16 bytes: the staged SpMV copies 16-byte
  // aligned windows that may end up to 15 bytes past the last element
  CK(cudaMalloc((void **)&A->block_rowptr, (size_t)(np + 1) * sizeof(int32_t) + 16),
     "alloc block_rowptr");
  CK(cudaMalloc((void **)&A->panel_vptr, (size_t)(np + 1) * sizeof(int32_t) + 16),
     "alloc panel_vptr");
  CK(cudaMalloc(&A->values, (size_t)nnz * vsize + 16), "alloc values");
  CK(cudaMalloc((void **)&A->value_src, (size_t)nnz * sizeof(int32_t) + 16), "alloc value_src");
  CK(cudaMalloc((void **)&A->dev_error, sizeof(uint32_t)), "alloc error word");
  CK(cudaMemsetAsync(A->dev_error, 0, sizeof(uint32_t), s), "zero error word");
  A->device_bytes = (int64_t)(2 * (np + 1) * sizeof(int32_t) + 32 + nnz * vsize + 16 +
                             nnz * sizeof(int32_t) + 16);

  if (nnz == 0) {
    CK(cudaMemsetAsync(A->block_rowptr, 0, (size_t)(np + 1) * sizeof(int32_t), s), "zero brp");
    CK(cudaMemsetAsync(A->panel_vptr, 0, (size_t)(np + 1) * sizeof(int32_t), s), "zero vptr");
    CK(cudaMalloc((void **)&A->block_colidx, 16), "alloc colidx");
    CK(cudaMalloc(&A->masks, 16), "alloc masks");
    A->nblocks = 0;
    A->device_bytes += 32;
    spc5_status pst = plan_tiles(A, nullptr, nullptr, s);
    if (pst != SPC5_OK) return pst;
    CK(cudaStreamSynchronize(s), "sync");
    return SPC5_OK;
  }

  // 2. merged ranks and the panel unions
  DevBuf<int32_t> merged(s), elem_pos(s), uidx(s), U(s);
  DevBuf<uint8_t> flags(s), ustart(s);
  CK(merged.alloc(nnz), "alloc merged");
  CK(elem_pos.alloc(nnz), "alloc elem_pos");
  CK(uidx.alloc(nnz), "alloc uidx");
  CK(flags.alloc(nnz), "alloc flags");
  k_merge_rank<<<grid_for(nnz), kThreads, 0, s>>>(nnz, n, r, rowptr, colidx, rowid.p, merged.p,
                                                 flags.p, elem_pos.p);
  CK(device_scan<int32_t>(nnz, FlagFirst{flags.p}, WriteI32{uidx.p}, AddI32{}, 0, true,
                          scan_tmp.p, s),
     "scan union");
  int32_t nu32 = 0;
  CK(cudaMemcpyAsync(&nu32, uidx.p + nnz - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
     "read nu");
  CK(cudaStreamSynchronize(s), "sync nu");
  const int64_t nu = nu32;
  CK(U.alloc(nu), "alloc U");
  CK(ustart.alloc(nu), "alloc ustart");
  k_compact_union<<<grid_for(nnz), kThreads, 0, s>>>(nnz, merged.p, flags.p, uidx.p, U.p,
                                                    ustart.p);

  // 3. chains of block starts
  const int64_t nchunks = (nu + 31) / 32;
  DevBuf<ChainMap> maps(s), map_tmp(s);
  DevBuf<uint8_t> entry(s);
  DevBuf<int32_t> is_start(s), bidx(s);
  CK(maps.alloc(nchunks), "alloc maps");
  CK(map_tmp.alloc(scan_tmp_elems(nchunks)), "alloc map tmp");
  CK(entry.alloc(nchunks), "alloc entry");
  CK(is_start.alloc(nu), "alloc is_start");
  CK(bidx.alloc(nu), "alloc bidx");
  unsigned chunk_blocks = (unsigned)((nchunks + kChunkWarps - 1) / kChunkWarps);
  k_chain_maps<<<chunk_blocks, 32 * kChunkWarps, 0, s>>>(nu, c, U.p, ustart.p, maps.p);
  CK(device_scan<ChainMap>(nchunks, MapIn{maps.p}, MapOutEntry{entry.p}, ComposeMap{},
                           identity_map(), false, map_tmp.p, s),
     "scan chain maps");
  k_chain_marks<<<chunk_blocks, 32 * kChunkWarps, 0, s>>>(nu, c, U.p, ustart.p, entry.p,
                                                          is_start.p);
  CK(device_scan<int32_t>(nu, ReadI32{is_start.p}, WriteI32{bidx.p}, AddI32{}, 0, true,
                          scan_tmp.p, s),
     "scan starts");
  int32_t nb32 = 0;
  CK(cudaMemcpyAsync(&nb32, bidx.p + nu - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
     "read nb");
  CK(cudaStreamSynchronize(s), "sync nb");
  nb = nb32;
  A->nblocks = nb;

  // 4. block arrays, masks, values
  CK(cudaMalloc((void **)&A->block_colidx, (size_t)nb * sizeof(int32_t) + 16), "alloc colidx");
  CK(cudaMalloc(&A->masks, (size_t)nb * mask_bytes + 16), "alloc masks");
  CK(cudaMemsetAsync(A->block_colidx, 0, (size_t)nb * sizeof(int32_t) + 16, s), "zero colidx");
  CK(cudaMemsetAsync(A->masks, 0, (size_t)nb * mask_bytes + 16, s), "zero masks");
  A->device_bytes += (int64_t)(nb * sizeof(int32_t) + nb * mask_bytes + 32);
  k_block_colidx<<<grid_for(nu), kThreads, 0, s>>>(nu, U.p, is_start.p, bidx.p, A->block_colidx);
  k_panel_ptrs<<<grid_for(np + 1), kThreads, 0, s>>>(np, n, r, rowptr, uidx.p, bidx.p,
                                                    A->panel_vptr, A->block_rowptr);
  DevBuf<uint32_t> mask32(s);
  DevBuf<int32_t> boff(s);
  CK(mask32.alloc(nb), "alloc mask32");
  CK(boff.alloc(nb), "alloc boff");
  CK(cudaMemsetAsync(mask32.p, 0, (size_t)nb * sizeof(uint32_t), s), "zero mask32");
  k_masks<<<grid_for(nnz), kThreads, 0, s>>>(nnz, r, c, colidx, rowid.p, elem_pos.p, uidx.p,
                                            bidx.p, A->block_colidx, mask32.p, err.p);
  CK(device_scan<int32_t>(nb, PopcIn{mask32.p}, WriteI32{boff.p}, AddI32{}, 0, false,
                          scan_tmp.p, s),
     "scan popcounts");
  if (A->value_dtype == SPC5_F64)
    k_values<StoreF64><<<grid_for(nnz), kThreads, 0, s>>>(
        nnz, r, c, colidx, rowid.p, elem_pos.p, uidx.p, bidx.p, A->block_colidx, mask32.p,
        boff.p, vals, (double *)A->values, A->value_src);
  else if (A->value_dtype == SPC5_F32)
    k_values<StoreF32><<<grid_for(nnz), kThreads, 0, s>>>(
        nnz, r, c, colidx, rowid.p, elem_pos.p, uidx.p, bidx.p, A->block_colidx, mask32.p,
        boff.p, vals, (float *)A->values, A->value_src);
  else
    k_values<StoreBF16><<<grid_for(nnz), kThreads, 0, s>>>(
        nnz, r, c, colidx, rowid.p, elem_pos.p, uidx.p, bidx.p, A->block_colidx, mask32.p,
        boff.p, vals, (uint16_t *)A->values, A->value_src);
  if (mask_bytes == 1)
    k_pack_masks<uint8_t><<<grid_for(nb), kThreads, 0, s>>>(nb, mask32.p, (uint8_t *)A->masks);
  else if (mask_bytes == 2)
    k_pack_masks<uint16_t><<<grid_for(nb), kThreads, 0, s>>>(nb, mask32.p, (uint16_t *)A->masks);
  else
    k_pack_masks<uint32_t><<<grid_for(nb), kThreads, 0, s>>>(nb, mask32.p, (uint32_t *)A->masks);
  k_check_offsets<<<grid_for(np), kThreads, 0, s>>>(np, A->block_rowptr, A->panel_vptr, boff.p,
                                                   nb, err.p);
  spc5_status pst = plan_tiles(A, mask32.p, boff.p, s);
  if (pst != SPC5_OK) return pst;
  CK(cudaGetLastError(), "conversion kernels");
  CK(cudaMemcpyAsync(&herr, err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read err");
  CK(cudaStreamSynchronize(s), "sync conversion");
  if (herr) return err_to_status(herr);
  return SPC5_OK;
}

}  // namespace spc5
