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
#include <stdlib.h>

#include <algorithm>
#include <climits>
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
struct ReadI32Pad {  // m[i] for i < n, 0 at i == n (an exclusive scan of n + 1 gives the total)
  const int32_t *m;
  int64_t n;
  __device__ int32_t operator()(int64_t i) const { return i < n ? m[i] : 0; }
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

// ------------------------------------------------ panel-local conversion --
//
// When no panel holds more than kPanelCap entries (stencils, FEM meshes,
// uniform rows: every matrix whose rows are not very long; the kernel comes
// sized for panels of 256, 1024 and 2048 entries), one warp converts a whole
// panel in shared memory, with the rule of the flat passes above: the
// panel's columns merged in column order (a tree of pairwise merges of the
// sorted rows, each split among the lanes by merge path), the union U
// without repeats, the greedy block starts
// over U (a ballot finds the first union column not covered by the previous
// block, one step per block), then masks, the blocks' value offsets (prefix
// sum of popcounts) and the value scatter.  One pass over the panels: a
// panel's values start at its CSR offset e0 (it holds exactly its rows'
// entries), so values and value sources go to their final places at once;
// a panel has no more blocks than entries, so its blocks go to scratch
// arrays at e0, with the panel's block count.  A prefix sum of the counts
// then places every panel's blocks, and a compaction copies them there.
// The values are read once, the columns once (twice for r >= 4).
constexpr int kPanelCap = 2048;      // entries of a panel (capacities 256, 1024, 2048)
constexpr int kPanelBlockCap = 256;  // blocks of a panel

// Shared memory of one warp for panels of at most CAP entries.
template <int CAP>
struct PanelSmem {
  int32_t col[CAP];                  // the panel's columns, row after row (CSR order)
  int32_t uni[CAP];                  // merged columns (-1: not the first occurrence),
                                     // then the union U, then every entry's block
  int32_t bst[kPanelBlockCap];       // block starts
  uint32_t bmask[kPanelBlockCap];    // block masks
  int32_t boffs[kPanelBlockCap];     // block value offsets in the panel
};
// Warps per CTA: 40 KB of shared memory per CTA at CAP = 256 (four CTAs of
// eight warps per SM, registers capped for that), 33 KB at CAP = 1024 (six
// CTAs of three), 19 KB at CAP = 2048 (eleven CTAs of one).  Smaller panels
// leave room for more warps, which hide more of the searches' latency.
template <int CAP>
struct PanelWarps {
  static constexpr int v = CAP <= 256 ? 8 : (CAP <= 1024 ? 3 : 1);
  static constexpr int per_sm = CAP <= 256 ? 4 : (CAP <= 1024 ? 6 : 11);
};

// Row q of panel entry t (ro[q] <= t < ro[q + 1]) and ro[q].
template <int R>
__device__ __forceinline__ int panel_row(int32_t t, const int32_t (&ro)[R + 1], int nr,
                                         int32_t *rstart) {
  int q = 0;
  int32_t st = ro[0];
#pragma unroll
  for (int qq = 1; qq < R; ++qq) {
    if (qq < nr && t >= ro[qq]) {
      q = qq;
      st = ro[qq];
    }
  }
  *rstart = st;
  return q;
}

// Largest entry count of a panel.
__global__ void k_panel_max_entries(int64_t np, int64_t nrows, int r, const int32_t *rowptr,
                                    int32_t *out) {
  int32_t mx = 0;
  GRID_STRIDE(p, np) {
    const int64_t a = p * r, b = (a + r < nrows) ? a + r : nrows;
    const int32_t ne = rowptr[b] - rowptr[a];
    mx = ne > mx ? ne : mx;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// Every panel: cnt[p] = its blocks; its block starts, masks (as 32-bit
// words) and value offsets at [e0, e0 + cnt[p]) of tcol, tmask, tboff; its
// values and value sources at their final places.  A panel with a column
// out of range or out of order is reported in err[0] and left out; a panel
// of more than kPanelBlockCap blocks raises err[1] to its count and is left
// out (the host then takes the flat passes).
template <int CAP, int R, typename Store>
__global__ void __launch_bounds__(32 * PanelWarps<CAP>::v, CAP <= 256 ? PanelWarps<CAP>::per_sm : 1)
    k_panel_convert(int64_t np, int64_t nrows, int64_t ncols, int r, int c,
                    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                    const double *__restrict__ vals, int32_t *cnt, int32_t *tcol,
                    uint32_t *tmask, int32_t *tboff, typename Store::T *values,
                    int32_t *value_src, uint32_t *err) {
  constexpr int kW = PanelWarps<CAP>::v;
  __shared__ PanelSmem<CAP> sm_all[kW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  PanelSmem<CAP> &S = sm_all[warp];
  const int64_t nw = (int64_t)gridDim.x * kW;
  for (int64_t p = (int64_t)blockIdx.x * kW + warp; p < np; p += nw) {
    const int64_t r0 = p * r;
    const int nr = (int)((r0 + r <= nrows) ? r : nrows - r0);
    const int32_t rp = (lane <= nr) ? rowptr[r0 + lane] : 0;
    const int32_t e0 = __shfl_sync(0xffffffffu, rp, 0);
    int32_t ro[R + 1];
#pragma unroll
    for (int q = 0; q <= R; ++q) ro[q] = __shfl_sync(0xffffffffu, rp, q < nr ? q : nr) - e0;
    const int32_t ne = ro[R];
    __syncwarp();
    // eight loads in flight per lane (a loop that stores each load before
    // issuing the next waits one memory latency per 32 entries)
    for (int32_t t0 = 0; t0 < ne; t0 += 256) {
      int32_t v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int32_t t = t0 + i * 32 + lane;
        v[i] = t < ne ? colidx[e0 + t] : 0;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int32_t t = t0 + i * 32 + lane;
        if (t < ne) S.col[t] = v[i];
      }
    }
    __syncwarp();
    // the columns: in range and strictly ascending in every row
    uint32_t bad = 0;
    for (int32_t t = lane; t < ne; t += 32) {
      int32_t st;
      panel_row<R>(t, ro, nr, &st);
      const int32_t x = S.col[t];
      if (x < 0 || x >= ncols) bad |= kErrRange;
      if (t > st && S.col[t - 1] >= x) bad |= kErrUnsorted;
    }
    if (__any_sync(0xffffffffu, bad != 0u)) {
      if (bad) atomicOr(err, bad);
      if (lane == 0) cnt[p] = 0;
      __syncwarp();
      continue;
    }
    // the panel's columns in (column, row) order: a tree of pairwise merges
    // of sorted runs (rows, then pairs of rows, ...) between the two column
    // buffers.  Each merge of two runs A and B is split into 32 equal
    // pieces of its output (merge path): a lane finds how many of A's
    // entries precede its piece by one binary search along the piece's
    // diagonal (A's entry first on equal columns), then writes its piece
    // by a sequential merge, one comparison per entry.
    int32_t *src = S.col, *dst = S.uni;
#pragma unroll
    for (int h = 1; h < R; h <<= 1) {
      __syncwarp();
#pragma unroll
      for (int g = 0; g < R / (2 * h); ++g) {
        const int32_t a0 = ro[2 * g * h], b0 = ro[(2 * g + 1) * h], b1 = ro[(2 * g + 2) * h];
        const int32_t na = b0 - a0, nb = b1 - b0, n = na + nb;
        const int32_t K = (n + 31) >> 5;
        const int32_t d = min(lane * K, n), dend = min(d + K, n);
        int32_t lo = max(0, d - nb), hi = min(d, na);
        while (lo < hi) {
          const int32_t mid = (lo + hi) >> 1;
          if (src[a0 + mid] <= src[b0 + d - mid - 1])
            lo = mid + 1;
          else
            hi = mid;
        }
        int32_t i = lo, j = d - lo;
        int32_t va = i < na ? src[a0 + i] : INT_MAX;
        int32_t vb = j < nb ? src[b0 + j] : INT_MAX;
        for (int32_t o = d; o < dend; ++o) {
          const bool ta = va <= vb;
          dst[a0 + o] = ta ? va : vb;
          if (ta) {
            ++i;
            va = i < na ? src[a0 + i] : INT_MAX;
          } else {
            ++j;
            vb = j < nb ? src[b0 + j] : INT_MAX;
          }
        }
      }
      int32_t *tmp = src;
      src = dst;
      dst = tmp;
    }
    __syncwarp();
    // the union U: the merged columns without repeats, into uni (in place
    // when the merge ended there: the previous chunk's last column is kept
    // in a register, so no lane reads a slot already rewritten).  One row
    // (r = 1) is its own union: U is the row's columns, left in col.
    const int32_t *U = R == 1 ? S.col : S.uni;
    int32_t nu = R == 1 ? ne : 0, last = -1;
    for (int32_t base = 0; base < (R == 1 ? 0 : ne); base += 32) {
      const bool in = base + lane < ne;
      const int32_t v = in ? src[base + lane] : -1;
      int32_t prev = __shfl_up_sync(0xffffffffu, v, 1);
      if (lane == 0) prev = last;
      last = __shfl_sync(0xffffffffu, v, 31);
      const bool keep = in && v != prev;
      const uint32_t ball = __ballot_sync(0xffffffffu, keep);
      __syncwarp();
      if (keep) S.uni[nu + __popc(ball & lt)] = v;
      nu += __popc(ball);
      __syncwarp();
    }
    // greedy block starts: the first union column not covered opens a block.
    // For r = 1 every union column is an entry, and its block (the last
    // start opened at or before it) goes to uni for the masks and the scatter
    int32_t nbk = 0;
    long long thr = LLONG_MIN;
    for (int32_t base = 0; base < nu; base += 32) {
      const bool in = base + lane < nu;
      const int32_t u = in ? U[base + lane] : 0;
      int32_t mine = nbk - 1;
      while (true) {
        const uint32_t ball = __ballot_sync(0xffffffffu, in && (long long)u >= thr);
        if (!ball) break;
        const int32_t sb = __shfl_sync(0xffffffffu, u, __ffs(ball) - 1);
        if (lane == 0 && nbk < kPanelBlockCap) S.bst[nbk] = sb;
        if (u >= sb) mine = nbk;
        ++nbk;
        thr = (long long)sb + c;
      }
      if (R == 1 && in) S.uni[base + lane] = mine;
    }
    if (lane == 0) cnt[p] = nbk;
    if (nbk > kPanelBlockCap) {
      if (lane == 0) atomicMax((int32_t *)err + 1, nbk);
      __syncwarp();
      continue;
    }
    __syncwarp();
    if (R >= 4) {  // merges of two levels and more wrote over the CSR-order columns
      for (int32_t t0 = 0; t0 < ne; t0 += 256) {
        int32_t v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int32_t t = t0 + i * 32 + lane;
          v[i] = t < ne ? colidx[e0 + t] : 0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int32_t t = t0 + i * 32 + lane;
          if (t < ne) S.col[t] = v[i];
        }
      }
      __syncwarp();
    }
    for (int32_t i = lane; i < nbk; i += 32) {
      tcol[e0 + i] = S.bst[i];
      S.bmask[i] = 0u;
    }
    __syncwarp();
    // masks: an entry's block is the last start not after its column (the
    // columns are checked, so every entry lies in [bst[b], bst[b] + c));
    // kept per entry for the value scatter (the union is no longer needed).
    // Each lane takes a contiguous run of entries: within a row the columns
    // and so the blocks ascend, so the lane finds a row's first block by a
    // binary search and then steps forward (for r = 1 the greedy pass has
    // recorded every entry's block)
    {
      const int32_t K = (ne + 31) >> 5;
      const int32_t t0 = min(lane * K, ne), t1 = min(t0 + K, ne);
      int32_t b = 0, rowend = -1;
      int q = 0;
      for (int32_t t = t0; t < t1; ++t) {
        const int32_t x = S.col[t];
        if (R == 1) {
          b = S.uni[t];
        } else if (t >= rowend) {  // first entry of the run, or a new row
          int32_t st;
          q = panel_row<R>(t, ro, nr, &st);
#pragma unroll
          for (int qq = 0; qq < R; ++qq)
            if (qq == q) rowend = ro[qq + 1];
          int32_t lo = 0, hi = nbk;  // first start > x
          while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (S.bst[mid] <= x)
              lo = mid + 1;
            else
              hi = mid;
          }
          b = lo - 1;
          S.uni[t] = b;
        } else {
          while (b + 1 < nbk && S.bst[b + 1] <= x) ++b;
          S.uni[t] = b;
        }
        atomicOr(&S.bmask[b], 1u << (q * c + (x - S.bst[b])));
      }
    }
    __syncwarp();
    // the blocks' value offsets: exclusive prefix of the popcounts
    int32_t run = 0;
    for (int32_t base = 0; base < nbk; base += 32) {
      const bool in = base + lane < nbk;
      const uint32_t m = in ? S.bmask[base + lane] : 0u;
      const int pc = __popc(m);
      int incl = pc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t2 = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t2;
      }
      if (in) {
        S.boffs[base + lane] = run + incl - pc;
        tmask[e0 + base + lane] = m;
        tboff[e0 + base + lane] = e0 + run + incl - pc;
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    // values in (block, row, column) order, eight loads in flight per lane
    for (int32_t t0 = 0; t0 < ne; t0 += 256) {
      double v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int32_t t = t0 + i * 32 + lane;
        v[i] = t < ne ? vals[e0 + t] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int32_t t = t0 + i * 32 + lane;
        if (t < ne) {
          int32_t st;
          const int q = panel_row<R>(t, ro, nr, &st);
          const int32_t x = S.col[t];
          const int32_t b = S.uni[t];
          const int bit = q * c + (x - S.bst[b]);
          const int32_t dst = e0 + S.boffs[b] + __popc(S.bmask[b] & ((1u << bit) - 1u));
          values[dst] = Store::cvt(v[i]);
          value_src[dst] = e0 + t;
        }
      }
    }
    __syncwarp();
  }
}

// Moves every panel's blocks from its CSR offset to its place (brp =
// block_rowptr): block columns, masks (32-bit and packed), value offsets.
// Eight lanes per panel.
template <typename MaskT>
__global__ void k_panel_compact(int64_t np, int r, const int32_t *rowptr,
                                const int32_t *brp, const int32_t *tcol, const uint32_t *tmask,
                                const int32_t *tboff, int32_t *block_colidx, MaskT *masks,
                                uint32_t *mask32, int32_t *boff) {
  const int64_t gl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const int sl = threadIdx.x & 7;
  const int64_t ng = ((int64_t)gridDim.x * blockDim.x) >> 3;
  for (int64_t p = gl; p < np; p += ng) {
    const int32_t e0 = rowptr[p * r];
    const int32_t g0 = brp[p], n = brp[p + 1] - g0;
    for (int32_t i = sl; i < n; i += 8) {
      const uint32_t m = tmask[e0 + i];
      block_colidx[g0 + i] = tcol[e0 + i];
      masks[g0 + i] = (MaskT)m;
      mask32[g0 + i] = m;
      boff[g0 + i] = tboff[e0 + i];
    }
  }
}

__global__ void k_panel_vptr(int64_t np, int64_t nrows, int r, const int32_t *rowptr,
                             int32_t *panel_vptr) {
  GRID_STRIDE(p, np + 1) { panel_vptr[p] = rowptr[(p * r < nrows) ? p * r : nrows]; }
}

template <typename T>
struct DevBuf {
  T *p = nullptr;
  cudaStream_t s;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  cudaError_t alloc(int64_t n) { return scratch_alloc((void **)&p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), s); }
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

namespace {

// Output arrays of a conversion (every array padded by 16 bytes: the staged
// SpMV copies 16-byte aligned windows that may end up to 15 bytes past the
// last element): those sized by the entries, then those sized by the nb
// blocks.
spc5_status alloc_values(spc5_matrix *A, cudaStream_t s) {
  const int64_t nnz = A->nnz;
  const size_t vsize = A->value_dtype == SPC5_F64 ? 8 : A->value_dtype == SPC5_F32 ? 4 : 2;
  CK(cudaMalloc(&A->values, (size_t)nnz * vsize + 16), "alloc values");
  CK(cudaMalloc((void **)&A->value_src, (size_t)nnz * sizeof(int32_t) + 16), "alloc value_src");
  CK(cudaMalloc((void **)&A->dev_error, sizeof(uint32_t)), "alloc error word");
  CK(cudaMemsetAsync(A->dev_error, 0, sizeof(uint32_t), s), "zero error word");
  return SPC5_OK;
}

spc5_status alloc_blocks(spc5_matrix *A, int64_t nb, cudaStream_t s) {
  const int64_t nnz = A->nnz, np = A->npanels;
  const int mask_bytes = A->r * A->c / 8;
  const size_t vsize = A->value_dtype == SPC5_F64 ? 8 : A->value_dtype == SPC5_F32 ? 4 : 2;
  CK(cudaMalloc((void **)&A->block_colidx, (size_t)nb * sizeof(int32_t) + 16), "alloc colidx");
  CK(cudaMalloc(&A->masks, (size_t)nb * mask_bytes + 16), "alloc masks");
  CK(cudaMemsetAsync((char *)A->block_colidx + nb * sizeof(int32_t), 0, 16, s), "zero colidx pad");
  CK(cudaMemsetAsync((char *)A->masks + nb * mask_bytes, 0, 16, s), "zero masks pad");
  A->nblocks = nb;
  A->device_bytes = (int64_t)(2 * (np + 1) * sizeof(int32_t) + 32 + nnz * vsize + 16 +
                             nnz * sizeof(int32_t) + 16) +
                    (int64_t)(nb * sizeof(int32_t) + nb * mask_bytes + 32);
  return SPC5_OK;
}

void release(void **p) {
  cudaFree(*p);
  *p = nullptr;
}

// The panel-local conversion (every panel at most CAP entries; the row
// pointers already checked).  *flat is set, and nothing kept, when some
// panel has more than kPanelBlockCap blocks.
template <int CAP>
spc5_status convert_panels(spc5_matrix *A, const int32_t *rowptr, const int32_t *colidx,
                           const double *vals, uint32_t *err, cudaStream_t s, bool *flat) {
  *flat = false;
  const int64_t n = A->nrows, np = A->npanels, nnz = A->nnz;
  const int r = A->r, c = A->c;
  const int mask_bytes = r * c / 8;
  // the CTAs of 19 to 40 KB that one SM holds
  constexpr int kW = PanelWarps<CAP>::v;
  constexpr int kCtas = PanelWarps<CAP>::per_sm;
  const unsigned grid = (unsigned)std::min<int64_t>(std::max<int64_t>((np + kW - 1) / kW, 1),
                                                    (int64_t)device_sm_count() * kCtas);
  DevBuf<int32_t> cnt(s), scan_tmp(s), tcol(s), tboff(s);
  DevBuf<uint32_t> tmask(s);
  CK(cnt.alloc(np + 1), "alloc block counts");
  CK(scan_tmp.alloc(scan_tmp_elems(np + 1)), "alloc scan tmp");
  CK(tcol.alloc(nnz), "alloc block scratch");
  CK(tmask.alloc(nnz), "alloc block scratch");
  CK(tboff.alloc(nnz), "alloc block scratch");
  spc5_status st = alloc_values(A, s);
  if (st != SPC5_OK) return st;
  CK(cudaMalloc((void **)&A->block_rowptr, (size_t)(np + 1) * sizeof(int32_t) + 16),
     "alloc block_rowptr");
  CK(cudaMalloc((void **)&A->panel_vptr, (size_t)(np + 1) * sizeof(int32_t) + 16),
     "alloc panel_vptr");
#define PANEL_PASS(RR, STORE, T)                                                           \
  k_panel_convert<CAP, RR, STORE><<<grid, 32 * kW, 0, s>>>(                                  \
      np, n, A->ncols, r, c, rowptr, colidx, vals, cnt.p, tcol.p, tmask.p, tboff.p,          \
      (T *)A->values, A->value_src, err)
#define PANEL_PASS_R(RR)                        \
  if (A->value_dtype == SPC5_F64)               \
    PANEL_PASS(RR, StoreF64, double);           \
  else if (A->value_dtype == SPC5_F32)          \
    PANEL_PASS(RR, StoreF32, float);            \
  else                                          \
    PANEL_PASS(RR, StoreBF16, uint16_t)
  if (r == 1) {
    PANEL_PASS_R(1);
  } else if (r == 2) {
    PANEL_PASS_R(2);
  } else if (r == 4) {
    PANEL_PASS_R(4);
  } else {
    PANEL_PASS_R(8);
  }
#undef PANEL_PASS_R
#undef PANEL_PASS
  CK(device_scan<int32_t>(np + 1, ReadI32Pad{cnt.p, np}, WriteI32{A->block_rowptr}, AddI32{}, 0,
                          false, scan_tmp.p, s),
     "scan block counts");
  k_panel_vptr<<<grid_for(np + 1), kThreads, 0, s>>>(np, n, r, rowptr, A->panel_vptr);
  uint32_t h[2] = {0, 0};
  int32_t nb32 = 0;
  CK(cudaMemcpyAsync(h, err, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read err");
  CK(cudaMemcpyAsync(&nb32, A->block_rowptr + np, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
     "read nb");
  CK(cudaStreamSynchronize(s), "sync panel pass");
  if (h[0]) return err_to_status(h[0]);
  if ((int32_t)h[1] > kPanelBlockCap) {  // the flat passes allocate their own outputs
    release(&A->values);
    release((void **)&A->value_src);
    release((void **)&A->dev_error);
    release((void **)&A->block_rowptr);
    release((void **)&A->panel_vptr);
    *flat = true;
    return SPC5_OK;
  }
  const int64_t nb = nb32;
  st = alloc_blocks(A, nb, s);
  if (st != SPC5_OK) return st;
  DevBuf<uint32_t> mask32(s);
  DevBuf<int32_t> boff(s);
  CK(mask32.alloc(nb), "alloc mask32");
  CK(boff.alloc(nb), "alloc boff");
  const unsigned cgrid = (unsigned)std::min<int64_t>(std::max<int64_t>((np + 31) / 32, 1),
                                                     (int64_t)device_sm_count() * 8);
#define PANEL_COMPACT(MT)                                                                  \
  k_panel_compact<MT><<<cgrid, kThreads, 0, s>>>(np, r, rowptr, A->block_rowptr, tcol.p,  \
                                                 tmask.p, tboff.p, A->block_colidx,       \
                                                 (MT *)A->masks, mask32.p, boff.p)
  if (mask_bytes == 1)
    PANEL_COMPACT(uint8_t);
  else if (mask_bytes == 2)
    PANEL_COMPACT(uint16_t);
  else
    PANEL_COMPACT(uint32_t);
#undef PANEL_COMPACT
  spc5_status pst = plan_tiles(A, mask32.p, boff.p, s);
  if (pst != SPC5_OK) return pst;
  CK(cudaGetLastError(), "conversion kernels");
  uint32_t herr = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read err");
  CK(cudaStreamSynchronize(s), "sync conversion");
  if (herr) return err_to_status(herr);
  return SPC5_OK;
}

}  // namespace

spc5_status convert_device(spc5_matrix *A, const int32_t *rowptr, const int32_t *colidx,
                           const double *vals, cudaStream_t s) {
  const int64_t n = A->nrows, nnz = A->nnz, np = A->npanels;
  const int r = A->r, c = A->c;
  const int mask_bytes = r * c / 8;

  DevBuf<uint32_t> err(s);
  CK(err.alloc(2), "alloc err");
  CK(cudaMemsetAsync(err.p, 0, 2 * sizeof(uint32_t), s), "memset err");

  // 0. panel-local conversion when no panel is longer than a warp's share
  //    of shared memory (SPC5_CONVERT=flat forces the flat passes)
  if (nnz > 0 && np > 0) {
    const char *mode = getenv("SPC5_CONVERT");
    if (!(mode && mode[0] == 'f')) {
      k_check_rowptr<<<grid_for(std::max<int64_t>(n, 1)), kThreads, 0, s>>>(n, nnz, rowptr,
                                                                             err.p);
      k_panel_max_entries<<<grid_for(np), kThreads, 0, s>>>(np, n, r, rowptr,
                                                           (int32_t *)err.p + 1);
      uint32_t h[2] = {0, 0};
      CK(cudaMemcpyAsync(h, err.p, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read");
      CK(cudaStreamSynchronize(s), "sync rowptr check");
      if (h[0]) return err_to_status(h[0]);
      if ((int32_t)h[1] <= kPanelCap) {
        CK(cudaMemsetAsync(err.p + 1, 0, sizeof(uint32_t), s), "memset");
        bool flat = false;
        spc5_status st =
            (int32_t)h[1] <= 256
                ? convert_panels<256>(A, rowptr, colidx, vals, err.p, s, &flat)
                : (int32_t)h[1] <= 1024
                      ? convert_panels<1024>(A, rowptr, colidx, vals, err.p, s, &flat)
                      : convert_panels<2048>(A, rowptr, colidx, vals, err.p, s, &flat);
        if (st != SPC5_OK || !flat) return st;
      }
    }
  }

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
