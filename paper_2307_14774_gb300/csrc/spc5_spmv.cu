// y = alpha * A x + beta * y over beta(r,c) (Algorithm 1).
//
// Algorithm 1 walks a panel's blocks with one running value index idxVal,
// so a block's values cannot be located without the popcounts of all earlier
// blocks.  The converter stores every panel's first value offset
// (panel_vptr), which removes the dependency between panels; inside a panel
// the offsets come from popcounts.
//
// Lane mapping (both kernels): a warp works on PPW = 32 / (r * G) panels;
// lane (j, q, g) handles row q of panel j, and the G lanes of a row take the
// panel's blocks G at a time.  A round loads G blocks (start column and
// packed mask word), the G lanes exclusive-scan the blocks' popcounts, and a
// lane finds its row's values at
//     panel offset + scan + popc(mask bits of rows < q).
// The lane then multiplies its row's values by x[start + k] for every set
// bit k (Algorithm 1's scalar path; x is read through L1/L2, where the c
// columns of a block are shared by the r rows), and the G partial sums of a
// row are reduced with shuffles before one lane writes y (Section 3.2: one
// write of the reduced row result instead of r separate updates).
//
// Staged kernel (SPC5_KERNEL=1, FP64): persistent, one CTA per SM.  Warp 0 is a
// producer: for each tile of the work plan it issues bulk asynchronous
// copies (cp.async.bulk, completion counted on an mbarrier) of the tile's
// values, block columns, masks and panel pointers into a ring of shared
// memory stages.  The other warps are consumers: they take the tiles in
// order, wait on the stage's barrier, compute from shared memory, and
// release the stage.  HBM is read in large contiguous transfers, while the
// consumers' irregular accesses hit shared memory.  Panels too long for one
// stage were cut into pieces by the planner; their row sums go to a partial
// buffer that a fixup kernel adds in a fixed order.
//
// Direct kernel (default, SPC5_KERNEL=0): the same tiles and lane mapping
// reading global memory directly with many resident warps.  On GB300 the
// FP64 path is bound by the FP64 pipe (2 FMA per cycle per SM), which needs
// many warps in flight more than it needs shared-memory staging; the staged
// kernel (SPC5_KERNEL=1) stays available for comparison.
//
// For rows of very different lengths (spc5_info.flat) the lanes own work
// instead of rows: blocks dealt four per lane per round (k_spmv_flat, plan
// 1), each round's values split evenly over the lanes (k_spmv_vflat, plan
// 3), or each tile's values laid out row by row in shared memory and split
// evenly (k_spmv_expand, plan 2); row sums cut between lanes are completed
// by segmented warp scans.  Hybrid matrices add their scalar entries with
// k_spmv_scalars.  No kernel waits on another warp or CTA except the staged
// kernel, whose waits are bounded.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>

#include "spc5_flat.cuh"
#include "spc5_internal.h"
#include "spc5_ptx.cuh"
#include "spc5_reduce.cuh"

namespace spc5 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDirectThreads = 256;
constexpr long long kWaitBudget = 4000000000LL;  // SM cycles (about 2 s) before a wait gives up

enum : uint32_t { kErrProducerWait = 1u, kErrConsumerWait = 2u, kErrTileTooLarge = 4u };

// One row's contribution of one block: sum over set bits k of mq of
// vals[running index] * x[col + k], accumulated in AT (FP64 for FP64
// values; FP32 for FP32 and BF16 values).
template <int C, bool UNROLL, typename VT, typename AT>
__device__ __forceinline__ AT row_block(AT acc, uint32_t mq, const VT *vals,
                                        const AT *__restrict__ xp) {
  if (UNROLL) {
    int o = 0;
#pragma unroll
    for (int t = 0; t < C; ++t) {
      if ((mq >> t) & 1u) {
        acc = fma((AT)widen(vals[o]), __ldg(xp + t), acc);
        ++o;
      }
    }
  } else {
    while (mq) {
      const int k = __ffs(mq) - 1;
      mq &= mq - 1u;
      acc = fma((AT)widen(*vals++), __ldg(xp + k), acc);
    }
  }
  return acc;
}

// Same with x already staged in shared memory (xrow[k] = x[start + k]).
template <int C, bool UNROLL>
__device__ __forceinline__ double row_block_xs(double acc, uint32_t mq, const double *vals,
                                               const double *xrow) {
  if (UNROLL) {
    int o = 0;
#pragma unroll
    for (int t = 0; t < C; ++t) {
      if ((mq >> t) & 1u) {
        acc = fma(vals[o], xrow[t], acc);
        ++o;
      }
    }
  } else {
    while (mq) {
      const int k = __ffs(mq) - 1;
      mq &= mq - 1u;
      acc = fma(*vals++, xrow[k], acc);
    }
  }
  return acc;
}

// Columns of a block present in at least one of its R rows.
template <int R, int C>
__device__ __forceinline__ uint32_t union_mask(uint32_t m) {
  uint32_t u = 0;
#pragma unroll
  for (int q = 0; q < R; ++q) u |= (m >> (q * C)) & ((1u << C) - 1u);
  return u;
}

// Exclusive prefix of `pc` over the G lanes of a row group; *total gets the
// group's sum.
__device__ __forceinline__ int group_scan(int pc, int g, int G, int *total) {
  int incl = pc;
  for (int o = 1; o < G; o <<= 1) {
    int t = __shfl_up_sync(kFull, incl, o, G);
    if (g >= o) incl += t;
  }
  *total = (G > 1) ? __shfl_sync(kFull, incl, G - 1, G) : pc;
  return incl - pc;
}

template <typename AT>
__device__ __forceinline__ AT group_sum(AT acc, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o, G);
  return acc;
}

// ------------------------------------------------------------ direct kernel --

// Tile-scheduled kernel reading global memory directly.  Each warp walks the
// planner's tiles (warp w takes tiles w, w + nwarps, ...), prefetching the
// next tile's descriptor, and pipelines each round's block metadata one
// round ahead so that a round waits for one memory round trip (its values)
// instead of two (metadata, then values).  Many resident warps (48 per SM)
// keep the FP64 pipe and the memory system busy.
//
// Row-stream body for row-group tiles with one lane per row: the lane walks
// its row's values across the panel's blocks, one FMA per loop trip, so a
// warp issues as many FP64 FMAs as its longest row has values (plus one trip
// for every block in which a row has no value), instead of the sum over
// blocks of the largest per-block bit count.  A lane enters its panel's next
// block when its row bits in the current one are used up; the metadata of
// the block after it is loaded, and its values prefetched to L1, one block
// ahead.
template <int R, int C, bool SKIP, typename VT, typename AT, typename MaskT>
__device__ __forceinline__ AT row_stream(const MaskT *__restrict__ masks,
                                         const int32_t *__restrict__ block_colidx,
                                         const VT *__restrict__ vals, const AT *__restrict__ x,
                                         int32_t bl, int32_t nbp, int32_t v, int q) {
  const int qc = q * C;
  const uint32_t row_low = (1u << qc) - 1u;
  const uint32_t cmask = (1u << C) - 1u;
  uint32_t m1 = 0u;  // next block to enter: mask word and start column
  int32_t c1 = 0;
  if (nbp > 0) {
    m1 = (uint32_t)masks[bl];
    c1 = block_colidx[bl];
  }
  int32_t b = 0;  // blocks entered
  uint32_t mq = 0u;
  int32_t off = 0, col = 0;
  AT acc = 0;
  // two trips per vote: a trip of a lane whose row is done does nothing
  while (__any_sync(kFull, mq != 0u || b < nbp)) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      // SKIP: blocks in which the row has no value are passed within the
      // trip (the lane does not spend an FMA slot on them)
      for (int e = 0; mq == 0u && b < nbp && (SKIP || e < 1); ++e) {
        mq = (m1 >> qc) & cmask;
        off = v + __popc(m1 & row_low);
        v += __popc(m1);
        col = c1;
        ++b;
        m1 = 0u;
        if (b < nbp) {
          m1 = (uint32_t)masks[bl + b];
          c1 = block_colidx[bl + b];
          prefetch_l1(vals + v);  // the next block's values, needed a few trips later
        }
      }
      if (mq) {
        const int k = __ffs(mq) - 1;
        acc = fma((AT)widen(vals[off]), __ldg(x + col + k), acc);
        mq &= mq - 1u;
        ++off;
      }
    }
  }
  return acc;
}

// Pipelined row stream (passing empty blocks): the walk of row_stream, but
// the operands of a product (the value and its x) are loaded two trips
// before its FMA, into two register slots used in turn.  In row_stream a
// trip's FMA waits for loads issued in the same trip; here every warp keeps
// three trips of loads in flight, which pays off where the rows are regular
// (stencils) and the FMA waits on memory.
template <int R, int C, typename VT, typename AT, typename MaskT>
__device__ __forceinline__ AT row_pipe(const MaskT *__restrict__ masks,
                                       const int32_t *__restrict__ block_colidx,
                                       const VT *__restrict__ vals, const AT *__restrict__ x,
                                       int32_t bl, int32_t nbp, int32_t v, int q) {
  const int qc = q * C;
  const uint32_t row_low = (1u << qc) - 1u;
  const uint32_t cmask = (1u << C) - 1u;
  uint32_t m1 = 0u;  // next block to enter: mask word and start column
  int32_t c1 = 0;
  if (nbp > 0) {
    m1 = (uint32_t)masks[bl];
    c1 = block_colidx[bl];
  }
  int32_t b = 0;  // blocks entered
  uint32_t mq = 0u;
  int32_t off = 0, col = 0;
  // Moves the cursor to the row's next value (entering as many blocks as it
  // takes) and loads its operands into (pv, px); false when the row is done.
  auto fetch = [&](VT &pv, AT &px) -> bool {
    while (mq == 0u && b < nbp) {
      mq = (m1 >> qc) & cmask;
      off = v + __popc(m1 & row_low);
      v += __popc(m1);
      col = c1;
      ++b;
      m1 = 0u;
      if (b < nbp) {
        m1 = (uint32_t)masks[bl + b];
        c1 = block_colidx[bl + b];
        prefetch_l1(vals + v);
      }
    }
    if (mq == 0u) return false;
    const int k = __ffs(mq) - 1;
    mq &= mq - 1u;
    pv = vals[off];
    px = __ldg(x + col + k);
    ++off;
    return true;
  };
  VT va = VT(0), vb = VT(0);
  AT xa = AT(0), xb = AT(0);
  bool ha = fetch(va, xa);
  bool hb = fetch(vb, xb);
  AT acc = 0;
  while (__any_sync(kFull, ha || hb)) {
    {  // slot a was filled two trips ago
      const VT cv = va;
      const AT cx = xa;
      const bool ch = ha;
      ha = fetch(va, xa);
      if (ch) acc = fma((AT)widen(cv), cx, acc);
    }
    {  // slot b one trip ago
      const VT cv = vb;
      const AT cx = xb;
      const bool ch = hb;
      hb = fetch(vb, xb);
      if (ch) acc = fma((AT)widen(cv), cx, acc);
    }
  }
  return acc;
}

// Queued row-stream body (one lane per row): the lane loads the metadata of
// its panel's next four blocks at once and packs its row's bits of the four
// blocks into one word (block i at bits [i*c, (i+1)*c)), with each block's
// start column and the value index of the row's first value in it.  A loop
// trip then takes the lowest pending bit, selects its block's column and
// value index (branch-free selects over the four slots) and does one FMA;
// blocks in which the row has no value cost nothing, and the queue is
// refilled only every four blocks, so a trip is a few integer instructions
// around one FP64 FMA.
template <typename T>
__device__ __forceinline__ T sel4(int i, T a0, T a1, T a2, T a3) {
  const T lo = (i & 1) ? a1 : a0;
  const T hi = (i & 1) ? a3 : a2;
  return (i & 2) ? hi : lo;
}

template <int R, int C, typename VT, typename AT, typename MaskT>
__device__ __forceinline__ AT row_queue(const MaskT *__restrict__ masks,
                                        const int32_t *__restrict__ block_colidx,
                                        const VT *__restrict__ vals, const AT *__restrict__ x,
                                        int32_t bl, int32_t nbp, int32_t v, int q) {
  constexpr int LOG2C = C == 8 ? 3 : 2;
  const int qc = q * C;
  const uint32_t row_low = (1u << qc) - 1u;
  const uint32_t cmask = (1u << C) - 1u;
  int32_t b = 0;        // blocks queued so far
  uint32_t w = 0u;      // pending row bits of the queued blocks
  int32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;  // start columns of the queued blocks
  int32_t o0 = 0, o1 = 0, o2 = 0, o3 = 0;  // value index of the row's first value in each
  int slot = 0;
  int32_t off = 0, col = 0;
  AT acc = 0;
  for (;;) {
    const bool refill = (w == 0u) && (b < nbp);
    if (!__any_sync(kFull, refill || w != 0u)) break;
    if (refill) {
      uint32_t m[4];
      int32_t cc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool ok = b + i < nbp;
        m[i] = ok ? (uint32_t)masks[bl + b + i] : 0u;
        cc[i] = ok ? block_colidx[bl + b + i] : 0;
      }
      int32_t o[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        o[i] = v + __popc(m[i] & row_low);
        v += __popc(m[i]);
        w |= ((m[i] >> qc) & cmask) << (i * C);
      }
      c0 = cc[0], c1 = cc[1], c2 = cc[2], c3 = cc[3];
      o0 = o[0], o1 = o[1], o2 = o[2], o3 = o[3];
      b += 4;
      slot = -1;
    }
    if (w) {
      const int k = __ffs(w) - 1;
      const int i = k >> LOG2C;
      const bool fresh = i != slot;
      off = fresh ? sel4(i, o0, o1, o2, o3) : off;
      col = fresh ? sel4(i, c0, c1, c2, c3) : col;
      slot = i;
      acc = fma((AT)widen(vals[off]), __ldg(x + col + (k & (C - 1))), acc);
      ++off;
      w &= w - 1u;
    }
  }
  return acc;
}

// Four-block rounds (one lane per row): all lanes of the warp take their
// panel's next four blocks together, pack their row's bits of the four blocks
// into one word, and loop as many times as the largest bit count in the warp
// (one FMA per trip, predicated on the lane having a bit left); each trip
// selects its block's column and value index with branch-free selects.  The
// warp never diverges, the block traversal costs a few instructions per four
// blocks, and summing a row's bits over four blocks evens out the lanes'
// trip counts (the FMA instructions' idle lanes).
template <int R, int C, typename VT, typename AT, typename MaskT>
__device__ __forceinline__ AT row_rounds4(const MaskT *__restrict__ masks,
                                          const int32_t *__restrict__ block_colidx,
                                          const VT *__restrict__ vals, const AT *__restrict__ x,
                                          int32_t bl, int32_t nbp, int32_t v, int q) {
  constexpr int LOG2C = C == 8 ? 3 : 2;
  const int qc = q * C;
  const uint32_t row_low = (1u << qc) - 1u;
  const uint32_t cmask = (1u << C) - 1u;
  AT acc = 0;
  const int32_t maxnb = __reduce_max_sync(kFull, nbp);
  for (int32_t b = 0; b < maxnb; b += 4) {
    uint32_t m[4];
    int32_t cc[4], o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool ok = b + i < nbp;
      m[i] = ok ? (uint32_t)masks[bl + b + i] : 0u;
      cc[i] = ok ? block_colidx[bl + b + i] : 0;
    }
    uint32_t w = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[i] = v + __popc(m[i] & row_low);
      v += __popc(m[i]);
      w |= ((m[i] >> qc) & cmask) << (i * C);
    }
    const int trips = __reduce_max_sync(kFull, __popc(w));
    int slot = -1;
    int32_t off = 0, col = 0;
    for (int it = 0; it < trips; ++it) {
      if (w) {
        const int k = __ffs(w) - 1;
        const int i = k >> LOG2C;
        const bool fresh = i != slot;
        off = fresh ? sel4(i, o[0], o[1], o[2], o[3]) : off;
        col = fresh ? sel4(i, cc[0], cc[1], cc[2], cc[3]) : col;
        slot = i;
        acc = fma((AT)widen(vals[off]), __ldg(x + col + (k & (C - 1))), acc);
        ++off;
        w &= w - 1u;
      }
    }
  }
  return acc;
}

// Launch shape of the row-group kernel: two CTAs of 24 warps per SM, so
// that 24 consecutive tiles (neighbouring rows, which share x) run on one
// SM's L1 at a time (the four-block body holds more registers: 5 x 8 warps;
// body 6 is the row stream at 2 x 32 warps, 32 registers, for matrices whose
// products wait on memory more than on issue).
template <int BODY>
struct TileThreads {
  static constexpr int v = BODY == 4 ? 256 : (BODY == 6 ? 1024 : 768);
};
template <int BODY>
struct TileBlocksPerSM {
  static constexpr int v = BODY == 4 ? 5 : 2;
};

template <int R, int C, int BODY, bool DYN, typename VT, typename AT>
__global__ void __launch_bounds__(TileThreads<BODY>::v, TileBlocksPerSM<BODY>::v)
    k_spmv_tiles(const Tile *__restrict__ tiles, int64_t ntiles, uint32_t *sched,
                 const int32_t *__restrict__ block_rowptr, const int32_t *__restrict__ panel_vptr,
                 const int32_t *__restrict__ block_colidx,
                 const typename MaskType<R, C>::T *__restrict__ masks,
                 const VT *__restrict__ vals, const AT *__restrict__ x, AT *__restrict__ y,
                 AT *__restrict__ partial, Scale<AT> sc, int64_t nrows) {
  constexpr int LOG2R = Log2<R>::v;
  const int lane = threadIdx.x & 31;
  const uint32_t cmask = (1u << C) - 1u;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __shared__ Tile s_next_all[TileThreads<BODY>::v / 32];
  Tile *s_next = &s_next_all[threadIdx.x >> 5];
  // Tiles are dealt grid-stride (warp w takes w, w + nwarps, ...), or, with
  // DYN, taken from a counter two ahead: the index of the tile after next
  // is requested when a tile starts, so the atomic's latency is hidden; the
  // last warp to finish resets the counter for the next launch.  The counter
  // evens out uneven tiles but costs one atomic per tile on one address.
  uint32_t grab = 0;
  int64_t t;
  if (DYN) {
    if (lane == 0) grab = atomicAdd(&sched[0], 1u);
    t = (int64_t)__shfl_sync(kFull, grab, 0);
    if (lane == 0 && t < ntiles) grab = atomicAdd(&sched[0], 1u);
  } else {
    t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  }
  Tile cur{0, 0, 0, 0, 0, 0, 0, 0};
  if (t < ntiles) cur = tiles[t];
  while (t < ntiles) {
    int64_t tn;
    if (DYN) {
      tn = (int64_t)__shfl_sync(kFull, grab, 0);
      if (lane == 0 && tn < ntiles) grab = atomicAdd(&sched[0], 1u);
    } else {
      tn = t + nwarps;
    }
    // the next tile's descriptor waits in shared memory, not in registers
    __syncwarp();
    if (lane < 8)
      reinterpret_cast<int32_t *>(s_next)[lane] =
          tn < ntiles ? reinterpret_cast<const int32_t *>(tiles + tn)[lane] : 0;
    {  // start bringing the first 2 KB of the tile's values and 1 KB of its
       // block columns to L2: the tile's first rounds wait on them (more
       // would evict x from L2 on large tiles)
      constexpr int kLine = 128 / (int)sizeof(VT);
      if (lane < 16 && lane * kLine < cur.v1 - cur.v0) prefetch_l2(vals + cur.v0 + lane * kLine);
      if (lane >= 16 && lane < 24 && (lane - 16) * 32 < cur.b1 - cur.b0)
        prefetch_l2(block_colidx + cur.b0 + (lane - 16) * 32);
    }
    const bool segment = (cur.mode & kSegment) != 0;
    const int log2G = cur.mode & 15;
    const int G = 1 << log2G;
    const int shift_j = LOG2R + log2G;
    const int g = lane & (G - 1);
    const int q = (lane >> log2G) & (R - 1);
    const int j = lane >> shift_j;
    const uint32_t row_low = (q == 0) ? 0u : ((1u << (q * C)) - 1u);
    bool pvalid;
    int32_t bl, nbp, v;
    if (segment) {
      pvalid = (j == 0);
      bl = cur.b0;
      nbp = cur.b1 - cur.b0;
      v = cur.v0;
    } else {
      const int64_t p = (int64_t)cur.p0 + j;
      // a heavy panel (kSkip) has tiles of its own
      pvalid = p < cur.p1 && !((cur.mode & kSkip) && (((uint32_t)cur.slot >> j) & 1u));
      bl = pvalid ? block_rowptr[p] : 0;
      nbp = pvalid ? block_rowptr[p + 1] - bl : 0;
      v = pvalid ? panel_vptr[p] : 0;
    }
    AT acc = 0;
    if ((BODY == 2 || BODY == 5 || BODY == 6) && G == 1) {
      acc = row_stream<R, C, BODY == 5>(masks, block_colidx, vals, x, bl, nbp, v, q);
    } else if (BODY == 7 && G == 1) {
      acc = row_pipe<R, C>(masks, block_colidx, vals, x, bl, nbp, v, q);
    } else if (BODY == 3 && G == 1) {
      acc = row_queue<R, C>(masks, block_colidx, vals, x, bl, nbp, v, q);
    } else if (BODY == 4 && G == 1) {
      acc = row_rounds4<R, C>(masks, block_colidx, vals, x, bl, nbp, v, q);
    } else {
    constexpr bool UNROLL = BODY == 1;
    const int32_t maxnb = __reduce_max_sync(kFull, nbp);
    uint32_t m_next = 0u;
    int32_t c_next = 0;
    if (g < nbp) {
      m_next = (uint32_t)masks[bl + g];
      c_next = block_colidx[bl + g];
    }
    for (int32_t it = 0; it < maxnb; it += G) {
      const uint32_t m = m_next;
      const int32_t col = c_next;
      const int32_t idx2 = it + G + g;
      if (idx2 < nbp) {
        m_next = (uint32_t)masks[bl + idx2];
        c_next = block_colidx[bl + idx2];
      } else {
        m_next = 0u;
        c_next = 0;
      }
      const int pc = __popc(m);
      int total;
      const int excl = group_scan(pc, g, G, &total);
      const int32_t off = v + excl + __popc(m & row_low);
      acc = row_block<C, UNROLL>(acc, (m >> (q * C)) & cmask, vals + off, x + col);
      v += total;
    }
    }
    acc = group_sum(acc, G);
    if (pvalid && g == 0) {
      if (cur.mode & kPartial) {
        partial[(int64_t)cur.slot * R + q] = acc;
      } else {
        const int64_t row = ((int64_t)cur.p0 + j) * R + q;
        if (row < nrows) put_row(sc, y, row, acc);
      }
    }
    __syncwarp();
    cur = *s_next;
    t = tn;
  }
  // every warp has made its last grab: the last one to finish resets the counter
  if (DYN && lane == 0) {
    if (atomicAdd(&sched[1], 1u) == (uint32_t)nwarps - 1) {
      atomicExch(&sched[0], 0u);
      atomicExch(&sched[1], 0u);
    }
  }
}

// -------------------------------------------------------------- flat kernel --

// The tile body (flat_tile) and its helpers are in spc5_flat.cuh.
template <int R>
struct FlatBlocksPerSM {  // registers grow with the r row sums a lane keeps
  static constexpr int v = R == 1 ? 6 : (R == 2 ? 5 : (R == 4 ? 4 : 3));
};

template <int R, int C, typename VT, typename AT>
__global__ void __launch_bounds__(kDirectThreads, FlatBlocksPerSM<R>::v)
    k_spmv_flat(const Tile *__restrict__ tiles, int32_t ntiles, uint32_t *sched,
                const int32_t *__restrict__ brp, const int32_t *__restrict__ block_colidx,
                const typename MaskType<R, C>::T *__restrict__ masks,
                const VT *__restrict__ vals, const AT *__restrict__ x, AT *__restrict__ y,
                AT *__restrict__ partial, Scale<AT> sc, int64_t nrows) {
  __shared__ int32_t s_pid[kDirectThreads / 32][kFlatRound];
  int32_t *pid = s_pid[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  uint32_t grab = 0;
  if (lane == 0) grab = atomicAdd(&sched[0], 1u);
  int32_t t = (int32_t)__shfl_sync(kFull, grab, 0);
  while (t < ntiles) {
    if (lane == 0) grab = atomicAdd(&sched[0], 1u);  // next tile, used after this one
    flat_tile<R, C>(tiles[t], lane, pid, brp, block_colidx, masks, vals, x, y, partial, sc,
                    nrows);
    t = (int32_t)__shfl_sync(kFull, grab, 0);
  }
  // every warp has made its last grab: the last one to finish resets the counters
  if (lane == 0) {
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(&sched[1], 1u) == nwarps - 1) {
      atomicExch(&sched[0], 0u);
      atomicExch(&sched[1], 0u);
    }
  }
}

// ------------------------------------------- value-balanced flat kernel --

// Value-balanced variant of the block-balanced kernel (plan 3), same tiles.
// A round stages up to kVRound consecutive blocks in shared memory (masks,
// block columns, each block's value offset in the round, and the id of the
// panel a block ends); the round's values are then split into 32 equal
// runs, one per lane, so a warp issues about values / 32 FMA instructions
// per round whatever the blocks' fill.  A lane finds its run's first block
// by a binary search of the offsets, walks the blocks one set bit per trip
// (a block holds at least one value), picks the row's sum by selects, and
// at the end of a block that ends a panel writes the panel's rows if the
// panel started in its run, else keeps them as the head.  The lanes' last
// partial sums are completed by the segmented warp scan of the
// block-balanced kernel; the open panel carries into the next round.
// Rounds of 256 blocks pay the scan's adds half as often as rounds of 128.
constexpr int kVRound = 256;
constexpr int kVPerLane = kVRound / 32;

template <int R>
struct VFlatBlocksPerSM {
  static constexpr int v = R <= 2 ? 5 : (R == 4 ? 4 : 3);
};

struct VFlatWarpSmem {
  uint32_t m[kVRound];
  int32_t c[kVRound];
  int32_t o[kVRound];    // value offset of the block in the round
  int32_t pid[kVRound];  // panel the block ends, -1 if none
};

template <int R, int C, typename VT, typename AT>
__global__ void __launch_bounds__(kDirectThreads, VFlatBlocksPerSM<R>::v)
    k_spmv_vflat(const Tile *__restrict__ tiles, int32_t ntiles, uint32_t *sched,
                 const int32_t *__restrict__ brp, const int32_t *__restrict__ block_colidx,
                 const typename MaskType<R, C>::T *__restrict__ masks,
                 const VT *__restrict__ vals, const AT *__restrict__ x, AT *__restrict__ y,
                 AT *__restrict__ partial, Scale<AT> sc, int64_t nrows) {
  __shared__ VFlatWarpSmem s_all[kDirectThreads / 32];
  VFlatWarpSmem &S = s_all[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  constexpr int LOG2C = C == 8 ? 3 : 2;
  uint32_t grab = 0;
  if (lane == 0) grab = atomicAdd(&sched[0], 1u);
  int32_t t = (int32_t)__shfl_sync(kFull, grab, 0);
  while (t < ntiles) {
    if (lane == 0) grab = atomicAdd(&sched[0], 1u);  // next tile, used after this one
    const Tile cur = tiles[t];
    if (cur.mode & kPartial) {
      flat_piece<R, C>(cur, lane, block_colidx, masks, vals, x, partial);
    } else {
      flat_empty_rows<R>(cur, lane, brp, y, sc, nrows);
      int32_t v = cur.v0;  // value index of the round's first value
      AT carry = 0;        // lane q < R: row q's sum of the panel still open
      bool open = false;   // a panel continues from the previous round
      int32_t pcur = cur.p0;
      for (int32_t base = cur.b0; base < cur.b1; base += kVRound) {
        const int32_t lim = (base + kVRound < cur.b1) ? base + kVRound : cur.b1;
        const int nbr = lim - base;
        // 1. stage the round's blocks, kVPerLane consecutive blocks per lane
        int cnt = 0;
        uint32_t mm[kVPerLane];
#pragma unroll
        for (int i = 0; i < kVPerLane; ++i) {
          const int32_t b = base + kVPerLane * lane + i;
          const bool ok = b < lim;
          mm[i] = ok ? (uint32_t)masks[b] : 0u;
          S.m[kVPerLane * lane + i] = mm[i];
          S.c[kVPerLane * lane + i] = ok ? block_colidx[b] : 0;
          S.pid[kVPerLane * lane + i] = -1;
          cnt += __popc(mm[i]);
        }
        int V;
        int o = warp_excl_scan(cnt, lane, &V);
#pragma unroll
        for (int i = 0; i < kVPerLane; ++i) {
          S.o[kVPerLane * lane + i] = o;
          o += __popc(mm[i]);
        }
        __syncwarp();
        // 2. the panels whose last block lies in the round
        for (int32_t w = pcur;; w += 32) {
          const int32_t p = w + lane;
          const bool in = p < cur.p1;
          const int32_t st = in ? brp[p] : 0;
          const int32_t en = in ? brp[p + 1] : 0;
          if (in && en > st && en > base && en <= lim) S.pid[en - 1 - base] = p;
          const unsigned beyond = __ballot_sync(kFull, !in || en > lim);
          if (beyond) {
            pcur = w + __ffs(beyond) - 1;
            break;
          }
        }
        __syncwarp();
        // 3. the lane's run of values [lo, hi) of the round
        const int K = (V + 31) >> 5;
        const int lo = min(lane * K, V);
        const int n = min(lo + K, V) - lo;
        int b = 0;
        uint32_t mr = 0u;
        int32_t col = 0;
        bool fresh = true;  // the lane's current panel started in its run
        if (n > 0) {
          int a = 0, z = nbr - 1;  // the last block whose offset is <= lo
          while (a < z) {
            const int mid = (a + z + 1) >> 1;
            if (S.o[mid] <= lo) a = mid; else z = mid - 1;
          }
          b = a;
          const int rank = lo - S.o[b];
          const uint32_t mb = S.m[b];
          mr = rank ? mb & ~((1u << __fns(mb, 0, rank + 1)) - 1u) : mb;
          col = S.c[b];
          fresh = rank == 0 && (b == 0 ? !open : S.pid[b - 1] >= 0);
        }
        // lane 0 starts from the sums of the panel still open (0 if none)
        AT acc[R], head[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const AT cq = __shfl_sync(kFull, carry, q);
          acc[q] = lane == 0 ? cq : (AT)0;
          head[q] = 0;
        }
        bool has_head = false, ended = false;
        int32_t head_pid = 0;
        auto end_panel = [&](int bb) {  // block bb ends panel S.pid[bb]
          const int64_t p = S.pid[bb];
          if (fresh) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
              const int64_t row = p * R + q;
              if (row < nrows) put_row(sc, y, row, acc[q]);
            }
          } else {
#pragma unroll
            for (int q = 0; q < R; ++q) head[q] = acc[q];
            has_head = true;
            head_pid = (int32_t)p;
          }
#pragma unroll
          for (int q = 0; q < R; ++q) acc[q] = 0;
          fresh = true;
          ended = true;
        };
        int32_t off = v + lo;
        for (int tt = 0; tt < K; ++tt) {
          if (tt < n) {
            if (mr == 0u) {  // the run goes on in the next block
              if (S.pid[b] >= 0) end_panel(b);
              ++b;
              mr = S.m[b];
              col = S.c[b];
            }
            const int kf = __ffs(mr) - 1;
            mr &= mr - 1u;
            const int q = kf >> LOG2C;
            AT tq = acc[0];
#pragma unroll
            for (int qq = 1; qq < R; ++qq) tq = (q == qq) ? acc[qq] : tq;
            tq = fma((AT)widen(vals[off]), __ldg(x + col + (kf & (C - 1))), tq);
#pragma unroll
            for (int qq = 0; qq < R; ++qq) acc[qq] = (q == qq) ? tq : acc[qq];
            ++off;
          }
        }
        if (n > 0 && mr == 0u && S.pid[b] >= 0) end_panel(b);  // run ends with a panel
        // segmented scan of the lanes' last partial sums (stops at the first
        // step where no lane can add)
        const uint32_t endl = __ballot_sync(kFull, ended);
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
          const bool same =
              lane >= o2 && ((endl >> (lane - o2 + 1)) & ((1u << o2) - 1u)) == 0u;
          if (!__any_sync(kFull, same)) break;
#pragma unroll
          for (int q = 0; q < R; ++q) {
            const AT tq = __shfl_up_sync(kFull, acc[q], o2);
            if (same) acc[q] += tq;
          }
        }
        // panels cut between lanes: the head plus the scanned partial before
        // it (lane 0's head already holds the open panel's sums)
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const AT cin = __shfl_up_sync(kFull, acc[q], 1);
          if (has_head) {
            const int64_t row = (int64_t)head_pid * R + q;
            if (row < nrows) put_row(sc, y, row, lane == 0 ? head[q] : head[q] + cin);
          }
        }
        // the panel open at the end of the round: its sums are those of the
        // lane holding the round's last value
        open = S.pid[nbr - 1] < 0;
        const int ll = (V - 1) / K;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const AT sl = __shfl_sync(kFull, acc[q], ll);
          if (lane == q) carry = open ? sl : (AT)0;
        }
        v += V;
        __syncwarp();
      }
    }
    t = (int32_t)__shfl_sync(kFull, grab, 0);
  }
  // every warp has made its last grab: the last one to finish resets the counters
  if (lane == 0) {
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(&sched[1], 1u) == nwarps - 1) {
      atomicExch(&sched[0], 0u);
      atomicExch(&sched[1], 0u);
    }
  }
}

// ---------------------------------------------------------- expanded kernel --

// Expanded kernel.  On GB300 the FP64 pipe executes two FMAs per cycle per SM,
// and an FMA instruction costs its 16 cycles whether 32 lanes or one lane
// use it; with lanes owning rows, lanes idle whenever rows (or a row's bits
// in a block) have uneven lengths, and power-law rows leave most lanes idle.
// This kernel separates the integer work from the FP64 work:
//   1. each tile's row starts in a row-major layout of its values were
//      computed when the plan was built (k_ex_row_starts: per-row counts
//      from a segmented warp scan of packed per-row bit counts, then an
//      exclusive scan); rows without values get y = beta y here;
//   2. scatter: the tile's blocks are dealt to the lanes one per lane per
//      round; a lane finds its block's panel by a binary search in the
//      tile's block_rowptr (staged in shared memory), and a value's
//      destination is its row's cursor plus its rank among the row's values
//      of the round (the same packed segmented scan) plus its rank among the
//      row's bits in the block; its value index is the running value offset
//      (Algorithm 1's idxVal) plus an exclusive warp scan of the blocks'
//      popcounts; the column index and the value index go to shared memory;
//   3. FP64: the tile's values, now row by row, are split into 32 equal runs,
//      one per lane; a lane multiplies its run's values by x with one FMA per
//      value (all lanes busy), writes the rows that start and end inside its
//      run (one write per row, Section 3.2), and a segmented warp scan of the
//      lanes' last partial sums completes the rows cut between lanes.
// The FP64 work per tile is ceil(values / 32) FMA instructions plus six adds.
// A piece of a long panel (mode & kPartial) writes its r row sums to the
// partial buffer for the fixup kernel.  Warps take tiles from a counter; the
// last warp to finish resets it for the next launch.
constexpr int kExpandWarps = 4;
constexpr int kExpandBlocksPerSM = 7;


// Per-row bit counts of a block, row q in bits [q * 64/R, (q + 1) * 64/R).
template <int R, int C>
__device__ __forceinline__ uint64_t packed_counts(uint32_t m) {
  constexpr int F = 64 / R;
  uint64_t w = 0;
#pragma unroll
  for (int q = 0; q < R; ++q) w |= (uint64_t)__popc((m >> (q * C)) & ((1u << C) - 1u)) << (q * F);
  return w;
}

template <int R>
__device__ __forceinline__ int32_t packed_field(uint64_t w, int q) {
  if constexpr (R == 1) {
    return (int32_t)w;
  } else {
    constexpr int F = 64 / R;
    return (int32_t)((w >> (q * F)) & ((1ull << F) - 1ull));
  }
}

// Inclusive scan of `w` over lanes with the same key (keys ascend with the lane).
__device__ __forceinline__ uint64_t seg_scan_u64(uint64_t w, int32_t key, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(kFull, w, o);
    const int32_t k = __shfl_up_sync(kFull, key, o);
    if (lane >= o && k == key) w += t;
  }
  return w;
}

// Per-row value counts of an expanded tile's blocks [b0, b1) (panels
// [0, np_t) of the tile, block_rowptr slice in s_brp) added to s_row[j*R+q]:
// blocks are dealt to the lanes one per lane per round; a lane finds its
// block's panel by a binary search in s_brp and packs the block's per-row bit
// counts into one 64-bit word; a segmented warp scan of the packed words by
// panel gives, at the last lane of each panel in the round, the round's
// per-row counts.
template <int R, int C>
__device__ __forceinline__ void ex_count_rows(int lane, int32_t b0, int32_t b1, int32_t np_t,
                                              const int32_t *s_brp, int32_t *s_row,
                                              const typename MaskType<R, C>::T *__restrict__ masks) {
  constexpr int32_t kNoPanel = 0x7fffffff;
  for (int32_t base = b0; base < b1; base += 32) {
    const int32_t b = base + lane;
    const bool valid = b < b1;
    const uint32_t m = valid ? (uint32_t)masks[b] : 0u;
    int32_t j = kNoPanel;
    if (valid) {
      int lo = 0, hi = np_t - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_brp[mid] <= b) lo = mid; else hi = mid - 1;
      }
      j = lo;
    }
    const uint64_t inc = seg_scan_u64(packed_counts<R, C>(m), j, lane);
    const int32_t jn = __shfl_down_sync(kFull, j, 1);
    if (valid && (lane == 31 || jn != j)) {
#pragma unroll
      for (int q = 0; q < R; ++q) s_row[j * R + q] += packed_field<R>(inc, q);
    }
    __syncwarp();
  }
}

// Row starts of every expanded tile, computed once when the plan is built:
// rowoff[base + r] = index of tile row r's first value in the tile's
// row-major layout, base = p0 * r for a tile of whole panels and
// (npanels + slot) * r for a piece of a long panel.  One warp per tile.
template <int R, int C>
__global__ void __launch_bounds__(32 * kExpandWarps)
    k_ex_row_starts(const Tile *__restrict__ tiles, int32_t ntiles, int64_t npanels,
                    const int32_t *__restrict__ brp,
                    const typename MaskType<R, C>::T *__restrict__ masks, uint16_t *rowoff) {
  __shared__ int32_t s_row_all[kExpandWarps][kExpandRows];
  __shared__ int32_t s_brp_all[kExpandWarps][kExpandRows + 1];
  const int wid = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int32_t *s_row = s_row_all[wid];
  int32_t *s_brp = s_brp_all[wid];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles;
       t += nwarps) {
    const Tile cur = tiles[t];
    const bool piece = (cur.mode & kPartial) != 0;
    const int32_t np_t = piece ? 1 : cur.p1 - cur.p0;
    const int rows_t = np_t * R;
    for (int j = lane; j <= np_t; j += 32)
      s_brp[j] = piece ? (j == 0 ? cur.b0 : cur.b1) : brp[cur.p0 + j];
    for (int r = lane; r < rows_t; r += 32) s_row[r] = 0;
    __syncwarp();
    ex_count_rows<R, C>(lane, cur.b0, cur.b1, np_t, s_brp, s_row, masks);
    const int r0 = lane * (kExpandRows / 32);
    int cnt[kExpandRows / 32];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < kExpandRows / 32; ++i) {
      cnt[i] = (r0 + i < rows_t) ? s_row[r0 + i] : 0;
      sum += cnt[i];
    }
    int total;
    int start = warp_excl_scan(sum, lane, &total);
    const int64_t base = piece ? (npanels + cur.slot) * R : (int64_t)cur.p0 * R;
#pragma unroll
    for (int i = 0; i < kExpandRows / 32; ++i) {
      if (r0 + i < rows_t) rowoff[base + r0 + i] = (uint16_t)start;
      start += cnt[i];
    }
    __syncwarp();
  }
}

template <int R, int C, typename VT, typename AT>
__global__ void __launch_bounds__(32 * kExpandWarps, kExpandBlocksPerSM)
    k_spmv_expand(const Tile *__restrict__ tiles, int32_t ntiles, uint32_t *sched,
                  const int32_t *__restrict__ brp, const int32_t *__restrict__ block_colidx,
                  const typename MaskType<R, C>::T *__restrict__ masks,
                  const VT *__restrict__ vals, const AT *__restrict__ x, AT *__restrict__ y,
                  AT *__restrict__ partial, Scale<AT> sc, int64_t nrows,
                  const uint16_t *__restrict__ rowoff, int64_t npanels) {
  __shared__ int32_t s_col_all[kExpandWarps][kExpandCap];
  __shared__ uint16_t s_vid_all[kExpandWarps][kExpandCap];
  __shared__ int32_t s_row_all[kExpandWarps][kExpandRows];
  __shared__ int32_t s_brp_all[kExpandWarps][kExpandRows + 1];
  const int wid = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int32_t *s_col = s_col_all[wid];
  uint16_t *s_vid = s_vid_all[wid];
  int32_t *s_row = s_row_all[wid];
  int32_t *s_brp = s_brp_all[wid];
  constexpr int32_t kNoPanel = 0x7fffffff;
  using MaskT = typename MaskType<R, C>::T;

  uint32_t grab = 0;
  if (lane == 0) grab = atomicAdd(&sched[0], 1u);
  int32_t t = (int32_t)__shfl_sync(kFull, grab, 0);
  while (t < ntiles) {
    if (lane == 0) grab = atomicAdd(&sched[0], 1u);  // next tile, used after this one
    const Tile cur = tiles[t];
    const bool piece = (cur.mode & kPartial) != 0;
    const int32_t np_t = piece ? 1 : cur.p1 - cur.p0;
    const int rows_t = np_t * R;
    const int32_t nv = cur.v1 - cur.v0;
    {  // start bringing the tile's masks and block columns (step 2) and its
       // values (step 3) to L2; shared memory leaves little room in L1
      constexpr int kLine = 128 / (int)sizeof(VT);
      constexpr int kLineM = 128 / (int)sizeof(MaskT);
      const int32_t nbt = cur.b1 - cur.b0;
      for (int32_t o = lane * kLine; o < nv; o += 32 * kLine) prefetch_l2(vals + cur.v0 + o);
      for (int32_t o = lane * kLineM; o < nbt; o += 32 * kLineM) prefetch_l2(masks + cur.b0 + o);
      for (int32_t o = lane * 32; o < nbt; o += 32 * 32) prefetch_l2(block_colidx + cur.b0 + o);
    }
    // tile rows' starts (computed when the plan was built)
    const int64_t rbase = piece ? (npanels + cur.slot) * R : (int64_t)cur.p0 * R;
    for (int j = lane; j <= np_t; j += 32)
      s_brp[j] = piece ? (j == 0 ? cur.b0 : cur.b1) : brp[cur.p0 + j];
    for (int r = lane; r < rows_t; r += 32) s_row[r] = rowoff[rbase + r];
    __syncwarp();

    // tile row of a value: global row (or partial slot) of tile row r
    auto emit = [&](int r, AT v) {
      const int j = r / R, q = r - j * R;
      if (piece) {
        partial[(int64_t)cur.slot * R + q] = v;
      } else {
        const int64_t row = ((int64_t)cur.p0 + j) * R + q;
        if (row < nrows) put_row(sc, y, row, v);
      }
    };
    // panel (index within the tile) of block b: the last j with s_brp[j] <= b
    auto panel_of = [&](int32_t b) {
      int lo = 0, hi = np_t - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_brp[mid] <= b) lo = mid; else hi = mid - 1;
      }
      return lo;
    };

    // rows without values
    for (int r = lane; r < rows_t; r += 32) {
      const int32_t next = (r + 1 < rows_t) ? s_row[r + 1] : nv;
      if (next == s_row[r]) {
        if (piece) emit(r, (AT)0);
        else {
          const int64_t row = ((int64_t)cur.p0 + r / R) * R + r % R;
          if (row < nrows) put_empty_row(sc, y, row);
        }
      }
    }
    __syncwarp();
    // 2. scatter (s_row holds each row's cursor)
    {
      int32_t vrun = 0;
      for (int32_t base = cur.b0; base < cur.b1; base += 32) {
        const int32_t b = base + lane;
        const bool valid = b < cur.b1;
        const uint32_t m = valid ? (uint32_t)masks[b] : 0u;
        const int32_t col = valid ? block_colidx[b] : 0;
        const int32_t j = valid ? panel_of(b) : kNoPanel;
        const uint64_t own = packed_counts<R, C>(m);
        const uint64_t inc = seg_scan_u64(own, j, lane);
        int total;
        int vi = vrun + warp_excl_scan(__popc(m), lane, &total);
        vrun += total;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          uint32_t mq = (m >> (q * C)) & ((1u << C) - 1u);
          if (mq) {
            int dst = s_row[j * R + q] + packed_field<R>(inc, q) - packed_field<R>(own, q);
            while (mq) {
              const int k = __ffs(mq) - 1;
              mq &= mq - 1u;
              s_col[dst] = col + k;
              s_vid[dst] = (uint16_t)vi;
              ++dst;
              ++vi;
            }
          }
        }
        __syncwarp();
        const int32_t jn = __shfl_down_sync(kFull, j, 1);
        if (valid && (lane == 31 || jn != j)) {
#pragma unroll
          for (int q = 0; q < R; ++q) s_row[j * R + q] += packed_field<R>(inc, q);
        }
        __syncwarp();
      }
    }
    // 3. FP64 (or FP32) products: s_row[r] is now the end of row r
    {
      // an odd run length keeps the lanes' shared-memory reads on distinct banks
      const int32_t K = ((nv + 31) >> 5) | 1;
      const int32_t lo = min(lane * K, nv), hi = min(lo + K, nv);
      const VT *__restrict__ tv = vals + cur.v0;
      AT acc = 0, head_val = 0;
      int head_row = -1, tail_row = -1;
      if (lo < hi) {
        int a = 0, bnd = rows_t - 1;  // first row ending after lo
        while (a < bnd) {
          const int mid = (a + bnd) >> 1;
          if (s_row[mid] > lo) bnd = mid; else a = mid + 1;
        }
        int r = a;
        int32_t rend = s_row[r];
        bool started_here = (r == 0 ? 0 : s_row[r - 1]) >= lo;
        // four values at a time: their loads are issued together
        for (int32_t i0 = lo; i0 < hi; i0 += 4) {
          AT av[4], xv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (i0 + u < hi) {
              av[u] = (AT)widen(tv[s_vid[i0 + u]]);
              xv[u] = __ldg(x + s_col[i0 + u]);
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int32_t i = i0 + u;
            if (i < hi) {
              acc = fma(av[u], xv[u], acc);
              if (i + 1 == rend) {
                if (started_here) {
                  emit(r, acc);
                } else {
                  head_row = r;
                  head_val = acc;
                }
                acc = 0;
                if (i + 1 < nv) {
                  do {
                    ++r;
                  } while (s_row[r] <= i + 1);
                  rend = s_row[r];
                  started_here = true;
                }
              }
            }
          }
        }
        if (hi < nv) tail_row = r;
      }
      // rows cut between lanes: segmented scan of the lanes' last partial sums
      AT sv = (tail_row >= 0) ? acc : (AT)0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {  // tail rows ascend with the lane
        const AT tsv = __shfl_up_sync(kFull, sv, o);
        const int kr = __shfl_up_sync(kFull, tail_row, o);
        const bool add = lane >= o && kr == tail_row && tail_row >= 0;
        if (!__any_sync(kFull, add)) break;
        if (add) sv += tsv;
      }
      const AT cin = __shfl_up_sync(kFull, sv, 1);
      if (head_row >= 0) emit(head_row, head_val + cin);
    }
    __syncwarp();
    t = (int32_t)__shfl_sync(kFull, grab, 0);
  }
  // every warp has made its last grab: the last one to finish resets the counters
  if (lane == 0) {
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(&sched[1], 1u) == nwarps - 1) {
      atomicExch(&sched[0], 0u);
      atomicExch(&sched[1], 0u);
    }
  }
}

// ----------------------------------------------------------- scalar kernel --

// Scalars of a hybrid matrix: y += alpha * S x for the CSR of single-value
// blocks, after the block part wrote y.  The scalars are already row by row,
// so this is the FP64 step of the expanded kernel reading global memory:
// tiles of whole rows (at most kExpandCap values and kExpandRows rows) split
// into 32 equal runs of values, one per lane, one FMA per value; a lane adds
// the rows that start and end in its run to y, and a segmented warp scan of
// the lanes' last partial sums completes the rows cut between lanes.  A piece
// of a long row writes its sum to the partial buffer.
template <typename VT, typename AT>
__global__ void __launch_bounds__(32 * kExpandWarps)
    k_spmv_scalars(const Tile *__restrict__ tiles, int32_t ntiles, uint32_t *sched,
                   const int32_t *__restrict__ s_rowptr, const int32_t *__restrict__ s_colidx,
                   const VT *__restrict__ s_vals, const AT *__restrict__ x, AT *__restrict__ y,
                   AT *__restrict__ partial, AT alpha) {
  __shared__ int32_t s_row_all[kExpandWarps][kExpandRows];
  const int wid = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int32_t *s_row = s_row_all[wid];
  uint32_t grab = 0;
  if (lane == 0) grab = atomicAdd(&sched[0], 1u);
  int32_t t = (int32_t)__shfl_sync(kFull, grab, 0);
  while (t < ntiles) {
    if (lane == 0) grab = atomicAdd(&sched[0], 1u);  // next tile, used after this one
    const Tile cur = tiles[t];
    const bool piece = (cur.mode & kPartial) != 0;
    const int rows_t = piece ? 1 : cur.p1 - cur.p0;
    const int32_t nv = cur.v1 - cur.v0;
    // end of each tile row's values, relative to the tile's first value
    for (int r = lane; r < rows_t; r += 32)
      s_row[r] = (piece ? cur.v1 : s_rowptr[cur.p0 + r + 1]) - cur.v0;
    __syncwarp();
    auto emit = [&](int r, AT v) {
      if (piece) partial[cur.slot] = v;
      else {
        const int64_t row = (int64_t)cur.p0 + r;
        y[row] = fma(alpha, v, y[row]);
      }
    };
    const int32_t K = ((nv + 31) >> 5) | 1;
    const int32_t lo = min(lane * K, nv), hi = min(lo + K, nv);
    const VT *__restrict__ tv = s_vals + cur.v0;
    const int32_t *__restrict__ tc = s_colidx + cur.v0;
    AT acc = 0, head_val = 0;
    int head_row = -1, tail_row = -1;
    if (lo < hi) {
      int a = 0, bnd = rows_t - 1;  // first row ending after lo
      while (a < bnd) {
        const int mid = (a + bnd) >> 1;
        if (s_row[mid] > lo) bnd = mid; else a = mid + 1;
      }
      int r = a;
      int32_t rend = s_row[r];
      bool started_here = (r == 0 ? 0 : s_row[r - 1]) >= lo;
      for (int32_t i0 = lo; i0 < hi; i0 += 4) {
        AT av[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (i0 + u < hi) {
            av[u] = (AT)widen(tv[i0 + u]);
            xv[u] = __ldg(x + tc[i0 + u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int32_t i = i0 + u;
          if (i < hi) {
            acc = fma(av[u], xv[u], acc);
            if (i + 1 == rend) {
              if (started_here) {
                emit(r, acc);
              } else {
                head_row = r;
                head_val = acc;
              }
              acc = 0;
              if (i + 1 < nv) {
                do {
                  ++r;
                } while (s_row[r] <= i + 1);
                rend = s_row[r];
                started_here = true;
              }
            }
          }
        }
      }
      if (hi < nv) tail_row = r;
    }
    AT sv = (tail_row >= 0) ? acc : (AT)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {  // tail rows ascend with the lane
      const AT tsv = __shfl_up_sync(kFull, sv, o);
      const int kr = __shfl_up_sync(kFull, tail_row, o);
      const bool add = lane >= o && kr == tail_row && tail_row >= 0;
      if (!__any_sync(kFull, add)) break;
      if (add) sv += tsv;
    }
    const AT cin = __shfl_up_sync(kFull, sv, 1);
    if (head_row >= 0) emit(head_row, head_val + cin);
    __syncwarp();
    t = (int32_t)__shfl_sync(kFull, grab, 0);
  }
  if (lane == 0) {
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(&sched[1], 1u) == nwarps - 1) {
      atomicExch(&sched[0], 0u);
      atomicExch(&sched[1], 0u);
    }
  }
}

// y[row] += alpha * (sum of the row's pieces) for rows of scalars cut into
// pieces, one warp per row as in k_fixup.
template <typename AT>
__global__ void k_fixup_add(int64_t nlong, const int32_t *long_rows, const int32_t *long_slots,
                            const AT *partial, AT *y, AT alpha) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < nlong; l += nw) {
    const int64_t first = (int64_t)long_slots[2 * l] + lane;
    const int64_t end = long_slots[2 * l + 1];
    AT acc = first < end ? strided_sum(partial + first, (end - first + 31) / 32, 32) : (AT)0;
    acc = warp_sum(acc);
    if (lane == 0) {
      const int64_t row = long_rows[l];
      y[row] = fma(alpha, acc, y[row]);
    }
  }
}

// ------------------------------------------------------------ staged kernel --

// Written by the producer before it arms the stage's barrier.  `seq` is the
// tile sequence number of the CTA: a consumer waits for its own number
// before waiting on the barrier, because a parity wait cannot tell a phase
// two laps behind from a completed one.
struct StageHdr {
  Tile t;
  int32_t voff, coff, moff, roff, pvoff, valid, seq, pad1;
};
static_assert(sizeof(StageHdr) == 64, "stage header is 64 bytes");

struct StagedParams {
  const Tile *tiles;
  int32_t ntiles;
  const int32_t *brp, *vptr, *colidx;
  const uint8_t *masks;
  const double *vals, *x;
  double *y, *partial;
  double alpha, beta;
  int64_t nrows;
  int32_t stages, stage_bytes, stage_base;
  int32_t off_vals, off_col, off_mask, off_brp, off_vptr;
  int32_t cap_vals, cap_col, cap_mask, cap_ptr;  // section capacities in bytes
  int32_t xs_base;                               // byte offset of the x windows (BODY >= 2)
  uint32_t *err;
};

// Body variants of the staged kernel's consumers:
//   0: set-bit loop, x from global;  1: predicated loop over the c bits, x
//   from global;  2 / 3: like 0 / 1 with x staged per window in shared memory.
// x staging: a window covers kXsRounds rounds of block loads; every lane
// loads the x values of its share of columns of its own blocks (about 32
// independent loads per lane), then the window is computed from shared
// memory.  Per-panel stride is odd (in doubles) so the panels of a warp hit
// different banks.
constexpr int kXsDoubles = 1024;
constexpr int kXsPerConsumer = kXsDoubles + 32;

// A 16-byte aligned window covering elements [first, last) of `elem` bytes.
struct Span {
  int64_t lo;
  uint32_t bytes;
  int32_t off;
};
__device__ __forceinline__ Span span_of(int64_t first, int64_t last, int elem) {
  Span sp;
  int64_t b0 = first * elem, b1 = last * elem;
  sp.lo = b0 & ~(int64_t)15;
  int64_t hi = (b1 + 15) & ~(int64_t)15;
  sp.bytes = (b1 > b0) ? (uint32_t)(hi - sp.lo) : 0u;
  sp.off = (int32_t)((b0 - sp.lo) / elem);
  return sp;
}

template <int R, int C>
__device__ void producer(const StagedParams &P, uint8_t *stage0, uint64_t *full, uint64_t *empty,
                         int my_ntiles) {
  constexpr int MB = R * C / 8;
  const int lane = threadIdx.x & 31;
  const int S = P.stages;
  int issued = 0;
  bool abort = false;
  for (int base = 0; base < my_ntiles && !abort; base += 32) {
    const int kk = base + lane;
    Tile mine{0, 0, 0, 0, 0, 0, 0, 0};
    if (kk < my_ntiles) mine = P.tiles[blockIdx.x + (int64_t)kk * gridDim.x];
    const int nbatch = min(32, my_ntiles - base);
    for (int i = 0; i < nbatch; ++i) {
      const int k = base + i;
      const int s = k % S;
      const uint32_t ph = (uint32_t)(k / S) & 1u;
      const bool ok = __all_sync(kFull, mbar_wait(&empty[s], ph ^ 1u, kWaitBudget));
      if (!ok) {
        if (lane == 0) atomicOr(P.err, kErrProducerWait);
        abort = true;
        break;
      }
      Tile t;
      t.p0 = __shfl_sync(kFull, mine.p0, i);
      t.p1 = __shfl_sync(kFull, mine.p1, i);
      t.b0 = __shfl_sync(kFull, mine.b0, i);
      t.b1 = __shfl_sync(kFull, mine.b1, i);
      t.v0 = __shfl_sync(kFull, mine.v0, i);
      t.v1 = __shfl_sync(kFull, mine.v1, i);
      t.slot = __shfl_sync(kFull, mine.slot, i);
      t.mode = __shfl_sync(kFull, mine.mode, i);
      if (lane == 0) {
        uint8_t *st = stage0 + (size_t)s * P.stage_bytes;
        const bool segment = (t.mode & kSegment) != 0;
        Span sv = span_of(t.v0, t.v1, 8);
        Span sc = span_of(t.b0, t.b1, 4);
        Span sm = span_of(t.b0, t.b1, MB);
        Span sr{0, 0u, 0}, sp{0, 0u, 0};
        if (!segment) {
          sr = span_of(t.p0, (int64_t)t.p1 + 1, 4);
          sp = span_of(t.p0, (int64_t)t.p1 + 1, 4);
        }
        const bool fits = sv.bytes <= (uint32_t)P.cap_vals && sc.bytes <= (uint32_t)P.cap_col &&
                          sm.bytes <= (uint32_t)P.cap_mask && sr.bytes <= (uint32_t)P.cap_ptr &&
                          (segment || (t.p1 - t.p0) <= 32);
        StageHdr *h = reinterpret_cast<StageHdr *>(st);
        h->t = t;
        h->voff = sv.off;
        h->coff = sc.off;
        h->moff = sm.off;
        h->roff = sr.off;
        h->pvoff = sp.off;
        h->valid = fits ? 1 : 0;
        h->seq = k;
        if (!fits) {
          atomicOr(P.err, kErrTileTooLarge);
          mbar_arrive_expect_tx(&full[s], 0u);
        } else {
          mbar_arrive_expect_tx(&full[s], sv.bytes + sc.bytes + sm.bytes + sr.bytes + sp.bytes);
          if (sv.bytes)
            bulk_g2s(st + P.off_vals, reinterpret_cast<const uint8_t *>(P.vals) + sv.lo, sv.bytes,
                     &full[s]);
          if (sc.bytes)
            bulk_g2s(st + P.off_col, reinterpret_cast<const uint8_t *>(P.colidx) + sc.lo,
                     sc.bytes, &full[s]);
          if (sm.bytes)
            bulk_g2s(st + P.off_mask, P.masks + sm.lo, sm.bytes, &full[s]);
          if (sr.bytes)
            bulk_g2s(st + P.off_brp, reinterpret_cast<const uint8_t *>(P.brp) + sr.lo, sr.bytes,
                     &full[s]);
          if (sp.bytes)
            bulk_g2s(st + P.off_vptr, reinterpret_cast<const uint8_t *>(P.vptr) + sp.lo,
                     sp.bytes, &full[s]);
        }
      }
      ++issued;
      __syncwarp();
    }
  }
  // Do not leave while copies issued by this warp may still be landing in
  // shared memory: wait (bounded) for the last phase of every used stage.
  const int first = issued > S ? issued - S : 0;
  for (int k = first; k < issued; ++k) {
    const bool ok = __all_sync(kFull, mbar_wait(&full[k % S], (uint32_t)(k / S) & 1u, kWaitBudget));
    if (!ok) {
      if (lane == 0) atomicOr(P.err, kErrProducerWait);
      break;
    }
  }
}

template <int R, int C, int BODY>
__device__ void consumer(const StagedParams &P, uint8_t *stage0, uint64_t *full, uint64_t *empty,
                         int *counter, int my_ntiles, double *xs) {
  constexpr bool UNROLL = (BODY & 1) != 0;
  constexpr bool XS = BODY >= 2;
  constexpr int CPL = (C + R - 1) / R;  // columns staged per lane and block
  using MaskT = typename MaskType<R, C>::T;
  constexpr int LOG2R = Log2<R>::v;
  const int lane = threadIdx.x & 31;
  const int S = P.stages;
  const uint32_t cmask = (1u << C) - 1u;
  for (;;) {
    int k = 0;
    if (lane == 0) k = atomicAdd(counter, 1);
    k = __shfl_sync(kFull, k, 0);
    if (k >= my_ntiles) break;
    const int s = k % S;
    const uint8_t *st = stage0 + (size_t)s * P.stage_bytes;
    // 1. wait until the producer has stamped this stage with tile k (then the
    //    barrier is in tile k's phase), 2. wait for that phase to complete.
    bool ok = true;
    if (lane == 0) {
      const volatile int32_t *seq = &reinterpret_cast<const StageHdr *>(st)->seq;
      const long long t0 = clock64();
      while (*seq != k) {
        if (clock64() - t0 > kWaitBudget) {
          ok = false;
          break;
        }
      }
    }
    ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
    ok = ok && __all_sync(kFull, mbar_wait(&full[s], (uint32_t)(k / S) & 1u, kWaitBudget));
    if (!ok) {
      if (lane == 0) atomicOr(P.err, kErrConsumerWait);
      break;
    }
    const StageHdr h = *reinterpret_cast<const StageHdr *>(st);
    if (h.valid) {
      const Tile &t = h.t;
      const bool segment = (t.mode & kSegment) != 0;
      const int log2G = t.mode & 15;
      const int G = 1 << log2G;
      const int shift_j = LOG2R + log2G;
      const int g = lane & (G - 1);
      const int q = (lane >> log2G) & (R - 1);
      const int j = lane >> shift_j;
      const uint32_t row_low = (q == 0) ? 0u : ((1u << (q * C)) - 1u);
      const double *vs = reinterpret_cast<const double *>(st + P.off_vals) + h.voff;
      const int32_t *cs = reinterpret_cast<const int32_t *>(st + P.off_col) + h.coff;
      const MaskT *ms = reinterpret_cast<const MaskT *>(st + P.off_mask) + h.moff;
      bool pvalid;
      int32_t bl, bh, v;
      if (segment) {
        pvalid = (j == 0);
        bl = 0;
        bh = t.b1 - t.b0;
        v = 0;
      } else {
        const int32_t *rs = reinterpret_cast<const int32_t *>(st + P.off_brp) + h.roff;
        const int32_t *ps = reinterpret_cast<const int32_t *>(st + P.off_vptr) + h.pvoff;
        pvalid = j < (t.p1 - t.p0);
        bl = pvalid ? rs[j] - t.b0 : 0;
        bh = pvalid ? rs[j + 1] - t.b0 : 0;
        v = pvalid ? ps[j] - t.v0 : 0;
      }
      const int32_t nbp = bh - bl;
      const int32_t maxnb = __reduce_max_sync(kFull, nbp);
      double acc = 0.0;
      if (!XS) {
        for (int32_t it = 0; it < maxnb; it += G) {
          const int32_t idx = it + g;
          const bool valid = idx < nbp;
          const int32_t b = bl + idx;
          const uint32_t m = valid ? (uint32_t)ms[b] : 0u;
          const int32_t col = valid ? cs[b] : 0;
          const int pc = __popc(m);
          int total;
          const int excl = group_scan(pc, g, G, &total);
          const int32_t off = v + excl + __popc(m & row_low);
          acc = row_block<C, UNROLL, double, double>(acc, (m >> (q * C)) & cmask, vs + off,
                                                     P.x + col);
          v += total;
        }
      } else {
        // rounds per window: the window holds 32 * W / R blocks of C doubles
        constexpr int W = (kXsDoubles * R) / (32 * C);
        const int xstride = W * G * C + 1;
        double *xw = xs + j * xstride;
        for (int32_t it0 = 0; it0 < maxnb; it0 += W * G) {
          for (int w = 0; w < W; ++w) {
            const int32_t idx = it0 + w * G + g;
            if (it0 + w * G >= maxnb) break;
            const bool valid = idx < nbp;
            const int32_t b = bl + idx;
            const uint32_t um = valid ? union_mask<R, C>((uint32_t)ms[b]) : 0u;
            const int32_t col = valid ? cs[b] : 0;
            double *dst = xw + (w * G + g) * C;
#pragma unroll
            for (int t = 0; t < CPL; ++t) {
              const int k = q * CPL + t;
              if (k < C && ((um >> k) & 1u)) dst[k] = __ldg(P.x + col + k);
            }
          }
          __syncwarp();
          for (int w = 0; w < W; ++w) {
            if (it0 + w * G >= maxnb) break;
            const int32_t idx = it0 + w * G + g;
            const bool valid = idx < nbp;
            const int32_t b = bl + idx;
            const uint32_t m = valid ? (uint32_t)ms[b] : 0u;
            const int pc = __popc(m);
            int total;
            const int excl = group_scan(pc, g, G, &total);
            const int32_t off = v + excl + __popc(m & row_low);
            acc = row_block_xs<C, UNROLL>(acc, (m >> (q * C)) & cmask, vs + off,
                                          xw + (w * G + g) * C);
            v += total;
          }
          __syncwarp();
        }
      }
      acc = group_sum(acc, G);
      if (pvalid && g == 0) {
        if (t.mode & kPartial) {
          P.partial[(int64_t)t.slot * R + q] = acc;
        } else {
          const int64_t row = ((int64_t)t.p0 + j) * R + q;
          if (row < P.nrows) {
            double out = P.alpha * acc;
            if (P.beta != 0.0) out = fma(P.beta, P.y[row], out);
            P.y[row] = out;
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <int R, int C, int BODY>
__global__ void __launch_bounds__(32 * 17, 1) k_spmv_staged(const StagedParams P) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);
  uint64_t *empty = full + P.stages;
  int *counter = reinterpret_cast<int *>(empty + P.stages);
  uint8_t *stage0 = smem + P.stage_base;
  const int warp = threadIdx.x >> 5;
  const int my_ntiles =
      (P.ntiles > (int)blockIdx.x) ? (P.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      reinterpret_cast<StageHdr *>(stage0 + (size_t)s * P.stage_bytes)->seq = -1;
    }
    *counter = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (warp == 0)
    producer<R, C>(P, stage0, full, empty, my_ntiles);
  else
    consumer<R, C, BODY>(P, stage0, full, empty, counter, my_ntiles,
                         reinterpret_cast<double *>(smem + P.xs_base) +
                             (size_t)(warp - 1) * kXsPerConsumer);
}

// y rows of panels that were cut into pieces.  One warp per split panel:
// the panel's partials are R values per slot, slot-major, so lane j adds
// elements j, j + 32, ... (all of row j % R) and the lanes of each row are
// then added, a fixed order for every launch.
template <int R, typename AT>
__global__ void k_fixup(int64_t nlong, const int32_t *long_panels, const int32_t *long_slots,
                        const AT *partial, AT *y, Scale<AT> sc, int64_t nrows) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < nlong; l += nw) {
    const int64_t first = (int64_t)long_slots[2 * l] * R + lane;
    const int64_t end = (int64_t)long_slots[2 * l + 1] * R;
    AT acc = first < end ? strided_sum(partial + first, (end - first + 31) / 32, 32) : (AT)0;
    for (int o = 16; o >= R; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane < R) {
      const int64_t row = (int64_t)long_panels[l] * R + lane;
      if (row < nrows) put_row(sc, y, row, acc);
    }
  }
}

int num_sms() { return device_sm_count(); }

// Blocks of 256 threads for a fixup over n split panels (one warp each).
int fixup_blocks(int64_t n) {
  return (int)std::min<int64_t>((n + 7) / 8, (int64_t)num_sms() * 8);
}

template <int R, int C, int BODY>
cudaError_t launch_staged(const spc5_matrix *A, const double *x, double *y, double alpha,
                          double beta, cudaStream_t s, double *partial) {
  constexpr int MB = R * C / 8;
  auto r16 = [](int v) { return (v + 15) / 16 * 16; };
  StagedParams P;
  P.tiles = A->tiles;
  P.ntiles = (int32_t)A->ntiles;
  P.brp = A->block_rowptr;
  P.vptr = A->panel_vptr;
  P.colidx = A->block_colidx;
  P.masks = reinterpret_cast<const uint8_t *>(A->masks);
  P.vals = reinterpret_cast<const double *>(A->values);
  P.x = x;
  P.y = y;
  P.partial = partial;
  P.alpha = alpha;
  P.beta = beta;
  P.nrows = A->nrows;
  P.stages = A->stages;
  P.cap_vals = r16(A->vcap * 8 + 16);
  P.cap_col = r16(A->bcap * 4 + 16);
  P.cap_mask = r16(A->bcap * MB + 16);
  P.cap_ptr = r16((A->group_panels + 1) * 4 + 16);
  P.off_vals = 64;
  P.off_col = P.off_vals + P.cap_vals;
  P.off_mask = P.off_col + P.cap_col;
  P.off_brp = P.off_mask + P.cap_mask;
  P.off_vptr = P.off_brp + P.cap_ptr;
  P.stage_bytes = P.off_vptr + P.cap_ptr;
  P.stage_base = (16 * A->stages + 16 + 127) / 128 * 128;
  P.err = A->dev_error;
  P.xs_base = P.stage_base + A->stages * P.stage_bytes;
  const size_t smem = (size_t)P.xs_base +
                      (BODY >= 2 ? (size_t)A->consumers * kXsPerConsumer * sizeof(double) : 0);
  // the attribute belongs to the device's context: remember it per device
  static size_t configured[kMaxDevices] = {};  // per instantiation
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices || smem > configured[dev]) {
    e = cudaFuncSetAttribute(k_spmv_staged<R, C, BODY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) configured[dev] = smem;
  }
  if (A->ntiles > 0) {
    int grid = (int)std::min<int64_t>(num_sms(), A->ntiles);
    k_spmv_staged<R, C, BODY><<<grid, 32 * (1 + A->consumers), smem, s>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (A->nlong > 0) {
    const int blocks = fixup_blocks(A->nlong);
    k_fixup<R, double><<<blocks, 256, 0, s>>>(A->nlong, A->long_panels, A->long_slots, partial,
                                              y, make_scale<double>(alpha, beta), A->nrows);
    e = cudaGetLastError();
  }
  return e;
}

template <int R, int C, int BODY, typename VT, typename AT>
cudaError_t launch_direct(const spc5_matrix *A, const AT *x, AT *y, double alpha, double beta,
                          cudaStream_t s, AT *partial, uint32_t *sched) {
  using MaskT = typename MaskType<R, C>::T;
  cudaError_t e = cudaSuccess;
  if (A->ntiles > 0) {
    const int warps_per_block = TileThreads<BODY>::v / 32;
    int64_t blocks = (A->ntiles + warps_per_block - 1) / warps_per_block;
    const int64_t resident = (int64_t)num_sms() * TileBlocksPerSM<BODY>::v;
    if (blocks > resident) blocks = resident;
    if (A->dynamic)
      k_spmv_tiles<R, C, BODY, true, VT, AT><<<(unsigned)blocks, TileThreads<BODY>::v, 0, s>>>(
          A->tiles, A->ntiles, sched, A->block_rowptr, A->panel_vptr, A->block_colidx,
          (const MaskT *)A->masks, (const VT *)A->values, x, y, partial,
          make_scale<AT>(alpha, beta), A->nrows);
    else
      k_spmv_tiles<R, C, BODY, false, VT, AT><<<(unsigned)blocks, TileThreads<BODY>::v, 0, s>>>(
          A->tiles, A->ntiles, sched, A->block_rowptr, A->panel_vptr, A->block_colidx,
          (const MaskT *)A->masks, (const VT *)A->values, x, y, partial,
          make_scale<AT>(alpha, beta), A->nrows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (A->nlong > 0) {
    const int fblocks = fixup_blocks(A->nlong);
    k_fixup<R, AT><<<fblocks, 256, 0, s>>>(A->nlong, A->long_panels, A->long_slots, partial, y,
                                           make_scale<AT>(alpha, beta), A->nrows);
    e = cudaGetLastError();
  }
  return e;
}

template <int R, int C, typename VT, typename AT>
cudaError_t launch_flat(const spc5_matrix *A, const AT *x, AT *y, double alpha, double beta,
                        cudaStream_t s, AT *partial, uint32_t *sched) {
  using MaskT = typename MaskType<R, C>::T;
  cudaError_t e = cudaSuccess;
  if (A->fntiles > 0) {
    const int warps_per_block = kDirectThreads / 32;
    int64_t blocks = (A->fntiles + warps_per_block - 1) / warps_per_block;
    const int64_t resident = (int64_t)num_sms() * FlatBlocksPerSM<R>::v;
    if (blocks > resident) blocks = resident;
    k_spmv_flat<R, C, VT, AT><<<(unsigned)blocks, kDirectThreads, 0, s>>>(
        A->ftiles, (int32_t)A->fntiles, sched, A->block_rowptr, A->block_colidx,
        (const MaskT *)A->masks, (const VT *)A->values, x, y, partial,
        make_scale<AT>(alpha, beta), A->nrows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (A->fnlong > 0) {
    const int fblocks = fixup_blocks(A->fnlong);
    k_fixup<R, AT><<<fblocks, 256, 0, s>>>(A->fnlong, A->flong_panels, A->flong_slots, partial,
                                           y, make_scale<AT>(alpha, beta), A->nrows);
    e = cudaGetLastError();
  }
  return e;
}

template <int R, int C, typename VT, typename AT>
cudaError_t launch_vflat(const spc5_matrix *A, const AT *x, AT *y, double alpha, double beta,
                         cudaStream_t s, AT *partial, uint32_t *sched) {
  using MaskT = typename MaskType<R, C>::T;
  cudaError_t e = cudaSuccess;
  if (A->fntiles > 0) {
    const int warps_per_block = kDirectThreads / 32;
    int64_t blocks = (A->fntiles + warps_per_block - 1) / warps_per_block;
    const int64_t resident = (int64_t)num_sms() * VFlatBlocksPerSM<R>::v;
    if (blocks > resident) blocks = resident;
    k_spmv_vflat<R, C, VT, AT><<<(unsigned)blocks, kDirectThreads, 0, s>>>(
        A->ftiles, (int32_t)A->fntiles, sched, A->block_rowptr, A->block_colidx,
        (const MaskT *)A->masks, (const VT *)A->values, x, y, partial,
        make_scale<AT>(alpha, beta), A->nrows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (A->fnlong > 0) {
    const int fblocks = fixup_blocks(A->fnlong);
    k_fixup<R, AT><<<fblocks, 256, 0, s>>>(A->fnlong, A->flong_panels, A->flong_slots, partial,
                                           y, make_scale<AT>(alpha, beta), A->nrows);
    e = cudaGetLastError();
  }
  return e;
}

template <int R, int C, typename VT, typename AT>
cudaError_t launch_expand(const spc5_matrix *A, const AT *x, AT *y, double alpha, double beta,
                          cudaStream_t s, AT *partial, uint32_t *sched) {
  using MaskT = typename MaskType<R, C>::T;
  cudaError_t e = cudaSuccess;
  if (A->fntiles > 0) {
    int64_t blocks = (A->fntiles + kExpandWarps - 1) / kExpandWarps;
    const int64_t resident = (int64_t)num_sms() * kExpandBlocksPerSM;
    if (blocks > resident) blocks = resident;
    k_spmv_expand<R, C, VT, AT><<<(unsigned)blocks, 32 * kExpandWarps, 0, s>>>(
        A->ftiles, (int32_t)A->fntiles, sched, A->block_rowptr, A->block_colidx,
        (const MaskT *)A->masks, (const VT *)A->values, x, y, partial,
        make_scale<AT>(alpha, beta), A->nrows, A->frowoff, A->npanels);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (A->fnlong > 0) {
    const int fblocks = fixup_blocks(A->fnlong);
    k_fixup<R, AT><<<fblocks, 256, 0, s>>>(A->fnlong, A->flong_panels, A->flong_slots, partial,
                                           y, make_scale<AT>(alpha, beta), A->nrows);
    e = cudaGetLastError();
  }
  return e;
}

template <int R, int C>
cudaError_t launch_row_starts(spc5_matrix *A, cudaStream_t s) {
  using MaskT = typename MaskType<R, C>::T;
  if (A->fntiles == 0) return cudaSuccess;
  int64_t blocks = (A->fntiles + kExpandWarps - 1) / kExpandWarps;
  if (blocks > 65536) blocks = 65536;
  k_ex_row_starts<R, C><<<(unsigned)blocks, 32 * kExpandWarps, 0, s>>>(
      A->ftiles, (int32_t)A->fntiles, A->npanels, A->block_rowptr, (const MaskT *)A->masks,
      A->frowoff);
  return cudaGetLastError();
}

template <int R, int C, typename VT, typename AT>
cudaError_t launch_direct_body(const spc5_matrix *A, const void *x, void *y, double alpha,
                               double beta, cudaStream_t s, void *partial, uint32_t *sched) {
  const AT *xa = (const AT *)x;
  AT *ya = (AT *)y, *pa = (AT *)partial;
  switch (A->body) {
    case 1: return launch_direct<R, C, 1, VT, AT>(A, xa, ya, alpha, beta, s, pa, sched);
    case 2: return launch_direct<R, C, 2, VT, AT>(A, xa, ya, alpha, beta, s, pa, sched);
    case 3: return launch_direct<R, C, 3, VT, AT>(A, xa, ya, alpha, beta, s, pa, sched);
    case 4: return launch_direct<R, C, 4, VT, AT>(A, xa, ya, alpha, beta, s, pa, sched);
    case 5: return launch_direct<R, C, 5, VT, AT>(A, xa, ya, alpha, beta, s, pa, sched);
    case 6: return launch_direct<R, C, 6, VT, AT>(A, xa, ya, alpha, beta, s, pa, sched);
    case 7: return launch_direct<R, C, 7, VT, AT>(A, xa, ya, alpha, beta, s, pa, sched);
    default: return launch_direct<R, C, 0, VT, AT>(A, xa, ya, alpha, beta, s, pa, sched);
  }
}

template <int R, int C>
cudaError_t launch(const spc5_matrix *A, const void *x, void *y, double alpha, double beta,
                   cudaStream_t s, void *partial, uint32_t *sched) {
  if (A->flat == 1) {
    if (A->value_dtype == SPC5_F32)
      return launch_flat<R, C, float, float>(A, (const float *)x, (float *)y, alpha, beta, s,
                                             (float *)partial, sched);
    if (A->value_dtype == SPC5_BF16)
      return launch_flat<R, C, uint16_t, float>(A, (const float *)x, (float *)y, alpha, beta, s,
                                                (float *)partial, sched);
    return launch_flat<R, C, double, double>(A, (const double *)x, (double *)y, alpha, beta, s,
                                             (double *)partial, sched);
  }
  if (A->flat == 3) {
    if (A->value_dtype == SPC5_F32)
      return launch_vflat<R, C, float, float>(A, (const float *)x, (float *)y, alpha, beta, s,
                                              (float *)partial, sched);
    if (A->value_dtype == SPC5_BF16)
      return launch_vflat<R, C, uint16_t, float>(A, (const float *)x, (float *)y, alpha, beta,
                                                 s, (float *)partial, sched);
    return launch_vflat<R, C, double, double>(A, (const double *)x, (double *)y, alpha, beta,
                                              s, (double *)partial, sched);
  }
  if (A->flat == 2) {
    if (A->value_dtype == SPC5_F32)
      return launch_expand<R, C, float, float>(A, (const float *)x, (float *)y, alpha, beta, s,
                                               (float *)partial, sched);
    if (A->value_dtype == SPC5_BF16)
      return launch_expand<R, C, uint16_t, float>(A, (const float *)x, (float *)y, alpha, beta,
                                                  s, (float *)partial, sched);
    return launch_expand<R, C, double, double>(A, (const double *)x, (double *)y, alpha, beta, s,
                                               (double *)partial, sched);
  }
  if (A->value_dtype == SPC5_F32)
    return launch_direct_body<R, C, float, float>(A, x, y, alpha, beta, s, partial, sched);
  if (A->value_dtype == SPC5_BF16)
    return launch_direct_body<R, C, uint16_t, float>(A, x, y, alpha, beta, s, partial, sched);
  if (A->kernel == 0)
    return launch_direct_body<R, C, double, double>(A, x, y, alpha, beta, s, partial, sched);
  const double *xd = (const double *)x;
  double *yd = (double *)y, *pd = (double *)partial;
  switch (A->body) {
    case 0: return launch_staged<R, C, 0>(A, xd, yd, alpha, beta, s, pd);
    case 1: return launch_staged<R, C, 1>(A, xd, yd, alpha, beta, s, pd);
    case 2: return launch_staged<R, C, 2>(A, xd, yd, alpha, beta, s, pd);
    default: return launch_staged<R, C, 3>(A, xd, yd, alpha, beta, s, pd);
  }
}

}  // namespace

int spmv_launches(const spc5_matrix *A) {
  if (A->nrows == 0) return 0;
  const int sc = A->hybrid ? (A->sntiles > 0 ? 1 : 0) + (A->snlong > 0 ? 1 : 0) : 0;
  if (A->flat) return (A->fntiles > 0 ? 1 : 0) + (A->fnlong > 0 ? 1 : 0) + sc;
  return (A->ntiles > 0 ? 1 : 0) + (A->nlong > 0 ? 1 : 0) + sc;
}

int64_t spmv_pieces(const spc5_matrix *A) { return A->flat ? A->fnpieces : A->npieces; }

spc5_status expand_row_starts(spc5_matrix *A, cudaStream_t s) {
  cudaError_t e;
  switch (A->r * 100 + A->c) {
    case 108: e = launch_row_starts<1, 8>(A, s); break;
    case 204: e = launch_row_starts<2, 4>(A, s); break;
    case 208: e = launch_row_starts<2, 8>(A, s); break;
    case 404: e = launch_row_starts<4, 4>(A, s); break;
    case 408: e = launch_row_starts<4, 8>(A, s); break;
    case 804: e = launch_row_starts<8, 4>(A, s); break;
    default:
      set_error("unsupported block shape");
      return SPC5_EUNSUPPORTED_RC;
  }
  return cuda_check(e, "expanded tiles' row starts");
}

spc5_status spmv_device_scratch(const spc5_matrix *A, const void *x, void *y, double alpha,
                                double beta, cudaStream_t s, void *partial, uint32_t *sched) {
  if (A->nrows == 0) return SPC5_OK;
  cudaError_t e;
  switch (A->r * 100 + A->c) {
    case 108: e = launch<1, 8>(A, x, y, alpha, beta, s, partial, sched); break;
    case 204: e = launch<2, 4>(A, x, y, alpha, beta, s, partial, sched); break;
    case 208: e = launch<2, 8>(A, x, y, alpha, beta, s, partial, sched); break;
    case 404: e = launch<4, 4>(A, x, y, alpha, beta, s, partial, sched); break;
    case 408: e = launch<4, 8>(A, x, y, alpha, beta, s, partial, sched); break;
    case 804: e = launch<8, 4>(A, x, y, alpha, beta, s, partial, sched); break;
    default:
      set_error("unsupported block shape");
      return SPC5_EUNSUPPORTED_RC;
  }
  return cuda_check(e, "spmv launch");
}

namespace {
template <typename VT, typename AT>
cudaError_t launch_scalars(const spc5_matrix *A, const AT *x, AT *y, double alpha,
                           cudaStream_t s, AT *partial, uint32_t *sched) {
  cudaError_t e = cudaSuccess;
  if (A->sntiles > 0) {
    int64_t blocks = (A->sntiles + kExpandWarps - 1) / kExpandWarps;
    const int64_t resident = (int64_t)num_sms() * 16;
    if (blocks > resident) blocks = resident;
    k_spmv_scalars<VT, AT><<<(unsigned)blocks, 32 * kExpandWarps, 0, s>>>(
        A->stiles, (int32_t)A->sntiles, sched, A->s_rowptr, A->s_colidx, (const VT *)A->s_vals,
        x, y, partial, (AT)alpha);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (A->snlong > 0) {
    const int blocks = fixup_blocks(A->snlong);
    k_fixup_add<AT><<<blocks, 256, 0, s>>>(A->snlong, A->slong_rows, A->slong_slots, partial, y,
                                           (AT)alpha);
    e = cudaGetLastError();
  }
  return e;
}
}  // namespace

spc5_status spmv_scalars(const spc5_matrix *A, const void *x, void *y, double alpha,
                         cudaStream_t s, void *partial, uint32_t *sched) {
  if (!A->hybrid || A->nrows == 0 || alpha == 0.0) return SPC5_OK;
  cudaError_t e;
  if (A->value_dtype == SPC5_F64)
    e = launch_scalars<double, double>(A, (const double *)x, (double *)y, alpha, s,
                                       (double *)partial, sched);
  else if (A->value_dtype == SPC5_F32)
    e = launch_scalars<float, float>(A, (const float *)x, (float *)y, alpha, s,
                                     (float *)partial, sched);
  else
    e = launch_scalars<uint16_t, float>(A, (const float *)x, (float *)y, alpha, s,
                                        (float *)partial, sched);
  return cuda_check(e, "scalar spmv launch");
}

spc5_status spmv_device(const spc5_matrix *A, const void *x, void *y, double alpha, double beta,
                        cudaStream_t s) {
  spc5_status st = spmv_device_scratch(A, x, y, alpha, beta, s,
                                       A->flat ? A->fpartial : A->partial, A->fsched);
  if (st != SPC5_OK || !A->hybrid) return st;
  return spmv_scalars(A, x, y, alpha, s, A->spartial, A->fsched);
}

}  // namespace spc5
