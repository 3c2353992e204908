// Block-balanced tile body (plan 1), shared by the standalone kernel
// (spc5_spmv.cu) and the batched kernel (spc5_batch.cu), with the row-update
// helpers it uses.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spc5_internal.h"

namespace spc5 {
namespace {

constexpr unsigned kFlatFull = 0xffffffffu;

// y = alpha * acc + beta * y with the FP64 operations the arguments need:
// mode 0 (alpha = 1, beta = 0) stores acc, mode 1 (beta = 0) scales it,
// mode 2 reads y.  On GB300 every FP64 instruction, even a compare, takes a
// slot of the FP64 pipe that the products need, so the mode is decided on
// the host.
template <typename AT>
struct Scale {
  AT alpha, beta;
  int mode;
};

template <typename AT>
Scale<AT> make_scale(double alpha, double beta) {
  return Scale<AT>{(AT)alpha, (AT)beta, beta != 0.0 ? 2 : (alpha != 1.0 ? 1 : 0)};
}

template <typename AT>
__device__ __forceinline__ void put_row(const Scale<AT> &sc, AT *y, int64_t row, AT acc) {
  if (sc.mode == 0)
    y[row] = acc;
  else if (sc.mode == 1)
    y[row] = sc.alpha * acc;
  else
    y[row] = fma(sc.beta, y[row], sc.alpha * acc);
}

template <typename AT>
__device__ __forceinline__ void put_empty_row(const Scale<AT> &sc, AT *y, int64_t row) {
  y[row] = (sc.mode == 2) ? sc.beta * y[row] : (AT)0;
}

// -------------------------------------------------------------- flat kernel --

// Block-balanced kernel for matrices whose panels hold very different
// numbers of blocks (power-law rows): with lanes owning rows, a warp waits
// for its longest row while the other lanes idle.  Here the blocks of a tile
// (consecutive whole panels) are dealt to the lanes four consecutive blocks
// per lane per round, so every lane has work whatever the row lengths:
//   - the value offset of a lane's blocks is the running offset plus the
//     exclusive warp scan of the lanes' popcounts (Algorithm 1's idxVal);
//   - a lane accumulates its blocks' r row sums with one FMA per set bit
//     (x through L1/L2);
//   - the panels ending inside the round are found from block_rowptr (a
//     window of up to 32 panels per step, marked in a 128-bit mask by warp
//     OR-reductions, their ids passed to the lanes through shared memory);
//   - a lane writes the rows of the panels that start and end among its own
//     blocks (one write per row, as in Section 3.2); the partial sums of
//     panels cut between lanes are completed by a segmented warp scan of the
//     lanes' last partial sums, and the panel still open at the end of the
//     round carries its sums into the next round.
// On GB300 every FP64 instruction costs a 16-cycle slot of the FP64 pipe
// whatever its active lanes: the scan's adds are paid once per 128 blocks.
// A piece of a long panel (mode & kPartial) holds one panel only: the lanes
// keep private row sums over all rounds, reduce them with shuffles at the
// end and write them to the partial buffer for the fixup kernel.
// Warps take tiles from a counter (dynamic scheduling); the last warp to
// finish resets the counter for the next launch.
constexpr int kFlatKB = 4;                // blocks per lane per round
constexpr int kFlatRound = 32 * kFlatKB;  // blocks per round

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int *total) {
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFlatFull, incl, o);
    if (lane >= o) incl += t;
  }
  *total = __shfl_sync(kFlatFull, incl, 31);
  return incl - v;
}

template <typename AT>
__device__ __forceinline__ AT warp_sum(AT v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFlatFull, v, o);
  return v;
}


// Adds the block's products to s[q] (q < R): values packed row by row,
// ascending bit within a row (Algorithm 1's order).  One loop over all the
// block's set bits, the row's sum chosen by selects, so a warp issues as
// many FMA instructions as its fullest block has values (a loop per row
// would issue, for every row, as many as the block fullest in that row).
template <int R, int C, typename VT, typename AT>
__device__ __forceinline__ void block_rows(AT (&s)[R], uint32_t m, const VT *__restrict__ vals,
                                           const AT *__restrict__ xp) {
  constexpr int LOG2C = C == 8 ? 3 : 2;
  int o = 0;
  if constexpr (R == 1) {
    AT acc = s[0];
    while (m) {
      const int k = __ffs(m) - 1;
      m &= m - 1u;
      acc = fma((AT)widen(vals[o]), __ldg(xp + k), acc);
      ++o;
    }
    s[0] = acc;
    return;
  }
  while (m) {
    const int kf = __ffs(m) - 1;
    m &= m - 1u;
    const int q = kf >> LOG2C;
    AT t = s[0];
#pragma unroll
    for (int qq = 1; qq < R; ++qq) t = (q == qq) ? s[qq] : t;
    t = fma((AT)widen(vals[o]), __ldg(xp + (kf & (C - 1))), t);
#pragma unroll
    for (int qq = 0; qq < R; ++qq) s[qq] = (q == qq) ? t : s[qq];
    ++o;
  }
}

// A piece of a long panel (block-balanced plans): the lanes keep private row
// sums over all rounds of four blocks per lane, reduce them with shuffles
// and write them to the partial buffer for the fixup kernel.
template <int R, int C, typename VT, typename AT>
__device__ __forceinline__ void flat_piece(const Tile &cur, int lane,
                                           const int32_t *__restrict__ block_colidx,
                                           const typename MaskType<R, C>::T *__restrict__ masks,
                                           const VT *__restrict__ vals,
                                           const AT *__restrict__ x, AT *__restrict__ partial) {
  int32_t v = cur.v0;
  AT s[R];
#pragma unroll
  for (int q = 0; q < R; ++q) s[q] = 0;
  for (int32_t base = cur.b0; base < cur.b1; base += kFlatRound) {
    uint32_t m[kFlatKB];
    int32_t cb[kFlatKB];
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < kFlatKB; ++i) {
      const int32_t b = base + kFlatKB * lane + i;
      const bool ok = b < cur.b1;
      m[i] = ok ? (uint32_t)masks[b] : 0u;
      cb[i] = ok ? block_colidx[b] : 0;
      cnt += __popc(m[i]);
    }
    int total;
    int32_t off = v + warp_excl_scan(cnt, lane, &total);
    v += total;
#pragma unroll
    for (int i = 0; i < kFlatKB; ++i) {
      block_rows<R, C>(s, m[i], vals + off, x + cb[i]);
      off += __popc(m[i]);
    }
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const AT tot = warp_sum(s[q]);
    if (lane == q) partial[(int64_t)cur.slot * R + q] = tot;
  }
}

// Rows of a tile's empty panels (block-balanced plans).
template <int R, typename AT>
__device__ __forceinline__ void flat_empty_rows(const Tile &cur, int lane,
                                                const int32_t *__restrict__ brp, AT *y,
                                                const Scale<AT> &sc, int64_t nrows) {
  for (int32_t p = cur.p0 + lane; p < cur.p1; p += 32) {
    if (brp[p] == brp[p + 1]) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int64_t row = (int64_t)p * R + q;
        if (row < nrows) put_empty_row(sc, y, row);
      }
    }
  }
}


// One block-balanced tile: whole panels [p0, p1) whose blocks [b0, b1) are
// dealt to the lanes in rounds, or (mode & kPartial) a piece of one long
// panel.  pid: the warp's kFlatRound ints of shared memory.
template <int R, int C, typename VT, typename AT>
__device__ __forceinline__ void flat_tile(const Tile &cur, int lane, int32_t *pid,
                                          const int32_t *__restrict__ brp,
                                          const int32_t *__restrict__ block_colidx,
                                          const typename MaskType<R, C>::T *__restrict__ masks,
                                          const VT *__restrict__ vals, const AT *__restrict__ x,
                                          AT *__restrict__ y, AT *__restrict__ partial,
                                          const Scale<AT> &sc, int64_t nrows) {
  int32_t v = cur.v0;
  if (cur.mode & kPartial) {
    flat_piece<R, C>(cur, lane, block_colidx, masks, vals, x, partial);
  } else {
    flat_empty_rows<R>(cur, lane, brp, y, sc, nrows);
    AT carry = 0;       // lane q < R: row q's sum of the panel still open
    bool open = false;  // a panel continues from the previous round
    int32_t pcur = cur.p0;
    for (int32_t base = cur.b0; base < cur.b1; base += kFlatRound) {
      const int32_t lim = (base + kFlatRound < cur.b1) ? base + kFlatRound : cur.b1;
      uint32_t m[kFlatKB];
      int32_t cb[kFlatKB];
      int cnt = 0;
#pragma unroll
      for (int i = 0; i < kFlatKB; ++i) {
        const int32_t b = base + kFlatKB * lane + i;
        const bool ok = b < lim;
        m[i] = ok ? (uint32_t)masks[b] : 0u;
        cb[i] = ok ? block_colidx[b] : 0;
        cnt += __popc(m[i]);
      }
      int total;
      int32_t off = v + warp_excl_scan(cnt, lane, &total);
      v += total;
      // panels whose last block lies in [base, lim): bit (end - 1 - base)
      uint32_t e0 = 0u, e1 = 0u, e2 = 0u, e3 = 0u;
      for (int32_t w = pcur;; w += 32) {
        const int32_t p = w + lane;
        const bool in = p < cur.p1;
        const int32_t st = in ? brp[p] : 0;
        const int32_t en = in ? brp[p + 1] : 0;
        const bool mark = in && en > st && en > base && en <= lim;
        const int pos = mark ? en - 1 - base : 0;
        if (mark) pid[pos] = p;
        const uint32_t bit = mark ? (1u << (pos & 31)) : 0u;
        const int wd = pos >> 5;
        e0 |= __reduce_or_sync(kFlatFull, wd == 0 ? bit : 0u);
        e1 |= __reduce_or_sync(kFlatFull, wd == 1 ? bit : 0u);
        e2 |= __reduce_or_sync(kFlatFull, wd == 2 ? bit : 0u);
        e3 |= __reduce_or_sync(kFlatFull, wd == 3 ? bit : 0u);
        const unsigned beyond = __ballot_sync(kFlatFull, !in || en > lim);
        if (beyond) {
          pcur = w + __ffs(beyond) - 1;
          break;
        }
      }
      __syncwarp();
      auto endbit = [&](int pos) -> bool {
        const int wd = pos >> 5;
        const uint32_t e = wd == 0 ? e0 : (wd == 1 ? e1 : (wd == 2 ? e2 : e3));
        return (e >> (pos & 31)) & 1u;
      };
      uint32_t ef = 0u;  // the lane's blocks that end a panel
#pragma unroll
      for (int i = 0; i < kFlatKB; ++i) ef |= (endbit(kFlatKB * lane + i) ? 1u : 0u) << i;
      // does the lane's first block start a panel?
      bool fresh = (lane == 0) ? !open : endbit(kFlatKB * lane - 1);
      // lane 0 starts from the sums of the panel still open (0 if none),
      // so carrying them costs no adds
      AT acc[R], head[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const AT cq = __shfl_sync(kFlatFull, carry, q);
        acc[q] = lane == 0 ? cq : (AT)0;
        head[q] = 0;
      }
      bool has_head = false;
      int32_t head_pid = 0;
      // block i was the lane's last block of a panel: write the panel's rows
      // if it started here, else keep them as the head for the scan
      auto end_block = [&](int i) {
        if ((ef >> i) & 1u) {
          const int64_t p = pid[kFlatKB * lane + i];
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
        }
      };
      if (R <= 2) {
#pragma unroll
        for (int i = 0; i < kFlatKB; ++i) {
          block_rows<R, C>(acc, m[i], vals + off, x + cb[i]);
          off += __popc(m[i]);
          end_block(i);
        }
      } else {
        // one FMA per trip over all the set bits of the lane's blocks, so
        // a warp issues as many FMA instructions as its fullest lane has
        // values (blocks hold at least one value; the round's padding
        // blocks hold none and end no panel); for r <= 2 the loop per
        // block measured faster
        const int trips = __reduce_max_sync(kFlatFull, cnt);
        int i = 0;
        uint32_t mc = m[0];
        int32_t cc = cb[0];
        for (int t = 0; t < trips; ++t) {
          while (mc == 0u && i < kFlatKB - 1) {
            end_block(i);
            ++i;
#pragma unroll
            for (int j = 1; j < kFlatKB; ++j) {
              mc = (i == j) ? m[j] : mc;
              cc = (i == j) ? cb[j] : cc;
            }
          }
          if (mc) {
            constexpr int LOG2C = C == 8 ? 3 : 2;
            const int kf = __ffs(mc) - 1;
            mc &= mc - 1u;
            const int q = kf >> LOG2C;
            AT tq = acc[0];
#pragma unroll
            for (int qq = 1; qq < R; ++qq) tq = (q == qq) ? acc[qq] : tq;
            tq = fma((AT)widen(vals[off]), __ldg(x + cc + (kf & (C - 1))), tq);
#pragma unroll
            for (int qq = 0; qq < R; ++qq) acc[qq] = (q == qq) ? tq : acc[qq];
            ++off;
          }
        }
        end_block(i);
      }
      // segmented scan of the lanes' last partial sums: lane adds lane - o
      // when no lane in (lane - o, lane] ends a panel; once no lane can,
      // no longer step can either
      const uint32_t endl = __ballot_sync(kFlatFull, ef != 0u);
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const bool same =
            lane >= o && ((endl >> (lane - o + 1)) & ((1u << o) - 1u)) == 0u;
        if (!__any_sync(kFlatFull, same)) break;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const AT tq = __shfl_up_sync(kFlatFull, acc[q], o);
          if (same) acc[q] += tq;
        }
      }
      // panels cut between lanes: the head plus the scanned partial before
      // it (lane 0's head already holds the open panel's sums)
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const AT cin = __shfl_up_sync(kFlatFull, acc[q], 1);
        if (has_head) {
          const int64_t row = (int64_t)head_pid * R + q;
          if (row < nrows) put_row(sc, y, row, lane == 0 ? head[q] : head[q] + cin);
        }
      }
      // the panel open at the end of the round
      const int lastpos = lim - 1 - base;
      open = !endbit(lastpos);
      const int ll = lastpos / kFlatKB;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const AT sl = __shfl_sync(kFlatFull, acc[q], ll);
        if (lane == q) carry = open ? sl : (AT)0;
      }
      __syncwarp();
    }
  }
}

}  // namespace
}  // namespace spc5
