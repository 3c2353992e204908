// Batched products: many converted matrices, each with k right-hand sides,
// in one kernel launch (plus one launch that adds the pieces of split
// panels).
//
// spc5_batch_create gathers, once, a device table with every matrix's
// arrays and vectors and a map from a global tile index to its matrix; the
// global tile list is the concatenation of the matrices' own work plans.
// spc5_batch_run then launches the persistent kernel over all tiles: a warp
// takes chunks of consecutive global tiles from a counter (consecutive tiles
// mostly belong to one matrix, so the warp reads the matrix's table entry
// once per chunk, and uneven matrices are balanced across the warps), and
// runs each tile with the lane mapping of that matrix's row-group plan: the
// matrix's block shape (a warp-uniform switch over the six shapes) and its
// tuned body (the row stream for one lane per row, else the per-block loop),
// with k accumulators per lane: every stored value meets k x values, read as
// one contiguous run (X row-major [n][k]) with vector loads when the vectors
// are 16-byte aligned.  Running allocates nothing and copies nothing from
// the host, so it can be captured in a CUDA graph; the tile counter is left
// at zero by every launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "spc5_flat.cuh"
#include "spc5_internal.h"
#include "spc5_reduce.cuh"

namespace spc5 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

struct MatDesc {
  const Tile *tiles;
  const int32_t *brp, *vptr, *colidx;
  const void *masks, *values;
  const void *x;
  void *y;
  void *partial;  // npieces * r * k slots
  const int32_t *long_panels, *long_slots;
  int64_t nrows;
  int64_t tile_base;
  int32_t r, c, ntiles, nlong;
  int32_t body;  // the matrix's row-group body (2, 6: row stream; 5, 7: passing empty blocks)
  int32_t flat;  // 1: the tiles are the matrix's block-balanced plan (k = 1, r <= 2)
};

constexpr int kBatchChunk = 8;  // consecutive tiles per counter grab

// The K values of one row of a row-major [n][K] vector block: vector loads
// when the block is 16-byte aligned (VEC), else K scalar loads.
template <int K, bool VEC, typename AT>
__device__ __forceinline__ void load_row(const AT *__restrict__ p, AT (&v)[K]) {
  if constexpr (VEC && sizeof(AT) == 4 && K % 4 == 0) {
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
      const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + i);
      v[4 * i] = t.x;
      v[4 * i + 1] = t.y;
      v[4 * i + 2] = t.z;
      v[4 * i + 3] = t.w;
    }
  } else if constexpr (VEC && sizeof(AT) == 4 && K == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    v[0] = t.x;
    v[1] = t.y;
  } else if constexpr (VEC && sizeof(AT) == 8 && K % 2 == 0) {
#pragma unroll
    for (int i = 0; i < K / 2; ++i) {
      const double2 t = __ldg(reinterpret_cast<const double2 *>(p) + i);
      v[2 * i] = t.x;
      v[2 * i + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = __ldg(p + i);
  }
}

// Row-stream body with K right-hand sides (one lane per row): the lane walks
// its row's values across the panel's blocks, one value (K FMAs) per trip,
// entering the next block when its row bits in the current one are used up;
// the next block's mask and start column are loaded one block ahead.
template <int R, int C, int K, bool VEC, typename VT, typename AT, typename MaskT>
__device__ __forceinline__ void row_stream_k(const MaskT *__restrict__ masks,
                                             const int32_t *__restrict__ colidx,
                                             const VT *__restrict__ vals,
                                             const AT *__restrict__ x, int32_t bl, int32_t nbp,
                                             int32_t v, int q, bool skip, AT (&acc)[K]) {
  const int qc = q * C;
  const uint32_t row_low = (1u << qc) - 1u;
  const uint32_t cmask = (1u << C) - 1u;
  uint32_t m1 = 0u;
  int32_t c1 = 0;
  if (nbp > 0) {
    m1 = (uint32_t)masks[bl];
    c1 = colidx[bl];
  }
  int32_t b = 0;
  uint32_t mq = 0u;
  int32_t off = 0, col = 0;
  while (__any_sync(kFull, mq != 0u || b < nbp)) {
    // with `skip`, blocks in which the row has no value are passed in one trip
    for (int e = 0; mq == 0u && b < nbp && (skip || e < 1); ++e) {
      mq = (m1 >> qc) & cmask;
      off = v + __popc(m1 & row_low);
      v += __popc(m1);
      col = c1;
      ++b;
      m1 = 0u;
      if (b < nbp) {
        m1 = (uint32_t)masks[bl + b];
        c1 = colidx[bl + b];
      }
    }
    if (mq) {
      const int k = __ffs(mq) - 1;
      const AT a = (AT)widen(vals[off]);
      AT xv[K];
      load_row<K, VEC>(x + (int64_t)(col + k) * K, xv);
#pragma unroll
      for (int i = 0; i < K; ++i) acc[i] = fma(a, xv[i], acc[i]);
      mq &= mq - 1u;
      ++off;
    }
  }
}


// One tile of one matrix with K right-hand sides.
template <int R, int C, int K, bool VEC, typename VT, typename AT>
__device__ __forceinline__ void batch_tile(const MatDesc &d, const Tile &cur, int lane, AT alpha,
                                           AT beta) {
  using MT = typename MaskType<R, C>::T;
  const MT *__restrict__ masks = (const MT *)d.masks;
  const VT *__restrict__ vals = (const VT *)d.values;
  const AT *__restrict__ x = (const AT *)d.x;
  AT *__restrict__ y = (AT *)d.y;
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
  if (segment) {
    pvalid = (j == 0);
    bl = cur.b0;
    nbp = cur.b1 - cur.b0;
    v = cur.v0;
  } else {
    const int64_t p = (int64_t)cur.p0 + j;
    // a heavy panel (kSkip) has tiles of its own
    pvalid = p < cur.p1 && !((cur.mode & kSkip) && (((uint32_t)cur.slot >> j) & 1u));
    bl = pvalid ? d.brp[p] : 0;
    nbp = pvalid ? d.brp[p + 1] - bl : 0;
    v = pvalid ? d.vptr[p] : 0;
  }
  AT acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = 0;
  if ((d.body == 2 || d.body == 5 || d.body == 6 || d.body == 7) && G == 1) {
    row_stream_k<R, C, K, VEC>(masks, d.colidx, vals, x, bl, nbp, v, q,
                               d.body == 5 || d.body == 7, acc);
  } else {
  const int32_t maxnb = __reduce_max_sync(kFull, nbp);
  for (int32_t it = 0; it < maxnb; it += G) {
    const int32_t idx = it + g;
    const bool valid = idx < nbp;
    const uint32_t m = valid ? (uint32_t)masks[bl + idx] : 0u;
    const int32_t col = valid ? d.colidx[bl + idx] : 0;
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
      const AT a = (AT)widen(vals[off++]);
      AT xv[K];
      load_row<K, VEC>(x + (int64_t)(col + k) * K, xv);
#pragma unroll
      for (int i = 0; i < K; ++i) acc[i] = fma(a, xv[i], acc[i]);
    }
    v += total;
  }
  }
#pragma unroll
  for (int i = 0; i < K; ++i)
    for (int o = G >> 1; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(kFull, acc[i], o, G);
  if (pvalid && g == 0) {
    if (cur.mode & kPartial) {
      AT *part = (AT *)d.partial + ((int64_t)cur.slot * R + q) * K;
#pragma unroll
      for (int i = 0; i < K; ++i) part[i] = acc[i];
    } else {
      const int64_t row = ((int64_t)cur.p0 + j) * R + q;
      if (row < d.nrows) {
        AT *yr = y + row * K;
#pragma unroll
        for (int i = 0; i < K; ++i) {
          AT out = alpha * acc[i];
          if (beta != (AT)0) out = fma(beta, yr[i], out);
          yr[i] = out;
        }
      }
    }
  }
}

// CTAs of 256 threads per SM that the registers allow: 48 warps for one or
// two FP32 right-hand sides, fewer as the k accumulators grow (and for FP64).
template <int K, typename AT>
struct BatchBlocksPerSM {
  static constexpr int v = sizeof(AT) == 4 ? (K <= 2 ? 6 : (K <= 4 ? 5 : (K <= 8 ? 4 : 3)))
                                           : (K <= 2 ? 5 : (K <= 4 ? 4 : (K <= 8 ? 3 : 2)));
};

template <int K, bool VEC, typename VT, typename AT>
__global__ void __launch_bounds__(kThreads, BatchBlocksPerSM<K, AT>::v)
    k_batch(const MatDesc *__restrict__ table, const int32_t *__restrict__ tile_mat,
            int64_t ntiles, uint32_t *sched, AT alpha, AT beta) {
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (ntiles + kBatchChunk - 1) / kBatchChunk;
  // chunks come from the counter one ahead: the grab for the next chunk is
  // issued when a chunk starts
  uint32_t grab = 0;
  if (lane == 0) grab = atomicAdd(&sched[0], 1u);
  int64_t ch = (int64_t)__shfl_sync(kFull, grab, 0);
  // the current matrix's table entry, kept in shared memory (registers are
  // needed for the k accumulators)
  __shared__ MatDesc s_desc[kThreads / 32];
  static_assert(sizeof(MatDesc) % 4 == 0 && sizeof(MatDesc) <= 128, "table entry size");
  MatDesc &d = s_desc[threadIdx.x >> 5];
  int cur_m = -1;
  while (ch < nchunks) {
    if (lane == 0) grab = atomicAdd(&sched[0], 1u);
    const int64_t t1 = min((ch + 1) * kBatchChunk, ntiles);
    for (int64_t t = ch * kBatchChunk; t < t1; ++t) {
      const int m = tile_mat[t];
      if (m != cur_m) {  // uniform over the warp
        __syncwarp();
        if (lane < (int)(sizeof(MatDesc) / 4))
          reinterpret_cast<uint32_t *>(&d)[lane] =
              reinterpret_cast<const uint32_t *>(table + m)[lane];
        __syncwarp();
        cur_m = m;
      }
      const Tile cur = d.tiles[t - d.tile_base];
      switch (d.r * 100 + d.c) {
        case 108: batch_tile<1, 8, K, VEC, VT, AT>(d, cur, lane, alpha, beta); break;
        case 204: batch_tile<2, 4, K, VEC, VT, AT>(d, cur, lane, alpha, beta); break;
        case 208: batch_tile<2, 8, K, VEC, VT, AT>(d, cur, lane, alpha, beta); break;
        case 404: batch_tile<4, 4, K, VEC, VT, AT>(d, cur, lane, alpha, beta); break;
        case 408: batch_tile<4, 8, K, VEC, VT, AT>(d, cur, lane, alpha, beta); break;
        default: batch_tile<8, 4, K, VEC, VT, AT>(d, cur, lane, alpha, beta); break;
      }
    }
    ch = (int64_t)__shfl_sync(kFull, grab, 0);
  }
  // every warp has made its last grab: the last one to finish resets the counter
  if (lane == 0) {
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(&sched[1], 1u) == nwarps - 1) {
      atomicExch(&sched[0], 0u);
      atomicExch(&sched[1], 0u);
    }
  }
}

// The members whose product runs the block-balanced plan (one right-hand
// side, r <= 2): a second persistent launch over their tiles, with the
// standalone kernel's tile body.  A warp takes chunks of kBatchChunk tiles
// from its own counter and runs consecutive whole-panel tiles of one matrix
// as one range (the plan cuts a small matrix into tiles of 64 blocks, sized
// for a launch of its own; the tile body takes any run of whole panels).
template <typename VT, typename AT>
__global__ void __launch_bounds__(kThreads, 4)
    k_batch_flat(const MatDesc *__restrict__ table, const int32_t *__restrict__ tile_mat,
                 int64_t ntiles, uint32_t *sched, AT alpha, AT beta) {
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (ntiles + kBatchChunk - 1) / kBatchChunk;
  __shared__ MatDesc s_desc[kThreads / 32];
  __shared__ int32_t s_pid[kThreads / 32][kFlatRound];
  MatDesc &d = s_desc[threadIdx.x >> 5];
  int32_t *pid = s_pid[threadIdx.x >> 5];
  const Scale<AT> sc{alpha, beta, beta != (AT)0 ? 2 : (alpha != (AT)1 ? 1 : 0)};
  uint32_t grab = 0;
  if (lane == 0) grab = atomicAdd(&sched[0], 1u);
  int64_t ch = (int64_t)__shfl_sync(kFull, grab, 0);
  int cur_m = -1;
  while (ch < nchunks) {
    if (lane == 0) grab = atomicAdd(&sched[0], 1u);
    const int64_t t1 = min((ch + 1) * kBatchChunk, ntiles);
    for (int64_t t = ch * kBatchChunk; t < t1;) {
      const int m = tile_mat[t];
      if (m != cur_m) {
        __syncwarp();
        if (lane < (int)(sizeof(MatDesc) / 4))
          reinterpret_cast<uint32_t *>(&d)[lane] =
              reinterpret_cast<const uint32_t *>(table + m)[lane];
        __syncwarp();
        cur_m = m;
      }
      Tile cur = d.tiles[t - d.tile_base];
      ++t;
      while (!(cur.mode & kPartial) && t < t1 && tile_mat[t] == m) {
        const Tile nx = d.tiles[t - d.tile_base];
        if (nx.mode & kPartial) break;
        cur.p1 = nx.p1;
        cur.b1 = nx.b1;
        cur.v1 = nx.v1;
        ++t;
      }
      const VT *vals = (const VT *)d.values;
      const AT *x = (const AT *)d.x;
      AT *y = (AT *)d.y, *part = (AT *)d.partial;
      switch (d.r * 100 + d.c) {
        case 108:
          flat_tile<1, 8>(cur, lane, pid, d.brp, d.colidx,
                          (const typename MaskType<1, 8>::T *)d.masks, vals, x, y, part, sc,
                          d.nrows);
          break;
        case 204:
          flat_tile<2, 4>(cur, lane, pid, d.brp, d.colidx,
                          (const typename MaskType<2, 4>::T *)d.masks, vals, x, y, part, sc,
                          d.nrows);
          break;
        default:
          flat_tile<2, 8>(cur, lane, pid, d.brp, d.colidx,
                          (const typename MaskType<2, 8>::T *)d.masks, vals, x, y, part, sc,
                          d.nrows);
          break;
      }
    }
    ch = (int64_t)__shfl_sync(kFull, grab, 0);
  }
  // every warp has made its last grab: the last one to finish resets the counter
  if (lane == 0) {
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(&sched[1], 1u) == nwarps - 1) {
      atomicExch(&sched[0], 0u);
      atomicExch(&sched[1], 0u);
    }
  }
}

// Split panels, one warp per panel: the panel's partials are W = r * k
// values per slot (slot-major, row q and RHS j at q * k + j).  For W <= 32
// lane t adds elements t, t + 32, ... (all of element t % W) and the lanes of
// each element are then added; for W > 32 each lane adds its elements' slots.
// lp_mat / lp_idx: matrix and local long-panel index of every global entry.
template <int K, typename AT>
__global__ void k_batch_fixup(const MatDesc *__restrict__ table,
                              const int32_t *__restrict__ lp_mat,
                              const int32_t *__restrict__ lp_idx, int64_t nlong_total, AT alpha,
                              AT beta) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nlong_total;
       e += nw) {
    const MatDesc d = table[lp_mat[e]];
    const int l = lp_idx[e];
    const int W = d.r * K;
    const AT *p = (const AT *)d.partial;
    const int64_t s0 = d.long_slots[2 * l];
    const int64_t n = d.long_slots[2 * l + 1] - s0;
    auto put = [&](int t, AT acc) {
      const int64_t row = (int64_t)d.long_panels[l] * d.r + t / K;
      if (row < d.nrows) {
        AT *yr = (AT *)d.y + row * K + t % K;
        AT out = alpha * acc;
        if (beta != (AT)0) out = fma(beta, *yr, out);
        *yr = out;
      }
    };
    if (W <= 32) {
      const int64_t first = s0 * W + lane, end = (s0 + n) * W;
      AT acc = first < end ? strided_sum(p + first, (end - first + 31) / 32, 32) : (AT)0;
      for (int o = 16; o >= W; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
      if (lane < W) put(lane, acc);
    } else {
      for (int t = lane; t < W; t += 32) put(t, strided_sum(p + s0 * W + t, n, W));
    }
  }
}

__global__ void k_fill(int32_t *dst, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = v;
}
__global__ void k_iota(int32_t *dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (int32_t)i;
}

int sm_count() { return device_sm_count(); }

}  // namespace
}  // namespace spc5

using namespace spc5;

struct spc5_batch {
  int nmat = 0, k = 0, device = 0;
  int vec = 0;              // every X and Y 16-byte aligned: vector loads of the k values
  uint32_t *sched = nullptr;  // [4] tile-chunk counter and finished warps of the row-group
                              // launch, then of the block-balanced launch (reset by them)
  spc5_dtype dtype = SPC5_F64;
  int64_t ntiles = 0, nlong = 0;
  int64_t fntiles = 0;               // tiles of the block-balanced members
  MatDesc *table = nullptr;
  int32_t *ftile_mat = nullptr;      // their tile -> matrix map
  int32_t *tile_mat = nullptr;
  int32_t *lp_mat = nullptr, *lp_idx = nullptr;
  void *partial = nullptr;
};

namespace {

void free_batch(spc5_batch *B) {
  if (!B) return;
  cudaFree(B->table);
  cudaFree(B->tile_mat);
  cudaFree(B->ftile_mat);
  cudaFree(B->lp_mat);
  cudaFree(B->lp_idx);
  cudaFree(B->partial);
  cudaFree(B->sched);
  delete B;
}

template <int K, typename VT, typename AT>
cudaError_t run_batch(const spc5_batch *B, double alpha, double beta, cudaStream_t s) {
  if (B->ntiles > 0) {
    const int64_t nchunks = (B->ntiles + kBatchChunk - 1) / kBatchChunk;
    int64_t blocks = (nchunks + (kThreads / 32) - 1) / (kThreads / 32);
    blocks = std::min<int64_t>(blocks, (int64_t)sm_count() * BatchBlocksPerSM<K, AT>::v);
    if (B->vec)
      k_batch<K, true, VT, AT><<<(unsigned)blocks, kThreads, 0, s>>>(
          B->table, B->tile_mat, B->ntiles, B->sched, (AT)alpha, (AT)beta);
    else
      k_batch<K, false, VT, AT><<<(unsigned)blocks, kThreads, 0, s>>>(
          B->table, B->tile_mat, B->ntiles, B->sched, (AT)alpha, (AT)beta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if constexpr (K == 1) {
    if (B->fntiles > 0) {
      const int64_t nchunks = (B->fntiles + kBatchChunk - 1) / kBatchChunk;
      int64_t blocks = (nchunks + (kThreads / 32) - 1) / (kThreads / 32);
      blocks = std::min<int64_t>(blocks, (int64_t)sm_count() * 4);
      k_batch_flat<VT, AT><<<(unsigned)blocks, kThreads, 0, s>>>(
          B->table, B->ftile_mat, B->fntiles, B->sched + 2, (AT)alpha, (AT)beta);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  if (B->nlong > 0) {
    const int blocks = (int)std::min<int64_t>((B->nlong + 7) / 8, (int64_t)sm_count() * 8);
    k_batch_fixup<K, AT><<<blocks, 256, 0, s>>>(B->table, B->lp_mat, B->lp_idx, B->nlong,
                                                (AT)alpha, (AT)beta);
  }
  return cudaGetLastError();
}

template <typename VT, typename AT>
cudaError_t run_k(const spc5_batch *B, double alpha, double beta, cudaStream_t s) {
  switch (B->k) {
    case 1: return run_batch<1, VT, AT>(B, alpha, beta, s);
    case 2: return run_batch<2, VT, AT>(B, alpha, beta, s);
    case 4: return run_batch<4, VT, AT>(B, alpha, beta, s);
    case 8: return run_batch<8, VT, AT>(B, alpha, beta, s);
    default: return run_batch<16, VT, AT>(B, alpha, beta, s);
  }
}

}  // namespace

extern "C" spc5_status spc5_batch_create(int nmat, const spc5_matrix *const *A,
                                         const void *const *X, void *const *Y, int k,
                                         void *stream, spc5_batch **out) {
  if (!out || nmat < 1 || !A || !X || !Y) {
    set_error("invalid argument");
    return SPC5_EINVAL;
  }
  if (k != 1 && k != 2 && k != 4 && k != 8 && k != 16) {
    set_error("k must be 1, 2, 4, 8 or 16");
    return SPC5_EUNSUPPORTED;
  }
  for (int m = 0; m < nmat; ++m) {
    if (!A[m] || (A[m]->ncols > 0 && !X[m]) || (A[m]->nrows > 0 && !Y[m])) {
      set_error("NULL matrix or vector in the batch");
      return SPC5_EINVAL;
    }
    if (A[m]->hybrid) {
      set_error("the batched product does not take hybrid matrices");
      return SPC5_EUNSUPPORTED;
    }
    if (A[m]->value_dtype != A[0]->value_dtype || A[m]->device != A[0]->device) {
      set_error("all matrices of a batch share one value dtype and one device");
      return SPC5_EINVAL;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  spc5_batch *B = new (std::nothrow) spc5_batch();
  if (!B) {
    set_error("host allocation failed");
    return SPC5_ENOMEM;
  }
  B->nmat = nmat;
  B->k = k;
  B->device = A[0]->device;
  B->dtype = A[0]->value_dtype;
  const size_t slot = B->dtype == SPC5_F64 ? 8 : 4;
  std::vector<MatDesc> table(nmat);
  int64_t tiles = 0, ftiles = 0, nlong = 0, pslots = 0;
  std::vector<int64_t> pbase(nmat);
  for (int m = 0; m < nmat; ++m) {
    const spc5_matrix *M = A[m];
    MatDesc &d = table[m];
    // one right-hand side: a matrix whose product runs the block-balanced
    // plan (skewed rows, r <= 2) runs it in the batch's second launch
    const bool fl = k == 1 && M->flat == 1 && M->r <= 2;
    d.tiles = fl ? M->ftiles : M->tiles;
    d.brp = M->block_rowptr;
    d.vptr = M->panel_vptr;
    d.colidx = M->block_colidx;
    d.masks = M->masks;
    d.values = M->values;
    d.x = X[m];
    d.y = Y[m];
    d.long_panels = fl ? M->flong_panels : M->long_panels;
    d.long_slots = fl ? M->flong_slots : M->long_slots;
    d.nrows = M->nrows;
    d.r = M->r;
    d.c = M->c;
    d.ntiles = (int32_t)(fl ? M->fntiles : M->ntiles);
    d.nlong = (int32_t)(fl ? M->fnlong : M->nlong);
    d.body = M->body;
    d.flat = fl ? 1 : 0;
    d.tile_base = fl ? ftiles : tiles;
    pbase[m] = pslots;
    pslots += (fl ? M->fnpieces : M->npieces) * M->r * k;
    (fl ? ftiles : tiles) += d.ntiles;
    nlong += d.nlong;
  }
  B->ntiles = tiles;
  B->fntiles = ftiles;
  B->nlong = nlong;
  B->vec = 1;
  for (int m = 0; m < nmat; ++m)
    if ((reinterpret_cast<uintptr_t>(X[m]) | reinterpret_cast<uintptr_t>(Y[m])) & 15u) B->vec = 0;
  spc5_status st = cuda_check(cudaMalloc(&B->partial, (size_t)std::max<int64_t>(pslots, 1) * slot),
                              "alloc batch partials");
  if (st == SPC5_OK)
    st = cuda_check(cudaMalloc((void **)&B->sched, 4 * sizeof(uint32_t)), "alloc batch counter");
  if (st == SPC5_OK)
    st = cuda_check(cudaMemsetAsync(B->sched, 0, 4 * sizeof(uint32_t), s), "zero batch counter");
  for (int m = 0; m < nmat; ++m) table[m].partial = (char *)B->partial + pbase[m] * slot;
  if (st == SPC5_OK)
    st = cuda_check(cudaMalloc((void **)&B->table, sizeof(MatDesc) * nmat), "alloc batch table");
  if (st == SPC5_OK)
    st = cuda_check(cudaMalloc((void **)&B->tile_mat, sizeof(int32_t) * std::max<int64_t>(tiles, 1)),
                    "alloc tile map");
  if (st == SPC5_OK)
    st = cuda_check(
        cudaMalloc((void **)&B->ftile_mat, sizeof(int32_t) * std::max<int64_t>(ftiles, 1)),
        "alloc flat tile map");
  if (st == SPC5_OK)
    st = cuda_check(cudaMalloc((void **)&B->lp_mat, sizeof(int32_t) * std::max<int64_t>(nlong, 1)),
                    "alloc long map");
  if (st == SPC5_OK)
    st = cuda_check(cudaMalloc((void **)&B->lp_idx, sizeof(int32_t) * std::max<int64_t>(nlong, 1)),
                    "alloc long map");
  if (st == SPC5_OK)
    st = cuda_check(cudaMemcpyAsync(B->table, table.data(), sizeof(MatDesc) * nmat,
                                    cudaMemcpyHostToDevice, s),
                    "copy batch table");
  int64_t lbase = 0;
  for (int m = 0; st == SPC5_OK && m < nmat; ++m) {
    const int64_t mt = table[m].ntiles, ml = table[m].nlong;
    if (mt > 0)
      k_fill<<<(unsigned)std::min<int64_t>((mt + 255) / 256, 4096), 256, 0, s>>>(
          (table[m].flat ? B->ftile_mat : B->tile_mat) + table[m].tile_base, mt, m);
    if (ml > 0) {
      k_fill<<<(unsigned)std::min<int64_t>((ml + 255) / 256, 4096), 256, 0, s>>>(
          B->lp_mat + lbase, ml, m);
      k_iota<<<(unsigned)std::min<int64_t>((ml + 255) / 256, 4096), 256, 0, s>>>(
          B->lp_idx + lbase, ml);
      lbase += ml;
    }
  }
  if (st == SPC5_OK) st = cuda_check(cudaStreamSynchronize(s), "sync batch create");
  if (st != SPC5_OK) {
    free_batch(B);
    return st;
  }
  *out = B;
  return SPC5_OK;
}

extern "C" spc5_status spc5_batch_run(const spc5_batch *B, double alpha, double beta,
                                      void *stream) {
  if (!B) {
    set_error("NULL batch");
    return SPC5_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (B->dtype == SPC5_F64)
    e = run_k<double, double>(B, alpha, beta, s);
  else if (B->dtype == SPC5_F32)
    e = run_k<float, float>(B, alpha, beta, s);
  else
    e = run_k<uint16_t, float>(B, alpha, beta, s);
  return cuda_check(e, "batch launch");
}

extern "C" spc5_status spc5_batch_destroy(spc5_batch *B) {
  free_batch(B);
  return SPC5_OK;
}

extern "C" spc5_status spc5_spmv_batched(int nmat, const spc5_matrix *const *A,
                                         const void *const *X, void *const *Y, int k,
                                         void *stream) {
  spc5_batch *B = nullptr;
  spc5_status st = spc5_batch_create(nmat, A, X, Y, k, stream, &B);
  if (st != SPC5_OK) return st;
  st = spc5_batch_run(B, 1.0, 0.0, stream);
  if (st == SPC5_OK) st = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "sync batch");
  free_batch(B);
  return st;
}
