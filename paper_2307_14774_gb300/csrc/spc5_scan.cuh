// Device-wide prefix scans for the conversion (reduce, scan the tile sums,
// scan each tile with its carry).  The operator need only be associative:
// the chain-map scan of the converter composes functions, which does not
// commute, so every combine keeps left-to-right order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spc5 {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide inclusive scan of one value per thread (Hillis-Steele in shared
// memory; any associative Op, order preserved).  Returns the thread's
// inclusive prefix; *total receives the block total.
template <typename T, typename Op>
__device__ T block_inclusive_scan(T v, Op op, T *smem, T *total) {
  const int t = threadIdx.x;
  smem[t] = v;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    T left = (t >= off) ? smem[t - off] : v;
    __syncthreads();
    if (t >= off) v = op(left, v);
    smem[t] = v;
    __syncthreads();
  }
  *total = smem[kScanThreads - 1];
  __syncthreads();
  return v;
}

// Pass 1: reduce every tile.
template <typename T, typename In, typename Op>
__global__ void __launch_bounds__(kScanThreads)
    scan_reduce_tiles(int64_t n, In in, Op op, T identity, T *tile_sums) {
  __shared__ T smem[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T acc = identity;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) acc = op(acc, in(base + i));
  T total;
  block_inclusive_scan(acc, op, smem, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Pass 2: exclusive scan of the tile sums in one block (sequential over
// chunks of kScanThreads with a running carry).
template <typename T, typename Op>
__global__ void __launch_bounds__(kScanThreads)
    scan_tile_sums(int64_t ntiles, Op op, T identity, T *tile_sums) {
  __shared__ T smem[kScanThreads];
  T carry = identity;
  for (int64_t base = 0; base < ntiles; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    T v = (i < ntiles) ? tile_sums[i] : identity;
    T total;
    T incl = block_inclusive_scan(v, op, smem, &total);
    // exclusive prefix within the chunk: inclusive of the left neighbour
    smem[threadIdx.x] = incl;
    __syncthreads();
    T excl = (threadIdx.x == 0) ? identity : smem[threadIdx.x - 1];
    __syncthreads();
    if (i < ntiles) tile_sums[i] = op(carry, excl);
    carry = op(carry, total);
    __syncthreads();
  }
}

// Pass 3: scan every tile with its carry and write the result.
template <typename T, typename In, typename Out, typename Op>
__global__ void __launch_bounds__(kScanThreads)
    scan_tiles(int64_t n, In in, Out out, Op op, T identity, const T *tile_carry,
               bool inclusive) {
  __shared__ T smem[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T items[kScanItems];
  T acc = identity;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    items[i] = (base + i < n) ? in(base + i) : identity;
    acc = op(acc, items[i]);
  }
  T total;
  T incl = block_inclusive_scan(acc, op, smem, &total);
  smem[threadIdx.x] = incl;
  __syncthreads();
  T run = (threadIdx.x == 0) ? identity : smem[threadIdx.x - 1];
  run = op(tile_carry[blockIdx.x], run);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) {
      T next = op(run, items[i]);
      out(base + i, inclusive ? next : run);
      run = next;
    }
  }
}

// Element access of the tile-sum array when the tile sums are themselves
// scanned by the three passes (more tile sums than one block scans quickly).
template <typename T>
struct ArrIn {
  const T *a;
  __device__ T operator()(int64_t i) const { return a[i]; }
};
template <typename T>
struct ArrOut {
  T *a;
  __device__ void operator()(int64_t i, T v) const { a[i] = v; }
};

// Tile sums up to this count are scanned by one block (pass 2 above);
// beyond it, by the three passes again, recursively.
constexpr int64_t kScanOneBlock = (int64_t)kScanThreads * 32;

// Elements of T that device_scan needs in `tmp` for n elements: the tile
// sums of every level of the recursion.
inline int64_t scan_tmp_elems(int64_t n) {
  int64_t total = 0, m = n <= 0 ? 1 : n;
  do {
    m = (m + kScanTile - 1) / kScanTile;
    total += m;
  } while (m > kScanOneBlock);
  return total + 1;
}

// Host driver: scan n elements read through `in(i)`, written through
// `out(i, v)`; `tmp` must hold scan_tmp_elems(n) elements of T.  Pass 2 runs
// in one block while the tile sums are few; for more tile sums (a conversion
// of 10^8 entries has about 10^5 tiles) they are scanned in place by the same
// three passes, so no pass walks more than kScanOneBlock elements serially.
template <typename T, typename In, typename Out, typename Op>
cudaError_t device_scan(int64_t n, In in, Out out, Op op, T identity, bool inclusive, T *tmp,
                        cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  scan_reduce_tiles<T><<<(unsigned)ntiles, kScanThreads, 0, stream>>>(n, in, op, identity, tmp);
  if (ntiles <= kScanOneBlock) {
    scan_tile_sums<T><<<1, kScanThreads, 0, stream>>>(ntiles, op, identity, tmp);
  } else {
    cudaError_t e = device_scan<T>(ntiles, ArrIn<T>{tmp}, ArrOut<T>{tmp}, op, identity, false,
                                   tmp + ntiles, stream);
    if (e != cudaSuccess) return e;
  }
  scan_tiles<T><<<(unsigned)ntiles, kScanThreads, 0, stream>>>(n, in, out, op, identity, tmp,
                                                               inclusive);
  return cudaGetLastError();
}

struct AddI32 {
  __device__ int32_t operator()(int32_t a, int32_t b) const { return a + b; }
};

}  // namespace spc5
