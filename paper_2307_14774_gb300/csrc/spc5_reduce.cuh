// Reductions shared by the SpMV and batched kernels' fixups of split panels.
#pragma once

#include <stdint.h>

namespace spc5 {

// Sum of p[k * stride] for k < n with eight independent accumulators, so
// that eight loads are in flight per lane (split panels can have thousands
// of pieces).
template <typename AT>
__device__ __forceinline__ AT strided_sum(const AT *__restrict__ p, int64_t n, int64_t stride) {
  AT a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0, a6 = 0, a7 = 0;
  int64_t k = 0;
  for (; k + 8 <= n; k += 8, p += 8 * stride) {
    a0 += p[0];
    a1 += p[stride];
    a2 += p[2 * stride];
    a3 += p[3 * stride];
    a4 += p[4 * stride];
    a5 += p[5 * stride];
    a6 += p[6 * stride];
    a7 += p[7 * stride];
  }
  for (; k < n; ++k, p += stride) a0 += p[0];
  return ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

}  // namespace spc5
