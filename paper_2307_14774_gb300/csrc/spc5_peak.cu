// Measured FMA rate of the current device, the denominator of the
// arithmetic roofline that the SpMV kernels are reported against.
//
// Every thread runs eight independent dependency chains a = a * b + c
// (FP64 or FP32), so each SM sub-partition always has independent FMAs to
// issue; the grid fills every SM with eight 256-thread CTAs.  b and c are
// kernel arguments (no constant folding) chosen so the chains stay normal
// numbers: b = 1 - 2^-20, c = 2^-10, a converging to c / (1 - b).  The result
// is written once per thread so the chains cannot be removed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "spc5_internal.h"

namespace spc5 {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chains(int iters, T b, T c, T *out) {
  T a[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) a[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < kPeakChains; ++i) a[i] = fma(a[i], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += a[i];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
spc5_status measure(cudaStream_t s, double *tflops) {
  int dev = 0, nsm = 0;
  spc5_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != SPC5_OK) return st;
  st = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev),
                  "cudaDeviceGetAttribute");
  if (st != SPC5_OK) return st;
  const int blocks = nsm * 8;
  T *out = nullptr;
  st = cuda_check(cudaMallocAsync((void **)&out, sizeof(T) * blocks * kPeakThreads, s),
                  "cudaMallocAsync(peak)");
  if (st != SPC5_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // FP64: about 10 ms per launch on a 152-SM GB300; FP32 runs 64x faster, so
  // it takes more iterations for the same duration.
  const int iters = sizeof(T) == 8 ? 256 : 8192;
  const T b = (T)(1.0 - 1.0 / 1048576.0), c = (T)(1.0 / 1024.0);
  double best = 0.0;
  for (int rep = 0; rep < 6 && st == SPC5_OK; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<blocks, kPeakThreads, 0, s>>>(iters, b, c, out);
    cudaEventRecord(e1, s);
    st = cuda_check(cudaEventSynchronize(e1), "peak kernel");
    if (st != SPC5_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kPeakChains * 16.0 * iters * (double)blocks * kPeakThreads;
    if (rep > 0 && ms > 0.f) best = best > flops / (ms * 1e-3) ? best : flops / (ms * 1e-3);
  }
  if (st == SPC5_OK) st = cuda_check(cudaGetLastError(), "peak kernel launch");
  cudaFreeAsync(out, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == SPC5_OK) *tflops = best / 1e12;
  return st;
}

}  // namespace
}  // namespace spc5

extern "C" spc5_status spc5_measure_fma_peak(spc5_dtype dtype, void *stream, double *tflops) {
  spc5::set_error("");
  if (!tflops) {
    spc5::set_error("tflops is NULL");
    return SPC5_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == SPC5_F64) return spc5::measure<double>(s, tflops);
  if (dtype == SPC5_F32) return spc5::measure<float>(s, tflops);
  spc5::set_error("dtype must be SPC5_F64 or SPC5_F32");
  return SPC5_EUNSUPPORTED;
}
