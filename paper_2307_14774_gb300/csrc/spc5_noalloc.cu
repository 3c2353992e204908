// spc5_spmv_noalloc: the SpMV for callers that must not allocate.
//
// Some callers cannot call cudaMalloc at the moment they need a product: a
// real-time loop that must not hit the allocator (or the device-wide
// synchronisation a cudaFree implies), a library that may only use memory
// its host application hands it, or code running under a device-memory
// budget fixed at start-up.  spc5_spmv itself allocates nothing for device
// vectors either, but it writes the partial sums of panels split into pieces
// to a buffer owned by the matrix handle, and the expanded plan schedules
// its tiles through a counter owned by the handle.  This entry point uses
// instead a fixed array and a fixed counter pair compiled into the library
// (file-scope __device__ storage), so the whole call allocates nothing and
// touches neither of those per-matrix buffers.  (The staged kernel, when a
// plan selects it, still reports a timed-out wait through the handle's
// error word.)
//
// The array holds kNoallocScratchDoubles doubles (1 MiB); every GPU that
// loads the library keeps it until the process exits.  A matrix whose split
// panels need more partial sums is rejected with SPC5_EOVERFLOW.  The
// counters start at zero and every launch leaves them at zero.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "spc5_internal.h"
#include "spc5_pointer.h"

namespace spc5 {
namespace {

constexpr int64_t kNoallocScratchDoubles = 131072;  // 1 MiB

// Shared by every call on a device.  Every slot a call reads is written
// earlier in the same call (each piece writes its own r sums before the
// fixup adds them), so nothing needs clearing; calls that overlap on the
// GPU race on it.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];
static __device__ uint32_t g_noalloc_sched[2];

std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {};
uint32_t *g_sched_addr[kMaxDevices] = {};

// Device address of the array on `dev`, looked up once per device with that
// device current.  (In host code the array's name is only a host-side
// stand-in, not a device address.)
spc5_status scratch_address(int dev, double **out, uint32_t **sched) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for spc5_spmv_noalloc");
    return SPC5_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    int cur = -1;
    spc5_status st = cuda_check(cudaGetDevice(&cur), "cudaGetDevice");
    if (st != SPC5_OK) return st;
    if (cur != dev) {
      st = cuda_check(cudaSetDevice(dev), "cudaSetDevice");
      if (st != SPC5_OK) return st;
    }
    void *p = nullptr, *q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_sched);
    if (cur != dev) cudaSetDevice(cur);
    st = cuda_check(e, "cudaGetSymbolAddress(noalloc scratch)");
    if (st != SPC5_OK) return st;
    g_scratch_addr[dev] = static_cast<double *>(p);
    g_sched_addr[dev] = static_cast<uint32_t *>(q);
  }
  *out = g_scratch_addr[dev];
  *sched = g_sched_addr[dev];
  return SPC5_OK;
}

// True when device `dev` can read `p` directly: its own device memory or
// managed memory (not host memory, not another GPU's memory).
bool device_readable(const void *p, int dev) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return placement_of((int)attr.type, attr.device, dev) == Placement::kDevice;
}

}  // namespace
}  // namespace spc5

using namespace spc5;

extern "C" spc5_status spc5_spmv_noalloc(const spc5_matrix *A, const void *x, void *y,
                                         double alpha, double beta, void *stream) {
  if (!A) {
    set_error("NULL handle");
    return SPC5_EINVAL;
  }
  if (A->nrows == 0) return SPC5_OK;
  if ((A->ncols > 0 && (!x || !device_readable(x, A->device))) || !y ||
      !device_readable(y, A->device)) {
    set_error("spc5_spmv_noalloc takes vectors in the matrix's device memory (or managed "
              "memory) only: host vectors need staging buffers");
    return SPC5_EINVAL;
  }
  const int64_t need = spmv_pieces(A) * A->r + (A->hybrid ? A->snpieces : 0);
  if (need > kNoallocScratchDoubles) {
    set_error("the matrix's split panels need " + std::to_string(need) +
              " partial sums; spc5_spmv_noalloc holds at most " +
              std::to_string(kNoallocScratchDoubles));
    return SPC5_EOVERFLOW;
  }
  double *scratch = nullptr;
  uint32_t *sched = nullptr;
  spc5_status st = scratch_address(A->device, &scratch, &sched);
  if (st != SPC5_OK) return st;
  int cur = -1;
  st = cuda_check(cudaGetDevice(&cur), "cudaGetDevice");
  if (st != SPC5_OK) return st;
  if (cur != A->device) {
    st = cuda_check(cudaSetDevice(A->device), "cudaSetDevice");
    if (st != SPC5_OK) return st;
  }
  st = spmv_device_scratch(A, x, y, alpha, beta, (cudaStream_t)stream, scratch, sched);
  if (st == SPC5_OK && A->hybrid)  // the scalars' partial sums follow the blocks'
    st = spmv_scalars(A, x, y, alpha, (cudaStream_t)stream,
                      (char *)scratch + spmv_pieces(A) * A->r * sizeof(double), sched);
  if (cur != A->device) cudaSetDevice(cur);
  return st;
}
