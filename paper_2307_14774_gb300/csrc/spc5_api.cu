// C-ABI entry points: argument checks, host/device pointer handling, and
// the lifetime of spc5_matrix handles.  The arithmetic lives in
// spc5_convert.cu and spc5_spmv.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "spc5_internal.h"
#include "spc5_pointer.h"

namespace spc5 {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

spc5_status cuda_check(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return SPC5_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return SPC5_ENOMEM;
  return SPC5_ECUDA;
}

int device_sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (dev < 0 || dev >= kMaxDevices) dev = 0;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
  static std::atomic<cudaMemPool_t> pools[kMaxDevices];
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaMallocAsync(p, bytes, s);
  cudaMemPool_t pool = pools[dev].load(std::memory_order_acquire);
  if (!pool) {
    std::lock_guard<std::mutex> lock(mu);
    pool = pools[dev].load(std::memory_order_relaxed);
    if (!pool) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pool, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = kScratchKeep;
      e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
      }
      pools[dev].store(pool, std::memory_order_release);
    }
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

bool supported_rc(int r, int c) {
  return (r == 1 && c == 8) || (r == 2 && c == 4) || (r == 2 && c == 8) || (r == 4 && c == 4) ||
         (r == 4 && c == 8) || (r == 8 && c == 4);
}

namespace {

// Where `p` lives relative to device `dev`: host memory (pageable or
// pinned), memory the device reads directly (its own device memory, or
// managed memory), or device memory of another GPU.  *mapped (if given)
// receives the device address of pinned (page-locked, mapped) host memory,
// nullptr otherwise.
Placement locate(const void *p, int dev, void **mapped = nullptr) {
  if (mapped) *mapped = nullptr;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return placement_of(-1, -1, dev);
  }
  if (mapped && attr.type == cudaMemoryTypeHost) *mapped = attr.devicePointer;
  return placement_of((int)attr.type, attr.device, dev);
}


struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void free_matrix(spc5_matrix *A) {
  if (!A) return;
  DeviceGuard g(A->device);
  free_matrix(A->transpose);
  cudaFree(A->block_rowptr);
  cudaFree(A->panel_vptr);
  cudaFree(A->block_colidx);
  cudaFree(A->masks);
  cudaFree(A->values);
  cudaFree(A->value_src);
  cudaFree(A->csr_rowptr);
  cudaFree(A->x_stage);
  cudaFree(A->y_stage);
  cudaFree(A->tiles);
  cudaFree(A->long_panels);
  cudaFree(A->long_slots);
  cudaFree(A->partial);
  cudaFree(A->ftiles);
  cudaFree(A->flong_panels);
  cudaFree(A->flong_slots);
  cudaFree(A->fpartial);
  cudaFree(A->fsched);
  cudaFree(A->frowoff);
  cudaFree(A->s_rowptr);
  cudaFree(A->s_colidx);
  cudaFree(A->s_vals);
  cudaFree(A->stiles);
  cudaFree(A->slong_rows);
  cudaFree(A->slong_slots);
  cudaFree(A->spartial);
  cudaFree(A->dev_error);
  delete A;
}

}  // namespace
}  // namespace spc5

using namespace spc5;

#define RETURN_IF(cond, code, msg) \
  do {                             \
    if (cond) {                    \
      set_error(msg);              \
      return (code);               \
    }                              \
  } while (0)

extern "C" {

const char *spc5_status_str(spc5_status s) {
  switch (s) {
    case SPC5_OK: return "SPC5_OK";
    case SPC5_EINVAL: return "SPC5_EINVAL";
    case SPC5_EUNSORTED: return "SPC5_EUNSORTED";
    case SPC5_EUNSUPPORTED_RC: return "SPC5_EUNSUPPORTED_RC";
    case SPC5_EOVERFLOW: return "SPC5_EOVERFLOW";
    case SPC5_ECUDA: return "SPC5_ECUDA";
    case SPC5_ENOMEM: return "SPC5_ENOMEM";
    case SPC5_EDEVICE: return "SPC5_EDEVICE";
    case SPC5_ERANGE: return "SPC5_ERANGE";
    case SPC5_EROWPTR: return "SPC5_EROWPTR";
    case SPC5_EUNSUPPORTED: return "SPC5_EUNSUPPORTED";
  }
  return "SPC5_UNKNOWN";
}

const char *spc5_last_error(void) { return g_last_error.c_str(); }

spc5_status spc5_convert_csr(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t *rowptr,
                             const int32_t *colidx, const void *vals, spc5_dtype vals_dtype,
                             spc5_dtype store_dtype, int r, int c, void *stream,
                             spc5_matrix **out) {
  g_last_error.clear();
  RETURN_IF(!out, SPC5_EINVAL, "out is NULL");
  RETURN_IF(nrows < 0 || ncols < 0 || nnz < 0, SPC5_EINVAL, "negative size");
  RETURN_IF(!rowptr, SPC5_EINVAL, "rowptr is NULL");
  RETURN_IF(nnz > 0 && (!colidx || !vals), SPC5_EINVAL, "colidx or vals is NULL");
  RETURN_IF(!supported_rc(r, c), SPC5_EUNSUPPORTED_RC,
            "block shape must be one of (1,8) (2,4) (2,8) (4,4) (4,8) (8,4)");
  RETURN_IF(nrows >= INT32_MAX || ncols >= INT32_MAX || nnz >= INT32_MAX, SPC5_EOVERFLOW,
            "sizes must stay below 2^31");
  RETURN_IF(vals_dtype != SPC5_F64, SPC5_EUNSUPPORTED, "input values must be FP64");
  RETURN_IF(store_dtype != SPC5_F64 && store_dtype != SPC5_F32 && store_dtype != SPC5_BF16,
            SPC5_EINVAL, "unknown storage dtype");
  cudaStream_t s = (cudaStream_t)stream;

  spc5_matrix *A = new (std::nothrow) spc5_matrix();
  RETURN_IF(!A, SPC5_ENOMEM, "host allocation failed");
  A->nrows = nrows;
  A->ncols = ncols;
  A->nnz = nnz;
  A->r = r;
  A->c = c;
  A->npanels = (nrows + r - 1) / r;
  A->value_dtype = store_dtype;
  spc5_status st = cuda_check(cudaGetDevice(&A->device), "cudaGetDevice");
  if (st != SPC5_OK) {
    delete A;
    return st;
  }

  // Host inputs are staged through temporary device copies.
  const int32_t *d_rowptr = rowptr, *d_colidx = colidx;
  const double *d_vals = (const double *)vals;
  void *tmp[3] = {nullptr, nullptr, nullptr};
  auto stage = [&](const void *src, size_t bytes, int slot, const void **dst) -> spc5_status {
    if (!src) return SPC5_OK;
    const Placement pl = locate(src, A->device);
    if (pl == Placement::kOtherDevice) {
      set_error("a CSR array is device memory of another GPU than the current one");
      return SPC5_EINVAL;
    }
    if (pl == Placement::kDevice) return SPC5_OK;
    spc5_status e = cuda_check(scratch_alloc(&tmp[slot], bytes > 0 ? bytes : 4, s), "alloc staging");
    if (e != SPC5_OK) return e;
    e = cuda_check(cudaMemcpyAsync(tmp[slot], src, bytes, cudaMemcpyHostToDevice, s), "copy CSR");
    if (e != SPC5_OK) return e;
    *dst = tmp[slot];
    return SPC5_OK;
  };
  st = stage(rowptr, (size_t)(nrows + 1) * sizeof(int32_t), 0, (const void **)&d_rowptr);
  if (st == SPC5_OK && nnz > 0)
    st = stage(colidx, (size_t)nnz * sizeof(int32_t), 1, (const void **)&d_colidx);
  if (st == SPC5_OK && nnz > 0)
    st = stage(vals, (size_t)nnz * sizeof(double), 2, (const void **)&d_vals);
  if (st == SPC5_OK) st = convert_device(A, d_rowptr, d_colidx, d_vals, s);
  if (st == SPC5_OK) {  // kept for the values gradient (4 bytes per row)
    st = cuda_check(cudaMalloc((void **)&A->csr_rowptr, (size_t)(nrows + 1) * sizeof(int32_t)),
                    "alloc CSR row pointer");
    if (st == SPC5_OK)
      st = cuda_check(cudaMemcpyAsync(A->csr_rowptr, d_rowptr, (size_t)(nrows + 1) * 4,
                                      cudaMemcpyDeviceToDevice, s),
                      "copy CSR row pointer");
    if (st == SPC5_OK) A->device_bytes += (nrows + 1) * 4;
  }
  for (void *p : tmp)
    if (p) cudaFreeAsync(p, s);
  if (st == SPC5_OK) st = cuda_check(cudaStreamSynchronize(s), "sync conversion");
  if (st != SPC5_OK) {
    free_matrix(A);
    return st;
  }
  *out = A;
  return SPC5_OK;
}

spc5_status spc5_convert_hybrid(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t *rowptr,
                                const int32_t *colidx, const void *vals, spc5_dtype vals_dtype,
                                spc5_dtype store_dtype, int r, int c, void *stream,
                                spc5_matrix **out) {
  spc5_matrix *A = nullptr;
  spc5_status st = spc5_convert_csr(nrows, ncols, nnz, rowptr, colidx, vals, vals_dtype,
                                    store_dtype, r, c, stream, &A);
  if (st != SPC5_OK) return st;
  {
    DeviceGuard g(A->device);
    st = hybrid_split(A, (cudaStream_t)stream);
  }
  if (st != SPC5_OK) {
    free_matrix(A);
    return st;
  }
  *out = A;
  return SPC5_OK;
}

spc5_status spc5_export_hybrid(const spc5_matrix *A, const int32_t **s_rowptr,
                               const int32_t **s_colidx, const void **s_vals) {
  RETURN_IF(!A, SPC5_EINVAL, "NULL handle");
  RETURN_IF(!A->hybrid, SPC5_EINVAL, "not a hybrid matrix");
  if (s_rowptr) *s_rowptr = A->s_rowptr;
  if (s_colidx) *s_colidx = A->s_colidx;
  if (s_vals) *s_vals = A->s_vals;
  return SPC5_OK;
}

spc5_status spc5_matrix_info(const spc5_matrix *A, spc5_info *info) {
  RETURN_IF(!A || !info, SPC5_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->nrows = A->nrows;
  info->ncols = A->ncols;
  info->nnz = A->nnz;
  info->r = A->r;
  info->c = A->c;
  info->npanels = A->npanels;
  info->nblocks = A->nblocks;
  info->filling = A->nblocks ? (double)A->nnz / ((double)A->nblocks * A->r * A->c) : 0.0;
  info->value_dtype = A->value_dtype;
  info->mask_bytes = A->r * A->c / 8;
  info->device_bytes = A->device_bytes;
  info->device = A->device;
  info->lanes_per_row = 1 << A->log2_group_lanes;
  info->launches_per_spmv = spmv_launches(A);
  info->ntiles = A->flat ? A->fntiles : A->ntiles;
  info->long_panels = A->flat ? A->fnlong : A->nlong;
  info->stages = A->stages;
  info->consumers = A->consumers;
  uint32_t derr = 0;
  if (A->dev_error) {
    DeviceGuard g(A->device);
    if (cudaMemcpy(&derr, A->dev_error, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      derr = 0xffffffffu;
  }
  info->device_error = derr;
  info->tuned_us = A->tuned_us;
  info->tuned_rows_us = A->tuned_rows_us;
  info->flat = A->flat;
  info->group_efficiency = A->group_efficiency;
  info->hybrid = A->hybrid;
  info->nscalars = A->nscalars;
  info->pieces = spmv_pieces(A);
  info->scalar_pieces = A->hybrid ? A->snpieces : 0;
  info->body = A->body;
  info->dynamic = A->dynamic;
  info->transposed = A->transpose ? 1 : 0;
  info->halves = A->halves;
  info->nnz = A->nnz + A->nscalars;
  info->filling = A->nblocks ? (double)A->nnz / ((double)A->nblocks * A->r * A->c) : 0.0;
  return SPC5_OK;
}

spc5_status spc5_export(const spc5_matrix *A, const int32_t **block_rowptr,
                        const int32_t **panel_vptr, const int32_t **block_colidx,
                        const void **block_masks, const void **values) {
  RETURN_IF(!A, SPC5_EINVAL, "NULL handle");
  if (block_rowptr) *block_rowptr = A->block_rowptr;
  if (panel_vptr) *panel_vptr = A->panel_vptr;
  if (block_colidx) *block_colidx = A->block_colidx;
  if (block_masks) *block_masks = A->masks;
  if (values) *values = A->values;
  return SPC5_OK;
}

spc5_status spc5_spmv(const spc5_matrix *A, const void *x, void *y, double alpha, double beta,
                      void *stream) {
  RETURN_IF(!A, SPC5_EINVAL, "NULL handle");
  RETURN_IF((A->ncols > 0 && !x) || (A->nrows > 0 && !y), SPC5_EINVAL, "NULL vector");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard guard(A->device);
  void *y_mapped = nullptr;
  const Placement px = A->ncols > 0 ? locate(x, A->device) : Placement::kDevice;
  const Placement py = A->nrows > 0 ? locate(y, A->device, &y_mapped) : Placement::kDevice;
  RETURN_IF(px == Placement::kOtherDevice || py == Placement::kOtherDevice, SPC5_EINVAL,
            "x or y is device memory of another GPU than the matrix's");
  const bool host_x = px == Placement::kHost;
  const bool host_y = py == Placement::kHost;
  if (!host_x && !host_y) return spmv_device(A, x, y, alpha, beta, s);
  // pinned y is written in place by the kernels (through its mapping), so
  // the result reaches the host while the product runs; pageable y goes
  // through a device buffer and a copy back
  const bool stage_y = host_y && !y_mapped;

  const size_t es = A->value_dtype == SPC5_F64 ? sizeof(double) : sizeof(float);
  spc5_matrix *M = const_cast<spc5_matrix *>(A);
  spc5_status st = SPC5_OK;
  if (host_x && !M->x_stage)
    st = cuda_check(cudaMalloc(&M->x_stage, (size_t)A->ncols * es + 16), "alloc x staging");
  if (st == SPC5_OK && stage_y && !M->y_stage)
    st = cuda_check(cudaMalloc(&M->y_stage, (size_t)A->nrows * es + 16), "alloc y staging");
  if (st != SPC5_OK) return st;
  const void *dx = x;
  void *dy = y;
  if (host_x) {
    st = cuda_check(cudaMemcpyAsync(M->x_stage, x, (size_t)A->ncols * es, cudaMemcpyHostToDevice,
                                    s),
                    "copy x");
    if (st != SPC5_OK) return st;
    dx = M->x_stage;
  }
  if (y_mapped) dy = y_mapped;
  if (stage_y) {
    if (beta != 0.0) {
      st = cuda_check(cudaMemcpyAsync(M->y_stage, y, (size_t)A->nrows * es,
                                      cudaMemcpyHostToDevice, s),
                      "copy y");
      if (st != SPC5_OK) return st;
    }
    dy = M->y_stage;
  }
  st = spmv_device(A, dx, dy, alpha, beta, s);
  if (st != SPC5_OK) return st;
  if (stage_y) {
    st = cuda_check(cudaMemcpyAsync(y, dy, (size_t)A->nrows * es, cudaMemcpyDeviceToHost, s),
                    "copy y back");
    if (st != SPC5_OK) return st;
  }
  return cuda_check(cudaStreamSynchronize(s), "sync spmv");
}

spc5_status spc5_destroy(spc5_matrix *A) {
  if (!A) return SPC5_OK;
  free_matrix(A);
  return SPC5_OK;
}

}  // extern "C"
