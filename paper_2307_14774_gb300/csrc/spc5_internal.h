// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "spc5.h"

// A converted matrix.  Every array is device memory owned by the handle.
struct spc5_matrix {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int r = 0, c = 0;
  int64_t npanels = 0, nblocks = 0;
  int device = 0;
  spc5_dtype value_dtype = SPC5_F64;
  int32_t *block_rowptr = nullptr;  // npanels + 1
  int32_t *panel_vptr = nullptr;    // npanels + 1
  int32_t *block_colidx = nullptr;  // nblocks (+16 bytes of padding)
  void *masks = nullptr;            // nblocks * r * c / 8 bytes (+16 bytes of padding)
  void *values = nullptr;           // nnz values (+16 bytes of padding)
  int log2_lanes_per_row = 0;       // SpMV mapping: 2^k lanes share one row
  int64_t device_bytes = 0;
  // staging for host vectors in spc5_spmv
  double *x_stage = nullptr;
  double *y_stage = nullptr;
};

namespace spc5 {

// Thread-local last error text.
void set_error(const std::string &msg);

// Status of the last CUDA call; records a message on failure.
spc5_status cuda_check(cudaError_t e, const char *what);

// Supported block shapes.
bool supported_rc(int r, int c);

// Conversion: fills A (sizes set by the caller) from a device CSR.
spc5_status convert_device(spc5_matrix *A, const int32_t *d_rowptr, const int32_t *d_colidx,
                           const double *d_vals, cudaStream_t stream);

// SpMV launch on device vectors.
spc5_status spmv_device(const spc5_matrix *A, const double *x, double *y, double alpha,
                        double beta, cudaStream_t stream);

}  // namespace spc5
