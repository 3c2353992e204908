"""GB300-native SPC5: beta(r,c) sparse matrix-vector product (sm_103a CUDA).

The library ``libspc5.so`` (``include/spc5.h``) converts CSR to the SPC5
beta(r,c) format and computes y = alpha*A*x + beta*y on the GPU.  This
package is its Python binding (``spc5``) plus the build script.
"""
from . import autograd, partition
from .spc5 import (EXPORTS, SPC5_BF16, SPC5_F32, SPC5_F64, STATUS, SUPPORTED_RC, Matrix,
                   SPC5Error, export_tensors, load, spc5_convert_csr, spc5_destroy, spc5_export,
                   spc5_last_error, spc5_matrix_info, spc5_spmv, spc5_spmv_noalloc,
                   spc5_spmv_t, spc5_build_transpose, spc5_values_grad, spc5_set_values,
                   spc5_tune, spc5_convert_tuned, spc5_convert_tuned_ex, spc5_spmv_batched, Batch,
                   spc5_ircg,
                   spc5_convert_hybrid, spc5_export_hybrid, spc5_status_str,
                   spc5_measure_fma_peak)

__all__ = ["EXPORTS", "SPC5_BF16", "SPC5_F32", "SPC5_F64", "STATUS", "SUPPORTED_RC", "Matrix",
           "SPC5Error", "export_tensors", "load", "spc5_convert_csr", "spc5_destroy",
           "spc5_export", "spc5_last_error", "spc5_matrix_info", "spc5_spmv",
           "spc5_spmv_noalloc", "spc5_spmv_t", "spc5_build_transpose", "spc5_values_grad",
           "spc5_set_values",
           "spc5_tune", "spc5_convert_tuned", "spc5_convert_tuned_ex", "spc5_spmv_batched",
           "Batch", "spc5_ircg",
           "spc5_convert_hybrid", "spc5_export_hybrid", "spc5_status_str",
           "spc5_measure_fma_peak"]
