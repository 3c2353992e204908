"""torch.autograd.Function for y = A(vals) x over a converted SPC5 matrix.

Forward stores `vals` (CSR order of the conversion) into the matrix and
computes y = A x; backward computes dx = A^T dy (spc5_spmv_t) and
dvals[e] = dy[row(e)] * x[col(e)] over the stored entries
(spc5_values_grad).  Argument marshalling only: the arithmetic runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import spc5 as _c


class SpMVFunction(torch.autograd.Function):
    """y = SpMVFunction.apply(M, vals, x) with M an spc5.Matrix converted from
    the same CSR pattern; vals [nnz] FP64 (CSR order), x [ncols]."""

    @staticmethod
    def forward(ctx, M, vals, x):
        info = M.info()
        dt = torch.float64 if info["value_dtype"] == _c.SPC5_F64 else torch.float32
        vals_c = vals.detach().to(torch.float64).contiguous()
        x_c = x.detach().to(dt).contiguous()
        _c.spc5_set_values(M, vals_c)
        y = torch.empty(info["nrows"], dtype=dt, device=x.device)
        _c.spc5_spmv(M, x_c, y)
        ctx.M = M
        ctx.nnz = info["nnz"]
        ctx.ncols = info["ncols"]
        ctx.save_for_backward(x_c)
        return y

    @staticmethod
    def backward(ctx, gy):
        (x_c,) = ctx.saved_tensors
        gy = gy.to(x_c.dtype).contiguous()
        dvals = dx = None
        if ctx.needs_input_grad[1]:
            dvals = torch.empty(ctx.nnz, dtype=x_c.dtype, device=x_c.device)
            _c.spc5_values_grad(ctx.M, gy, x_c, dvals)
        if ctx.needs_input_grad[2]:
            dx = torch.empty(ctx.ncols, dtype=x_c.dtype, device=x_c.device)
            _c.spc5_spmv_t(ctx.M, gy, dx)
        return None, dvals, dx


def spmv(M, vals, x):
    """Differentiable y = A(vals) x."""
    return SpMVFunction.apply(M, vals, x)
