"""Helpers for the GPU parity tests: move a synthetic CSR to the device,
convert it through the C-ABI, and read the library's arrays back."""
from __future__ import annotations

import numpy as np

import paper_2307_14774_gb300 as spc5

FP64_TOL = 1e-13  # |y - y_ref| <= 1e-13 * sum_j |a_ij x_j| per row


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def to_device(A):
    torch = torch_cuda()
    return (torch.from_numpy(np.ascontiguousarray(A.rowptr)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.colidx)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.vals)).cuda())


def convert(A, r, c, dev=None):
    rowptr, colidx, vals = dev if dev is not None else to_device(A)
    M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rowptr, colidx, vals, r=r, c=c)
    return M


def exported(M) -> dict:
    t = spc5.export_tensors(M)
    torch = torch_cuda()
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in t.items()}
    return out


def spmv(M, x: np.ndarray, y0: np.ndarray | None = None, alpha=1.0, beta=0.0) -> np.ndarray:
    torch = torch_cuda()
    dx = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    nrows = M.info()["nrows"]
    dy = (torch.from_numpy(np.ascontiguousarray(y0)).cuda() if y0 is not None
          else torch.full((nrows,), float("nan"), dtype=torch.float64, device="cuda"))
    spc5.spc5_spmv(M, dx, dy, alpha, beta)
    torch.cuda.synchronize()
    return dy.cpu().numpy()


def assert_conversion_equal(M, S, A):
    """GPU arrays must equal the oracle's byte for byte."""
    g = exported(M)
    info = M.info()
    assert info["nblocks"] == S.nblocks
    assert np.array_equal(g["block_rowptr"].astype(np.int64), S.block_rowptr)
    npanels = S.npanels
    first_rows = np.minimum(np.arange(npanels + 1) * S.r, A.nrows)
    assert np.array_equal(g["panel_vptr"].astype(np.int64), A.rowptr[first_rows].astype(np.int64))
    assert np.array_equal(g["block_colidx"], S.block_colidx)
    packed = S.packed_masks()
    assert np.array_equal(g["block_masks"].view(np.uint8).reshape(packed.shape), packed)
    assert np.array_equal(g["values"].view(np.uint64), S.values.view(np.uint64))


def assert_within_tol(y, y_ref, scale, tol=FP64_TOL, extra=None):
    bound = tol * scale if extra is None else tol * (scale + extra)
    err = np.abs(y - y_ref)
    bad = np.flatnonzero(~(err <= bound))
    assert bad.size == 0, (f"{bad.size} rows out of tolerance; worst row {bad[0]}: "
                           f"y={y[bad[0]]!r} ref={y_ref[bad[0]]!r} bound={bound[bad[0]]!r}")
