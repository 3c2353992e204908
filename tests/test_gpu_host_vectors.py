"""spc5_spmv with host vectors: pageable x and y go through device buffers;
a pinned y is written in place by the kernels through its device mapping
(and read there when beta != 0).  The kernels and their inputs are the same
as with device vectors, so y must be bit-identical in all three cases, for
every plan, with alpha and beta, and within the FP64 tolerance of the
oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, convert, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("plan", ["0", "1", "3"])
@pytest.mark.parametrize("r,c", [(1, 8), (4, 8)])
def test_pinned_pageable_and_device_vectors_agree(monkeypatch, r, c, plan):
    torch = torch_cuda()
    monkeypatch.setenv("SPC5_FLAT", plan)
    A = synth.powerlaw(40_000, seed=8)
    M = convert(A, r, c)
    assert M.info()["flat"] == int(plan)
    x = synth.vector_uniform(A.ncols, seed=3)
    y0 = synth.vector_normal(A.nrows, seed=5)
    y_ref, scale = oracle.csr_spmv(A, x)
    for alpha, beta in ((1.0, 0.0), (0.5, -1.5)):
        dy = torch.from_numpy(y0.copy()).cuda()
        spc5.spc5_spmv(M, torch.from_numpy(x).cuda(), dy, alpha, beta)
        torch.cuda.synchronize()
        y_dev = dy.cpu().numpy()
        y_pageable = y0.copy()
        spc5.spc5_spmv(M, x, y_pageable, alpha, beta)
        px = torch.from_numpy(x).pin_memory()
        py = torch.from_numpy(y0.copy()).pin_memory()
        spc5.spc5_spmv(M, px, py, alpha, beta)
        y_pinned = py.numpy()
        assert np.array_equal(y_pageable.view(np.uint64), y_dev.view(np.uint64))
        assert np.array_equal(y_pinned.view(np.uint64), y_dev.view(np.uint64))
        assert_within_tol(y_pinned, alpha * y_ref + beta * y0, abs(alpha) * scale,
                          extra=np.abs(beta * y0))


def test_pinned_y_with_device_x_and_fp32_storage():
    torch = torch_cuda()
    A = synth.stencil27(20, 21, 22, values="normal")
    rp, ci, vv = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals))
    M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, store_dtype=spc5.SPC5_F32,
                              r=4, c=8)
    x32 = synth.vector_uniform(A.ncols, seed=1).astype(np.float32)
    dx = torch.from_numpy(x32).cuda()
    dy = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
    spc5.spc5_spmv(M, dx, dy)
    torch.cuda.synchronize()
    py = torch.empty(A.nrows, dtype=torch.float32).pin_memory()
    spc5.spc5_spmv(M, dx, py)
    assert np.array_equal(py.numpy().view(np.uint32), dy.cpu().numpy().view(np.uint32))
