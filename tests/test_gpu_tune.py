"""Autotuner: spc5_tune re-plans a converted matrix for each lanes-per-row
candidate and keeps the fastest; spc5_convert_tuned also picks the block
shape.  Whatever it picks, the product must stay within the FP64 tolerance
of the oracle and the stored arrays must stay those of the chosen shape."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_conversion_equal, assert_within_tol, convert, spmv, to_device, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("r,c", [(1, 8), (4, 8), (8, 4)])
def test_tune_keeps_results(r, c):
    torch = torch_cuda()
    A = synth.powerlaw(60_000, seed=13)
    M = convert(A, r, c)
    x = synth.vector_uniform(A.ncols, seed=2)
    dx = torch.from_numpy(x).cuda()
    dy = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    info = spc5.spc5_tune(M, dx, dy, iters=3)
    assert info["tuned_us"] > 0
    assert info["lanes_per_row"] in (1, 2, 4, 8)
    y_ref, scale = oracle.csr_spmv(A, x)
    assert_within_tol(spmv(M, x), y_ref, scale)
    assert_conversion_equal(M, oracle.convert(A, r, c), A)


@pytest.mark.parametrize("dtype", [spc5.SPC5_F64, spc5.SPC5_F32])
def test_convert_tuned_picks_a_valid_shape(dtype):
    torch = torch_cuda()
    A = synth.stencil27(30, 30, 30, values="normal")
    rp, ci, vv = to_device(A)
    M = spc5.spc5_convert_tuned(A.nrows, A.ncols, A.nnz, rp, ci, vv, store_dtype=dtype,
                                shapes=[(1, 8), (4, 8), (2, 4)], iters=3)
    info = M.info()
    assert (info["r"], info["c"]) in [(1, 8), (4, 8), (2, 4)]
    assert info["tuned_us"] > 0
    x = synth.vector_uniform(A.ncols, seed=4)
    y_ref, scale = oracle.csr_spmv(A, x)
    if dtype == spc5.SPC5_F64:
        assert_within_tol(spmv(M, x), y_ref, scale)
    else:
        dxx = torch.from_numpy(x.astype(np.float32)).cuda()
        dyy = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
        spc5.spc5_spmv(M, dxx, dyy)
        torch.cuda.synchronize()
        assert_within_tol(dyy.cpu().numpy().astype(np.float64), y_ref, scale, tol=2e-6)


def test_convert_tuned_ex_ranks_by_the_row_group_plan():
    """rows_plan ranks the shapes by their fastest row-group plan: the shape
    kept has the smallest tuned_rows_us among the shapes, each tuned alone
    (allowing 50 % for timing noise between tuning runs on a shared GPU),
    and it serves the batched kernel."""
    torch = torch_cuda()
    A = synth.powerlaw(80_000, seed=21)
    rp, ci, vv = to_device(A)
    shapes = [(1, 8), (4, 4), (8, 4)]
    M = spc5.spc5_convert_tuned_ex(A.nrows, A.ncols, A.nnz, rp, ci, vv, shapes=shapes, iters=5,
                                   rows_plan=True)
    info = M.info()
    assert (info["r"], info["c"]) in shapes
    assert 0 < info["tuned_rows_us"] and 0 < info["tuned_us"] <= info["tuned_rows_us"]
    x = synth.vector_uniform(A.ncols, seed=5)
    dx = torch.from_numpy(x).cuda()
    dy = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    alone = {}
    for r, c in shapes:
        Ms = convert(A, r, c)
        alone[(r, c)] = spc5.spc5_tune(Ms, dx, dy, iters=5)["tuned_rows_us"]
    assert info["tuned_rows_us"] <= 1.5 * min(alone.values())
    y_ref, scale = oracle.csr_spmv(A, x)
    assert_within_tol(spmv(M, x), y_ref, scale)
    Y = torch.full((A.nrows, 1), float("nan"), dtype=torch.float64, device="cuda")
    spc5.spc5_spmv_batched([M], [dx.reshape(-1, 1)], [Y], 1)
    torch.cuda.synchronize()
    assert_within_tol(Y.cpu().numpy()[:, 0], y_ref, scale)
