"""Parity at the benchmark's full sizes, with the same matrices and calls the
benchmark times: 27-point stencil on 100^3, FEM 3x3 blocks on 1e6 nodes,
power-law rows on 2e6 rows, uniform columns on 1e6 rows, every beta(r,c).
The conversion is compared with the oracle's byte for byte and every row of
y within the FP64 tolerance, under the planner's default mapping and under
the mapping spc5_tune picks (the benchmark tunes every matrix before timing
it).  The FP32 and BF16 storage forms the benchmark times (27-point and FEM,
every beta, tuned) are checked against the FP64 oracle at their stated
tolerances and, for the kernel's own FP32 arithmetic, against the oracle on
the stored (rounded) values."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import (assert_conversion_equal, assert_within_tol, convert, spmv, to_device,
                        torch_cuda)

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]
WORKLOADS = ["stencil27", "fem3d", "powerlaw", "uniform"]
TUNE_ITERS = 3  # as in the benchmark


@pytest.fixture(scope="module", params=WORKLOADS)
def workload(request):
    torch = torch_cuda()
    A = synth.workload(request.param, "full")
    x = synth.vector_uniform(A.ncols, seed=1)
    y_ref, scale = oracle.csr_spmv(A, x)
    dev = to_device(A)
    yield A, x, y_ref, scale, dev
    del dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("r,c", BETAS)
def test_fullsize(workload, r, c):
    A, x, y_ref, scale, dev = workload
    M = convert(A, r, c, dev)
    assert_within_tol(spmv(M, x), y_ref, scale)
    assert_conversion_equal(M, oracle.convert(A, r, c), A)


@pytest.mark.parametrize("r,c", BETAS)
def test_fullsize_tuned(workload, r, c):
    torch = torch_cuda()
    A, x, y_ref, scale, dev = workload
    M = convert(A, r, c, dev)
    dx = torch.from_numpy(x).cuda()
    dy = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    info = spc5.spc5_tune(M, dx, dy, iters=TUNE_ITERS)
    assert info["tuned_us"] > 0
    assert_within_tol(spmv(M, x), y_ref, scale)


REDUCED = {"f32": (spc5.SPC5_F32, 2e-6), "bf16": (spc5.SPC5_BF16, 1e-2)}


@pytest.fixture(scope="module", params=["stencil27", "fem3d"])
def reduced_workload(request):
    torch = torch_cuda()
    A = synth.workload(request.param, "full")
    x = synth.vector_uniform(A.ncols, seed=1)
    x32 = x.astype(np.float32)
    y_ref, scale = oracle.csr_spmv(A, x)
    dq = {}
    for dt in REDUCED:
        q = oracle.quantize(A.vals, dt)
        v = q.astype(np.float64) if dt == "f32" else oracle.bf16_to_f64(q)
        dq[dt] = oracle.csr_spmv(synth.CSR(A.nrows, A.ncols, A.rowptr, A.colidx, v),
                                 x32.astype(np.float64))
    dev = to_device(A)
    yield A, x32, y_ref, scale, dq, dev
    del dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", list(REDUCED))
@pytest.mark.parametrize("r,c", BETAS)
def test_fullsize_reduced_precision_tuned(reduced_workload, dtype, r, c):
    torch = torch_cuda()
    A, x32, y_ref, scale, dq, dev = reduced_workload
    code, tol = REDUCED[dtype]
    M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *dev, store_dtype=code, r=r, c=c)
    dx = torch.from_numpy(x32).cuda()
    dy = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
    spc5.spc5_tune(M, dx, dy, iters=TUNE_ITERS)
    dy.fill_(float("nan"))
    spc5.spc5_spmv(M, dx, dy)
    torch.cuda.synchronize()
    y = dy.cpu().numpy().astype(np.float64)
    assert_within_tol(y, y_ref, scale, tol=tol)
    y_dq, scale_dq = dq[dtype]
    k = np.diff(A.rowptr).astype(np.float64)
    assert np.all(np.abs(y - y_dq) <= (k + 2) * 2.0 ** -24 * scale_dq)
