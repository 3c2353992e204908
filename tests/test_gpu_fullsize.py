"""Parity at the benchmark's full sizes, with the same matrices and calls the
benchmark times: 27-point stencil on 100^3, FEM 3x3 blocks on 1e6 nodes,
power-law rows on 2e6 rows, uniform columns on 1e6 rows, every beta(r,c).
The conversion is compared with the oracle's byte for byte and every row of
y within the FP64 tolerance."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpuhelpers import (assert_conversion_equal, assert_within_tol, convert, spmv, to_device,
                        torch_cuda)

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]
WORKLOADS = ["stencil27", "fem3d", "powerlaw", "uniform"]


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
