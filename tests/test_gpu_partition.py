"""Row-partitioned SpMV on one GPU (every part converted and multiplied on
its own, y assembled from the parts) against the CPU oracle: several part
counts including more parts than panels, every block shape, alpha and
beta."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpuhelpers import assert_within_tol, torch_cuda
from paper_2307_14774_gb300 import partition

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]


@pytest.mark.parametrize("r,c", BETAS)
def test_partitioned_product_matches_oracle(r, c):
    torch = torch_cuda()
    for A, nparts in ((synth.powerlaw(20_000, seed=3), 3), (synth.fem3d(1500, seed=2), 4),
                      (synth.laplace2d(5, 3), 9)):
        P = partition.PartitionedMatrix(A.nrows, A.ncols, A.rowptr, A.colidx, A.vals, r, c,
                                        nparts)
        x = synth.vector_uniform(A.ncols, seed=5)
        y0 = synth.vector_normal(A.nrows, seed=6)
        dx = torch.from_numpy(x).cuda()
        dy = torch.from_numpy(y0.copy()).cuda()
        P.spmv(dx, dy, 2.0, -1.0)
        torch.cuda.synchronize()
        y_ref, scale = oracle.csr_spmv(A, x)
        assert_within_tol(dy.cpu().numpy(), 2.0 * y_ref - y0, 2.0 * scale, extra=np.abs(y0))
