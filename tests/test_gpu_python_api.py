"""The binding's convenience layer: Matrix.from_csr on a torch sparse CSR
tensor, A @ x for a vector and for k right-hand sides, A.t() @ g, checked
against the oracle (FP64 tolerance |y - y_ref| <= 1e-13 * sum_j |a_ij x_j|)
and the converted arrays against the oracle converter."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_conversion_equal, assert_within_tol, torch_cuda

pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore:Sparse CSR tensor support is in beta")]


def _sparse(A, torch):
    return torch.sparse_csr_tensor(torch.from_numpy(A.rowptr.astype(np.int64)),
                                   torch.from_numpy(A.colidx.astype(np.int64)),
                                   torch.from_numpy(A.vals), size=(A.nrows, A.ncols),
                                   dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("r,c", [(1, 8), (4, 8), (8, 4)])
def test_from_csr_matmul_and_transpose(r, c):
    torch = torch_cuda()
    A = synth.powerlaw(30_000, seed=9)
    M = spc5.Matrix.from_csr(_sparse(A, torch), r=r, c=c)
    assert M.shape == (A.nrows, A.ncols) and M.t().shape == (A.ncols, A.nrows)
    assert_conversion_equal(M, oracle.convert(A, r, c), A)
    x = synth.vector_uniform(A.ncols, seed=2)
    y_ref, scale = oracle.csr_spmv(A, x)
    y = M @ torch.from_numpy(x).cuda()
    assert_within_tol(y.cpu().numpy(), y_ref, scale)
    # A^T g against the oracle's product with the transposed CSR
    g = synth.vector_normal(A.nrows, seed=3)
    dx_ref, dscale = oracle.csr_spmv(_transposed(A), g)
    dx = M.t() @ torch.from_numpy(g).cuda()
    assert_within_tol(dx.cpu().numpy(), dx_ref, dscale)


def _transposed(A):
    """CSR of A^T: the entries sorted by (column, row)."""
    rows = np.repeat(np.arange(A.nrows, dtype=np.int64), np.diff(A.rowptr))
    order = np.lexsort((rows, A.colidx))
    counts = np.bincount(A.colidx, minlength=A.ncols)
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return synth.CSR(A.ncols, A.nrows, rowptr, rows[order].astype(np.int32),
                     A.vals[order], "transposed")


@pytest.mark.parametrize("k", [3, 4])
def test_matmul_several_right_hand_sides(k):
    torch = torch_cuda()
    A = synth.stencil27(12, 11, 10, values="normal")
    M = spc5.Matrix.from_csr(_sparse(A, torch), r=2, c=4)
    X = synth.vector_uniform(A.ncols * k, seed=4).reshape(A.ncols, k)
    Y = (M @ torch.from_numpy(X).cuda()).cpu().numpy()
    assert Y.shape == (A.nrows, k)
    for j in range(k):
        y_ref, scale = oracle.csr_spmv(A, np.ascontiguousarray(X[:, j]))
        assert_within_tol(Y[:, j], y_ref, scale)


def test_from_csr_rejects_other_layouts():
    torch = torch_cuda()
    with pytest.raises(TypeError):
        spc5.Matrix.from_csr(torch.zeros(4, 4, device="cuda"))
