"""Rows far longer than a tile: a panel cut into hundreds of pieces, whose
partial sums a fixup adds.  y = A x within |y - y_ref| <= 1e-13 *
sum_j |a_ij x_j| for every plan, the hybrid form (a row of isolated values
becomes hundreds of scalar pieces) and the batched path with k right-hand
sides (r * k partials per piece, up to 128), against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, convert, spmv, to_device, torch_cuda

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]


def _long_rows(nrows=70, ncols=400_000, seed=11):
    """Rows 0, 5 and 17: about 300,000 random columns each; row 33: every
    8th column (single-value blocks); the rest: up to 40 random columns."""
    rng = np.random.default_rng(seed)
    rp, ci = [0], []
    for i in range(nrows):
        if i in (0, 5, 17):
            cols = np.flatnonzero(rng.random(ncols) < 0.75)
        elif i == 33:
            cols = np.arange(3, ncols, 8)
        else:
            cols = np.sort(rng.choice(ncols, int(rng.integers(0, 41)), replace=False))
        ci.append(cols.astype(np.int32))
        rp.append(rp[-1] + len(cols))
    colidx = np.concatenate(ci)
    vals = rng.normal(size=len(colidx))
    return synth.CSR(nrows, ncols, np.array(rp, np.int32), colidx, vals, "long_rows")


@pytest.fixture(scope="module")
def long_rows():
    torch_cuda()
    return _long_rows()


@pytest.mark.parametrize("plan", ["0", "1", "2", "3"])
@pytest.mark.parametrize("r,c", BETAS)
def test_long_rows_every_plan(monkeypatch, long_rows, r, c, plan):
    monkeypatch.setenv("SPC5_FLAT", plan)
    A = long_rows
    x = synth.vector_uniform(A.ncols, seed=4)
    y_ref, scale = oracle.csr_spmv(A, x)
    for hybrid in (False, True):
        conv = spc5.spc5_convert_hybrid if hybrid else spc5.spc5_convert_csr
        M = conv(A.nrows, A.ncols, A.nnz, *to_device(A), r=r, c=c)
        info = M.info()
        assert info["long_panels"] > 0
        if hybrid:
            assert info["nscalars"] >= 49_000
        assert_within_tol(spmv(M, x), y_ref, scale)
        y0 = synth.vector_normal(A.nrows, seed=6)
        assert_within_tol(spmv(M, x, y0.copy(), 0.75, -2.0), 0.75 * y_ref - 2.0 * y0,
                          0.75 * scale, extra=np.abs(2.0 * y0))


@pytest.mark.parametrize("k", [1, 16])
def test_long_rows_batched(long_rows, k):
    torch = torch_cuda()
    A = long_rows
    Ms = [spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *to_device(A), r=r, c=c)
          for r, c in BETAS]
    X = synth.vector_uniform(A.ncols * k, seed=9).reshape(A.ncols, k)
    dX = [torch.from_numpy(X).cuda().contiguous() for _ in Ms]
    dY = [torch.full((A.nrows, k), float("nan"), dtype=torch.float64, device="cuda")
          for _ in Ms]
    spc5.spc5_spmv_batched(Ms, dX, dY, k)
    torch.cuda.synchronize()
    for Y in dY:
        Yh = Y.cpu().numpy()
        for j in range(k):
            y_ref, scale = oracle.csr_spmv(A, X[:, j])
            assert_within_tol(Yh[:, j], y_ref, scale)


@pytest.mark.parametrize("r,c", [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)])
def test_small_dense_matrix_is_cut_into_pieces(monkeypatch, r, c):
    """A small matrix with long rows (dense 600 x 700) gives few row groups;
    the planner cuts its panels into pieces so that every SM gets work, and
    the pieces' partial sums are added by the fixup kernel: same result as
    the oracle, every row written (y starts as NaN)."""
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", "0")
    for key in ("SPC5_VCAP", "SPC5_BCAP", "SPC5_BODY", "SPC5_LOG2G_GROUP"):
        monkeypatch.delenv(key, raising=False)
    A = synth.dense(600, 700, values="normal")
    x = synth.vector_uniform(A.ncols, seed=9)
    y_ref, scale = oracle.csr_spmv(A, x)
    M = convert(A, r, c)
    info = M.info()
    assert info["long_panels"] == info["npanels"] and info["pieces"] >= 2 * info["npanels"]
    for _ in range(2):
        assert_within_tol(spmv(M, x), y_ref, scale)
