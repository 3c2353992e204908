"""The transposed copy (spc5_build_transpose): A^T converted to beta(r,c) on
the device from A's stored blocks, after which spc5_spmv_t is an ordinary
product over it.  Checked through the C ABI against the oracle's transposed
CSR product (|dx - dx_ref| <= tol * sum_i |a_ij g_i|), bit for bit against
spc5_spmv over a matrix converted from the oracle's transposed CSR, for
run-to-run determinism, after spc5_set_values, and for its rejections."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, convert, spmv, to_device, torch_cuda

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]
TOL = {"f64": 1e-13, "f32": 2e-6, "bf16": 1e-2}


def _mats():
    return [synth.stencil27(12, 11, 10, values="normal"), synth.fem3d(900, seed=1),
            synth.powerlaw(30_000, seed=5), synth.uniform(5_000, 16, seed=4),
            synth.bernoulli(70, 130, 0.2, seed=4, integer_values=False),   # rectangular
            synth.bernoulli(301, 157, 0.02, seed=7, integer_values=False),  # empty rows/columns
            synth.laplace2d(37, 29)]


@pytest.fixture(scope="module")
def mats():
    torch_cuda()
    return _mats()


def _spmv_t(M, g, ncols, dtype):
    torch = torch_cuda()
    dg = torch.from_numpy(g).cuda().to(dtype)
    dx = torch.full((ncols,), float("nan"), dtype=dtype, device="cuda")
    spc5.spc5_spmv_t(M, dg, dx)
    torch.cuda.synchronize()
    return dx.double().cpu().numpy()


@pytest.mark.parametrize("r,c", BETAS)
def test_transposed_product_fp64(mats, r, c):
    torch = torch_cuda()
    for A in mats:
        g = synth.vector_uniform(A.nrows, seed=3)
        M = convert(A, r, c)
        spc5.spc5_build_transpose(M)
        assert M.info()["transposed"] == 1
        dx = _spmv_t(M, g, A.ncols, torch.float64)
        ref, scale = oracle.csr_spmv_t(A, g)
        assert_within_tol(dx, ref, scale)
        assert np.array_equal(dx, _spmv_t(M, g, A.ncols, torch.float64))   # deterministic
        # the same product as a matrix converted from the transposed CSR
        T = oracle.transpose(A)
        T = synth.CSR(T.nrows, T.ncols, T.rowptr, T.colidx, T.vals, "transpose")
        assert np.array_equal(dx, spmv(convert(T, r, c), g))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("r,c", [(1, 8), (2, 4), (4, 8), (8, 4)])
def test_transposed_product_reduced_precision(mats, r, c, dtype):
    torch = torch_cuda()
    code = {"f32": spc5.SPC5_F32, "bf16": spc5.SPC5_BF16}[dtype]
    for A in mats:
        g = synth.vector_uniform(A.nrows, seed=5)
        M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *to_device(A), store_dtype=code,
                                  r=r, c=c)
        spc5.spc5_build_transpose(M)
        dx = _spmv_t(M, g.astype(np.float32).astype(np.float64), A.ncols, torch.float32)
        ref, scale = oracle.csr_spmv_t(A, g.astype(np.float32).astype(np.float64))
        assert_within_tol(dx, ref, scale, tol=TOL[dtype])
        assert np.array_equal(dx, _spmv_t(M, g, A.ncols, torch.float32))


@pytest.mark.parametrize("r,c", [(1, 8), (4, 8), (8, 4)])
def test_set_values_refreshes_the_transposed_copy(mats, r, c):
    torch = torch_cuda()
    for A in mats[:4]:
        M = convert(A, r, c)
        spc5.spc5_build_transpose(M)
        new = synth.vector_normal(A.nnz, seed=9)
        spc5.spc5_set_values(M, torch.from_numpy(new).cuda())
        B = synth.CSR(A.nrows, A.ncols, A.rowptr, A.colidx, new, "new values")
        g = synth.vector_uniform(A.nrows, seed=4)
        ref, scale = oracle.csr_spmv_t(B, g)
        assert_within_tol(_spmv_t(M, g, A.ncols, torch.float64), ref, scale)
        x = synth.vector_uniform(A.ncols, seed=6)
        y_ref, yscale = oracle.csr_spmv(B, x)
        assert_within_tol(spmv(M, x), y_ref, yscale)


def test_long_columns():
    """Columns of more than 1024 entries (ranked by a CTA each): a dense
    block of 2000 rows in the first columns."""
    torch = torch_cuda()
    n, w = 2000, 40
    rowptr = np.arange(0, (n + 1) * w, w, dtype=np.int32)
    colidx = np.tile(np.arange(w, dtype=np.int32) * 3, n)
    A = synth.CSR(n, 3 * w, rowptr, colidx, synth.vector_normal(n * w, seed=1), "tall")
    for r, c in [(1, 8), (4, 8)]:
        M = convert(A, r, c)
        spc5.spc5_build_transpose(M)
        g = synth.vector_uniform(n, seed=2)
        ref, scale = oracle.csr_spmv_t(A, g)
        dx = _spmv_t(M, g, A.ncols, torch.float64)
        assert_within_tol(dx, ref, scale)
        T = oracle.transpose(A)
        T = synth.CSR(T.nrows, T.ncols, T.rowptr, T.colidx, T.vals, "transpose")
        assert np.array_equal(dx, spmv(convert(T, r, c), g))


def test_rejections_leave_the_atomic_product():
    torch = torch_cuda()
    # a column of 70000 entries: more than the column sort takes
    n = 70_000
    rowptr = np.arange(n + 1, dtype=np.int32)
    colidx = np.zeros(n, dtype=np.int32)
    A = synth.CSR(n, 4, rowptr, colidx, synth.vector_normal(n, seed=1), "one column")
    M = convert(A, 4, 8)
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_build_transpose(M)
    assert ei.value.name == "SPC5_EUNSUPPORTED"
    assert M.info()["transposed"] == 0
    g = synth.vector_uniform(n, seed=2)
    ref, scale = oracle.csr_spmv_t(A, g)
    assert_within_tol(_spmv_t(M, g, A.ncols, torch.float64), ref, scale)
    H = synth.powerlaw(20_000, seed=3)
    Mh = spc5.spc5_convert_hybrid(H.nrows, H.ncols, H.nnz, *to_device(H), r=4, c=8)
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_build_transpose(Mh)
    assert ei.value.name == "SPC5_EUNSUPPORTED"
