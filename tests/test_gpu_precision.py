"""FP32 and BF16 value storage (FP32 x, y and accumulation).

Conversion: the stored values equal the oracle's beta(r,c) values rounded
by the oracle's own quantizer, bit for bit.  SpMV: against the FP64 oracle
on the original FP64 values and x,
    |y - y_ref| <= 2e-6 * S_i   (FP32 storage)
    |y - y_ref| <= 1e-2 * S_i   (BF16 storage),   S_i = sum_j |a_ij x_j|,
and, to isolate the kernel's arithmetic, against the FP64 oracle on the
dequantized values and x: |y - y_dq| <= (k_i + 2) * 2^-24 * S_i' for a row
of k_i entries (sequential FP32 accumulation bound)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, exported, to_device, torch_cuda

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]
DTYPES = {"f32": (spc5.SPC5_F32, 2e-6), "bf16": (spc5.SPC5_BF16, 1e-2)}


def _convert(A, r, c, dtype):
    rowptr, colidx, vals = to_device(A)
    return spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rowptr, colidx, vals,
                                 store_dtype=DTYPES[dtype][0], r=r, c=c)


def _spmv32(M, x32, nrows, y0=None, alpha=1.0, beta=0.0):
    torch = torch_cuda()
    dx = torch.from_numpy(x32).cuda()
    dy = (torch.from_numpy(y0.astype(np.float32)).cuda() if y0 is not None
          else torch.full((nrows,), float("nan"), dtype=torch.float32, device="cuda"))
    spc5.spc5_spmv(M, dx, dy, alpha, beta)
    torch.cuda.synchronize()
    return dy.cpu().numpy().astype(np.float64)


def _dequantized(A, dtype):
    q = oracle.quantize(A.vals, dtype)
    v = q.astype(np.float64) if dtype == "f32" else oracle.bf16_to_f64(q)
    return synth.CSR(A.nrows, A.ncols, A.rowptr, A.colidx, v)


def _mats():
    return [synth.stencil27(20, 21, 22, values="normal"), synth.fem3d(3000, seed=2),
            synth.powerlaw(40_000, seed=3), synth.laplace2d(50, 37),
            synth.bernoulli(101, 333, 0.05, seed=3, integer_values=False)]


@pytest.fixture(scope="module")
def mats():
    torch_cuda()
    return _mats()


@pytest.mark.parametrize("dtype", list(DTYPES))
@pytest.mark.parametrize("r,c", BETAS)
def test_quantized_conversion_bit_exact(mats, dtype, r, c):
    for A in mats:
        M = _convert(A, r, c, dtype)
        S = oracle.convert(A, r, c)
        g = exported(M)
        assert np.array_equal(g["block_colidx"], S.block_colidx)
        assert np.array_equal(g["block_masks"].view(np.uint8).reshape(S.nblocks, -1),
                              S.packed_masks())
        expect = oracle.quantize(S.values, dtype)
        raw = g["values"].view(np.uint8).view(expect.dtype)  # raw bytes of the stored values
        assert np.array_equal(raw, expect)


@pytest.mark.parametrize("dtype", list(DTYPES))
@pytest.mark.parametrize("r,c", BETAS)
def test_reduced_precision_spmv_error(mats, dtype, r, c):
    tol = DTYPES[dtype][1]
    for A in mats:
        x = synth.vector_uniform(A.ncols, seed=11)
        x32 = x.astype(np.float32)
        M = _convert(A, r, c, dtype)
        y = _spmv32(M, x32, A.nrows)
        y_ref, scale = oracle.csr_spmv(A, x)
        assert_within_tol(y, y_ref, scale, tol=tol)
        Adq = _dequantized(A, dtype)
        y_dq, scale_dq = oracle.csr_spmv(Adq, x32.astype(np.float64))
        k = np.diff(A.rowptr).astype(np.float64)
        assert np.all(np.abs(y - y_dq) <= (k + 2) * 2.0 ** -24 * scale_dq)


@pytest.mark.parametrize("body", ["0", "1", "2", "3", "4", "5", "6", "7"])
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_reduced_precision_integer_exact(monkeypatch, dtype, body):
    monkeypatch.setenv("SPC5_FLAT", "0")
    monkeypatch.setenv("SPC5_BODY", body)
    for seed in range(3):
        A = synth.bernoulli(77, 300, 0.4, seed=seed, integer_values=True)
        x = synth.vector_int(A.ncols, -3, 3, seed=seed).astype(np.float32)
        for r, c in BETAS:
            y = _spmv32(_convert(A, r, c, dtype), x, A.nrows)
            assert np.array_equal(y, A.todense() @ x.astype(np.float64))


@pytest.mark.parametrize("flat", ["0", "1", "2", "3"])
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_reduced_precision_pieces_alpha_beta_host(monkeypatch, dtype, flat):
    monkeypatch.setenv("SPC5_FLAT", flat)
    monkeypatch.setenv("SPC5_VCAP", "2048")
    monkeypatch.setenv("SPC5_BCAP", "256")
    tol = DTYPES[dtype][1]
    A = synth.powerlaw(50_000, seed=7)
    M = _convert(A, 4, 8, dtype)
    assert M.info()["long_panels"] > 0
    assert M.info()["flat"] == int(flat)
    x = synth.vector_uniform(A.ncols, seed=2)
    x32 = x.astype(np.float32)
    y0 = synth.vector_normal(A.nrows, seed=5).astype(np.float32)
    y_ref, scale = oracle.csr_spmv(A, x)
    y = _spmv32(M, x32, A.nrows, y0, 0.5, -2.0)
    assert_within_tol(y, 0.5 * y_ref - 2.0 * y0.astype(np.float64), 0.5 * scale, tol=tol,
                      extra=np.abs(2.0 * y0.astype(np.float64)) * 1e-3 / tol)
    y_host = np.zeros(A.nrows, np.float32)
    spc5.spc5_spmv(M, x32, y_host)  # host vectors
    assert np.array_equal(y_host.astype(np.float64), _spmv32(M, x32, A.nrows))
