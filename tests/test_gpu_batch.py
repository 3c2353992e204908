"""Batched products: many matrices of different sizes and block shapes, k
right-hand sides each, one launch (spc5_spmv_batched, spc5_batch_*),
checked column by column against the oracle; the batch run captured in a
CUDA graph and replayed."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, to_device, torch_cuda

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]


def _batch_mats(seed=0, count=12):
    mats = []
    for i in range(count):
        kind = (i + seed) % 4
        if kind == 0:
            mats.append(synth.laplace2d(20 + 7 * i, 13 + i))
        elif kind == 1:
            mats.append(synth.stencil27(6 + i, 5 + i % 3, 7, values="normal"))
        elif kind == 2:
            mats.append(synth.powerlaw(2000 + 1500 * i, seed=i))
        else:
            mats.append(synth.uniform(1000 + 300 * i, 16, seed=i))
    return mats


def _convert_all(mats, dtype, monkeypatch=None):
    out = []
    for i, A in enumerate(mats):
        r, c = BETAS[i % 6]
        if monkeypatch is not None:
            if i % 3 == 0:
                monkeypatch.setenv("SPC5_VCAP", "2048")
                monkeypatch.setenv("SPC5_BCAP", "256")
            else:
                monkeypatch.delenv("SPC5_VCAP", raising=False)
                monkeypatch.delenv("SPC5_BCAP", raising=False)
        rp, ci, vv = to_device(A)
        out.append(spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, store_dtype=dtype,
                                         r=r, c=c))
    return out


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_matches_oracle(monkeypatch, k, dtype):
    torch = torch_cuda()
    code = {"f64": spc5.SPC5_F64, "f32": spc5.SPC5_F32}[dtype]
    tdt = {"f64": torch.float64, "f32": torch.float32}[dtype]
    tol = {"f64": 1e-13, "f32": 2e-6}[dtype]
    mats = _batch_mats(seed=k)
    Ms = _convert_all(mats, code, monkeypatch)
    assert any(M.info()["long_panels"] > 0 for M in Ms)
    Xs = [synth.vector_uniform(A.ncols * k, seed=m).reshape(A.ncols, k) for m, A in enumerate(mats)]
    dX = [torch.from_numpy(X).to(tdt).cuda().contiguous() for X in Xs]
    dY = [torch.full((A.nrows, k), float("nan"), dtype=tdt, device="cuda") for A in mats]
    spc5.spc5_spmv_batched(Ms, dX, dY, k)
    for A, X, Y in zip(mats, Xs, dY):
        Yh = Y.double().cpu().numpy()
        if dtype == "f32":
            # the kernel's own FP32 arithmetic, against the oracle on the
            # stored (rounded) values and the FP32 x it was given
            Xq = X.astype(np.float32).astype(np.float64)
            Adq = synth.CSR(A.nrows, A.ncols, A.rowptr, A.colidx,
                            oracle.quantize(A.vals, "f32").astype(np.float64))
            nrow = np.diff(A.rowptr).astype(np.float64)
        for j in range(k):
            y_ref, scale = oracle.csr_spmv(A, X[:, j])
            assert_within_tol(Yh[:, j], y_ref, scale, tol=tol)
            if dtype == "f32":
                y_dq, scale_dq = oracle.csr_spmv(Adq, Xq[:, j])
                assert np.all(np.abs(Yh[:, j] - y_dq) <= (nrow + 2) * 2.0 ** -24 * scale_dq)


def test_batch_reuse_alpha_beta_and_graph_capture():
    torch = torch_cuda()
    k = 4
    mats = _batch_mats(seed=1, count=9)
    Ms = _convert_all(mats, spc5.SPC5_F64)
    Xs = [synth.vector_uniform(A.ncols * k, seed=m + 7).reshape(A.ncols, k) for m, A in enumerate(mats)]
    Y0 = [synth.vector_normal(A.nrows * k, seed=m).reshape(A.nrows, k) for m, A in enumerate(mats)]
    dX = [torch.from_numpy(X).cuda() for X in Xs]
    dY = [torch.from_numpy(Y.copy()).cuda() for Y in Y0]
    B = spc5.Batch(Ms, dX, dY, k)
    B.run(2.0, -1.0)
    torch.cuda.synchronize()
    expect = []
    for A, X, Y, Yd in zip(mats, Xs, Y0, dY):
        Yh = Yd.cpu().numpy()
        cols = []
        for j in range(k):
            y_ref, scale = oracle.csr_spmv(A, X[:, j])
            assert_within_tol(Yh[:, j], 2.0 * y_ref - Y[:, j], 2.0 * scale, extra=np.abs(Y[:, j]))
            cols.append((y_ref, scale))
        expect.append(cols)
    # capture y = A x in a CUDA graph, replay after changing the inputs in place
    for Yd in dY:
        Yd.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.run(1.0, 0.0, stream=s)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        B.run(1.0, 0.0, stream=torch.cuda.current_stream())
    for X, Xd in zip(Xs, dX):
        Xd.copy_(torch.from_numpy(-X))
    for Yd in dY:
        Yd.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    for cols, Yd in zip(expect, dY):
        Yh = Yd.cpu().numpy()
        for j, (y_ref, scale) in enumerate(cols):
            assert_within_tol(Yh[:, j], -y_ref, scale)


def test_batch_rejections():
    torch = torch_cuda()
    A = synth.laplace2d(10, 10)
    rp, ci, vv = to_device(A)
    M64 = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, r=4, c=8)
    M32 = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, store_dtype=spc5.SPC5_F32,
                                r=4, c=8)
    x = torch.zeros(100, 3, dtype=torch.float64, device="cuda")
    y = torch.zeros(100, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_spmv_batched([M64], [x], [y], 3)
    assert ei.value.name == "SPC5_EUNSUPPORTED"
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_spmv_batched([M64, M32], [x, x], [y, y], 1)
    assert ei.value.name == "SPC5_EINVAL"
