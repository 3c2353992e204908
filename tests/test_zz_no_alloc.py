"""spc5_spmv_noalloc, the entry point for callers that cannot allocate device
memory during a product (a loop that must never reach the allocator, a
library limited to the memory its application hands it): its partial sums
live in a fixed array inside the library.  Checked through the C ABI
against spc5_spmv on two calls in a row, plus its size limit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, convert, torch_cuda

pytestmark = pytest.mark.gpu


def _run(fn, M, x, nrows, alpha=1.0, beta=0.0, y0=None):
    torch = torch_cuda()
    dx = torch.from_numpy(x).cuda()
    dy = (torch.from_numpy(y0.copy()).cuda() if y0 is not None
          else torch.full((nrows,), float("nan"), dtype=torch.float64, device="cuda"))
    fn(M, dx, dy, alpha, beta)
    torch.cuda.synchronize()
    return dy.cpu().numpy()


@pytest.mark.parametrize("plan", ["rows", "staged", "flat", "expanded", "vflat", "hybrid"])
def test_noalloc_matches_spmv_twice(monkeypatch, plan):
    monkeypatch.setenv("SPC5_KERNEL", "1" if plan == "staged" else "0")
    monkeypatch.setenv("SPC5_FLAT", {"flat": "1", "expanded": "2", "vflat": "3",
                                          "hybrid": "1"}.get(plan, "0"))
    A = synth.powerlaw(200_000, seed=17)          # long rows: split into pieces
    if plan == "hybrid":                          # scalar rows cut into pieces too
        from gpuhelpers import to_device
        M = spc5.spc5_convert_hybrid(A.nrows, A.ncols, A.nnz, *to_device(A), r=4, c=8)
    else:
        M = convert(A, 4, 8)
    info = M.info()
    assert info["long_panels"] > 0               # the scratch array is used
    assert info["pieces"] > 0
    if plan == "hybrid":                         # and its region after the blocks' sums
        assert info["scalar_pieces"] > 0
    assert info["pieces"] * 4 + info["scalar_pieces"] <= 131072
    assert info["flat"] == {"flat": 1, "expanded": 2, "vflat": 3, "hybrid": 1}.get(plan, 0)
    for call, seed in enumerate((1, 2)):         # two calls in a row, different x
        x = synth.vector_uniform(A.ncols, seed=seed)
        y_ref, scale = oracle.csr_spmv(A, x)
        y_alloc = _run(spc5.spc5_spmv, M, x, A.nrows)
        y_noalloc = _run(spc5.spc5_spmv_noalloc, M, x, A.nrows)
        assert_within_tol(y_noalloc, y_alloc, scale)
        assert_within_tol(y_noalloc, y_ref, scale)
        y0 = synth.vector_normal(A.nrows, seed=call)
        y_ab = _run(spc5.spc5_spmv_noalloc, M, x, A.nrows, 2.0, -0.5, y0)
        assert_within_tol(y_ab, _run(spc5.spc5_spmv, M, x, A.nrows, 2.0, -0.5, y0),
                          2.0 * scale, extra=np.abs(0.5 * y0))


def test_noalloc_rejects_oversized_scratch_and_host_vectors(monkeypatch):
    torch = torch_cuda()
    monkeypatch.setenv("SPC5_KERNEL", "1")
    monkeypatch.setenv("SPC5_VCAP", "512")
    monkeypatch.setenv("SPC5_BCAP", "128")
    A = synth.dense(16, 600_000, values="normal")   # 2 panels of 8 rows cut into ~20000 pieces
    M = convert(A, 8, 4)
    info = M.info()
    assert info["long_panels"] > 0
    assert info["pieces"] * 8 > 131072           # more partial sums than the array holds
    x = torch.from_numpy(synth.vector_uniform(A.ncols, seed=3)).cuda()
    y = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_spmv_noalloc(M, x, y)
    assert ei.value.name == "SPC5_EOVERFLOW"
    assert "131072" in str(ei.value)
    small = convert(synth.laplace2d(64, 64), 4, 8)
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_spmv_noalloc(small, np.ones(4096), np.zeros(4096))
    assert ei.value.name == "SPC5_EINVAL"
    # the library still works afterwards
    spc5.spc5_spmv(M, x, y)
    torch.cuda.synchronize()
    y_ref, scale = oracle.csr_spmv(A, x.cpu().numpy())
    assert_within_tol(y.cpu().numpy(), y_ref, scale)
