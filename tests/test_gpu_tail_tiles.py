"""The last round of the row-group kernel's tile dealing: when the tiles
left over after whole rounds over the resident warps would fill at most half
of them, the planner can cut those last groups into two tiles of half the
panels with twice the lanes per row (SPC5_HALVES=1 here; spc5_tune takes it
when faster).  On the 27-point 65^3 stencil at
beta(4,8) (68,657 panels, 8,583 group tiles) the plan must hold those half
tiles, and every consumer of the plan must still match the oracle: the SpMV
under several bodies and storage types, the transposed product and the
values gradient."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, convert, spmv, to_device, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stencil():
    torch_cuda()
    return synth.stencil27(65, 65, 65, values="normal", seed=3)


def _expected_tiles(torch, np_, gp):
    """Group tiles, plus one for every halved group with more than gp / 2
    panels (the last group may hold fewer)."""
    warps = torch.cuda.get_device_properties(0).multi_processor_count * 48
    t = -(-np_ // gp)
    rem = t % warps
    if not (t > warps and 0 < rem and 2 * rem <= warps):
        return t
    return t + sum(1 for g in range(t - rem, t) if np_ - g * gp > gp // 2)


@pytest.mark.parametrize("body", ["0", "2", "7"])
def test_half_tiles_fp64(monkeypatch, stencil, body):
    torch = torch_cuda()
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", "0")
    monkeypatch.setenv("SPC5_LOG2G_GROUP", "0")
    monkeypatch.setenv("SPC5_BODY", body)
    monkeypatch.setenv("SPC5_HALVES", "1")
    A = stencil
    x = synth.vector_uniform(A.ncols, seed=1)
    y_ref, scale = oracle.csr_spmv(A, x)
    M = convert(A, 4, 8)
    info = M.info()
    assert info["ntiles"] == _expected_tiles(torch, info["npanels"], 8)
    assert_within_tol(spmv(M, x), y_ref, scale)
    monkeypatch.setenv("SPC5_HALVES", "0")
    M0 = convert(A, 4, 8)
    assert M0.info()["ntiles"] == -(-info["npanels"] // 8)
    assert_within_tol(spmv(M0, x), y_ref, scale)
    if body == "0":
        g = synth.vector_uniform(A.nrows, seed=2)
        ref_t, scale_t = oracle.csr_spmv_t(A, g)
        dx = torch.zeros(A.ncols, dtype=torch.float64, device="cuda")
        spc5.spc5_spmv_t(M, torch.from_numpy(g).cuda(), dx)
        dv = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
        spc5.spc5_values_grad(M, torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda(), dv)
        torch.cuda.synchronize()
        assert_within_tol(dx.cpu().numpy(), ref_t, scale_t)
        assert np.array_equal(dv.cpu().numpy(), oracle.values_grad(A, g, x))


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-6), ("bf16", 1e-2)])
def test_half_tiles_reduced_precision(monkeypatch, stencil, dtype, tol):
    torch = torch_cuda()
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", "0")
    monkeypatch.setenv("SPC5_LOG2G_GROUP", "0")
    monkeypatch.setenv("SPC5_BODY", "0")
    monkeypatch.setenv("SPC5_HALVES", "1")
    A = stencil
    code = {"f32": spc5.SPC5_F32, "bf16": spc5.SPC5_BF16}[dtype]
    M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *to_device(A), store_dtype=code, r=4, c=8)
    info = M.info()
    assert info["ntiles"] == _expected_tiles(torch, info["npanels"], 8)
    x = synth.vector_uniform(A.ncols, seed=4).astype(np.float32)
    y = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
    spc5.spc5_spmv(M, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    y_ref, scale = oracle.csr_spmv(A, x.astype(np.float64))
    assert_within_tol(y.double().cpu().numpy(), y_ref, scale, tol=tol)
