"""FP32 and BF16 storage under every work mapping the autotuner can pick:
the row-group plan with every lanes-per-row count G in {1, 2, 4, 8} and every
row body (set-bit loop, predicated loop over the c bits, row stream, queued
row stream, four-block rounds, row stream passing empty blocks within a
trip, row stream at 64 warps per SM), with and without long panels cut into
pieces, and the block-balanced, expanded and value-balanced plans, for every
beta(r,c).  Each product is checked against the FP64 oracle on the original
values at the stated tolerance (2e-6 / 1e-2 * sum_j |a_ij x_j|) and, for the
kernel's FP32 arithmetic, against the oracle on the stored values and the
FP32 x: |y - y_dq| <= (k_i + 2) * 2^-24 * S_i' for a row of k_i entries."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, to_device, torch_cuda

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]
REDUCED = {"f32": (spc5.SPC5_F32, 2e-6), "bf16": (spc5.SPC5_BF16, 1e-2)}


@pytest.fixture(scope="module")
def case():
    torch_cuda()
    A = synth.powerlaw(30_000, seed=12)   # skewed rows: long panels and short ones
    x32 = synth.vector_uniform(A.ncols, seed=4).astype(np.float32)
    y_ref, scale = oracle.csr_spmv(A, x32.astype(np.float64))
    dq = {}
    for dt in REDUCED:
        q = oracle.quantize(A.vals, dt)
        v = q.astype(np.float64) if dt == "f32" else oracle.bf16_to_f64(q)
        dq[dt] = oracle.csr_spmv(synth.CSR(A.nrows, A.ncols, A.rowptr, A.colidx, v),
                                 x32.astype(np.float64))
    return A, x32, y_ref, scale, dq, to_device(A)


def _check(case, dtype, r, c):
    torch = torch_cuda()
    A, x32, y_ref, scale, dq, dev = case
    code, tol = REDUCED[dtype]
    M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *dev, store_dtype=code, r=r, c=c)
    dx = torch.from_numpy(x32).cuda()
    dy = torch.full((A.nrows,), float("nan"), dtype=torch.float32, device="cuda")
    spc5.spc5_spmv(M, dx, dy)
    torch.cuda.synchronize()
    y = dy.cpu().numpy().astype(np.float64)
    assert_within_tol(y, y_ref, scale, tol=tol)
    y_dq, scale_dq = dq[dtype]
    k = np.diff(A.rowptr).astype(np.float64)
    assert np.all(np.abs(y - y_dq) <= (k + 2) * 2.0 ** -24 * scale_dq)
    return M.info()


@pytest.mark.parametrize("dtype", list(REDUCED))
@pytest.mark.parametrize("log2g", [0, 1, 2, 3])
def test_row_groups_every_lane_count_and_body(monkeypatch, case, dtype, log2g):
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", "0")
    monkeypatch.setenv("SPC5_LOG2G_GROUP", str(log2g))
    for r, c in BETAS:
        for body in ("0", "1", "2", "3", "4", "5", "6", "7"):
            for vcap in ("", "2048"):
                monkeypatch.setenv("SPC5_BODY", body)
                if vcap:
                    monkeypatch.setenv("SPC5_VCAP", vcap)
                    monkeypatch.setenv("SPC5_BCAP", "256")
                else:
                    monkeypatch.delenv("SPC5_VCAP", raising=False)
                    monkeypatch.delenv("SPC5_BCAP", raising=False)
                info = _check(case, dtype, r, c)
                assert info["flat"] == 0
                assert info["lanes_per_row"] == 1 << min(log2g, 5 - {1: 0, 2: 1, 4: 2, 8: 3}[r])
                if vcap:
                    assert info["long_panels"] > 0


@pytest.mark.parametrize("dtype", list(REDUCED))
@pytest.mark.parametrize("plan", ["1", "2", "3"])
def test_skewed_row_plans_every_shape(monkeypatch, case, dtype, plan):
    monkeypatch.setenv("SPC5_FLAT", plan)
    for r, c in BETAS:
        info = _check(case, dtype, r, c)
        assert info["flat"] == int(plan)
