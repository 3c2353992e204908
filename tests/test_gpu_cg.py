"""Mixed-precision iterative-refinement CG (spc5_ircg) on the SPD 27-point
Poisson matrix (26 on the diagonal, -1 off it): the final FP64 residual,
recomputed by the CPU oracle, must satisfy ||b - A x|| / ||b|| <= 1e-10 for
every inner precision (FP32 and BF16 storage are exact for these values)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import to_device, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("inner", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("r,c", [(4, 8), (1, 8)])
def test_ircg_reaches_1e_10(inner, r, c):
    torch = torch_cuda()
    A = synth.stencil27(24, 22, 20, values="poisson")
    rp, ci, vv = to_device(A)
    A64 = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, r=r, c=c)
    code = {"f32": spc5.SPC5_F32, "bf16": spc5.SPC5_BF16, "f64": spc5.SPC5_F64}[inner]
    Alo = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, store_dtype=code, r=r, c=c)
    b = synth.vector_uniform(A.nrows, seed=7)
    db = torch.from_numpy(b).cuda()
    dx = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    rep = spc5.spc5_ircg(A64, Alo, db, dx, tol=1e-10, max_outer=30, inner_tol=1e-3,
                         max_inner=500)
    x = dx.cpu().numpy()
    Ax, _ = oracle.csr_spmv(A, x)
    relres = np.linalg.norm(b - Ax) / np.linalg.norm(b)
    assert relres <= 1e-10, (rep, relres)
    assert rep["relres"] <= 1e-10
    assert 1 <= rep["outer_iters"] <= 30 and rep["inner_iters"] >= rep["outer_iters"]


def test_ircg_zero_rhs_and_rejections():
    torch = torch_cuda()
    A = synth.stencil27(8, 8, 8, values="poisson")
    rp, ci, vv = to_device(A)
    A64 = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, r=4, c=8)
    A32 = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, store_dtype=spc5.SPC5_F32,
                                r=4, c=8)
    db = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    dx = torch.ones(A.nrows, dtype=torch.float64, device="cuda")
    rep = spc5.spc5_ircg(A64, A32, db, dx)
    assert rep["outer_iters"] == 0 and float(dx.abs().max()) == 0.0
    with pytest.raises(spc5.SPC5Error):
        spc5.spc5_ircg(A32, A32, db, dx)  # the outer matrix must be FP64


def test_ircg_is_deterministic():
    """Two solves of one system give the same iterates bit for bit: every
    reduction sums its per-block partials in block order (the last block to
    finish does it), and the SpMV is deterministic."""
    torch = torch_cuda()
    A = synth.stencil27(30, 30, 30, values="poisson")
    rp, ci, vv = to_device(A)
    A64 = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, r=4, c=8)
    A32 = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rp, ci, vv, store_dtype=spc5.SPC5_F32,
                                r=4, c=8)
    db = torch.from_numpy(synth.vector_uniform(A.nrows, seed=5)).cuda()
    xs, reps = [], []
    for _ in range(2):
        dx = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        reps.append(spc5.spc5_ircg(A64, A32, db, dx, tol=1e-10, max_outer=30, inner_tol=1e-3,
                                   max_inner=500))
        xs.append(dx.cpu().numpy())
    assert reps[0] == reps[1]
    assert np.array_equal(xs[0], xs[1])
