"""Differentiation of y = A(vals) x through the C ABI:
dx = A^T g (spc5_spmv_t), dvals[e] = g[row(e)] * x[col(e)] (spc5_values_grad),
spc5_set_values, and the torch.autograd.Function built on them, checked
against the oracle, against central finite differences in FP64 (y is
bilinear in (vals, x), so the difference quotient is exact up to rounding)
and against torch.autograd.gradcheck."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, convert, spmv, torch_cuda
from paper_2307_14774_gb300.autograd import SpMVFunction

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]


def _mats():
    return [synth.stencil27(12, 11, 10, values="normal"), synth.powerlaw(30_000, seed=5),
            synth.bernoulli(70, 130, 0.2, seed=4, integer_values=False), synth.fem3d(900, seed=1)]


@pytest.mark.parametrize("r,c", BETAS)
def test_spmv_t_matches_oracle(r, c):
    torch = torch_cuda()
    for A in _mats():
        g = synth.vector_uniform(A.nrows, seed=3)
        dx0 = synth.vector_normal(A.ncols, seed=4)
        M = convert(A, r, c)
        ref, scale = oracle.csr_spmv_t(A, g)
        dg = torch.from_numpy(g).cuda()
        for alpha, beta in [(1.0, 0.0), (-0.5, 2.0)]:
            dx = torch.from_numpy(dx0.copy()).cuda()
            spc5.spc5_spmv_t(M, dg, dx, alpha, beta)
            torch.cuda.synchronize()
            assert_within_tol(dx.cpu().numpy(), alpha * ref + beta * dx0, abs(alpha) * scale,
                              extra=np.abs(beta * dx0))


@pytest.mark.parametrize("r,c", BETAS)
def test_values_grad_exact(r, c):
    """One rounded product per entry on both sides: bit-exact in FP64."""
    torch = torch_cuda()
    for A in _mats():
        g = synth.vector_normal(A.nrows, seed=5)
        x = synth.vector_uniform(A.ncols, seed=6)
        M = convert(A, r, c)
        dv = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
        spc5.spc5_values_grad(M, torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda(), dv)
        torch.cuda.synchronize()
        assert np.array_equal(dv.cpu().numpy(), oracle.values_grad(A, g, x))


@pytest.mark.parametrize("r,c", [(1, 8), (4, 8), (8, 4)])
def test_set_values(r, c):
    torch = torch_cuda()
    A = synth.powerlaw(20_000, seed=8)
    M = convert(A, r, c)
    new = synth.vector_normal(A.nnz, seed=9)
    spc5.spc5_set_values(M, torch.from_numpy(new).cuda())
    B = synth.CSR(A.nrows, A.ncols, A.rowptr, A.colidx, new)
    x = synth.vector_uniform(A.ncols, seed=1)
    y_ref, scale = oracle.csr_spmv(B, x)
    assert_within_tol(spmv(M, x), y_ref, scale)


def test_autograd_matches_finite_differences_and_dense_gradient():
    """27-point stencil on 16^3 (FP64): f = <w, A(vals) x>."""
    torch = torch_cuda()
    A = synth.stencil27(16, 16, 16, values="normal")
    M = convert(A, 4, 8)
    vals = torch.from_numpy(A.vals.copy()).cuda().requires_grad_(True)
    x = torch.from_numpy(synth.vector_uniform(A.ncols, seed=2)).cuda().requires_grad_(True)
    w = torch.from_numpy(synth.vector_normal(A.nrows, seed=3)).cuda()
    y = SpMVFunction.apply(M, vals, x)
    (y * w).sum().backward()
    gv, gx = vals.grad.cpu().numpy(), x.grad.cpu().numpy()
    wn, xn = w.cpu().numpy(), x.detach().cpu().numpy()
    # dense reference gradient
    D = A.todense()
    assert np.allclose(gx, D.T @ wn, rtol=0, atol=1e-12)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    assert np.array_equal(gv, wn[rows] * xn[A.colidx])

    def f(v, xx):
        with torch.no_grad():
            return float((SpMVFunction.apply(M, v, xx) * w).sum())

    h = 1e-3
    rng = np.random.default_rng(0)
    v0 = vals.detach().clone()
    for e in rng.choice(A.nnz, 40, replace=False):
        vp, vm = v0.clone(), v0.clone()
        vp[e] += h
        vm[e] -= h
        fd = (f(vp, x.detach()) - f(vm, x.detach())) / (2 * h)
        assert abs(fd - gv[e]) <= 1e-8 * (1 + abs(gv[e]))
    x0 = x.detach().clone()
    for j in rng.choice(A.ncols, 40, replace=False):
        xp, xm = x0.clone(), x0.clone()
        xp[j] += h
        xm[j] -= h
        fd = (f(v0, xp) - f(v0, xm)) / (2 * h)
        assert abs(fd - gx[j]) <= 1e-8 * (1 + abs(gx[j]))


def test_autograd_gradcheck_small():
    torch = torch_cuda()
    A = synth.bernoulli(23, 19, 0.3, seed=11, integer_values=False)
    M = convert(A, 2, 4)
    vals = torch.from_numpy(A.vals.copy()).cuda().requires_grad_(True)
    x = torch.from_numpy(synth.vector_uniform(A.ncols, seed=1)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v, xx: SpMVFunction.apply(M, v, xx), (vals, x),
                                    eps=1e-6, atol=1e-9)


def test_autograd_fp32_storage_against_dense_gradient():
    """FP32 value storage (the differentiation workload's precision): the
    gradients, computed in FP32, against the dense FP64 gradient of the same
    function on the FP32-rounded values and x, within FP32 rounding of
    sum |terms|; values gradient per stored entry, in CSR order."""
    torch = torch_cuda()
    A = synth.stencil27(16, 16, 16, values="normal")
    rowptr, colidx, vv = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals))
    M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rowptr, colidx, vv,
                              store_dtype=spc5.SPC5_F32, r=4, c=8)
    vals = torch.from_numpy(A.vals.copy()).cuda().requires_grad_(True)
    x32 = synth.vector_uniform(A.ncols, seed=2).astype(np.float32)
    x = torch.from_numpy(x32).cuda().requires_grad_(True)
    w = torch.from_numpy(synth.vector_normal(A.nrows, seed=3).astype(np.float32)).cuda()
    y = SpMVFunction.apply(M, vals, x)
    assert y.dtype == torch.float32
    (y * w).sum().backward()
    assert vals.grad.dtype == torch.float64 and x.grad.dtype == torch.float32
    gv, gx = vals.grad.cpu().numpy(), x.grad.cpu().numpy().astype(np.float64)
    wn = w.cpu().numpy().astype(np.float64)
    q = oracle.quantize(A.vals, "f32").astype(np.float64)
    Aq = synth.CSR(A.nrows, A.ncols, A.rowptr, A.colidx, q)
    D = Aq.todense()
    # dx = A^T w: FP32 accumulation of at most 27 terms per column
    bound = 30 * 2.0 ** -24 * (np.abs(D.T) @ np.abs(wn))
    assert np.all(np.abs(gx - D.T @ wn) <= bound)
    # dvals[e] = w[row] * x[col]: one FP32 product, exactly rounded
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    exact = wn[rows] * x32.astype(np.float64)[A.colidx]
    assert np.array_equal(gv, exact.astype(np.float32).astype(np.float64))
