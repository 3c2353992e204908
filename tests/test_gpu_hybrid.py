"""Hybrid beta(r,c) (single-value blocks as scalar CSR entries) through the C
ABI: the GPU split equals the oracle's byte for byte (block part and
scalars), and y = A x within the FP64 tolerance |y - y_ref| <= 1e-13 *
sum_j |a_ij x_j| (FP32/BF16 bounds for reduced storage), exact on integer
data, with every block-part plan, scalar rows longer than a tile (pieces),
empty rows, a block part with no blocks (every block a single value) and
no scalars (dense)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, exported, spmv, to_device, torch_cuda

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]


def _sparse_rows(n=5000, ncols=900, seed=3):
    rng = np.random.default_rng(seed)
    rp, ci, vv = [0], [], []
    for i in range(n):
        if i % 7 == 0 or i % 11 == 0:
            k = int(rng.integers(1, 9))
            ci += sorted(rng.choice(ncols, k, replace=False).tolist())
            vv += rng.normal(size=k).tolist()
        rp.append(len(ci))
    return synth.CSR(n, ncols, np.array(rp, np.int32), np.array(ci, np.int32),
                     np.array(vv, np.float64))


def _mats():
    return [synth.powerlaw(60_000, seed=3), synth.uniform(20_000, 16, seed=4), _sparse_rows(),
            synth.bernoulli(301, 157, 0.02, seed=7, integer_values=False),
            synth.stencil27(14, 13, 12, values="normal"), synth.dense(40, 300, values="normal")]


@pytest.fixture(scope="module")
def mats():
    torch_cuda()
    return _mats()


def _convert(A, r, c, store=spc5.SPC5_F64):
    rowptr, colidx, vals = to_device(A)
    return spc5.spc5_convert_hybrid(A.nrows, A.ncols, A.nnz, rowptr, colidx, vals,
                                    store_dtype=store, r=r, c=c)


def _panel_vptr(B):
    pc = np.array([sum(bin(int(w)).count("1") for w in row) for row in B.block_masks], np.int64)
    cum = np.concatenate([[0], np.cumsum(pc)])
    return cum[B.block_rowptr]


@pytest.mark.parametrize("r,c", BETAS)
def test_hybrid_split_bit_exact(mats, r, c):
    for A in mats:
        M = _convert(A, r, c)
        info = M.info()
        B, Sc = oracle.hybrid_split(oracle.convert(A, r, c))
        g = exported(M)
        assert info["hybrid"] == 1 and info["nnz"] == A.nnz
        assert info["nscalars"] == len(Sc.vals) and info["nblocks"] == B.nblocks
        assert np.array_equal(g["block_rowptr"].astype(np.int64), B.block_rowptr)
        assert np.array_equal(g["panel_vptr"].astype(np.int64), _panel_vptr(B))
        assert np.array_equal(g["block_colidx"], B.block_colidx)
        assert np.array_equal(g["block_masks"].view(np.uint8).reshape(-1),
                              B.packed_masks().reshape(-1))
        assert np.array_equal(g["values"].view(np.uint64), B.values.view(np.uint64))
        assert np.array_equal(g["s_rowptr"], Sc.rowptr)
        assert np.array_equal(g["s_colidx"], Sc.colidx)
        assert np.array_equal(g["s_vals"].view(np.uint64), Sc.vals.view(np.uint64))


@pytest.mark.parametrize("plan", ["0", "1", "2", "3"])
@pytest.mark.parametrize("r,c", BETAS)
def test_hybrid_spmv_fp64(monkeypatch, mats, r, c, plan):
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", plan)
    for A in mats:
        M = _convert(A, r, c)
        x = synth.vector_uniform(A.ncols, seed=5)
        y_ref, scale = oracle.csr_spmv(A, x)
        assert_within_tol(spmv(M, x), y_ref, scale)
        y0 = synth.vector_normal(A.nrows, seed=2)
        assert_within_tol(spmv(M, x, y0.copy(), -1.5, 0.5), -1.5 * y_ref + 0.5 * y0,
                          1.5 * scale, extra=np.abs(0.5 * y0))


@pytest.mark.parametrize("r,c", BETAS)
def test_hybrid_integer_exact(r, c):
    torch_cuda()
    for A in (synth.bernoulli(40, 20_000, 0.01, seed=9, integer_values=True),
              synth.bernoulli(3000, 400, 0.01, seed=4, integer_values=True)):
        x = synth.vector_int(A.ncols, -3, 3, seed=1)
        M = _convert(A, r, c)
        assert M.info()["nscalars"] > 0
        assert np.array_equal(spmv(M, x), A.todense() @ x)


@pytest.mark.parametrize("dtype,code,tol", [("f32", spc5.SPC5_F32, 2e-6),
                                            ("bf16", spc5.SPC5_BF16, 1e-2)])
@pytest.mark.parametrize("r,c", [(1, 8), (4, 8), (8, 4)])
def test_hybrid_reduced_precision(mats, dtype, code, tol, r, c):
    torch = torch_cuda()
    for A in mats[:4]:
        M = _convert(A, r, c, code)
        _, Sc = oracle.hybrid_split(oracle.convert(A, r, c))
        g = exported(M)
        expect = oracle.quantize(Sc.vals, dtype)
        assert np.array_equal(g["s_vals"].view(np.uint8).view(expect.dtype), expect)
        x32 = synth.vector_uniform(A.ncols, seed=7).astype(np.float32)
        dy = torch.full((A.nrows,), float("nan"), dtype=torch.float32, device="cuda")
        spc5.spc5_spmv(M, torch.from_numpy(x32).cuda(), dy)
        torch.cuda.synchronize()
        y_ref, scale = oracle.csr_spmv(A, x32.astype(np.float64))
        assert_within_tol(dy.cpu().numpy().astype(np.float64), y_ref, scale, tol=tol)


def test_hybrid_unsupported_operations():
    torch = torch_cuda()
    A = synth.powerlaw(5000, seed=2)
    M = _convert(A, 4, 8)
    x = torch.zeros(A.ncols, dtype=torch.float64, device="cuda")
    y = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    for call in (lambda: spc5.spc5_spmv_t(M, y, x),
                 lambda: spc5.spc5_values_grad(M, y, x, torch.zeros(A.nnz, dtype=torch.float64,
                                                                   device="cuda")),
                 lambda: spc5.spc5_set_values(M, torch.from_numpy(A.vals).cuda()),
                 lambda: spc5.spc5_spmv_batched([M], [x], [y])):
        with pytest.raises(spc5.SPC5Error) as ei:
            call()
        assert ei.value.name == "SPC5_EUNSUPPORTED"
    plain = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *to_device(A), r=4, c=8)
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_export_hybrid(plain)
    assert ei.value.name == "SPC5_EINVAL"
    # the handle still works
    y_ref, scale = oracle.csr_spmv(A, np.ones(A.ncols))
    assert_within_tol(spmv(M, np.ones(A.ncols)), y_ref, scale)


def test_hybrid_tune_and_ircg():
    """The tuner and the refinement solver take hybrid matrices."""
    torch = torch_cuda()
    A = synth.powerlaw(30_000, seed=5)
    M = _convert(A, 2, 4)
    x = synth.vector_uniform(A.ncols, seed=3)
    dx, dy = torch.from_numpy(x).cuda(), torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    spc5.spc5_tune(M, dx, dy, iters=2)
    y_ref, scale = oracle.csr_spmv(A, x)
    assert_within_tol(spmv(M, x), y_ref, scale)
    P = synth.stencil27(20, 20, 20, values="poisson")
    rp, ci, vv = to_device(P)
    A64 = spc5.spc5_convert_hybrid(P.nrows, P.ncols, P.nnz, rp, ci, vv, r=8, c=4)
    A32 = spc5.spc5_convert_hybrid(P.nrows, P.ncols, P.nnz, rp, ci, vv,
                                   store_dtype=spc5.SPC5_F32, r=8, c=4)
    b = torch.from_numpy(synth.vector_uniform(P.nrows, seed=8)).cuda()
    sol = torch.zeros(P.nrows, dtype=torch.float64, device="cuda")
    rep = spc5.spc5_ircg(A64, A32, b, sol, tol=1e-10, max_outer=40, inner_tol=1e-3,
                         max_inner=2000)
    assert rep["relres"] <= 1e-10
