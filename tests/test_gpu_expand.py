"""The three plans for skewed rows.  Block-balanced (SPC5_FLAT=1): the
blocks of runs of whole panels dealt to the lanes four blocks per lane per
round, row sums by a segmented warp scan, long panels cut into pieces of a
fixed block count.  Value-balanced (SPC5_FLAT=3): the same tiles, each
round of 256 blocks staged in shared memory and its values split into 32
equal runs.  Expanded (SPC5_FLAT=2): runs of whole panels (at most 1024
values and 128 rows) whose values a warp lays out row by row in shared
memory and splits evenly over its lanes; panels of more than 1024 values
cut into pieces.  Pieces' row sums are added by a fixup kernel.

Checked through the C ABI against the CPU oracle at the FP64 tolerance
|y - y_ref| <= 1e-13 * sum_j |a_ij x_j| (and the FP32/BF16 bounds of the
precision tests), bit-exact on integer data, over matrices with skewed row
lengths, runs of empty rows and panels, ragged last panels, rows cut between
lanes and tiles of one to many rounds of blocks."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, convert, spmv, to_device, torch_cuda

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]
PLANS = ["1", "2", "3"]


def _sparse_rows(n=6000, ncols=700, seed=9):
    """Rows mostly empty: long runs of empty panels inside one round."""
    rng = np.random.default_rng(seed)
    rp, ci, vv = [0], [], []
    for i in range(n):
        if i % 97 == 0 or (i > n // 2 and i % 5 == 0):
            k = int(rng.integers(1, 12))
            ci += sorted(rng.choice(ncols, k, replace=False).tolist())
            vv += rng.normal(size=k).tolist()
        rp.append(len(ci))
    return synth.CSR(n, ncols, np.array(rp, np.int32), np.array(ci, np.int32),
                     np.array(vv, np.float64))


def _mats():
    return [
        synth.powerlaw(60_000, seed=3),
        synth.powerlaw(20_000, sigma=50.0, long_row=150, seed=8),
        _sparse_rows(),
        synth.bernoulli(301, 157, 0.02, seed=7, integer_values=False),
        synth.laplace2d(37, 29),
        synth.stencil27(17, 18, 19, values="normal"),
        synth.fem3d(3000, seed=2),
        synth.uniform(20_000, 16, seed=4),
        synth.dense(70, 3000, values="normal"),
    ]


@pytest.fixture(scope="module")
def mats():
    torch_cuda()
    return _mats()


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("r,c", BETAS)
def test_skewed_plans_fp64_tolerance(monkeypatch, mats, r, c, plan):
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", plan)
    saw_pieces = False
    for A in mats:
        M = convert(A, r, c)
        info = M.info()
        assert info["flat"] == int(plan)
        saw_pieces |= info["long_panels"] > 0
        x = synth.vector_uniform(A.ncols, seed=5)
        y_ref, scale = oracle.csr_spmv(A, x)
        assert_within_tol(spmv(M, x), y_ref, scale)
        y0 = synth.vector_normal(A.nrows, seed=2)
        assert_within_tol(spmv(M, x, y0.copy(), -1.5, 0.5), -1.5 * y_ref + 0.5 * y0,
                          1.5 * scale, extra=np.abs(0.5 * y0))
    assert saw_pieces


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("r,c", BETAS)
def test_skewed_plans_integer_exact(monkeypatch, r, c, plan):
    """Integer data: every order of summation gives the exact result."""
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", plan)
    for A in (synth.bernoulli(40, 20_000, 0.3, seed=9, integer_values=True),
              synth.bernoulli(3000, 400, 0.01, seed=4, integer_values=True)):
        x = synth.vector_int(A.ncols, -3, 3, seed=1)
        M = convert(A, r, c)
        assert M.info()["flat"] == int(plan)
        assert np.array_equal(spmv(M, x), A.todense() @ x)


def test_skewed_plans_default_choice():
    """The converter picks a block-balanced plan for skewed rows (values split
    over the lanes for r >= 4) and keeps row groups for a stencil."""
    torch_cuda()
    for r, c in BETAS:
        skewed = convert(synth.powerlaw(60_000, seed=3), r, c).info()
        assert skewed["group_efficiency"] >= 0.7 or skewed["flat"] == (3 if r >= 4 else 1)
    assert convert(synth.powerlaw(60_000, seed=3), 1, 8).info()["group_efficiency"] < 0.7
    regular = convert(synth.stencil27(20, 20, 20, values="normal"), 4, 8).info()
    assert regular["group_efficiency"] >= 0.7 and regular["flat"] == 0


@pytest.mark.parametrize("plan", PLANS)
def test_skewed_plans_counter_resets_across_launches_and_graph_replay(monkeypatch, plan):
    """Tiles are taken from a counter that each launch resets: back-to-back
    launches and CUDA-graph replays give the same y."""
    torch = torch_cuda()
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", plan)
    A = synth.powerlaw(50_000, seed=6)
    M = convert(A, 2, 8)
    x = synth.vector_uniform(A.ncols, seed=9)
    y_ref, scale = oracle.csr_spmv(A, x)
    dx = torch.from_numpy(x).cuda()
    dy = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    first = None
    for _ in range(5):
        dy.fill_(float("nan"))
        spc5.spc5_spmv(M, dx, dy)
        torch.cuda.synchronize()
        y = dy.cpu().numpy()
        assert_within_tol(y, y_ref, scale)
        if first is None:
            first = y
        assert np.array_equal(y, first)   # the same tiles, the same order of sums
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        spc5.spc5_spmv(M, dx, dy)      # warm-up on the capture stream
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        spc5.spc5_spmv(M, dx, dy)
    for _ in range(3):
        dy.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(dy.cpu().numpy(), first)


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("dtype,tol", [("f32", 2e-6), ("bf16", 1e-2)])
@pytest.mark.parametrize("r,c", BETAS)
def test_skewed_plans_reduced_precision(monkeypatch, mats, dtype, tol, r, c, plan):
    torch = torch_cuda()
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", plan)
    code = spc5.SPC5_F32 if dtype == "f32" else spc5.SPC5_BF16
    for A in mats[:4]:
        rowptr, colidx, vals = to_device(A)
        M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, rowptr, colidx, vals,
                                  store_dtype=code, r=r, c=c)
        assert M.info()["flat"] == int(plan)
        x32 = synth.vector_uniform(A.ncols, seed=7).astype(np.float32)
        dy = torch.full((A.nrows,), float("nan"), dtype=torch.float32, device="cuda")
        spc5.spc5_spmv(M, torch.from_numpy(x32).cuda(), dy)
        torch.cuda.synchronize()
        y_ref, scale = oracle.csr_spmv(A, x32.astype(np.float64))
        assert_within_tol(dy.cpu().numpy().astype(np.float64), y_ref, scale, tol=tol)
