"""GPU parity against the CPU oracle, through the C-ABI: conversion bit-exact,
SpMV within the FP64 tolerance |y - y_ref| <= 1e-13 * sum_j |a_ij x_j|.

Sizes span many tiles, ragged tails (rows not a multiple of r, empty rows
and panels, panels longer than a warp's round) and the degenerate cases."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import (assert_conversion_equal, assert_within_tol, convert, exported, spmv,
                        to_device, torch_cuda)

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]


def _mats():
    return [
        synth.laplace2d(128, 128),                       # the 5-point configuration
        synth.laplace2d(37, 29),                         # n not a multiple of 8
        synth.stencil27(24, 23, 22, values="normal"),
        synth.fem3d(6000, seed=2),
        synth.powerlaw(60_000, seed=3),                  # long rows, empty-free but skewed
        synth.uniform(20_000, 16, seed=4),
        synth.bernoulli(301, 157, 0.02, seed=7, integer_values=False),  # empty rows/panels
        synth.bernoulli(97, 300, 0.6, seed=8, integer_values=False),
        synth.dense(200, values="normal"),
    ]


@pytest.fixture(scope="module")
def mats():
    torch_cuda()
    return _mats()


@pytest.mark.parametrize("conv", ["auto", "flat"])
@pytest.mark.parametrize("r,c", BETAS)
def test_conversion_bit_exact(monkeypatch, mats, r, c, conv):
    """Both converters: the panel-local one (taken when no panel holds more
    than 1024 entries) and the flat passes (the other matrices, or forced)."""
    if conv == "flat":
        monkeypatch.setenv("SPC5_CONVERT", "flat")
    for A in mats:
        M = convert(A, r, c)
        S = oracle.convert(A, r, c)
        assert_conversion_equal(M, S, A)
        assert M.info()["filling"] == pytest.approx(S.filling(), rel=0, abs=1e-15)


@pytest.mark.parametrize("r,c", BETAS)
def test_conversion_many_blocks_per_panel(r, c):
    """Panels of a few hundred entries, each entry a block of its own (columns
    nine apart): more blocks per panel than the panel-local converter keeps
    in shared memory (256), so the conversion falls back to the flat passes
    after counting; bit-exact all the same."""
    torch_cuda()
    rng = np.random.default_rng(12)
    rp, ci = [0], []
    for i in range(40):
        k = 300 if i % 3 else 20
        cols = np.sort(rng.choice(5000, k, replace=False)) * 9
        ci.append(cols.astype(np.int32))
        rp.append(rp[-1] + k)
    colidx = np.concatenate(ci)
    A = synth.CSR(40, 45_000, np.array(rp, np.int32), colidx, rng.normal(size=len(colidx)),
                  "spread")
    M = convert(A, r, c)
    assert M.info()["nblocks"] > 256
    assert_conversion_equal(M, oracle.convert(A, r, c), A)
    x = synth.vector_uniform(A.ncols, seed=5)
    y_ref, scale = oracle.csr_spmv(A, x)
    assert_within_tol(spmv(M, x), y_ref, scale)


@pytest.mark.parametrize("r,c", BETAS)
def test_spmv_fp64_tolerance(mats, r, c):
    for A in mats:
        x = synth.vector_uniform(A.ncols, seed=11)
        M = convert(A, r, c)
        y = spmv(M, x)
        y_ref, scale = oracle.csr_spmv(A, x)
        assert_within_tol(y, y_ref, scale)


@pytest.mark.parametrize("r,c", BETAS)
def test_spmv_integer_matrices_exact(r, c):
    """Integer values and x: every partial sum is exact in FP64 in any
    order, so the GPU must equal the dense product bit for bit."""
    for seed, (nr, nc, d) in enumerate([(64, 64, 0.3), (129, 77, 0.5), (33, 500, 0.9)]):
        A = synth.bernoulli(nr, nc, d, seed=seed, integer_values=True)
        x = synth.vector_int(nc, -7, 7, seed=seed)
        y = spmv(convert(A, r, c), x)
        assert np.array_equal(y, A.todense() @ x)


@pytest.mark.parametrize("r,c", BETAS)
def test_laplacian_times_ones(r, c):
    A = synth.stencil27(21, 19, 17, values="poisson")
    y = spmv(convert(A, r, c), np.ones(A.ncols))
    assert np.array_equal(y, 26.0 - (np.diff(A.rowptr) - 1))


@pytest.mark.parametrize("r,c", [(1, 8), (4, 8), (8, 4)])
def test_alpha_beta(r, c):
    A = synth.fem3d(3000, seed=5)
    x = synth.vector_uniform(A.ncols, seed=1)
    y0 = synth.vector_normal(A.nrows, seed=2)
    M = convert(A, r, c)
    y_ref, scale = oracle.csr_spmv(A, x)
    for alpha, beta in [(1.0, 0.0), (-2.5, 0.0), (1.0, 1.0), (0.5, -3.0), (0.0, 2.0)]:
        y = spmv(M, x, y0.copy(), alpha, beta)
        expect = alpha * y_ref + beta * y0
        assert_within_tol(y, expect, abs(alpha) * scale, extra=np.abs(beta * y0))
    # beta == 0 never reads y: NaN in y must not propagate
    y = spmv(M, x, np.full(A.nrows, np.nan), 1.0, 0.0)
    assert np.all(np.isfinite(y))


def test_host_vectors_match_device_vectors():
    A = synth.stencil27(20, 20, 20, values="normal")
    M = convert(A, 4, 8)
    x = synth.vector_uniform(A.ncols, seed=3)
    y_dev = spmv(M, x)
    y_host = np.full(A.nrows, np.nan)
    spc5.spc5_spmv(M, x, y_host)  # numpy: host pointers
    assert np.array_equal(y_host, y_dev)
    y0 = synth.vector_normal(A.nrows, seed=1)
    y_host = y0.copy()
    spc5.spc5_spmv(M, x, y_host, 2.0, -1.0)
    assert np.array_equal(y_host, spmv(M, x, y0.copy(), 2.0, -1.0))


def test_host_csr_input_matches_device_csr_input():
    A = synth.powerlaw(20_000, seed=9)
    M_host = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, A.rowptr, A.colidx, A.vals, r=2, c=8)
    M_dev = convert(A, 2, 8)
    gh, gd = exported(M_host), exported(M_dev)
    for k in gh:
        assert np.array_equal(gh[k], gd[k])


@pytest.mark.parametrize("plan", ["0", "1", "2", "3"])
@pytest.mark.parametrize("r,c", BETAS)
def test_degenerate_shapes(monkeypatch, r, c, plan):
    monkeypatch.setenv("SPC5_FLAT", plan)
    cases = [
        synth.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0])),
        synth.CSR(5, 9, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0)),  # no entries
        synth.CSR(3, 1, np.array([0, 1, 1, 2], np.int32), np.array([0, 0], np.int32),
                  np.array([2.0, -1.0])),                                          # one column
        synth.bernoulli(1, 1000, 0.7, seed=3, integer_values=False),               # one long row
        synth.bernoulli(9, 17, 0.0, seed=1),                                       # empty again
        synth.dense(1, 3000, values="normal"),                                     # one dense row
        synth.dense(3000, 1, values="normal"),                                     # one column
    ]
    for A in cases:
        M = convert(A, r, c)
        assert M.info()["flat"] == int(plan)
        assert_conversion_equal(M, oracle.convert(A, r, c), A)
        x = synth.vector_uniform(A.ncols, seed=2)
        y_ref, scale = oracle.csr_spmv(A, x)
        assert_within_tol(spmv(M, x), y_ref, scale)
        y0 = synth.vector_normal(A.nrows, seed=4)
        assert_within_tol(spmv(M, x, y0.copy(), 2.0, -1.0), 2.0 * y_ref - y0, 2.0 * scale,
                          extra=np.abs(y0))


def test_explicit_zeros_are_kept():
    A = synth.bernoulli(50, 50, 0.5, seed=4, integer_values=True)
    assert (A.vals == 0).any()
    S = oracle.convert(A, 4, 8)
    assert_conversion_equal(convert(A, 4, 8), S, A)


@pytest.mark.parametrize("conv", ["auto", "flat"])
def test_invalid_csr_is_rejected_on_device(monkeypatch, conv):
    torch = torch_cuda()
    if conv == "flat":
        monkeypatch.setenv("SPC5_CONVERT", "flat")
    A = synth.bernoulli(40, 40, 0.3, seed=5)
    row = int(np.argmax(np.diff(A.rowptr) >= 2))
    a = A.rowptr[row]
    bad_cols = A.colidx.copy()
    bad_cols[a], bad_cols[a + 1] = bad_cols[a + 1], bad_cols[a]
    out_cols = A.colidx.copy()
    out_cols[-1] = 40
    bad_rowptr = A.rowptr.copy()
    bad_rowptr[-1] += 1
    dec_rowptr = A.rowptr.copy()
    dec_rowptr[5] = dec_rowptr[6] + 1
    for rowptr, colidx, code in [(A.rowptr, bad_cols, "SPC5_EUNSORTED"),
                                 (A.rowptr, out_cols, "SPC5_ERANGE"),
                                 (bad_rowptr, A.colidx, "SPC5_EROWPTR"),
                                 (dec_rowptr, A.colidx, "SPC5_EROWPTR")]:
        with pytest.raises(spc5.SPC5Error) as ei:
            spc5.spc5_convert_csr(40, 40, A.nnz, torch.from_numpy(rowptr).cuda(),
                                  torch.from_numpy(colidx).cuda(),
                                  torch.from_numpy(A.vals).cuda(), r=4, c=8)
        assert ei.value.name == code
    # the context is still usable afterwards
    y = spmv(convert(A, 4, 8), np.ones(40))
    assert np.array_equal(y, A.todense() @ np.ones(40))


@pytest.mark.parametrize("log2g", [0, 1, 2, 3])
def test_direct_kernel_lane_mappings(monkeypatch, log2g):
    """The direct tile kernel with every lanes-per-row mapping and every row
    body (set-bit loop, predicated loop, row stream, queued row stream,
    four-block rounds, row stream passing empty blocks within a trip, row
    stream at 64 warps per SM, pipelined row stream), with and without
    long-panel pieces."""
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", "0")
    monkeypatch.setenv("SPC5_LOG2G_GROUP", str(log2g))
    A = synth.powerlaw(30_000, seed=12)
    x = synth.vector_uniform(A.ncols, seed=4)
    y_ref, scale = oracle.csr_spmv(A, x)
    for r, c in [(1, 8), (4, 4), (8, 4)]:
        for body in ("0", "1", "2", "3", "4", "5", "6", "7"):
            for vcap in ("", "2048"):
                monkeypatch.setenv("SPC5_BODY", body)
                if vcap:
                    monkeypatch.setenv("SPC5_VCAP", vcap)
                    monkeypatch.setenv("SPC5_BCAP", "256")
                else:
                    monkeypatch.delenv("SPC5_VCAP", raising=False)
                    monkeypatch.delenv("SPC5_BCAP", raising=False)
                M = convert(A, r, c)
                assert M.info()["lanes_per_row"] == 1 << min(log2g, 5 - {1: 0, 4: 2, 8: 3}[r])
                assert_within_tol(spmv(M, x), y_ref, scale)


STAGED_SETTINGS = [
    # (env, expect pieces) -- small stages force fat groups, segment tiles and pieces
    ({}, False),
    ({"SPC5_VCAP": "512", "SPC5_BCAP": "128"}, True),
    ({"SPC5_VCAP": "512", "SPC5_BCAP": "128", "SPC5_STAGES": "2", "SPC5_CONSUMERS": "5"}, True),
    ({"SPC5_LOG2G_GROUP": "2", "SPC5_BODY": "0"}, False),
    ({"SPC5_LOG2G_GROUP": "1", "SPC5_BODY": "1", "SPC5_STAGES": "3", "SPC5_CONSUMERS": "1"}, False),
    ({"SPC5_BODY": "2"}, False),
    ({"SPC5_BODY": "3", "SPC5_VCAP": "512", "SPC5_BCAP": "128", "SPC5_CONSUMERS": "3"}, True),
    ({"SPC5_BODY": "2", "SPC5_LOG2G_GROUP": "2", "SPC5_STAGES": "2", "SPC5_CONSUMERS": "6"}, False),
]


@pytest.mark.parametrize("setting", range(len(STAGED_SETTINGS)))
@pytest.mark.parametrize("r,c", BETAS)
def test_staged_kernel_plans(monkeypatch, setting, r, c):
    """The staged kernel under different plans: group tiles only, fat groups
    with segment tiles and long panels cut into pieces (fixup), a two-stage
    ring with more consumers than stages, both row bodies."""
    env, expect_pieces = STAGED_SETTINGS[setting]
    monkeypatch.setenv("SPC5_KERNEL", "1")
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    mats = [synth.powerlaw(40_000, seed=21), synth.fem3d(4000, seed=3),
            synth.bernoulli(333, 5000, 0.2, seed=2, integer_values=False)]
    saw_pieces = False
    for A in mats:
        x = synth.vector_uniform(A.ncols, seed=6)
        y_ref, scale = oracle.csr_spmv(A, x)
        M = convert(A, r, c)
        info = M.info()
        saw_pieces |= info["long_panels"] > 0
        y0 = synth.vector_normal(A.nrows, seed=3)
        assert_within_tol(spmv(M, x), y_ref, scale)
        assert_within_tol(spmv(M, x, y0.copy(), -1.5, 0.5), -1.5 * y_ref + 0.5 * y0,
                          1.5 * scale, extra=np.abs(0.5 * y0))
        assert M.info()["device_error"] == 0
    if expect_pieces:
        assert saw_pieces


@pytest.mark.parametrize("kernel", ["0", "1"])
def test_integer_exact_with_pieces(monkeypatch, kernel):
    """Integer data through pieces and fixup: bit-exact, both kernels."""
    monkeypatch.setenv("SPC5_KERNEL", kernel)
    monkeypatch.setenv("SPC5_FLAT", "0")
    monkeypatch.setenv("SPC5_VCAP", "512")
    monkeypatch.setenv("SPC5_BCAP", "128")
    A = synth.bernoulli(40, 20_000, 0.3, seed=9, integer_values=True)
    x = synth.vector_int(A.ncols, -3, 3, seed=1)
    for r, c in BETAS:
        M = convert(A, r, c)
        assert M.info()["long_panels"] > 0
        assert np.array_equal(spmv(M, x), A.todense() @ x)


@pytest.mark.parametrize("r,c", BETAS)
def test_row_groups_from_the_tile_counter(monkeypatch, r, c):
    """Row-group tiles taken from the self-resetting tile counter instead of
    grid-stride: every body, with and without pieces, three products in a
    row (the counter must be back at zero after each launch), through
    spc5_spmv and spc5_spmv_noalloc (which counts on the library's own
    counter)."""
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", "0")
    monkeypatch.setenv("SPC5_DYNAMIC", "1")
    A = synth.powerlaw(30_000, seed=21)
    x = synth.vector_uniform(A.ncols, seed=6)
    y_ref, scale = oracle.csr_spmv(A, x)
    torch = torch_cuda()
    for body in ("0", "1", "2", "3", "4", "5", "6", "7"):
        for vcap in ("", "2048"):
            monkeypatch.setenv("SPC5_BODY", body)
            if vcap:
                monkeypatch.setenv("SPC5_VCAP", vcap)
                monkeypatch.setenv("SPC5_BCAP", "256")
            else:
                monkeypatch.delenv("SPC5_VCAP", raising=False)
                monkeypatch.delenv("SPC5_BCAP", raising=False)
            M = convert(A, r, c)
            for _ in range(3):
                assert_within_tol(spmv(M, x), y_ref, scale)
            dx = torch.from_numpy(x).cuda()
            dy = torch.full((A.nrows,), float("nan"), dtype=torch.float64, device="cuda")
            for _ in range(2):
                spc5.spc5_spmv_noalloc(M, dx, dy)
                torch.cuda.synchronize()
                assert_within_tol(dy.cpu().numpy(), y_ref, scale)

