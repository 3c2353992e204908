"""Pins for the CPU oracle: brute force, closed forms, invariants and the
paper's printed values.  None of these compare the oracle with itself."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
import synth
from bruteforce import dense_pattern, grid_convert, pack_word

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIX_BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]
ODD_BETAS = [(3, 5), (1, 1), (5, 3), (8, 8), (1, 16)]


def _small_cases():
    cases = []
    for (nr, nc) in [(1, 1), (7, 9), (13, 29), (33, 40), (40, 17)]:
        for dens in (0.0, 0.08, 0.35, 0.8, 1.0):
            cases.append(synth.bernoulli(nr, nc, dens, seed=nr * 100 + int(dens * 10)))
    return cases


# ------------------------------------------------------------- CSR SpMV --

@pytest.mark.parametrize("seed", range(6))
def test_csr_spmv_equals_dense_matvec_exactly(seed):
    """Small integer values and x: every partial sum is an exact integer,
    so the oracle must equal the dense product bit for bit."""
    A = synth.bernoulli(31, 23, 0.3 + 0.1 * seed, seed=seed)
    x = synth.vector_int(A.ncols, -4, 4, seed=seed)
    y, scale = oracle.csr_spmv(A, x)
    D = A.todense()
    assert np.array_equal(y, D @ x)
    assert np.array_equal(scale, np.abs(D) @ np.abs(x))


def test_csr_spmv_is_correctly_rounded_sum_of_products():
    """Against math.fsum (exactly rounded) of the rounded products: the
    compensated sum is within about one rounding of the exact sum."""
    A = synth.powerlaw(3000, seed=11)
    x = synth.vector_uniform(A.ncols, seed=7)
    y, scale = oracle.csr_spmv(A, x)
    eps = np.finfo(np.float64).eps
    for i in range(A.nrows):
        lo, hi = A.rowptr[i], A.rowptr[i + 1]
        terms = [float(v) * float(x[j]) for v, j in zip(A.vals[lo:hi], A.colidx[lo:hi])]
        ref = math.fsum(terms)
        assert abs(y[i] - ref) <= 2 * eps * abs(ref) + 1e-30 * len(terms) * scale[i]


def test_csr_spmv_plain_matches_within_sequential_bound():
    A = synth.stencil27(12, 11, 10, values="normal")
    x = synth.vector_uniform(A.ncols, seed=3)
    y, scale = oracle.csr_spmv(A, x)
    yp = oracle.csr_spmv_plain(A, x)
    lens = np.diff(A.rowptr)
    assert np.all(np.abs(y - yp) <= lens * np.finfo(float).eps * scale)


def test_empty_rows_give_zero():
    A = synth.bernoulli(20, 20, 0.05, seed=9)
    assert (np.diff(A.rowptr) == 0).any()
    y, s = oracle.csr_spmv(A, np.ones(20))
    assert np.all(y[np.diff(A.rowptr) == 0] == 0.0)


# ------------------------------------------------------------ conversion --

@pytest.mark.parametrize("r,c", SIX_BETAS + ODD_BETAS)
def test_convert_equals_grid_scan(r, c):
    """The merge-based converter agrees byte for byte with an independent
    grid scan, on every density including empty and full, and on row counts
    that are not multiples of r."""
    for A in _small_cases():
        S = oracle.convert(A, r, c)
        brp, cols, masks, values = grid_convert(A, r, c)
        assert S.block_rowptr.tolist() == brp
        assert S.block_colidx.tolist() == cols
        assert S.block_masks.astype(np.uint64).tolist() == masks
        assert S.values.tolist() == values
        if r * c <= 64:
            nbytes = (r * c + 7) // 8
            expect = np.array([[(pack_word(m, c) >> (8 * t)) & 0xFF for t in range(nbytes)]
                               for m in masks], dtype=np.uint8).reshape(-1, nbytes)
            assert np.array_equal(S.packed_masks(), expect)


@pytest.mark.parametrize("r,c", SIX_BETAS + [(3, 5)])
def test_roundtrip_is_bit_exact(r, c):
    mats = [synth.laplace2d(31, 17), synth.stencil27(9, 7, 6, values="normal"),
            synth.powerlaw(5000, seed=5), synth.uniform(3000, 16, seed=6),
            synth.fem3d(800, seed=2), synth.bernoulli(50, 70, 0.4, seed=3)]
    for A in mats:
        S = oracle.convert(A, r, c)
        rowptr, colidx, vals = oracle.to_csr(S)
        assert np.array_equal(rowptr, A.rowptr)
        assert np.array_equal(colidx, A.colidx)
        assert np.array_equal(vals.view(np.uint64), A.vals.view(np.uint64))


@pytest.mark.parametrize("r,c", SIX_BETAS)
def test_mask_popcounts_sum_to_nnz_and_block_invariants(r, c):
    for A in [synth.powerlaw(4000, seed=8), synth.uniform(2000, 16, seed=1),
              synth.stencil27(10, 10, 10)]:
        S = oracle.convert(A, r, c)
        pop = sum(bin(int(m)).count("1") for m in S.block_masks.reshape(-1))
        assert pop == A.nnz
        assert S.nblocks <= A.nnz
        # blocks of a panel: ascending, disjoint, each starting on a stored column
        # of some row of the panel, bit 0 set in at least one row
        union0 = np.bitwise_or.reduce(S.block_masks, axis=1) & 1 if S.nblocks else []
        assert np.all(union0 == 1)
        for p in range(S.npanels):
            cols = S.block_colidx[S.block_rowptr[p]:S.block_rowptr[p + 1]].astype(np.int64)
            assert np.all(np.diff(cols) >= c)
            nnz_p = A.rowptr[min((p + 1) * r, A.nrows)] - A.rowptr[p * r]
            nb_p = len(cols)
            assert nb_p >= math.ceil(nnz_p / (r * c))
        # a set bit never points past the last column
        for b in range(S.nblocks):
            for q in range(r):
                m = int(S.block_masks[b, q])
                if m:
                    assert S.block_colidx[b] + m.bit_length() - 1 < A.ncols


@pytest.mark.parametrize("c", [4, 8])
def test_r1_values_are_the_csr_values(c):
    """Section 5: beta(1,*) leaves the array of values unchanged w.r.t. CSR."""
    for A in [synth.powerlaw(3000, seed=2), synth.fem3d(500), synth.uniform(1000, 16)]:
        S = oracle.convert(A, 1, c)
        assert np.array_equal(S.values.view(np.uint64), A.vals.view(np.uint64))


def test_table1_dense_row():
    """Table 1, row "dense": n = 2048, nnz = 4194304, 100% filling for every
    beta(r, VS).  Full blocks also fix nblocks = (2048/r) * (2048/VS)."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_dense.txt"))
            if ln.strip() and not ln.startswith("#")]
    meta = {k: int(v) for k, v in (r for r in rows if len(r) == 2)}
    A = synth.dense(meta["dim"], values="normal")
    assert A.nrows == meta["dim"] and A.nnz == meta["nnz"]
    assert A.nnz // A.nrows == meta["nnz_per_row"]
    for r, vs, fill in ((int(a), int(b), int(c)) for a, b, c in (r for r in rows if len(r) == 3)):
        S = oracle.convert(A, r, vs)
        assert S.nblocks == (2048 // r) * (2048 // vs)
        assert round(100 * S.filling()) == fill


def test_fig3_mask_1101():
    """Fig. 3: mask 1101 (drawn MSB to LSB) selects three elements; with
    Algorithm 1's bit test they sit at positions 0, 2 and 3."""
    line = [ln for ln in open(os.path.join(GOLDEN, "fig3_mask_1101.txt"))
            if ln.strip() and not ln.startswith("#")][0].split()
    mask = int(line[0], 2)
    count = int(line[1])
    positions = [int(t) for t in line[2:]]
    assert bin(mask).count("1") == count
    A = synth.CSR(1, 4, np.array([0, count], np.int32), np.array(positions, np.int32),
                  np.array([11.0, 22.0, 33.0]))
    S = oracle.convert(A, 1, 4)
    assert S.nblocks == 1 and S.block_colidx[0] == 0
    assert int(S.block_masks[0, 0]) == mask
    assert S.values.tolist() == [11.0, 22.0, 33.0]
    x = np.array([1.0, 10.0, 100.0, 1000.0])
    assert oracle.spc5_spmv(S, x)[0] == 11.0 * 1 + 22.0 * 100 + 33.0 * 1000


# closed forms: derived from the stencil structure, independent of any converter

def _count_27pt(n1, r, c):
    """Blocks of a 27-point stencil on n1^3 (x fastest) when r divides n1 and
    every panel's union in one (dy, dz) neighbour line spans at most
    r + 2 contiguous columns.  Each line neighbour group is one run of
    contiguous columns, so it needs ceil(width / c) blocks; summing over
    valid (dy, dz) gives (3*n1 - 2)^2 groups per x-panel position."""
    groups = (3 * n1 - 2) ** 2
    per_line = 0
    for x0 in range(0, n1, r):
        lo, hi = max(x0 - 1, 0), min(x0 + r, n1 - 1)
        per_line += math.ceil((hi - lo + 1) / c)
    return groups * per_line


@pytest.mark.parametrize("r,c", [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8)])
def test_closed_form_27pt_100(r, c):
    A = synth.stencil27(100, 100, 100, values="poisson")
    assert A.nnz == 298 ** 3
    S = oracle.convert(A, r, c)
    assert S.nblocks == _count_27pt(100, r, c)
    assert S.nblocks == {(1, 8): 8_880_400, (2, 4): 4_440_200, (2, 8): 4_440_200,
                         (4, 4): 4_440_200, (4, 8): 2_220_100}[(r, c)]


@pytest.mark.parametrize("r,c", [(1, 8), (4, 8), (2, 4), (8, 4)])
def test_closed_form_27pt_16(r, c):
    A = synth.stencil27(16, 16, 16, values="poisson")
    assert A.nnz == 46 ** 3
    S = oracle.convert(A, r, c)
    assert S.nblocks == _count_27pt(16, r, c)


def test_closed_form_5pt_128():
    """5-point stencil on 128^2: beta(1,8) has one block for (x-1, x, x+1)
    plus one per existing vertical neighbour: n + 2*128*127.  beta(4,8):
    panels stay inside a grid line (4 | 128); the union of 4 rows is
    x0-1..x0+4 (one block) plus the 4-wide runs above and below."""
    A = synth.laplace2d(128, 128)
    assert A.nnz == 81408
    assert oracle.convert(A, 1, 8).nblocks == 16384 + 2 * 128 * 127 == 48896
    assert oracle.convert(A, 4, 8).nblocks == 16384 // 4 + 2 * 32 * 127 == 12224


def test_27pt_8x4_straddling_panels_match_grid_scan():
    """beta(8,4) on 10^3: 8 does not divide 10, so panels straddle grid lines;
    no closed form, compare with the grid scan."""
    A = synth.stencil27(10, 10, 10, values="poisson")
    S = oracle.convert(A, 8, 4)
    brp, cols, masks, values = grid_convert(A, 8, 4)
    assert S.block_rowptr.tolist() == brp and S.block_colidx.tolist() == cols


# ------------------------------------------------------------ Algorithm 1 --

@pytest.mark.parametrize("r,c", SIX_BETAS + ODD_BETAS)
def test_algorithm1_equals_dense_matvec_exactly(r, c):
    for A in _small_cases():
        x = synth.vector_int(A.ncols, -5, 5, seed=A.nrows)
        S = oracle.convert(A, r, c)
        assert np.array_equal(oracle.spc5_spmv(S, x), A.todense() @ x)


@pytest.mark.parametrize("r,c", SIX_BETAS)
def test_laplacian_times_ones(r, c):
    """Stencil with diagonal = number of possible neighbours and -1 off it:
    A 1 is 0 in the interior and (possible - actual neighbours) on the
    boundary, exactly, in any summation order."""
    A = synth.laplace2d(40, 37)
    S = oracle.convert(A, r, c)
    y = oracle.spc5_spmv(S, np.ones(A.ncols))
    deg = np.diff(A.rowptr) - 1
    assert np.array_equal(y, 4.0 - deg)
    B = synth.stencil27(13, 11, 9, values="poisson")
    yb = oracle.spc5_spmv(oracle.convert(B, r, c), np.ones(B.ncols))
    assert np.array_equal(yb, 26.0 - (np.diff(B.rowptr) - 1))
    interior = (np.diff(B.rowptr) == 27)
    assert np.all(yb[interior] == 0.0)


@pytest.mark.parametrize("r,c", SIX_BETAS)
def test_algorithm1_matches_csr_within_fp64(r, c):
    for A in [synth.fem3d(2000), synth.powerlaw(6000, seed=4), synth.uniform(4000, 16)]:
        x = synth.vector_uniform(A.ncols, seed=9)
        y, scale = oracle.csr_spmv(A, x)
        y1 = oracle.spc5_spmv(oracle.convert(A, r, c), x)
        lens = np.diff(A.rowptr)
        assert np.all(np.abs(y1 - y) <= (lens + 2) * np.finfo(float).eps * scale)


# ------------------------------------------------------------ rejections --

def test_rejects_invalid_csr():
    good = synth.bernoulli(6, 6, 0.5, seed=1)
    assert oracle.check_csr(6, 6, good.rowptr, good.colidx) == 0
    unsorted = good.colidx.copy()
    row = int(np.argmax(np.diff(good.rowptr) >= 2))
    a = good.rowptr[row]
    unsorted[a], unsorted[a + 1] = unsorted[a + 1], unsorted[a]
    assert oracle.check_csr(6, 6, good.rowptr, unsorted) == 2
    dup = good.colidx.copy()
    dup[a + 1] = dup[a]
    assert oracle.check_csr(6, 6, good.rowptr, dup) == 2
    out = good.colidx.copy()
    out[-1] = 6
    assert oracle.check_csr(6, 6, good.rowptr, out) == 3
    bad = good.rowptr.copy()
    bad[2], bad[3] = bad[3] + 1, bad[2]
    assert oracle.check_csr(6, 6, bad, good.colidx) in (2, 3, 4)
    with pytest.raises(oracle.OracleError):
        oracle.convert(synth.CSR(6, 6, good.rowptr, unsorted, good.vals), 2, 4)


# ------------------------------------------------------------- gradients --

def test_transpose_pins():
    for seed, (nr, nc, d) in enumerate([(31, 23, 0.3), (5, 80, 0.7), (64, 1, 0.5), (9, 9, 0.0)]):
        A = synth.bernoulli(nr, nc, d, seed=seed, integer_values=True)
        T = oracle.transpose(A)
        assert np.array_equal(synth.CSR(T.nrows, T.ncols, T.rowptr, T.colidx, T.vals).todense(),
                              A.todense().T)
        TT = oracle.transpose(T)
        assert np.array_equal(TT.rowptr, A.rowptr) and np.array_equal(TT.colidx, A.colidx)
        assert np.array_equal(TT.vals, A.vals)
        g = synth.vector_int(nr, -4, 4, seed=seed)
        dx, _ = oracle.csr_spmv_t(A, g)
        assert np.array_equal(dx, A.todense().T @ g)


def test_values_grad_pin():
    A = synth.bernoulli(40, 30, 0.4, seed=2, integer_values=True)
    g = synth.vector_normal(40, seed=1)
    x = synth.vector_normal(30, seed=2)
    dv = oracle.values_grad(A, g, x)
    dense = np.outer(g, x)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    assert np.array_equal(dv, dense[rows, A.colidx])
