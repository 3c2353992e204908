"""The oracle's hybrid split (blocks holding one value become scalar CSR
entries, the paper's proposed mix of the block format with a scalar one),
pinned against the definition rebuilt here from the beta(r,c) arrays,
against the CSR it came from (exact round trip), and against special cases:
beta(1,1) turns every entry into a scalar (the split is CSR itself), a dense
matrix keeps every block."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth


def _mats():
    return [synth.bernoulli(13, 29, 0.1, seed=1), synth.bernoulli(33, 40, 0.3, seed=5),
            synth.powerlaw(800, seed=4), synth.stencil27(7, 6, 5, values="normal"),
            synth.uniform(300, 16, seed=2), synth.laplace2d(11, 9)]


def _expected(S):
    """Blocks with >= 2 set bits and the single-bit blocks' (row, col, value),
    straight from the definition."""
    keep, scalars, vals_keep = [], [], []
    idx = 0
    for p in range(S.npanels):
        for b in range(int(S.block_rowptr[p]), int(S.block_rowptr[p + 1])):
            bits = [(q, k) for q in range(S.r) for k in range(S.c)
                    if (int(S.block_masks[b, q]) >> k) & 1]
            if len(bits) == 1:
                q, k = bits[0]
                scalars.append((p * S.r + q, int(S.block_colidx[b]) + k, S.values[idx]))
            else:
                keep.append(b)
                vals_keep.extend(S.values[idx:idx + len(bits)])
            idx += len(bits)
    return keep, scalars, np.array(vals_keep)


@pytest.mark.parametrize("r,c", [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4), (3, 5)])
def test_split_matches_definition(r, c):
    for A in _mats():
        S = oracle.convert(A, r, c)
        B, Sc = oracle.hybrid_split(S)
        keep, scalars, vals_keep = _expected(S)
        # block part: the kept blocks, in order, with their values
        assert B.nblocks == len(keep)
        assert np.array_equal(B.block_colidx, S.block_colidx[keep])
        assert np.array_equal(B.block_masks, S.block_masks[keep])
        assert np.array_equal(B.values, vals_keep)
        kept_per_panel = [sum(1 for b in keep if S.block_rowptr[p] <= b < S.block_rowptr[p + 1])
                          for p in range(S.npanels)]
        assert np.array_equal(np.diff(B.block_rowptr), kept_per_panel)
        # scalars: CSR by row, ascending columns
        scalars.sort(key=lambda t: (t[0], t[1]))
        assert np.array_equal(np.diff(Sc.rowptr),
                              np.bincount([t[0] for t in scalars], minlength=A.nrows))
        assert np.array_equal(Sc.colidx, [t[1] for t in scalars])
        assert np.array_equal(Sc.vals, [t[2] for t in scalars])
        assert not any(len([1 for q in range(r) for k in range(c)
                            if (int(m[q]) >> k) & 1]) == 1 for m in B.block_masks)


@pytest.mark.parametrize("r,c", [(1, 8), (4, 4), (8, 4)])
def test_split_round_trip_is_exact(r, c):
    """Block part back to CSR, merged with the scalars, is the input CSR."""
    for A in _mats():
        B, Sc = oracle.hybrid_split(oracle.convert(A, r, c))
        rp, ci, vv = oracle.to_csr(B)
        rows = []
        for i in range(A.nrows):
            ent = list(zip(ci[rp[i]:rp[i + 1]], vv[rp[i]:rp[i + 1]]))
            ent += list(zip(Sc.colidx[Sc.rowptr[i]:Sc.rowptr[i + 1]],
                            Sc.vals[Sc.rowptr[i]:Sc.rowptr[i + 1]]))
            rows.append(sorted(ent))
        merged_rp = np.concatenate([[0], np.cumsum([len(e) for e in rows])])
        assert np.array_equal(merged_rp, A.rowptr)
        assert np.array_equal([col for e in rows for col, _ in e], A.colidx)
        assert np.array_equal([v for e in rows for _, v in e], A.vals)


def test_special_cases():
    A = synth.powerlaw(500, seed=9)
    B, Sc = oracle.hybrid_split(oracle.convert(A, 1, 1))   # every block holds one value
    assert B.nblocks == 0 and B.nnz == 0
    assert np.array_equal(Sc.rowptr, A.rowptr) and np.array_equal(Sc.colidx, A.colidx)
    assert np.array_equal(Sc.vals, A.vals)
    D = synth.dense(24, 40, values="normal")
    S = oracle.convert(D, 4, 8)
    B, Sc = oracle.hybrid_split(S)                          # full blocks: nothing moves
    assert len(Sc.vals) == 0 and B.nblocks == S.nblocks
    assert np.array_equal(B.values, S.values)


def test_hybrid_product_exact_on_integers():
    for A in [synth.bernoulli(40, 50, 0.15, seed=s, integer_values=True) for s in range(3)]:
        x = synth.vector_int(A.ncols, -4, 4, seed=1)
        for r, c in [(1, 8), (2, 4), (4, 8), (8, 4)]:
            B, Sc = oracle.hybrid_split(oracle.convert(A, r, c))
            y = oracle.spc5_spmv(B, x) + oracle.csr_spmv_plain(Sc, x)
            assert np.array_equal(y, A.todense() @ x)
