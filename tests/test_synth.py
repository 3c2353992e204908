"""The synthetic workloads (inputs only): benchmark sizes of the 27-point,
power-law and uniform matrices, the FEM mesh's link statistics, CSR
invariants, determinism under the seed and independence from the number of
OpenMP threads."""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check_csr(A):
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz
    assert np.all(np.diff(A.rowptr) >= 0)
    assert A.colidx.min(initial=0) >= 0 and A.colidx.max(initial=-1) < A.ncols
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    same_row = rows[1:] == rows[:-1]
    assert np.all(np.diff(A.colidx.astype(np.int64))[same_row] > 0)  # strictly ascending


def _digest(A) -> str:
    h = hashlib.sha256()
    for a in (A.rowptr, A.colidx, A.vals):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def test_benchmark_sizes():
    st = synth.workload("stencil27")
    assert (st.nrows, st.nnz) == (10**6, 26_463_592) == (10**6, 298**3)
    pl = synth.workload("powerlaw")
    assert (pl.nrows, pl.nnz) == (2 * 10**6, 39_648_070)
    lens = np.diff(pl.rowptr)
    assert lens.max() == pl.ncols                          # the longest row is dense
    assert 19.5 < lens.mean() < 20.5                       # rescaled to mean 20
    un = synth.workload("uniform")
    assert (un.nrows, un.nnz) == (10**6, 16 * 10**6)
    assert np.all(np.diff(un.rowptr) == 16)
    for A in (st, pl, un):
        _check_csr(A)


def test_powerlaw_columns_near_the_diagonal():
    A = synth.powerlaw(50_000, seed=3)
    lens = np.diff(A.rowptr)
    rows = np.repeat(np.arange(A.nrows), lens)
    short = np.repeat(lens <= 4000, lens)
    dist = np.abs(A.colidx[short].astype(np.int64) - rows[short])
    assert np.median(dist) < 1000                          # sigma 1000 around row i
    with pytest.raises(ValueError):                        # long_row must be <= 4 sigma
        synth.powerlaw(1000, sigma=50.0, long_row=500)


def test_fem_mesh_links_and_symmetry():
    A = synth.fem3d(20_000, seed=2)
    _check_csr(A)
    assert A.nrows == 3 * 20_000
    lens = np.diff(A.rowptr)
    assert np.all(lens % 3 == 0)                           # dense 3x3 node blocks
    assert np.array_equal(lens[0::3], lens[1::3]) and np.array_equal(lens[0::3], lens[2::3])
    links = lens[0::3] // 3                                # neighbours incl. self
    assert 23 < links.mean() < 27                          # about 26 (fewer at the boundary)
    D = np.zeros((3000, 3000), bool)                       # pattern symmetric: link i-j <=> j-i
    sub = synth.fem3d(1000, seed=5)
    rows = np.repeat(np.arange(sub.nrows), np.diff(sub.rowptr))
    D[rows, sub.colidx] = True
    assert np.array_equal(D, D.T)


def test_same_seed_same_matrix_other_seed_other_matrix():
    assert _digest(synth.powerlaw(30_000, seed=7)) == _digest(synth.powerlaw(30_000, seed=7))
    assert _digest(synth.powerlaw(30_000, seed=7)) != _digest(synth.powerlaw(30_000, seed=8))
    assert np.array_equal(synth.vector_uniform(1000, seed=3), synth.vector_uniform(1000, seed=3))


def test_results_do_not_depend_on_the_thread_count():
    code = ("import hashlib, numpy as np, synth\n"
            "A = synth.fem3d(5000, seed=4)\n"
            "h = hashlib.sha256()\n"
            "[h.update(np.ascontiguousarray(a).tobytes()) for a in (A.rowptr, A.colidx, A.vals)]\n"
            "print(h.hexdigest())\n")
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONPATH=ROOT)
    one = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=300, check=True).stdout.strip()
    assert one == _digest(synth.fem3d(5000, seed=4))
