"""Row-partitioned SpMV (the split of the product over several GPUs): the
panel ranges, the local rows, the x slices and their all-gather, checked on
the CPU; the exchange runs over two gloo ranks, each rank multiplying its
own rows (with the CPU oracle, as test infrastructure) by the gathered x,
and the parts' products must equal the oracle's product of the whole matrix
bit for bit (rows are independent and summed in the same order)."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2307_14774_gb300 import partition


@pytest.mark.parametrize("r", [1, 2, 4, 8])
@pytest.mark.parametrize("nparts", [1, 2, 3, 7])
def test_ranges_are_panel_aligned_contiguous_and_balanced(r, nparts):
    A = synth.powerlaw(5000, seed=3)
    ranges = partition.balanced_panel_ranges(A.rowptr, r, nparts)
    assert len(ranges) == nparts
    assert ranges[0][0] == 0 and ranges[-1][1] == A.nrows
    for (a0, a1), (b0, b1) in zip(ranges[:-1], ranges[1:]):
        assert a1 == b0 and a0 <= a1
    for a, b in ranges:
        assert a % r == 0 and (b % r == 0 or b == A.nrows)
    rp = A.rowptr.astype(np.int64)
    work = [int(rp[b] - rp[a]) + (b - a) for a, b in ranges]
    first = np.minimum(np.arange((A.nrows + r - 1) // r + 1) * r, A.nrows)
    panel_work = np.diff(rp[first] + first)
    assert max(work) <= sum(work) / nparts + panel_work.max()


def test_more_parts_than_panels_gives_empty_parts():
    A = synth.laplace2d(3, 3)  # 9 rows
    ranges = partition.balanced_panel_ranges(A.rowptr, 4, 5)  # 3 panels
    assert sum(b - a for a, b in ranges) == 9
    assert sum(1 for a, b in ranges if b == a) >= 2


def test_local_rows_reassemble_the_matrix():
    A = synth.fem3d(800, seed=2)
    parts = [partition.local_rows(A.rowptr, A.colidx, A.vals, a, b)
             for a, b in partition.balanced_panel_ranges(A.rowptr, 4, 3)]
    assert np.array_equal(np.concatenate([p[1] for p in parts]), A.colidx)
    assert np.array_equal(np.concatenate([p[2] for p in parts]), A.vals)
    lens = np.concatenate([np.diff(p[0]) for p in parts])
    assert np.array_equal(lens, np.diff(A.rowptr))


def test_slice_bounds_cover_x():
    for ncols, n in ((10, 3), (7, 7), (5, 8)):
        b = partition.slice_bounds(ncols, n)
        assert b[0][0] == 0 and b[-1][1] == ncols and all(x1 == y0 for (_, x1), (y0, _) in zip(b, b[1:]))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = synth.powerlaw(3000, seed=9)
        x = synth.vector_uniform(A.ncols, seed=4)
        c0, c1 = partition.slice_bounds(A.ncols, world)[rank]
        xg = partition.gather_x(torch.from_numpy(x[c0:c1].copy()), A.ncols).numpy()
        row0, row1 = partition.balanced_panel_ranges(A.rowptr, 4, world)[rank]
        lrp, lci, lv = partition.local_rows(A.rowptr, A.colidx, A.vals, row0, row1)
        y_local, _ = oracle.csr_spmv(synth.CSR(row1 - row0, A.ncols, lrp, lci, lv), xg)
        pieces = [None] * world
        dist.all_gather_object(pieces, (row0, y_local))
        out.put((rank, bool(np.array_equal(xg, x)), pieces if rank == 0 else None))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_x_and_multiply_their_rows():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=120) for _ in procs), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(g[1] for g in got)  # every rank has the whole x
    pieces = sorted(got[0][2])
    y = np.concatenate([yl for _, yl in pieces])
    A = synth.powerlaw(3000, seed=9)
    y_ref, _ = oracle.csr_spmv(A, synth.vector_uniform(A.ncols, seed=4))
    assert np.array_equal(y, y_ref)
