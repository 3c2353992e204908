"""Row-partitioned SpMV: the split a product over several GPUs would use.

The panels of beta(r,c) are independent units of work (Algorithm 1 walks
them one after another), so y = A x splits by rows: each part owns a
contiguous range of whole panels, converts its own rows (columns stay
global), and needs the whole of x, which is spread over the parts as
slices.  One product is then an all-gather of the x slices followed by
independent local products; y stays partitioned.  There is no reduction.

  balanced_panel_ranges  contiguous panel ranges of about equal work
                         (stored entries plus rows, a proxy for the values
                         and blocks a part streams)
  local_rows             the CSR rows of one part, columns global
  slice_bounds           the x slice each part holds
  gather_x               all-gather of the slices into the whole x
                         (torch.distributed; NCCL between GPUs)
  PartitionedMatrix      all parts on one GPU, for checking the split and
                         for replicas; PartMatrix one part on its own GPU

The paper runs its kernels on the cores of one node and splits rows among
threads naively (Section 4.3); this is the GPU counterpart at the level of
whole devices.  Every local product runs in the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np

from . import spc5 as _c


def balanced_panel_ranges(rowptr: np.ndarray, r: int, nparts: int) -> list[tuple[int, int]]:
    """Row ranges [row0, row1) of `nparts` parts, each a run of whole panels
    of r rows, cut where the running work (stored entries + rows) crosses
    k / nparts of the total.  Parts may be empty when there are fewer panels
    than parts."""
    if nparts < 1 or r < 1:
        raise ValueError("nparts and r must be positive")
    rowptr = np.asarray(rowptr, dtype=np.int64)
    n = rowptr.size - 1
    npanels = (n + r - 1) // r
    first = np.minimum(np.arange(npanels + 1) * r, n)
    work = rowptr[first] + first  # running work at every panel boundary
    total = work[-1]
    cuts = [0]
    for k in range(1, nparts):
        target = total * k / nparts
        p = int(np.searchsorted(work, target, side="left"))
        cuts.append(max(cuts[-1], min(p, npanels)))
    cuts.append(npanels)
    return [(int(first[a]), int(first[b])) for a, b in zip(cuts[:-1], cuts[1:])]


def local_rows(rowptr, colidx, vals, row0: int, row1: int):
    """CSR of rows [row0, row1): row pointers rebased to 0, columns global."""
    rowptr = np.asarray(rowptr)
    e0, e1 = int(rowptr[row0]), int(rowptr[row1])
    lrp = (rowptr[row0:row1 + 1] - e0).astype(np.int32)
    return lrp, np.ascontiguousarray(colidx[e0:e1]), np.ascontiguousarray(vals[e0:e1])


def slice_bounds(ncols: int, nparts: int) -> list[tuple[int, int]]:
    """The x slice [c0, c1) each part holds: nparts nearly equal slices."""
    edges = [(ncols * k) // nparts for k in range(nparts + 1)]
    return list(zip(edges[:-1], edges[1:]))


def gather_x(x_slice, ncols: int, group=None):
    """All-gather the parts' slices (part k holds slice_bounds(ncols, N)[k])
    into the whole x on every part.  Slices are padded to one length for the
    collective and trimmed after it."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    bounds = slice_bounds(ncols, world)
    width = max(b - a for a, b in bounds)
    buf = torch.zeros(width, dtype=x_slice.dtype, device=x_slice.device)
    buf[:x_slice.numel()] = x_slice
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:b - a] for p, (a, b) in zip(parts, bounds)])


class PartMatrix:
    """One part of a row-partitioned matrix on the current GPU: rows
    [row0, row1) converted to beta(r,c) (columns global)."""

    def __init__(self, nrows, ncols, rowptr, colidx, vals, row0, row1, r, c,
                 store_dtype=_c.SPC5_F64, stream=None):
        import torch
        self.row0, self.row1, self.ncols = int(row0), int(row1), int(ncols)
        lrp, lci, lv = local_rows(rowptr, colidx, vals, row0, row1)
        dev = [torch.from_numpy(a).cuda() for a in (lrp, lci, np.asarray(lv, np.float64))]
        self.matrix = _c.spc5_convert_csr(self.row1 - self.row0, ncols, int(lrp[-1]), *dev,
                                          store_dtype=store_dtype, r=r, c=c, stream=stream)

    def spmv(self, x_full, y_local, alpha=1.0, beta=0.0, stream=None):
        """y_local = alpha * A[row0:row1, :] x + beta * y_local (device vectors)."""
        if self.row1 > self.row0:
            _c.spc5_spmv(self.matrix, x_full, y_local, alpha, beta, stream)


class PartitionedMatrix:
    """A matrix split into `nparts` row parts on one GPU: the same split a
    multi-GPU product uses, each part converted and multiplied on its own;
    y is the concatenation of the parts' products."""

    def __init__(self, nrows, ncols, rowptr, colidx, vals, r, c, nparts,
                 store_dtype=_c.SPC5_F64, stream=None):
        self.nrows, self.ncols = int(nrows), int(ncols)
        self.ranges = balanced_panel_ranges(rowptr, r, nparts)
        self.parts = [PartMatrix(nrows, ncols, rowptr, colidx, vals, a, b, r, c, store_dtype,
                                 stream) for a, b in self.ranges]

    def spmv(self, x, y, alpha=1.0, beta=0.0, stream=None):
        """y = alpha * A x + beta * y, part by part (device vectors)."""
        for p in self.parts:
            p.spmv(x, y[p.row0:p.row1], alpha, beta, stream)
