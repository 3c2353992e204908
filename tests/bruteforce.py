"""Brute-force restatements used to pin the oracle (pure Python, tiny inputs).

These are written independently of ``oracle/spc5_oracle.c``: the block
builder here scans a dense occupancy grid column by column instead of
merging sorted row lists, and the products are plain dense algebra.
"""
from __future__ import annotations

import numpy as np


def dense_pattern(A):
    """(occupied[nrows][ncols] as lists of bools, values as lists)."""
    occ = [[False] * A.ncols for _ in range(A.nrows)]
    val = [[0.0] * A.ncols for _ in range(A.nrows)]
    for i in range(A.nrows):
        for e in range(int(A.rowptr[i]), int(A.rowptr[i + 1])):
            occ[i][int(A.colidx[e])] = True
            val[i][int(A.colidx[e])] = float(A.vals[e])
    return occ, val


def grid_convert(A, r: int, c: int):
    """beta(r,c) by scanning the occupancy grid of each panel left to right:
    an occupied column not covered by the previous block opens a block
    covering c columns; every row's bits and values are read off the grid.
    Returns (block_rowptr, block_colidx, masks[nblocks][r], values)."""
    occ, val = dense_pattern(A)
    n = A.nrows
    npanels = (n + r - 1) // r
    brp, cols, masks, values = [0], [], [], []
    for p in range(npanels):
        rows = [i for i in range(p * r, p * r + r) if i < n]
        covered_until = -1
        for j in range(A.ncols):
            if j <= covered_until or not any(occ[i][j] for i in rows):
                continue
            covered_until = j + c - 1
            cols.append(j)
            row_masks = []
            for q in range(r):
                i = p * r + q
                m = 0
                for k in range(c):
                    if i < n and j + k < A.ncols and occ[i][j + k]:
                        m |= 1 << k
                        values.append(val[i][j + k])
                row_masks.append(m)
            masks.append(row_masks)
        brp.append(len(cols))
    return brp, cols, masks, values


def pack_word(row_masks, c: int) -> int:
    w = 0
    for q, m in enumerate(row_masks):
        w |= int(m) << (q * c)
    return w
