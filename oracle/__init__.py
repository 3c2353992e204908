"""CPU oracle for the SPC5 beta(r,c) SpMV (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

The arithmetic lives in plain C (``spc5_oracle.c``), compiled with gcc on
first use (or by ``build()``), and follows the paper:

* ``csr_spmv``      y = A x from CSR in FP64 (Section 2.3), with the per-row
                    magnitude S_i = sum |a_ij x_j| that tolerances are
                    stated against.
* ``convert``       CSR -> beta(r,c) (Section 2.4, union-greedy blocks).
* ``spc5_spmv``     Algorithm 1, scalar path.
* ``to_csr``        beta(r,c) -> CSR.
* ``pack_masks``    per-block packed r*c-bit mask words.
* ``quantize``      FP64 -> FP32 / BF16 storage (round to nearest even;
                    BF16 through a round-to-odd FP32 intermediate).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spc5_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libspc5oracle.so")
_OMP_LIB_PATH = os.path.join(_OUT_DIR, "libspc5oracle_omp.so")
_lock = threading.Lock()

ERRORS = {1: "EINVAL", 2: "EUNSORTED", 3: "ERANGE", 4: "EROWPTR"}


class OracleError(ValueError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no OpenMP, no target-specific flags)."""
    return _compile(_LIB_PATH, [], force)


def build_omp(force: bool = False) -> str | None:
    """Compile the same source with OpenMP (-fopenmp): the two CSR products
    then run their rows on several host threads.  Used only to time the CPU
    baseline; None if the compiler has no OpenMP."""
    try:
        return _compile(_OMP_LIB_PATH, ["-fopenmp"], force)
    except subprocess.CalledProcessError:
        return None


def _compile(out: str, extra, force: bool) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *extra, _SRC, "-o", tmp, "-lm"],
                   check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def _p(dtype):
    return np.ctypeslib.ndpointer(dtype=dtype, flags="C_CONTIGUOUS")


def _bind(lib):
    i64, ci = ctypes.c_int64, ctypes.c_int
    i32p, f64p, i64p, u64p, u8p = (_p(np.int32), _p(np.float64), _p(np.int64),
                                  _p(np.uint64), _p(np.uint8))
    opt = ctypes.c_void_p
    lib.oracle_check_csr.argtypes = [i64, i64, i32p, i32p]
    lib.oracle_set_threads.argtypes = [ci]
    lib.oracle_set_threads.restype = ci
    lib.oracle_csr_spmv.argtypes = [i64, i32p, i32p, f64p, f64p, f64p, opt]
    lib.oracle_csr_spmv_plain.argtypes = [i64, i32p, i32p, f64p, f64p, f64p]
    lib.oracle_spc5_convert.argtypes = [i64, i64, i32p, i32p, opt, ci, ci, i64p,
                                        ctypes.POINTER(ctypes.c_int64), opt, opt, opt]
    lib.oracle_spc5_spmv.argtypes = [i64, ci, ci, i64p, i32p, u64p, f64p, f64p, f64p]
    lib.oracle_spc5_to_csr.argtypes = [i64, ci, ci, i64p, i32p, u64p, f64p, i32p, i32p, f64p]
    lib.oracle_pack_masks.argtypes = [i64, ci, ci, u64p, u8p]
    lib.oracle_quantize.argtypes = [i64, f64p, ci, opt]
    lib.oracle_csr_transpose.argtypes = [i64, i64, i32p, i32p, f64p, i32p, i32p, f64p]
    lib.oracle_values_grad.argtypes = [i64, i32p, i32p, f64p, f64p, f64p]
    lib.oracle_hybrid_split.argtypes = [i64, ci, ci, i64p, i32p, u64p, f64p, i64p, i32p, u64p,
                                        f64p, ctypes.POINTER(ctypes.c_int64), i32p, i32p, f64p,
                                        ctypes.POINTER(ctypes.c_int64)]
    for f in (lib.oracle_quantize, lib.oracle_csr_transpose, lib.oracle_values_grad,
              lib.oracle_hybrid_split, lib.oracle_check_csr, lib.oracle_csr_spmv,
              lib.oracle_csr_spmv_plain,
              lib.oracle_spc5_convert, lib.oracle_spc5_spmv, lib.oracle_spc5_to_csr,
              lib.oracle_pack_masks):
        f.restype = ci
    return lib


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc: int):
    if rc != 0:
        raise OracleError(rc)


@dataclass
class SPC5:
    """A matrix in beta(r,c) form as the oracle builds it.

    block_rowptr[npanels+1]  first block of each panel (int64)
    block_colidx[nblocks]    start column of each block
    block_masks[nblocks, r]  c-bit mask of each row of each block
    values[nnz]              packed values in Algorithm 1's idxVal order
    """
    nrows: int
    ncols: int
    r: int
    c: int
    block_rowptr: np.ndarray
    block_colidx: np.ndarray
    block_masks: np.ndarray
    values: np.ndarray
    lib: object = None

    @property
    def npanels(self) -> int:
        return (self.nrows + self.r - 1) // self.r

    @property
    def nblocks(self) -> int:
        return int(self.block_rowptr[-1])

    @property
    def nnz(self) -> int:
        return int(self.values.shape[0])

    def filling(self) -> float:
        """Share of block slots holding an entry: nnz / (nblocks * r * c)."""
        return self.nnz / (self.nblocks * self.r * self.c) if self.nblocks else 0.0

    def packed_masks(self) -> np.ndarray:
        """[nblocks, ceil(r*c/8)] uint8: one little-endian r*c-bit word per
        block, row q at bits [q*c, (q+1)*c)."""
        nbytes = (self.r * self.c + 7) // 8
        out = np.empty((self.nblocks, nbytes), np.uint8)
        lib = self.lib if self.lib is not None else _default().lib
        _check(lib.oracle_pack_masks(self.nblocks, self.r, self.c,
                                     _arr(self.block_masks.reshape(-1), np.uint64),
                                     out.reshape(-1)))
        return out


class Oracle:
    """The oracle functions bound to one compiled copy of spc5_oracle.c."""

    def __init__(self, path: str | None = None):
        self.lib = _bind(ctypes.CDLL(path or build()))

    def set_threads(self, n: int) -> int:
        """Host threads of the CSR products (1 unless this copy has OpenMP)."""
        return self.lib.oracle_set_threads(int(n))

    def check_csr(self, nrows, ncols, rowptr, colidx) -> int:
        """0 if the CSR pattern is valid, else the oracle's error code."""
        return self.lib.oracle_check_csr(nrows, ncols, _arr(rowptr, np.int32),
                                         _arr(colidx, np.int32))

    def csr_spmv(self, A, x):
        """y = A x (compensated FP64 sum) and S_i = sum_j |a_ij x_j|."""
        x = _arr(x, np.float64)
        y = np.empty(A.nrows, np.float64)
        scale = np.empty(A.nrows, np.float64)
        _check(self.lib.oracle_csr_spmv(A.nrows, _arr(A.rowptr, np.int32),
                                        _arr(A.colidx, np.int32), _arr(A.vals, np.float64),
                                        x, y, scale.ctypes.data_as(ctypes.c_void_p)))
        return y, scale

    def csr_spmv_plain(self, A, x):
        """Textbook sequential CSR SpMV in FP64."""
        x = _arr(x, np.float64)
        y = np.empty(A.nrows, np.float64)
        _check(self.lib.oracle_csr_spmv_plain(A.nrows, _arr(A.rowptr, np.int32),
                                              _arr(A.colidx, np.int32),
                                              _arr(A.vals, np.float64), x, y))
        return y

    def convert(self, A, r: int, c: int) -> SPC5:
        """CSR -> beta(r,c) following Section 2.4 (union-greedy blocks)."""
        lib = self.lib
        rowptr, colidx = _arr(A.rowptr, np.int32), _arr(A.colidx, np.int32)
        vals = _arr(A.vals, np.float64)
        npanels = (A.nrows + r - 1) // r
        brp = np.zeros(npanels + 1, np.int64)
        nb = ctypes.c_int64(0)
        _check(lib.oracle_spc5_convert(A.nrows, A.ncols, rowptr, colidx, None, r, c, brp,
                                       ctypes.byref(nb), None, None, None))
        nb = nb.value
        bcol = np.zeros(max(nb, 1), np.int32)
        masks = np.zeros((max(nb, 1), r), np.uint64)
        values = np.zeros(max(len(vals), 1), np.float64)
        _check(lib.oracle_spc5_convert(A.nrows, A.ncols, rowptr, colidx,
                                       vals.ctypes.data_as(ctypes.c_void_p), r, c, brp, None,
                                       bcol.ctypes.data_as(ctypes.c_void_p),
                                       masks.ctypes.data_as(ctypes.c_void_p),
                                       values.ctypes.data_as(ctypes.c_void_p)))
        return SPC5(A.nrows, A.ncols, r, c, brp, bcol[:nb], masks[:nb], values[:len(vals)],
                    lib)

    def spc5_spmv(self, S: SPC5, x) -> np.ndarray:
        """Algorithm 1 (scalar path): y = A x over beta(r,c)."""
        x = _arr(x, np.float64)
        y = np.zeros(S.nrows, np.float64)
        _check(self.lib.oracle_spc5_spmv(S.nrows, S.r, S.c, _arr(S.block_rowptr, np.int64),
                                         _arr(S.block_colidx, np.int32),
                                         _arr(S.block_masks.reshape(-1), np.uint64),
                                         _arr(S.values, np.float64), x, y))
        return y

    def quantize(self, values, dtype: str) -> np.ndarray:
        """FP64 -> "f32" (float32) or "bf16" (uint16 bit patterns)."""
        v = _arr(values, np.float64)
        code, out = {"f32": (1, np.empty(v.shape, np.float32)),
                     "bf16": (2, np.empty(v.shape, np.uint16))}[dtype]
        _check(self.lib.oracle_quantize(v.size, v, code, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def transpose(self, A):
        """A^T as a CSR with the same attribute names (nrows, ncols, rowptr, colidx, vals)."""
        from types import SimpleNamespace
        nnz = int(A.rowptr[-1])
        rp = np.zeros(A.ncols + 1, np.int32)
        ci = np.zeros(max(nnz, 1), np.int32)
        vv = np.zeros(max(nnz, 1), np.float64)
        _check(self.lib.oracle_csr_transpose(A.nrows, A.ncols, _arr(A.rowptr, np.int32),
                                             _arr(A.colidx, np.int32), _arr(A.vals, np.float64),
                                             rp, ci, vv))
        return SimpleNamespace(nrows=A.ncols, ncols=A.nrows, rowptr=rp, colidx=ci[:nnz],
                               vals=vv[:nnz])

    def csr_spmv_t(self, A, g):
        """dx = A^T g (compensated FP64) and S_j = sum_i |a_ij g_i|."""
        return self.csr_spmv(self.transpose(A), g)

    def values_grad(self, A, g, x) -> np.ndarray:
        """dvals[e] = g[row(e)] * x[col(e)] in CSR order."""
        out = np.empty(int(A.rowptr[-1]), np.float64)
        _check(self.lib.oracle_values_grad(A.nrows, _arr(A.rowptr, np.int32),
                                           _arr(A.colidx, np.int32), _arr(g, np.float64),
                                           _arr(x, np.float64), out))
        return out

    def hybrid_split(self, S: SPC5):
        """beta(r,c) -> (block part: SPC5 of the blocks holding two or more
        values, scalars: CSR namespace of the single-value blocks)."""
        from types import SimpleNamespace
        nb, nnz = S.nblocks, S.nnz
        brp = np.zeros(S.npanels + 1, np.int64)
        bcol = np.zeros(max(nb, 1), np.int32)
        masks = np.zeros((max(nb, 1), S.r), np.uint64)
        vals = np.zeros(max(nnz, 1), np.float64)
        srp = np.zeros(S.nrows + 1, np.int32)
        scol = np.zeros(max(nnz, 1), np.int32)
        svals = np.zeros(max(nnz, 1), np.float64)
        nbb, ns = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(self.lib.oracle_hybrid_split(S.nrows, S.r, S.c, _arr(S.block_rowptr, np.int64),
                                            _arr(S.block_colidx, np.int32),
                                            _arr(S.block_masks.reshape(-1), np.uint64),
                                            _arr(S.values, np.float64), brp, bcol,
                                            masks.reshape(-1), vals, ctypes.byref(nbb), srp,
                                            scol, svals, ctypes.byref(ns)))
        nbb, ns = nbb.value, ns.value
        blocks = SPC5(S.nrows, S.ncols, S.r, S.c, brp, bcol[:nbb], masks[:nbb],
                      vals[:nnz - ns], self.lib)
        scalars = SimpleNamespace(nrows=S.nrows, ncols=S.ncols, rowptr=srp, colidx=scol[:ns],
                                  vals=svals[:ns])
        return blocks, scalars

    def to_csr(self, S: SPC5):
        """beta(r,c) -> (rowptr, colidx, vals)."""
        nnz = S.nnz
        rowptr = np.zeros(S.nrows + 1, np.int32)
        colidx = np.zeros(max(nnz, 1), np.int32)
        vals = np.zeros(max(nnz, 1), np.float64)
        _check(self.lib.oracle_spc5_to_csr(S.nrows, S.r, S.c, _arr(S.block_rowptr, np.int64),
                                           _arr(S.block_colidx, np.int32),
                                           _arr(S.block_masks.reshape(-1), np.uint64),
                                           _arr(S.values, np.float64), rowptr, colidx, vals))
        return rowptr, colidx[:nnz], vals[:nnz]


_default_oracle = None


def _default() -> Oracle:
    global _default_oracle
    with _lock:
        if _default_oracle is None:
            _default_oracle = Oracle()
    return _default_oracle


def timing_oracle() -> Oracle | None:
    """The OpenMP build of the oracle (for timing the CPU baseline on all host
    cores), or None when the compiler cannot build it."""
    path = build_omp()
    return Oracle(path) if path else None


def check_csr(nrows, ncols, rowptr, colidx) -> int:
    return _default().check_csr(nrows, ncols, rowptr, colidx)


def csr_spmv(A, x):
    return _default().csr_spmv(A, x)


def csr_spmv_plain(A, x):
    return _default().csr_spmv_plain(A, x)


def convert(A, r: int, c: int) -> SPC5:
    return _default().convert(A, r, c)


def spc5_spmv(S: SPC5, x) -> np.ndarray:
    return _default().spc5_spmv(S, x)


def hybrid_split(S: SPC5):
    return _default().hybrid_split(S)


def to_csr(S: SPC5):
    return _default().to_csr(S)


def quantize(values, dtype: str) -> np.ndarray:
    return _default().quantize(values, dtype)


def transpose(A):
    return _default().transpose(A)


def csr_spmv_t(A, g):
    return _default().csr_spmv_t(A, g)


def values_grad(A, g, x) -> np.ndarray:
    return _default().values_grad(A, g, x)


def bf16_to_f64(bits) -> np.ndarray:
    """BF16 bit patterns -> exact FP64 values (a BF16 is the upper half of an FP32)."""
    b = np.asarray(bits, np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def panel_value_offsets(A, r: int) -> np.ndarray:
    """Offset of each panel's first value: the CSR row pointer of the
    panel's first row (a panel's values are a permutation of its rows')."""
    npanels = (A.nrows + r - 1) // r
    first_rows = np.minimum(np.arange(npanels + 1, dtype=np.int64) * r, A.nrows)
    return np.asarray(A.rowptr, np.int64)[first_rows]
