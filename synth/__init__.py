"""Seeded synthetic CSR matrices and vectors (inputs only).

This package draws the inputs that both the CPU oracle and the CUDA path
consume.  It holds none of the SPC5 arithmetic.  The generators are plain C
(``synth.c``) behind ctypes; the shared library is compiled with gcc on
first use (or by ``build()``) into ``synth/_build``.

Workloads and their recipes:

* ``laplace2d(nx, ny)``: 5-point stencil, 4 on the diagonal, -1 off it.
* ``stencil27(nx, ny, nz, values=...)``: 27-point stencil, values N(0,1)
  (``values="normal"``) or 26/-1 (``values="poisson"``).
* ``fem3d(nnodes)``: 3x3 dense node blocks on a random-geometric mesh with
  about 26 neighbours per node, Morton-ordered, values N(0,1).
* ``powerlaw(n)``: Zipf(2) row lengths rescaled to mean 20, columns near the
  diagonal (sigma 1000), rows longer than 4000 uniform; values N(0,1).
* ``uniform(n, per_row)``: distinct uniform columns; values N(0,1).
* ``dense(n)``: every entry stored (the paper's "dense" matrix).
* ``bernoulli(nrows, ncols, density)``: small random patterns.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libspc5synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library (gcc, OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CSR(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64),
                ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.POINTER(ctypes.c_int32)),
                ("colidx", ctypes.POINTER(ctypes.c_int32)),
                ("vals", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, dbl, ci = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                 ctypes.c_int)
            p = ctypes.POINTER(_CSR)
            sigs = {
                "synth_stencil2d_5pt": [i64, i64, ci, dbl, dbl, u64, p],
                "synth_stencil3d_27pt": [i64, i64, i64, ci, dbl, dbl, u64, p],
                "synth_dense": [i64, i64, ci, dbl, dbl, u64, p],
                "synth_bernoulli": [i64, i64, dbl, ci, u64, p],
                "synth_uniform": [i64, i64, i64, u64, p],
                "synth_powerlaw": [i64, dbl, dbl, dbl, i64, u64, p],
                "synth_fem3d": [i64, dbl, u64, p],
            }
            for name, args in sigs.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ci
            lib.synth_free.argtypes = [p]
            lib.synth_free.restype = None
            dp = ctypes.POINTER(ctypes.c_double)
            lib.synth_vector_uniform.argtypes = [i64, dbl, dbl, u64, u64, dp]
            lib.synth_vector_normal.argtypes = [i64, u64, u64, dp]
            lib.synth_vector_int.argtypes = [i64, i64, i64, u64, u64, dp]
            for f in (lib.synth_vector_uniform, lib.synth_vector_normal,
                      lib.synth_vector_int):
                f.restype = None
            _lib = lib
    return _lib


@dataclass
class CSR:
    """A CSR matrix in host memory: int32 row pointers and column indices
    (columns strictly ascending per row), float64 values."""
    nrows: int
    ncols: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def todense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols), dtype=np.float64)
        rows = np.repeat(np.arange(self.nrows), np.diff(self.rowptr))
        d[rows, self.colidx] = self.vals
        return d


def _call(fn_name: str, *args, name: str = "") -> CSR:
    lib = _load()
    out = _CSR()
    rc = getattr(lib, fn_name)(*args, ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"{fn_name} failed with code {rc}")
    try:
        n, nnz = out.nrows, out.nnz
        rowptr = np.ctypeslib.as_array(out.rowptr, shape=(n + 1,)).copy()
        if nnz > 0:
            colidx = np.ctypeslib.as_array(out.colidx, shape=(nnz,)).copy()
            vals = np.ctypeslib.as_array(out.vals, shape=(nnz,)).copy()
        else:
            colidx = np.zeros(0, np.int32)
            vals = np.zeros(0, np.float64)
        return CSR(int(n), int(out.ncols), rowptr, colidx, vals, name)
    finally:
        lib.synth_free(ctypes.byref(out))


_VALUE_MODES = {"constant": 0, "normal": 1}


def laplace2d(nx: int, ny: int, diag: float = 4.0, off: float = -1.0) -> CSR:
    return _call("synth_stencil2d_5pt", nx, ny, 0, diag, off, 0,
                 name=f"laplace2d_{nx}x{ny}")


def stencil27(nx: int, ny: int, nz: int, values: str = "normal", seed: int = 1,
              diag: float = 26.0, off: float = -1.0) -> CSR:
    if values == "poisson":
        mode, diag, off = 0, 26.0, -1.0
    else:
        mode = _VALUE_MODES[values]
    return _call("synth_stencil3d_27pt", nx, ny, nz, mode, diag, off, seed,
                 name=f"stencil27_{nx}x{ny}x{nz}")


def dense(nrows: int, ncols: int | None = None, values: str = "normal",
          seed: int = 5, diag: float = 1.0, off: float = 1.0) -> CSR:
    ncols = nrows if ncols is None else ncols
    return _call("synth_dense", nrows, ncols, _VALUE_MODES[values], diag, off, seed,
                 name=f"dense_{nrows}x{ncols}")


def bernoulli(nrows: int, ncols: int, density: float, seed: int = 0,
              integer_values: bool = True) -> CSR:
    return _call("synth_bernoulli", nrows, ncols, density,
                 2 if integer_values else 1, seed,
                 name=f"bernoulli_{nrows}x{ncols}_{density}_{seed}")


def uniform(nrows: int, per_row: int = 16, ncols: int | None = None,
            seed: int = 4) -> CSR:
    ncols = nrows if ncols is None else ncols
    return _call("synth_uniform", nrows, ncols, per_row, seed,
                 name=f"uniform_{nrows}_{per_row}")


def powerlaw(n: int, s: float = 2.0, mean: float = 20.0, sigma: float = 1000.0,
             long_row: int = 4000, seed: int = 3) -> CSR:
    """Zipf(s) row lengths rescaled to `mean`; rows of at most `long_row`
    entries take distinct columns round(i + N(0, sigma)), longer rows take
    distinct uniform columns.  Requires long_row <= 4 * sigma."""
    return _call("synth_powerlaw", n, s, mean, sigma, long_row, seed,
                 name=f"powerlaw_{n}")


def fem3d(nnodes: int, mean_nbrs: float = 26.0, seed: int = 2) -> CSR:
    return _call("synth_fem3d", nnodes, mean_nbrs, seed, name=f"fem3d_{nnodes}")


def vector_uniform(n: int, lo: float = -1.0, hi: float = 1.0, seed: int = 0,
                   stream: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_vector_uniform(n, lo, hi, seed, stream,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def vector_normal(n: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_vector_normal(n, seed, stream,
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def vector_int(n: int, lo: int = -3, hi: int = 3, seed: int = 0,
               stream: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_vector_int(n, lo, hi, seed, stream,
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


# Named workloads with the sizes of the benchmark configurations.
def workload(name: str, scale: str = "full") -> CSR:
    """Named workloads.  scale="full": the benchmark sizes; "small": reduced
    instances of the same generators for quick parity runs; "profile":
    instances still larger than the GPU's L2 cache (129 MB) but a quarter or
    less of the full size, for hardware-counter captures."""
    if scale not in ("full", "small", "profile"):
        raise ValueError(scale)
    pick = {"full": 0, "profile": 1, "small": 2}[scale]
    if name == "laplace2d_128":
        return laplace2d(128, 128)
    if name == "stencil27":
        k = (100, 90, 24)[pick]
        return stencil27(k, k, k, values="normal", seed=1)
    if name == "fem3d":
        return fem3d((1_000_000, 250_000, 20_000)[pick], seed=2)
    if name == "powerlaw":
        return powerlaw((2_000_000, 1_000_000, 40_000)[pick], seed=3)
    if name == "uniform":
        return uniform((1_000_000, 1_000_000, 30_000)[pick], 16, seed=4)
    if name == "poisson27_128":
        return stencil27(128, 128, 128, values="poisson")
    if name == "dense2048":
        return dense(2048, values="normal", seed=5)
    raise KeyError(name)
