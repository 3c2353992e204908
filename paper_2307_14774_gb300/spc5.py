"""Thin ctypes binding of libspc5.so: the C-ABI names, argument marshalling
only.  Every step of the conversion and of the product runs in the
library's CUDA kernels; there is no Python or CPU fallback.  If the library
is missing or fails to load, import raises.

Tensors are torch CUDA tensors (torch provides device memory and streams)
or host arrays (numpy or CPU tensors), passed by pointer.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SPC5_F64, SPC5_F32, SPC5_BF16 = 0, 1, 2
STATUS = {0: "SPC5_OK", 1: "SPC5_EINVAL", 2: "SPC5_EUNSORTED", 3: "SPC5_EUNSUPPORTED_RC",
          4: "SPC5_EOVERFLOW", 5: "SPC5_ECUDA", 6: "SPC5_ENOMEM", 7: "SPC5_EDEVICE",
          8: "SPC5_ERANGE", 9: "SPC5_EROWPTR", 10: "SPC5_EUNSUPPORTED"}
SUPPORTED_RC = ((1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4))

# Exported symbols declared in include/spc5.h.
EXPORTS = ("spc5_convert_csr", "spc5_matrix_info", "spc5_export", "spc5_spmv", "spc5_destroy",
           "spc5_status_str", "spc5_last_error", "spc5_spmv_t", "spc5_build_transpose",
           "spc5_values_grad",
           "spc5_set_values", "spc5_tune", "spc5_convert_tuned", "spc5_convert_tuned_ex",
           "spc5_spmv_batched",
           "spc5_batch_create", "spc5_batch_run", "spc5_batch_destroy", "spc5_ircg",
           "spc5_spmv_noalloc", "spc5_convert_hybrid", "spc5_export_hybrid",
           "spc5_measure_fma_peak")


class SPC5Error(RuntimeError):
    def __init__(self, code: int, detail: str = ""):
        super().__init__(f"{STATUS.get(code, code)}: {detail}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Info(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("r", ctypes.c_int32), ("c", ctypes.c_int32), ("npanels", ctypes.c_int64),
                ("nblocks", ctypes.c_int64), ("filling", ctypes.c_double),
                ("value_dtype", ctypes.c_int), ("mask_bytes", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("device", ctypes.c_int32),
                ("lanes_per_row", ctypes.c_int32), ("launches_per_spmv", ctypes.c_int32),
                ("ntiles", ctypes.c_int64), ("long_panels", ctypes.c_int64),
                ("stages", ctypes.c_int32), ("consumers", ctypes.c_int32),
                ("device_error", ctypes.c_uint32), ("tuned_us", ctypes.c_double),
                ("flat", ctypes.c_int32), ("group_efficiency", ctypes.c_double),
                ("hybrid", ctypes.c_int32), ("nscalars", ctypes.c_int64),
                ("tuned_rows_us", ctypes.c_double), ("pieces", ctypes.c_int64),
                ("scalar_pieces", ctypes.c_int64), ("body", ctypes.c_int32),
                ("dynamic", ctypes.c_int32), ("transposed", ctypes.c_int32),
                ("halves", ctypes.c_int32)]


class CGReport(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("relres", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load (building first if needed) libspc5.so and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is None:
            path = _build.build() if not _build.up_to_date() else _build.LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"libspc5.so not found at {path}")
        lib = ctypes.CDLL(path)
        vp, i64, ci, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.spc5_convert_csr.argtypes = [i64, i64, i64, vp, vp, vp, ci, ci, ci, ci, vp,
                                         ctypes.POINTER(vp)]
        lib.spc5_matrix_info.argtypes = [vp, ctypes.POINTER(Info)]
        lib.spc5_export.argtypes = [vp] + [ctypes.POINTER(vp)] * 5
        lib.spc5_spmv.argtypes = [vp, vp, vp, dbl, dbl, vp]
        lib.spc5_spmv_t.argtypes = [vp, vp, vp, dbl, dbl, vp]
        lib.spc5_build_transpose.argtypes = [vp, vp]
        lib.spc5_build_transpose.restype = ci
        lib.spc5_values_grad.argtypes = [vp, vp, vp, vp, dbl, vp]
        lib.spc5_set_values.argtypes = [vp, vp, vp]
        for f in (lib.spc5_spmv_t, lib.spc5_values_grad, lib.spc5_set_values):
            f.restype = ci
        lib.spc5_tune.argtypes = [vp, vp, vp, ci, vp]
        lib.spc5_tune.restype = ci
        lib.spc5_convert_tuned.argtypes = [i64, i64, i64, vp, vp, vp, ci, ci,
                                           ctypes.POINTER(ctypes.c_int), ci, ci, vp,
                                           ctypes.POINTER(vp)]
        lib.spc5_convert_tuned.restype = ci
        lib.spc5_convert_tuned_ex.argtypes = [i64, i64, i64, vp, vp, vp, ci, ci,
                                              ctypes.POINTER(ctypes.c_int), ci, ci, ci, vp,
                                              ctypes.POINTER(vp)]
        lib.spc5_convert_tuned_ex.restype = ci
        pvp = ctypes.POINTER(vp)
        lib.spc5_spmv_batched.argtypes = [ci, pvp, pvp, pvp, ci, vp]
        lib.spc5_batch_create.argtypes = [ci, pvp, pvp, pvp, ci, vp, pvp]
        lib.spc5_batch_run.argtypes = [vp, dbl, dbl, vp]
        lib.spc5_batch_destroy.argtypes = [vp]
        for f in (lib.spc5_spmv_batched, lib.spc5_batch_create, lib.spc5_batch_run,
                  lib.spc5_batch_destroy):
            f.restype = ci
        lib.spc5_ircg.argtypes = [vp, vp, vp, vp, dbl, ci, dbl, ci, vp, ctypes.POINTER(CGReport)]
        lib.spc5_ircg.restype = ci
        lib.spc5_spmv_noalloc.argtypes = [vp, vp, vp, dbl, dbl, vp]
        lib.spc5_spmv_noalloc.restype = ci
        lib.spc5_convert_hybrid.argtypes = lib.spc5_convert_csr.argtypes
        lib.spc5_convert_hybrid.restype = ci
        lib.spc5_export_hybrid.argtypes = [vp] + [ctypes.POINTER(vp)] * 3
        lib.spc5_export_hybrid.restype = ci
        lib.spc5_measure_fma_peak.argtypes = [ci, vp, ctypes.POINTER(dbl)]
        lib.spc5_measure_fma_peak.restype = ci
        lib.spc5_destroy.argtypes = [vp]
        for f in (lib.spc5_convert_csr, lib.spc5_matrix_info, lib.spc5_export, lib.spc5_spmv,
                  lib.spc5_destroy):
            f.restype = ci
        lib.spc5_status_str.argtypes = [ci]
        lib.spc5_status_str.restype = ctypes.c_char_p
        lib.spc5_last_error.argtypes = []
        lib.spc5_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        detail = load().spc5_last_error().decode(errors="replace")
        raise SPC5Error(rc, detail)


def _ptr(a) -> int | None:
    """Raw address of a torch tensor or numpy array (None for None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Matrix:
    """Owning wrapper of an spc5_matrix handle."""

    def __init__(self, handle: int, keepalive=()):
        self._h = ctypes.c_void_p(handle)
        self._keep = keepalive

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("matrix has been destroyed")
        return self._h

    def info(self) -> dict:
        return spc5_matrix_info(self)

    @classmethod
    def from_csr(cls, A, r: int = 4, c: int = 8, store_dtype=SPC5_F64, stream=None) -> "Matrix":
        """beta(r,c) from a torch sparse CSR tensor (indices narrowed to int32,
        values widened to FP64 for the conversion; the call synchronises)."""
        import torch
        if getattr(A, "layout", None) != torch.sparse_csr:
            raise TypeError("expected a torch.sparse_csr tensor")
        nrows, ncols = A.shape
        rowptr = A.crow_indices().to(torch.int32).contiguous()
        colidx = A.col_indices().to(torch.int32).contiguous()
        vals = A.values().to(torch.float64).contiguous()
        return spc5_convert_csr(nrows, ncols, vals.numel(), rowptr, colidx, vals,
                                store_dtype=store_dtype, r=r, c=c, stream=stream)

    @property
    def shape(self) -> tuple:
        info = self.info()
        return (info["nrows"], info["ncols"])

    def _vector_dtype(self):
        import torch
        return torch.float64 if self.info()["value_dtype"] == SPC5_F64 else torch.float32

    def __matmul__(self, x):
        """y = A x for x [ncols] or X [ncols][k] (torch tensors; k columns go
        through the batched kernel when k is 1, 2, 4, 8 or 16)."""
        import torch
        info = self.info()
        dt = self._vector_dtype()
        xc = x.to(dt).contiguous()
        if xc.dim() == 1:
            y = torch.empty(info["nrows"], dtype=dt, device=x.device)
            spc5_spmv(self, xc, y)
            return y
        if xc.dim() != 2:
            raise ValueError("x must be a vector or a matrix of right-hand sides")
        k = xc.shape[1]
        y = torch.empty((info["nrows"], k), dtype=dt, device=x.device)
        if k in (1, 2, 4, 8, 16) and not info["hybrid"] and x.is_cuda:
            spc5_spmv_batched([self], [xc], [y], k)
        else:
            for j in range(k):
                col = torch.empty(info["nrows"], dtype=dt, device=x.device)
                spc5_spmv(self, xc[:, j].contiguous(), col)
                y[:, j] = col
        return y

    def t(self) -> "_Transposed":
        """A^T, for products A^T g (spc5_spmv_t)."""
        return _Transposed(self)


class _Transposed:
    """A^T of a converted matrix: A.t() @ g = spc5_spmv_t(A, g)."""

    def __init__(self, A: "Matrix"):
        self.A = A

    @property
    def shape(self) -> tuple:
        return tuple(reversed(self.A.shape))

    def __matmul__(self, g):
        import torch
        info = self.A.info()
        dt = self.A._vector_dtype()
        gc = g.to(dt).contiguous()
        if gc.dim() != 1:
            raise ValueError("g must be a vector")
        dx = torch.empty(info["ncols"], dtype=dt, device=g.device)
        spc5_spmv_t(self.A, gc, dx)
        return dx

    def __del__(self):
        try:
            if self._h:
                load().spc5_destroy(self._h)
                self._h = ctypes.c_void_p(None)
        except Exception:
            pass


def spc5_convert_csr(nrows, ncols, nnz, rowptr, colidx, vals, vals_dtype=SPC5_F64,
                     store_dtype=SPC5_F64, r=4, c=8, stream=None) -> Matrix:
    """CSR -> beta(r,c) on the GPU; arrays in device or host memory."""
    lib = load()
    out = ctypes.c_void_p()
    _check(lib.spc5_convert_csr(nrows, ncols, nnz, _ptr(rowptr), _ptr(colidx), _ptr(vals),
                                vals_dtype, store_dtype, r, c, _stream_ptr(stream),
                                ctypes.byref(out)))
    return Matrix(out.value)


def spc5_convert_hybrid(nrows, ncols, nnz, rowptr, colidx, vals, vals_dtype=SPC5_F64,
                        store_dtype=SPC5_F64, r=4, c=8, stream=None) -> Matrix:
    """CSR -> hybrid beta(r,c): blocks of two or more values plus scalars."""
    lib = load()
    out = ctypes.c_void_p()
    _check(lib.spc5_convert_hybrid(nrows, ncols, nnz, _ptr(rowptr), _ptr(colidx), _ptr(vals),
                                   vals_dtype, store_dtype, r, c, _stream_ptr(stream),
                                   ctypes.byref(out)))
    return Matrix(out.value)


def spc5_export_hybrid(A: Matrix) -> dict:
    """Device pointers of a hybrid matrix's scalars (owned by A)."""
    lib = load()
    outs = [ctypes.c_void_p() for _ in range(3)]
    _check(lib.spc5_export_hybrid(A.handle, *[ctypes.byref(o) for o in outs]))
    return dict(zip(("s_rowptr", "s_colidx", "s_vals"), (o.value for o in outs)))


def spc5_matrix_info(A: Matrix) -> dict:
    info = Info()
    _check(load().spc5_matrix_info(A.handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in Info._fields_}


def spc5_export(A: Matrix) -> dict:
    """Device pointers of the converted arrays (owned by A)."""
    ptrs = [ctypes.c_void_p() for _ in range(5)]
    _check(load().spc5_export(A.handle, *[ctypes.byref(p) for p in ptrs]))
    names = ("block_rowptr", "panel_vptr", "block_colidx", "block_masks", "values")
    return {n: p.value for n, p in zip(names, ptrs)}


def spc5_spmv(A: Matrix, x, y, alpha: float = 1.0, beta: float = 0.0, stream=None) -> None:
    """y = alpha * A x + beta * y (FP64 vectors, device or host)."""
    _check(load().spc5_spmv(A.handle, _ptr(x), _ptr(y), float(alpha), float(beta),
                            _stream_ptr(stream)))


def spc5_spmv_t(A: Matrix, g, dx, alpha: float = 1.0, beta: float = 0.0, stream=None) -> None:
    """dx = alpha * A^T g + beta * dx (device vectors)."""
    _check(load().spc5_spmv_t(A.handle, _ptr(g), _ptr(dx), float(alpha), float(beta),
                              _stream_ptr(stream)))


def spc5_build_transpose(A: Matrix, stream=None) -> None:
    """Attach A^T in beta(r,c) to A: spc5_spmv_t then runs as a plain SpMV."""
    _check(load().spc5_build_transpose(A.handle, _stream_ptr(stream)))


def spc5_values_grad(A: Matrix, g, x, dvals, alpha: float = 1.0, stream=None) -> None:
    """dvals[e] = alpha * g[row(e)] * x[col(e)] in CSR order (device arrays)."""
    _check(load().spc5_values_grad(A.handle, _ptr(g), _ptr(x), _ptr(dvals), float(alpha),
                                   _stream_ptr(stream)))


def spc5_set_values(A: Matrix, vals, stream=None) -> None:
    """Replace the stored values with CSR-ordered FP64 device values."""
    _check(load().spc5_set_values(A.handle, _ptr(vals), _stream_ptr(stream)))


def spc5_measure_fma_peak(dtype: int = SPC5_F64, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (FP64 or FP32)."""
    out = ctypes.c_double(0.0)
    _check(load().spc5_measure_fma_peak(int(dtype), _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def spc5_tune(A: Matrix, x, y, iters: int = 5, stream=None) -> dict:
    """Autotune the lanes-per-row mapping on (x, y); returns the new info."""
    _check(load().spc5_tune(A.handle, _ptr(x), _ptr(y), int(iters), _stream_ptr(stream)))
    return spc5_matrix_info(A)


def spc5_convert_tuned(nrows, ncols, nnz, rowptr, colidx, vals, vals_dtype=SPC5_F64,
                       store_dtype=SPC5_F64, shapes=None, iters: int = 5,
                       stream=None) -> Matrix:
    """Convert into each block shape (default: all six), tune each, keep the fastest."""
    lib = load()
    out = ctypes.c_void_p()
    arr, n = _shape_array(shapes)
    _check(lib.spc5_convert_tuned(nrows, ncols, nnz, _ptr(rowptr), _ptr(colidx), _ptr(vals),
                                  vals_dtype, store_dtype, arr, n, int(iters),
                                  _stream_ptr(stream), ctypes.byref(out)))
    return Matrix(out.value)


def spc5_convert_tuned_ex(nrows, ncols, nnz, rowptr, colidx, vals, vals_dtype=SPC5_F64,
                          store_dtype=SPC5_F64, shapes=None, iters: int = 5,
                          rows_plan: bool = False, stream=None) -> Matrix:
    """spc5_convert_tuned; rows_plan ranks the shapes by their fastest
    row-group plan (the batched, transposed and gradient kernels' plan)."""
    lib = load()
    out = ctypes.c_void_p()
    arr, n = _shape_array(shapes)
    _check(lib.spc5_convert_tuned_ex(nrows, ncols, nnz, _ptr(rowptr), _ptr(colidx), _ptr(vals),
                                     vals_dtype, store_dtype, arr, n, int(iters),
                                     1 if rows_plan else 0, _stream_ptr(stream),
                                     ctypes.byref(out)))
    return Matrix(out.value)


def _shape_array(shapes):
    if shapes is None:
        return None, 0
    flat = [v for rc in shapes for v in rc]
    return (ctypes.c_int * len(flat))(*flat), len(shapes)


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, it in enumerate(items):
        arr[i] = it.handle.value if isinstance(it, Matrix) else _ptr(it)
    return arr


def spc5_spmv_batched(mats, X, Y, k: int = 1, stream=None) -> None:
    """Y[m] = A[m] X[m] (X[m]: [ncols][k], Y[m]: [nrows][k], row-major, device)."""
    _check(load().spc5_spmv_batched(len(mats), _ptr_array(mats), _ptr_array(X), _ptr_array(Y),
                                    int(k), _stream_ptr(stream)))


class Batch:
    """Owning wrapper of an spc5_batch handle (keeps matrices and vectors alive)."""

    def __init__(self, mats, X, Y, k: int = 1, stream=None):
        self._keep = (list(mats), list(X), list(Y))
        h = ctypes.c_void_p()
        _check(load().spc5_batch_create(len(mats), _ptr_array(mats), _ptr_array(X),
                                        _ptr_array(Y), int(k), _stream_ptr(stream),
                                        ctypes.byref(h)))
        self._h = h

    def run(self, alpha: float = 1.0, beta: float = 0.0, stream=None) -> None:
        _check(load().spc5_batch_run(self._h, float(alpha), float(beta), _stream_ptr(stream)))

    def __del__(self):
        try:
            if self._h:
                load().spc5_batch_destroy(self._h)
                self._h = ctypes.c_void_p(None)
        except Exception:
            pass


def spc5_ircg(A64: Matrix, Alo: Matrix, b, x, tol: float = 1e-10, max_outer: int = 50,
              inner_tol: float = 1e-3, max_inner: int = 1000, stream=None) -> dict:
    """Mixed-precision iterative-refinement CG; x (FP64, device) is updated in place."""
    rep = CGReport()
    _check(load().spc5_ircg(A64.handle, Alo.handle, _ptr(b), _ptr(x), float(tol), int(max_outer),
                            float(inner_tol), int(max_inner), _stream_ptr(stream),
                            ctypes.byref(rep)))
    return {"outer_iters": rep.outer_iters, "inner_iters": rep.inner_iters,
            "relres": rep.relres}


def spc5_spmv_noalloc(A: Matrix, x, y, alpha: float = 1.0, beta: float = 0.0,
                      stream=None) -> None:
    """y = alpha * A x + beta * y without any device allocation (device
    vectors only; partial sums in the library's fixed scratch array)."""
    _check(load().spc5_spmv_noalloc(A.handle, _ptr(x), _ptr(y), float(alpha), float(beta),
                                    _stream_ptr(stream)))


def spc5_destroy(A: Matrix) -> None:
    if A._h:
        _check(load().spc5_destroy(A._h))
        A._h = ctypes.c_void_p(None)


def spc5_status_str(code: int) -> str:
    return load().spc5_status_str(code).decode()


def spc5_last_error() -> str:
    return load().spc5_last_error().decode(errors="replace")


# ---------------------------------------------------------------- helpers --

class _DeviceArray:
    """A non-owning view of device memory exposed through the CUDA array
    interface, so torch can wrap the library's arrays without copying."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}
        self._owner = owner


def export_tensors(A: Matrix) -> dict:
    """The converted arrays as torch tensors viewing A's device memory."""
    import torch
    info = spc5_matrix_info(A)
    p = spc5_export(A)
    npan, nb = info["npanels"], info["nblocks"]
    nnz = info["nnz"] - info["nscalars"]  # values stored in blocks
    dev = torch.device("cuda", info["device"])

    def view(ptr, n, typestr):
        if n == 0:
            return torch.empty(0, device=dev, dtype={"<i4": torch.int32, "|u1": torch.uint8,
                                                     "<f8": torch.float64}[typestr])
        return torch.as_tensor(_DeviceArray(ptr, (n,), typestr, A), device=dev)

    out = {"block_rowptr": view(p["block_rowptr"], npan + 1, "<i4"),
            "panel_vptr": view(p["panel_vptr"], npan + 1, "<i4"),
            "block_colidx": view(p["block_colidx"], nb, "<i4"),
            # packed mask words as raw little-endian bytes, mask_bytes per block
            "block_masks": view(p["block_masks"], nb * info["mask_bytes"], "|u1"),
            # raw value storage: FP64, FP32 or BF16 bit patterns, as bytes for non-FP64
            "values": (view(p["values"], nnz, "<f8") if info["value_dtype"] == SPC5_F64 else
                       view(p["values"], nnz * (4 if info["value_dtype"] == SPC5_F32 else 2),
                            "|u1"))}
    if info["hybrid"]:
        h = spc5_export_hybrid(A)
        ns = info["nscalars"]
        out["s_rowptr"] = view(h["s_rowptr"], info["nrows"] + 1, "<i4")
        out["s_colidx"] = view(h["s_colidx"], ns, "<i4")
        out["s_vals"] = (view(h["s_vals"], ns, "<f8") if info["value_dtype"] == SPC5_F64 else
                         view(h["s_vals"], ns * (4 if info["value_dtype"] == SPC5_F32 else 2),
                              "|u1"))
    return out
