"""Python binding of libgrb.so, the GB300 nonblocking-GraphBLAS library.

Argument marshalling only: every function below calls the C entry point of
the same name declared in include/grb.h, and every step of the computation
runs in the library's CUDA kernels.  Importing the package loads libgrb.so
and raises if it has not been built (``python -c "import __graft_entry__ as
g; g.build()"``); there is no CPU fallback.

Handles are plain integers (the C pointers).  Host arrays are numpy arrays;
device arrays may be passed as torch CUDA tensors where a call accepts device
pointers.  Errors raise GrbError carrying the grb_info code.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [n for n in dir() if n.startswith("grb_") or n.startswith("GRB_")]

_HERE = os.path.dirname(os.path.abspath(__file__))
# GRB_CHECK_BOUNDS=1 in the environment selects the bounds-checked debug
# build of the same library (include/grb_debug.h)
CHECKED = os.environ.get("GRB_CHECK_BOUNDS", "0") == "1"
LIB_PATH = os.path.join(_HERE, "libgrb_checked.so" if CHECKED else "libgrb.so")

# ---------------------------------------------------------------- constants
GRB_SUCCESS, GRB_NO_VALUE = 0, 1
GRB_NULL_POINTER, GRB_INVALID_VALUE, GRB_INVALID_INDEX = -1, -2, -3
GRB_DOMAIN_MISMATCH, GRB_DIMENSION_MISMATCH, GRB_UNINITIALIZED_OBJECT = -4, -5, -6
GRB_NOT_IMPLEMENTED, GRB_INVALID_OBJECT = -7, -8
GRB_OUT_OF_MEMORY, GRB_INDEX_OUT_OF_BOUNDS, GRB_DEVICE_ERROR = -101, -102, -103
GRB_DEVICE_TIMEOUT, GRB_PANIC = -104, -105

GRB_BLOCKING, GRB_NONBLOCKING = 0, 1
GRB_INT32, GRB_FP32, GRB_FP64, GRB_BF16 = 1, 2, 3, 4
(GRB_FIRST, GRB_SECOND, GRB_PLUS, GRB_MINUS, GRB_TIMES, GRB_DIV, GRB_MAX, GRB_MIN,
 GRB_ABS_DIFF, GRB_MAX_DIV_BY) = range(1, 11)
GRB_IDENTITY, GRB_ABS, GRB_AINV, GRB_MINV = 1, 2, 3, 4
GRB_MONOID_PLUS, GRB_MONOID_MAX, GRB_MONOID_MIN, GRB_MONOID_TIMES = 1, 2, 3, 4
(GRB_PLUS_TIMES, GRB_PLUS_SECOND, GRB_PLUS_FIRST, GRB_MAX_TIMES, GRB_MIN_PLUS,
 GRB_MAX_SECOND) = range(1, 7)
GRB_DESC_DEFAULT, GRB_DESC_REPLACE, GRB_DESC_STRUCTURE, GRB_DESC_COMPLEMENT = 0, 1, 2, 4
GRB_BUILD_TRANSPOSE, GRB_BUILD_DROP_SELF, GRB_BUILD_DEDUP, GRB_BUILD_DEVICE_PTRS = 1, 2, 4, 8
GRB_WAIT_COMPLETE, GRB_WAIT_MATERIALIZE = 0, 1
GRB_OPT_FUSION, GRB_OPT_PERSISTENT, GRB_OPT_SPIN_LIMIT, GRB_OPT_MIXED_SWITCH, GRB_OPT_MIXED, GRB_OPT_RELABEL = 1, 2, 3, 4, 5, 6
GRB_OPT_HOT_BYTES = 7
GRB_OPT_TMA_STAGES = 8
GRB_OPT_ROW_BINS = 9
GRB_HOT_BYTES_MAX = 196608
GRB_FUSED_INDEX_LIMIT = 2130706432   # 2^31 - 2^24: nrows + nnz bound of the fused kernels

NP_TYPES = {GRB_INT32: np.int32, GRB_FP32: np.float32, GRB_FP64: np.float64, GRB_BF16: np.uint16}


class GrbError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        super().__init__(f"{where} failed with grb_info {code}" + (f": {msg}" if msg else ""))
        self.code = code


class grb_binop(ctypes.Structure):
    _fields_ = [("opcode", ctypes.c_int32), ("reserved", ctypes.c_int32), ("k", ctypes.c_double)]


class grb_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("kernel_launches", "fused_groups", "unfused_nodes",
                                              "elided_vectors", "persistent_loops", "replayed_loops",
                                              "device_bytes", "cache_hits", "last_loop_kernel_ns")]


class grb_serve_config(ctypes.Structure):
    _fields_ = [("damping", ctypes.c_double), ("tol", ctypes.c_double), ("itermax", ctypes.c_int64),
                ("chunk", ctypes.c_int64), ("slots", ctypes.c_int32), ("mem_fraction", ctypes.c_double),
                ("single_max", ctypes.c_int32)]


class grb_serve_result(ctypes.Structure):
    _fields_ = [("latency_s", ctypes.c_void_p), ("iters", ctypes.c_void_p), ("resid", ctypes.c_void_p),
                ("ranks", ctypes.c_void_p), ("slots", ctypes.c_int32), ("vector_width", ctypes.c_int32),
                ("steps", ctypes.c_int64),
                ("max_in_flight", ctypes.c_int64), ("wall_s", ctypes.c_double), ("single_queries", ctypes.c_int64)]


def binop(code: int, k: float = 0.0) -> grb_binop:
    return grb_binop(int(code), 0, float(k))


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

# ---------------------------------------------------------------- loading
_lock = threading.Lock()
_lib = None
_keep = {}   # allocator callbacks per context (must outlive the context)


def _declare(lib):
    V, I, U64, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    B = grb_binop
    sig = {
        "grb_context_new": [P(V), I, V, ALLOC_FN, FREE_FN, V],
        "grb_context_set": [V, I, I64],
        "grb_context_stats": [V, P(grb_stats)],
        "grb_context_wait": [V],
        "grb_matrix_build_csr": [P(V), V, I, U64, U64, V, V, V, U64, ctypes.c_uint32],
        "grb_matrix_nvals": [P(U64), V],
        "grb_matrix_nrows": [P(U64), V],
        "grb_matrix_export_csr": [V, V, V, V, I],
        "grb_matrix_col_degree": [V, V],
        "grb_vector_new": [P(V), V, I, U64],
        "grb_vector_fill": [V, D],
        "grb_vector_build": [V, V, V, U64, I],
        "grb_vector_copy": [V, V],
        "grb_vector_size": [P(U64), V],
        "grb_vector_nvals": [P(U64), V],
        "grb_vector_extract_dense": [V, V, V, I],
        "grb_scalar_new": [P(V), V, I],
        "grb_scalar_set": [V, D],
        "grb_scalar_get": [V, P(D)],
        "grb_scalar_apply_bind2nd": [V, B, V, D],
        "grb_apply": [V, V, P(B), I, V, ctypes.c_uint32],
        "grb_apply_bind2nd": [V, V, P(B), B, V, D, ctypes.c_uint32],
        "grb_apply_bind2nd_scalar": [V, V, P(B), B, V, V, ctypes.c_uint32],
        "grb_assign_scalar": [V, V, P(B), V, ctypes.c_uint32],
        "grb_mxv": [V, V, P(B), I, V, V, ctypes.c_uint32],
        "grb_ewise_add": [V, V, P(B), B, V, V, ctypes.c_uint32],
        "grb_ewise_mult": [V, V, P(B), B, V, V, ctypes.c_uint32],
        "grb_reduce": [V, P(B), I, V, ctypes.c_uint32],
        "grb_wait": [V, I],
        "grb_iterate_begin": [V],
        "grb_iterate_end": [V, V, D, I64, P(I64)],
        "grb_iterate_history": [V, P(D), P(D), I64, P(I64), P(ctypes.c_int32)],
        "grb_context_loop_times": [V, P(D), I64, P(I64)],
        "grb_free": [P(V)],
        "grb_error": [V],
        "grb_selftest_wait_timeout": [V, I64],
        "grb_reduce_dense_noalloc": [V, I, U64, I, V, V],
        "grb_ppr_new": [P(V), V, D, ctypes.c_int32],
        "grb_ppr_slots": [V, P(ctypes.c_int32)],
        "grb_ppr_tune": [V, I64, V, V],
        "grb_ppr_layout": [V, ctypes.c_int32],
        "grb_ppr_set": [V, ctypes.c_int32, V, I64, D, I64],
        "grb_ppr_clear": [V, ctypes.c_int32],
        "grb_ppr_run": [V, I64],
        "grb_ppr_status": [V, V, V, V],
        "grb_ppr_get": [V, ctypes.c_int32, V, I],
        "grb_ppr_serve": [V, P(grb_serve_config), I64, V, V, V, P(grb_serve_result)],
        "grb_prbatch_new": [P(V), V, ctypes.c_int32, V, D],
        "grb_prbatch_tune": [V, I64, V, ctypes.c_int32, V],
        "grb_prbatch_run": [V, D, I64, I64],
        "grb_prbatch_result": [V, V, V, V],
    }
    if CHECKED:
        # include/grb_debug.h: exported by the bounds-checked build only
        sig["grb_debug_check_csr"] = [V, V, V, U64, U64, U64, P(ctypes.c_int32), P(I64)]
        sig["grb_debug_set_col"] = [V, U64, ctypes.c_int32]
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "grb_error" else ctypes.c_int


def load():
    """Load libgrb.so, or libgrb_checked.so under GRB_CHECK_BOUNDS=1 (raises
    if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                                  "(__graft_entry__.build()); there is no CPU fallback")
            lib = ctypes.CDLL(LIB_PATH)
            _declare(lib)
            _lib = lib
    return _lib


def symbols():
    """Names of the entry points the binding declares (all of include/grb.h)."""
    lib = load()
    return [n for n in ("grb_context_new", "grb_context_set", "grb_context_stats", "grb_context_wait",
                        "grb_matrix_build_csr", "grb_matrix_nvals", "grb_matrix_nrows", "grb_matrix_export_csr",
                        "grb_matrix_col_degree", "grb_vector_new", "grb_vector_fill", "grb_vector_build",
                        "grb_vector_copy", "grb_vector_size", "grb_vector_nvals", "grb_vector_extract_dense",
                        "grb_scalar_new", "grb_scalar_set", "grb_scalar_get", "grb_scalar_apply_bind2nd",
                        "grb_apply", "grb_apply_bind2nd", "grb_apply_bind2nd_scalar", "grb_assign_scalar",
                        "grb_mxv", "grb_ewise_add", "grb_ewise_mult", "grb_reduce", "grb_wait",
                        "grb_iterate_begin", "grb_iterate_end", "grb_iterate_history", "grb_context_loop_times",
                        "grb_free", "grb_error",
                        "grb_selftest_wait_timeout", "grb_reduce_dense_noalloc", "grb_ppr_new", "grb_ppr_slots", "grb_ppr_tune",
                        "grb_ppr_layout",
                        "grb_ppr_set", "grb_ppr_clear", "grb_ppr_run", "grb_ppr_status", "grb_ppr_get",
                        "grb_ppr_serve", "grb_prbatch_new", "grb_prbatch_tune", "grb_prbatch_run",
                        "grb_prbatch_result")
            if hasattr(lib, n)]


def _check(rc: int, where: str, obj=None) -> int:
    if rc < 0:
        msg = ""
        if obj:
            try:
                msg = (load().grb_error(obj) or b"").decode()
            except Exception:
                msg = ""
        raise GrbError(rc, where, msg)
    return rc


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None for None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _acc(accum):
    return None if accum is None else ctypes.byref(accum)


# ---------------------------------------------------------------- context
def grb_context_new(mode: int = GRB_NONBLOCKING, stream=None, torch_allocator: bool = True, alloc_hook=None) -> int:
    """New context on the current CUDA device.  `stream` is a torch CUDA
    stream (default: torch's current stream).  With torch_allocator, device
    memory comes from torch's caching allocator; alloc_hook(nbytes) -> bool,
    when given, is asked before every allocation and a False answer makes
    that allocation fail (allocator-failure injection)."""
    import torch
    lib = load()
    if not torch.cuda.is_available():
        raise GrbError(GRB_DEVICE_ERROR, "grb_context_new", "no CUDA device")
    dev = torch.cuda.current_device()
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    handle = ctypes.c_void_p(st.cuda_stream)
    if torch_allocator:
        def _alloc(_ctx, nbytes, stream_ptr):
            if alloc_hook is not None and not alloc_hook(int(nbytes)):
                return None
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream_ptr or 0))
            except Exception:
                return None

        def _free(_ctx, ptr, _stream):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass
        fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    else:
        fa, ff = ALLOC_FN(), FREE_FN()
    out = ctypes.c_void_p()
    _check(lib.grb_context_new(ctypes.byref(out), int(mode), handle, fa, ff, None), "grb_context_new")
    _keep[out.value] = (fa, ff, st)
    return out.value


def grb_context_set(ctx: int, opt: int, value: int) -> None:
    _check(load().grb_context_set(ctx, int(opt), int(value)), "grb_context_set", ctx)


def grb_context_stats(ctx: int) -> dict:
    s = grb_stats()
    _check(load().grb_context_stats(ctx, ctypes.byref(s)), "grb_context_stats", ctx)
    return {n: getattr(s, n) for n, _ in grb_stats._fields_}


def grb_context_wait(ctx: int) -> None:
    _check(load().grb_context_wait(ctx), "grb_context_wait", ctx)


# ----------------------------------------------------------------- matrix
def grb_matrix_build_csr(ctx: int, type_: int, nrows: int, ncols: int, src, dst, vals=None,
                         flags: int = GRB_BUILD_TRANSPOSE | GRB_BUILD_DROP_SELF | GRB_BUILD_DEDUP) -> int:
    """CSR from COO.  src/dst: int32 numpy arrays or contiguous int32 torch
    CPU tensors (host; pinned tensors let the library's upload run as a
    direct DMA copy), or int32 torch CUDA tensors (device;
    GRB_BUILD_DEVICE_PTRS is then added)."""
    if _is_device(src):
        flags |= GRB_BUILD_DEVICE_PTRS
    elif hasattr(src, "data_ptr"):
        import torch

        for a in (src, dst):
            if a.dtype != torch.int32 or not a.is_contiguous():
                raise GrbError(GRB_INVALID_VALUE, "grb_matrix_build_csr", "host tensors must be contiguous int32")
        if vals is not None:
            vals = np.ascontiguousarray(vals.numpy() if hasattr(vals, "numpy") else vals, dtype=NP_TYPES[type_])
    else:
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        if vals is not None:
            vals = np.ascontiguousarray(vals, dtype=NP_TYPES[type_])
    out = ctypes.c_void_p()
    _check(load().grb_matrix_build_csr(ctypes.byref(out), ctx, int(type_), int(nrows), int(ncols), _ptr(src),
                                       _ptr(dst), _ptr(vals), len(src), int(flags)), "grb_matrix_build_csr", ctx)
    return out.value


def grb_matrix_nvals(A: int) -> int:
    n = ctypes.c_uint64()
    _check(load().grb_matrix_nvals(ctypes.byref(n), A), "grb_matrix_nvals")
    return n.value


def grb_matrix_nrows(A: int) -> int:
    n = ctypes.c_uint64()
    _check(load().grb_matrix_nrows(ctypes.byref(n), A), "grb_matrix_nrows")
    return n.value


def grb_matrix_export_csr(A: int):
    """(row_ptr, col_idx) as int32 numpy arrays."""
    n, nnz = grb_matrix_nrows(A), grb_matrix_nvals(A)
    rp = np.empty(n + 1, dtype=np.int32)
    ci = np.empty(max(nnz, 1), dtype=np.int32)
    _check(load().grb_matrix_export_csr(A, _ptr(rp), _ptr(ci), None, 0), "grb_matrix_export_csr", A)
    return rp, ci[:nnz]


def grb_matrix_col_degree(deg: int, A: int) -> None:
    _check(load().grb_matrix_col_degree(deg, A), "grb_matrix_col_degree", deg)


# ----------------------------------------------------------------- vector
def grb_vector_new(ctx: int, type_: int, n: int) -> int:
    out = ctypes.c_void_p()
    _check(load().grb_vector_new(ctypes.byref(out), ctx, int(type_), int(n)), "grb_vector_new", ctx)
    return out.value


def grb_vector_fill(v: int, value: float) -> None:
    _check(load().grb_vector_fill(v, float(value)), "grb_vector_fill", v)


def grb_vector_build(v: int, idx, vals) -> None:
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    _check(load().grb_vector_build(v, _ptr(idx), _ptr(vals), len(idx), 0), "grb_vector_build", v)


def grb_vector_copy(dst: int, src: int) -> None:
    _check(load().grb_vector_copy(dst, src), "grb_vector_copy", dst)


def grb_vector_size(v: int) -> int:
    n = ctypes.c_uint64()
    _check(load().grb_vector_size(ctypes.byref(n), v), "grb_vector_size", v)
    return n.value


def grb_vector_nvals(v: int) -> int:
    n = ctypes.c_uint64()
    _check(load().grb_vector_nvals(ctypes.byref(n), v), "grb_vector_nvals", v)
    return n.value


def grb_vector_extract_dense(v: int, type_: int, out=None, present: bool = True):
    """Values (numpy array of the vector's type, absent -> 0) and a uint8
    presence array.  With `out` (a contiguous torch tensor or numpy array of
    the vector's length and element size) the values are written there
    instead -- straight to the device for a CUDA tensor, by one copy from the
    device for a host buffer (pinned: at the link's full rate) -- and
    (out, None) is returned."""
    n = grb_vector_size(v)
    if out is not None:
        esize = out.element_size() if hasattr(out, "element_size") else out.itemsize
        contiguous = out.is_contiguous() if hasattr(out, "is_contiguous") else out.flags["C_CONTIGUOUS"]
        count = out.numel() if hasattr(out, "numel") else out.size
        if count != n:
            raise ValueError("out must hold one element per vector entry")
        if esize != np.dtype(NP_TYPES[type_]).itemsize or not contiguous:
            raise ValueError("out must be contiguous with the vector type's element size")
        dev = 1 if _is_device(out) else 0
        _check(load().grb_vector_extract_dense(v, _ptr(out), None, dev), "grb_vector_extract_dense", v)
        return out, None
    vals = np.empty(n, dtype=NP_TYPES[type_])
    pres = np.empty(n, dtype=np.uint8) if present else None
    _check(load().grb_vector_extract_dense(v, _ptr(vals), _ptr(pres), 0), "grb_vector_extract_dense", v)
    return vals, pres


# ----------------------------------------------------------------- scalar
def grb_scalar_new(ctx: int, type_: int = GRB_FP64) -> int:
    out = ctypes.c_void_p()
    _check(load().grb_scalar_new(ctypes.byref(out), ctx, int(type_)), "grb_scalar_new", ctx)
    return out.value


def grb_scalar_set(s: int, value: float) -> None:
    _check(load().grb_scalar_set(s, float(value)), "grb_scalar_set", s)


def grb_scalar_get(s: int):
    """The scalar's value, or None when it holds no value."""
    x = ctypes.c_double()
    rc = _check(load().grb_scalar_get(s, ctypes.byref(x)), "grb_scalar_get", s)
    return None if rc == GRB_NO_VALUE else x.value


def grb_scalar_apply_bind2nd(out: int, op: grb_binop, s: int, k: float) -> None:
    _check(load().grb_scalar_apply_bind2nd(out, op, s, float(k)), "grb_scalar_apply_bind2nd", out)


# ---------------------------------------------------------------- methods
def grb_apply(w, mask, accum, op, u, desc=0):
    _check(load().grb_apply(w, mask, _acc(accum), int(op), u, int(desc)), "grb_apply", w)


def grb_apply_bind2nd(w, mask, accum, op, u, s, desc=0):
    _check(load().grb_apply_bind2nd(w, mask, _acc(accum), op, u, float(s), int(desc)), "grb_apply_bind2nd", w)


def grb_apply_bind2nd_scalar(w, mask, accum, op, u, s, desc=0):
    _check(load().grb_apply_bind2nd_scalar(w, mask, _acc(accum), op, u, s, int(desc)), "grb_apply_bind2nd_scalar", w)


def grb_assign_scalar(w, mask, accum, s, desc=0):
    _check(load().grb_assign_scalar(w, mask, _acc(accum), s, int(desc)), "grb_assign_scalar", w)


def grb_mxv(w, mask, accum, semiring, A, u, desc=0):
    _check(load().grb_mxv(w, mask, _acc(accum), int(semiring), A, u, int(desc)), "grb_mxv", w)


def grb_ewise_add(w, mask, accum, op, u, v, desc=0):
    _check(load().grb_ewise_add(w, mask, _acc(accum), op, u, v, int(desc)), "grb_ewise_add", w)


def grb_ewise_mult(w, mask, accum, op, u, v, desc=0):
    _check(load().grb_ewise_mult(w, mask, _acc(accum), op, u, v, int(desc)), "grb_ewise_mult", w)


def grb_reduce(s, accum, monoid, u, desc=0):
    _check(load().grb_reduce(s, _acc(accum), int(monoid), u, int(desc)), "grb_reduce", s)


def grb_wait(obj, mode=GRB_WAIT_MATERIALIZE):
    _check(load().grb_wait(obj, int(mode)), "grb_wait", obj)


def grb_iterate_begin(ctx):
    _check(load().grb_iterate_begin(ctx), "grb_iterate_begin", ctx)


def grb_iterate_end(ctx, cond, tol, itermax) -> int:
    it = ctypes.c_int64()
    _check(load().grb_iterate_end(ctx, cond, float(tol), int(itermax), ctypes.byref(it)), "grb_iterate_end", ctx)
    return it.value


def grb_iterate_history(ctx, with_dang: bool = False):
    """(residual history of the last device loop, mixed-precision phase), or
    with with_dang (residuals, dangling masses, phase)."""
    n = ctypes.c_int64()
    ph = ctypes.c_int32()
    _check(load().grb_iterate_history(ctx, None, None, 0, ctypes.byref(n), ctypes.byref(ph)),
           "grb_iterate_history", ctx)
    h = np.empty(max(n.value, 1), dtype=np.float64)
    dg = np.empty(max(n.value, 1), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().grb_iterate_history(ctx, h.ctypes.data_as(dp), dg.ctypes.data_as(dp), n.value, ctypes.byref(n),
                                      ctypes.byref(ph)), "grb_iterate_history", ctx)
    if with_dang:
        return h[:n.value], dg[:n.value], ph.value
    return h[:n.value], ph.value


def grb_context_loop_times(ctx, cap: int = 64):
    """Device times (ms) of the last device loops, oldest first (waits for them)."""
    ms = np.zeros(max(int(cap), 1), np.float64)
    n = ctypes.c_int64()
    _check(load().grb_context_loop_times(ctx, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(cap),
                                         ctypes.byref(n)), "grb_context_loop_times", ctx)
    return ms[:n.value]


# ------------------------------------------- batched personalised PageRank
GRB_PPR_MAX_SLOTS = 128


def grb_ppr_new(AT: int, damping: float, slots: int) -> int:
    out = ctypes.c_void_p()
    _check(load().grb_ppr_new(ctypes.byref(out), AT, float(damping), int(slots)), "grb_ppr_new", AT)
    return out.value


def grb_ppr_slots(P: int) -> int:
    k = ctypes.c_int32()
    _check(load().grb_ppr_slots(P, ctypes.byref(k)), "grb_ppr_slots")
    return k.value


def grb_ppr_tune(P: int, trial_bodies: int = 2):
    """(ms per body for vector widths 1, 2, 4; chosen width).  Empties every slot."""
    ms = np.zeros(3, np.float64)
    vw = ctypes.c_int32()
    _check(load().grb_ppr_tune(P, int(trial_bodies), ms.ctypes.data, ctypes.byref(vw)), "grb_ppr_tune")
    return ms, vw.value


def grb_ppr_layout(P: int, vw: int) -> None:
    _check(load().grb_ppr_layout(P, int(vw)), "grb_ppr_layout")


def grb_ppr_set(P: int, slot: int, seeds, tol: float, itermax: int) -> None:
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    _check(load().grb_ppr_set(P, int(slot), seeds.ctypes.data, len(seeds), float(tol), int(itermax)), "grb_ppr_set")


def grb_ppr_clear(P: int, slot: int) -> None:
    _check(load().grb_ppr_clear(P, int(slot)), "grb_ppr_clear")


def grb_ppr_run(P: int, iters: int) -> None:
    _check(load().grb_ppr_run(P, int(iters)), "grb_ppr_run")


def grb_ppr_status(P: int):
    """(active[slots] int32, iters[slots] int64, resid[slots] float64)."""
    k = grb_ppr_slots(P)
    a = np.empty(k, np.int32)
    it = np.empty(k, np.int64)
    rs = np.empty(k, np.float64)
    _check(load().grb_ppr_status(P, a.ctypes.data, it.ctypes.data, rs.ctypes.data), "grb_ppr_status")
    return a, it, rs


def grb_ppr_get(P: int, slot: int, n: int, out=None):
    """Slot's ranks: into a new host float32 array, or into `out` (a device
    tensor of n float32)."""
    if out is not None:
        _check(load().grb_ppr_get(P, int(slot), _ptr(out), 1), "grb_ppr_get")
        return out
    r = np.empty(n, np.float32)
    _check(load().grb_ppr_get(P, int(slot), r.ctypes.data, 0), "grb_ppr_get")
    return r


def grb_ppr_serve(AT: int, arrival_s, seed_sets, damping: float = 0.85, tol: float = 1e-6, itermax: int = 1000,
                  chunk: int = 4, slots: int = 0, mem_fraction: float = 0.5, n: int | None = None,
                  want_ranks: bool = False, single_max: int = 0):
    """Run the serving loop on host arrival times and seed sets.  Returns a
    dict: latency_s, iters, resid (numpy, per query), ranks (nq x n float32
    when want_ranks), slots, steps, max_in_flight, wall_s, single_queries."""
    arrival = np.ascontiguousarray(arrival_s, dtype=np.float64)
    nq = len(arrival)
    ptr = np.zeros(nq + 1, np.int64)
    ptr[1:] = np.cumsum([len(s) for s in seed_sets])
    idx = np.ascontiguousarray(np.concatenate([np.asarray(s, np.int32) for s in seed_sets]) if nq else
                               np.zeros(1, np.int32), dtype=np.int32)
    lat = np.zeros(nq, np.float64)
    its = np.zeros(nq, np.int64)
    res = np.zeros(nq, np.float64)
    ranks = None
    if want_ranks:
        if n is None:
            n = grb_matrix_nrows(AT)
        ranks = np.zeros((nq, n), np.float32)
    cfg = grb_serve_config(float(damping), float(tol), int(itermax), int(chunk), int(slots), float(mem_fraction),
                           int(single_max))
    out = grb_serve_result(lat.ctypes.data, its.ctypes.data, res.ctypes.data,
                           ranks.ctypes.data if ranks is not None else None, 0, 0, 0, 0, 0.0, 0)
    _check(load().grb_ppr_serve(AT, ctypes.byref(cfg), nq, arrival.ctypes.data, ptr.ctypes.data, idx.ctypes.data,
                                ctypes.byref(out)), "grb_ppr_serve", AT)
    return {"latency_s": lat, "iters": its, "resid": res, "ranks": ranks, "slots": out.slots,
            "vector_width": out.vector_width, "steps": out.steps,
            "max_in_flight": out.max_in_flight, "wall_s": out.wall_s, "single_queries": out.single_queries}


# ------------------------------------------------ batch of independent graphs
def block_diagonal_edges(graphs):
    """Concatenate per-graph (n_g, src, dst) edge lists into one COO with
    vertex ids offset per graph; returns (n_total, src, dst, vptr)."""
    vptr = np.zeros(len(graphs) + 1, np.int64)
    vptr[1:] = np.cumsum([g[0] for g in graphs])
    src = np.concatenate([np.asarray(g[1], np.int64) + vptr[k] for k, g in enumerate(graphs)]).astype(np.int32)
    dst = np.concatenate([np.asarray(g[2], np.int64) + vptr[k] for k, g in enumerate(graphs)]).astype(np.int32)
    return int(vptr[-1]), src, dst, vptr


def grb_prbatch_new(AT: int, vptr, damping: float = 0.85) -> int:
    vptr = np.ascontiguousarray(vptr, dtype=np.int64)
    out = ctypes.c_void_p()
    _check(load().grb_prbatch_new(ctypes.byref(out), AT, len(vptr) - 1, vptr.ctypes.data, float(damping)),
           "grb_prbatch_new", AT)
    return out.value


def grb_prbatch_tune(B: int, trial_bodies: int = 3):
    """(ms per body for 1..k resident CTAs per SM, chosen CTAs per SM)."""
    ms = np.zeros(16, np.float64)
    ch = ctypes.c_int32()
    _check(load().grb_prbatch_tune(B, int(trial_bodies), ms.ctypes.data, 16, ctypes.byref(ch)), "grb_prbatch_tune")
    return ms[ms > 0], ch.value


def grb_prbatch_run(B: int, tol: float, itermax: int, chunk: int = 16) -> None:
    _check(load().grb_prbatch_run(B, float(tol), int(itermax), int(chunk)), "grb_prbatch_run")


def grb_prbatch_result(B: int, n: int, ngraphs: int):
    """(ranks float32[n], iters int64[ngraphs], resid float64[ngraphs])."""
    r = np.empty(n, np.float32)
    it = np.empty(ngraphs, np.int64)
    rs = np.empty(ngraphs, np.float64)
    _check(load().grb_prbatch_result(B, r.ctypes.data, it.ctypes.data, rs.ctypes.data), "grb_prbatch_result")
    return r, it, rs


def grb_free(obj) -> None:
    if not obj:
        return
    p = ctypes.c_void_p(obj)
    _check(load().grb_free(ctypes.byref(p)), "grb_free")
    _keep.pop(obj, None)


def grb_error(obj) -> str:
    return (load().grb_error(obj) or b"").decode()


GRB_NOALLOC_MAX_N = 16777216


def grb_reduce_dense_noalloc(x, type_: int, n: int, monoid: int, out, stream=None) -> int:
    """Allocation-free reduction of the dense device array `x` (torch CUDA
    tensor or raw device pointer) into the one-double device buffer `out`,
    asynchronously on `stream` (torch stream, raw handle, or None for
    torch's current stream).  Returns the grb_info code (no exception, so
    that callers can check the size limit themselves)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    xp = x if isinstance(x, int) else _ptr(x)
    op = out if isinstance(out, int) else _ptr(out)
    return load().grb_reduce_dense_noalloc(xp, int(type_), int(n), int(monoid), op, ctypes.c_void_p(handle))


def grb_selftest_wait_timeout(ctx, spin_limit: int) -> int:
    """Returns the grb_info code (GRB_DEVICE_TIMEOUT expected)."""
    return load().grb_selftest_wait_timeout(ctx, int(spin_limit))


def grb_debug_check_csr(ctx, row_ptr, col_idx, ncols: int):
    """Bounds-checked build only: the device structure check on host CSR
    arrays.  Returns (grb_info code, what, value) -- what 1: a column index
    outside [0, ncols) (value = the index), 2: a row_ptr entry out of order
    or outside [0, nnz] (value = its row)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    what, value = ctypes.c_int32(0), ctypes.c_int64(0)
    rc = load().grb_debug_check_csr(ctx, rp.ctypes.data, ci.ctypes.data if ci.size else None, rp.size - 1,
                                    int(ncols), ci.size, ctypes.byref(what), ctypes.byref(value))
    return rc, what.value, value.value


def grb_debug_set_col(A, k: int, col: int) -> None:
    """Bounds-checked build only: overwrite column index k of A (no check)."""
    _check(load().grb_debug_set_col(A, int(k), int(col)), "grb_debug_set_col", A)


__all__ = [n for n in list(globals()) if n.startswith("grb_") or n.startswith("GRB_")] + \
    ["GrbError", "binop", "load", "symbols", "NP_TYPES"]
