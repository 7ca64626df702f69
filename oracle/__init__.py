"""CPU oracle (FP64, blocking mode) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (including ``bench.py --impl reference``) may import this package.  The
GPU library never calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64), compiled on first use.
This wrapper only marshals numpy arrays.  Sparse vectors are ``(n, idx,
val)`` with ascending int64 ``idx`` and float64 ``val``; operators are named
by strings ("plus", "times", "div", "max", "min", "first", "second",
"minus", "abs_diff", ("max_div_by", k)).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, dense solves, brute-force adjacency, hand-checked
GraphBLAS semantics in ``tests/golden/``).  ``pagerank_par`` (``oracle_par.c``,
the same listing with OpenMP loops over the rows, for timing the oracle on
all host cores) is checked against ``pagerank`` there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC_PAR = os.path.join(_HERE, "oracle_par.c")
_LIB_PAR = os.path.join(_HERE, "liboracle_par.so")
_lock = threading.Lock()
_lib = None
_lib_par = None

_BINOPS = {"first": 1, "second": 2, "plus": 3, "minus": 4, "times": 5, "div": 6, "max": 7,
           "min": 8, "abs_diff": 9, "max_div_by": 10}
_UNOPS = {"identity": 1, "abs": 2, "ainv": 3, "minv": 4}
_MODES = {"gap": 0, "uniform": 1}

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


class _OVec(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nvals", ctypes.c_int64), ("idx", _i64p), ("val", _f64p)]


class _OBinop(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("k", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, single-threaded) and
    oracle_par.c into liboracle_par.so (OpenMP when gcc has it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    if force or not os.path.exists(_LIB_PAR) or os.path.getmtime(_LIB_PAR) < os.path.getmtime(_SRC_PAR):
        tmp = _LIB_PAR + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC_PAR, "-lm"]
        if subprocess.call(base[:2] + ["-fopenmp"] + base[2:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PAR)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            V = ctypes.POINTER(_OVec)
            B = ctypes.POINTER(_OBinop)
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            lib.oracle_ewise_add.argtypes = [V, B, V, V]
            lib.oracle_ewise_mult.argtypes = [V, B, V, V]
            lib.oracle_apply.argtypes = [V, ctypes.c_int, V]
            lib.oracle_apply_bind2nd.argtypes = [V, B, V, ctypes.c_double]
            lib.oracle_full.argtypes = [V, ctypes.c_int64, ctypes.c_double]
            lib.oracle_mxv.argtypes = [V, ctypes.c_int, B, ctypes.c_int64, ctypes.c_int64, _i64p, _i64p,
                                       _f64p, ctypes.c_double, V]
            lib.oracle_reduce.argtypes = [ctypes.c_int, V]
            lib.oracle_reduce.restype = ctypes.c_double
            lib.oracle_write.argtypes = [V, V, V, B, V, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_build_at.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(_i64p), ctypes.POINTER(_i64p), _i64p]
            lib.oracle_out_degree.argtypes = [ctypes.c_int64, _i64p, _i64p, _i64p]
            lib.oracle_pagerank.argtypes = [ctypes.c_int64, _i64p, _i64p, _i64p, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int64, ctypes.c_int, V, _f64p,
                                            _i64p, _f64p]
            for f in ("oracle_ewise_add", "oracle_ewise_mult", "oracle_apply", "oracle_apply_bind2nd",
                      "oracle_full", "oracle_mxv", "oracle_write", "oracle_build_at", "oracle_out_degree",
                      "oracle_pagerank"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


# ------------------------------------------------------------ marshalling

class SparseVec:
    """A materialised oracle vector: n, ascending int64 idx, float64 val."""

    __slots__ = ("n", "idx", "val")

    def __init__(self, n, idx, val):
        self.n = int(n)
        self.idx = np.ascontiguousarray(idx, dtype=np.int64)
        self.val = np.ascontiguousarray(val, dtype=np.float64)

    @staticmethod
    def full(values):
        values = np.asarray(values, dtype=np.float64)
        return SparseVec(len(values), np.arange(len(values)), values)

    def dense(self, fill=0.0):
        out = np.full(self.n, fill, dtype=np.float64)
        out[self.idx] = self.val
        return out

    def _c(self):
        return _OVec(self.n, len(self.idx), self.idx.ctypes.data_as(_i64p), self.val.ctypes.data_as(_f64p))


def _take(ov: _OVec) -> SparseVec:
    lib = _load()
    nv = ov.nvals
    idx = np.ctypeslib.as_array(ov.idx, shape=(max(nv, 1),))[:nv].copy()
    val = np.ctypeslib.as_array(ov.val, shape=(max(nv, 1),))[:nv].copy()
    lib.oracle_free(ctypes.cast(ov.idx, ctypes.c_void_p))
    lib.oracle_free(ctypes.cast(ov.val, ctypes.c_void_p))
    return SparseVec(ov.n, idx, val)


def _binop(op) -> _OBinop:
    if isinstance(op, tuple):
        return _OBinop(_BINOPS[op[0]], float(op[1]))
    return _OBinop(_BINOPS[op], 0.0)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------- methods

def ewise_add(op, u: SparseVec, v: SparseVec) -> SparseVec:
    out = _OVec(); b = _binop(op); cu, cv = u._c(), v._c()
    _check(_load().oracle_ewise_add(ctypes.byref(out), ctypes.byref(b), ctypes.byref(cu), ctypes.byref(cv)), "ewise_add")
    return _take(out)


def ewise_mult(op, u: SparseVec, v: SparseVec) -> SparseVec:
    out = _OVec(); b = _binop(op); cu, cv = u._c(), v._c()
    _check(_load().oracle_ewise_mult(ctypes.byref(out), ctypes.byref(b), ctypes.byref(cu), ctypes.byref(cv)), "ewise_mult")
    return _take(out)


def apply(unop: str, u: SparseVec) -> SparseVec:
    out = _OVec(); cu = u._c()
    _check(_load().oracle_apply(ctypes.byref(out), _UNOPS[unop], ctypes.byref(cu)), "apply")
    return _take(out)


def apply_bind2nd(op, u: SparseVec, s: float) -> SparseVec:
    out = _OVec(); b = _binop(op); cu = u._c()
    _check(_load().oracle_apply_bind2nd(ctypes.byref(out), ctypes.byref(b), ctypes.byref(cu), float(s)), "apply_bind2nd")
    return _take(out)


def full(n: int, s: float) -> SparseVec:
    out = _OVec()
    _check(_load().oracle_full(ctypes.byref(out), int(n), float(s)), "full")
    return _take(out)


def mxv(add: str, mul, ptr, col, u: SparseVec, aval=None, a_iso: float = 1.0, ncols=None) -> SparseVec:
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int64)
    nrows = len(ptr) - 1
    ncols = u.n if ncols is None else int(ncols)
    av = None if aval is None else np.ascontiguousarray(aval, dtype=np.float64)
    out = _OVec(); b = _binop(mul); cu = u._c()
    _check(_load().oracle_mxv(ctypes.byref(out), _BINOPS[add], ctypes.byref(b), nrows, ncols,
                              ptr.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p),
                              None if av is None else av.ctypes.data_as(_f64p), float(a_iso),
                              ctypes.byref(cu)), "mxv")
    return _take(out)


def reduce(add: str, u: SparseVec) -> float:
    cu = u._c()
    return float(_load().oracle_reduce(_BINOPS[add], ctypes.byref(cu)))


def write(w_old: SparseVec, t: SparseVec, accum=None, mask: SparseVec | None = None,
          structural: bool = False, complement: bool = False, replace: bool = False) -> SparseVec:
    out = _OVec(); cw, ct = w_old._c(), t._c()
    acc = None if accum is None else ctypes.byref(_binop(accum))
    cm = None if mask is None else ctypes.byref(mask._c())
    _check(_load().oracle_write(ctypes.byref(out), ctypes.byref(cw), ctypes.byref(ct), acc, cm,
                                int(structural), int(complement), int(replace)), "write")
    return _take(out)


def build_at(n: int, src, dst, drop_self: bool = True, dedup: bool = True):
    """CSR of A^T from COO edges: returns (row_ptr int64[n+1], col_idx int64[nnz])."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    p, c, k = _i64p(), _i64p(), ctypes.c_int64()
    lib = _load()
    _check(lib.oracle_build_at(int(n), len(src), src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               dst.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(drop_self),
                               int(dedup), ctypes.byref(p), ctypes.byref(c), ctypes.byref(k)), "build_at")
    nnz = k.value
    ptr = np.ctypeslib.as_array(p, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(c, shape=(max(nnz, 1),))[:nnz].copy()
    lib.oracle_free(ctypes.cast(p, ctypes.c_void_p))
    lib.oracle_free(ctypes.cast(c, ctypes.c_void_p))
    return ptr, col


def out_degree(ptr, col) -> np.ndarray:
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int64)
    n = len(ptr) - 1
    out = np.empty(n, dtype=np.int64)
    _check(_load().oracle_out_degree(n, ptr.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p),
                                     out.ctypes.data_as(_i64p)), "out_degree")
    return out


def pagerank(ptr, col, outdeg, damping: float = 0.85, tol: float = 1e-10, itermax: int = 100,
             mode: str = "uniform", personal: SparseVec | None = None):
    """pagerank_gap (§IV) in FP64 blocking mode.  Returns (r, iterations,
    rdiff_history)."""
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int64)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int64)
    n = len(ptr) - 1
    r = np.empty(n, dtype=np.float64)
    hist = np.zeros(max(int(itermax), 1), dtype=np.float64)
    iters = ctypes.c_int64()
    cp = None if personal is None else ctypes.byref(personal._c())
    _check(_load().oracle_pagerank(n, ptr.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p),
                                   outdeg.ctypes.data_as(_i64p), float(damping), float(tol), int(itermax),
                                   _MODES[mode], cp, r.ctypes.data_as(_f64p), ctypes.byref(iters),
                                   hist.ctypes.data_as(_f64p)), "pagerank")
    k = iters.value
    return r, k, hist[:k].copy()


def pagerank_edges(n: int, src, dst, **kw):
    """Convenience: build A^T and out-degrees from COO, then pagerank."""
    ptr, col = build_at(n, src, dst)
    return pagerank(ptr, col, out_degree(ptr, col), **kw)


def _load_par():
    global _lib_par
    with _lock:
        if _lib_par is None:
            build()
            lib = ctypes.CDLL(_LIB_PAR)
            lib.oracle_par_threads.argtypes = []
            lib.oracle_par_threads.restype = ctypes.c_int
            lib.oracle_pagerank_par.argtypes = [ctypes.c_int64, _i64p, _i64p, _i64p, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int64, ctypes.c_int, _f64p, _i64p, _f64p]
            lib.oracle_pagerank_par.restype = ctypes.c_int
            _lib_par = lib
    return _lib_par


def par_threads() -> int:
    """Threads the multi-core variant runs on (OMP_NUM_THREADS, else all cores)."""
    return int(_load_par().oracle_par_threads())


def pagerank_par(ptr, col, outdeg, damping: float = 0.85, tol: float = 1e-10, itermax: int = 100,
                 mode: str = "uniform"):
    """The same pagerank_gap listing with OpenMP loops over the rows (for
    timing on all host cores).  Returns (r, iterations, rdiff_history)."""
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int64)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int64)
    n = len(ptr) - 1
    r = np.empty(n, dtype=np.float64)
    hist = np.zeros(max(int(itermax), 1), dtype=np.float64)
    iters = ctypes.c_int64()
    _check(_load_par().oracle_pagerank_par(n, ptr.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p),
                                           outdeg.ctypes.data_as(_i64p), float(damping), float(tol), int(itermax),
                                           _MODES[mode], r.ctypes.data_as(_f64p), ctypes.byref(iters),
                                           hist.ctypes.data_as(_f64p)), "pagerank_par")
    k = iters.value
    return r, k, hist[:k].copy()
