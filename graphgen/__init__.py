"""Seeded synthetic inputs shared by the oracle and the GPU library.

This module is the only code that both sides use.  It holds no PageRank or
GraphBLAS arithmetic: it only turns seeds into edge lists, seed-vertex sets
and request arrival times.  The C generator (graphgen.c) is compiled on first
use; ``numpy_*`` functions restate the same counter-based definitions in numpy
so that tests can pin the C code on small sizes.

Workload shapes (synthetic stand-ins for the paper's GAP-web run, §IV):

* R-MAT (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), edge factor 16, labels
  scrambled by a seeded bijection.
* Erdos-Renyi: average out-degree 16 with ~2% of vertices forced dangling.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)
GAMMA = np.uint64(0x9E3779B97F4A7C15)
S_RMAT, S_PERM, S_ER_DANG, S_ER_SRC, S_ER_DST = 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, i32p = ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
            lib.gg_key.restype = u64
            lib.gg_key.argtypes = [u64, u64]
            lib.gg_draw.restype = u64
            lib.gg_draw.argtypes = [u64, u64]
            lib.gg_scramble.restype = u64
            lib.gg_scramble.argtypes = [u64, ctypes.c_int, u64]
            lib.gg_rmat_edges.restype = ctypes.c_int
            lib.gg_rmat_edges.argtypes = [ctypes.c_int, i64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, u64, ctypes.c_int, i32p, i32p]
            lib.gg_er_edges.restype = ctypes.c_int
            lib.gg_er_edges.argtypes = [i64, i64, ctypes.c_double, u64, i32p, i32p]
            lib.gg_er_is_dangling.restype = ctypes.c_int
            lib.gg_er_is_dangling.argtypes = [u64, i64, ctypes.c_double]
            lib.gg_draws.restype = None
            lib.gg_draws.argtypes = [u64, u64, i64, ctypes.POINTER(ctypes.c_uint64)]
            _lib = lib
    return _lib


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def rmat_edges(scale: int, edge_factor: int = 16, seed: int = 0, abc=RMAT_ABC,
               permute: bool = True, nedges: int | None = None):
    """R-MAT COO edge list (src, dst) as int32 arrays of 2^scale * edge_factor
    pairs (duplicates and self loops included; the CSR build removes them)."""
    m = int(nedges if nedges is not None else (1 << scale) * edge_factor)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _load().gg_rmat_edges(int(scale), m, float(abc[0]), float(abc[1]), float(abc[2]),
                               int(seed), int(bool(permute)), _i32p(src), _i32p(dst))
    if rc != 0:
        raise ValueError("gg_rmat_edges: invalid arguments")
    return src, dst


def er_edges(n: int, avg_degree: int = 16, p_dangling: float = 0.02, seed: int = 2,
             nedges: int | None = None):
    """Erdos-Renyi style COO edge list with ~p_dangling of vertices forced to
    out-degree 0."""
    m = int(nedges if nedges is not None else n * avg_degree)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _load().gg_er_edges(int(n), m, float(p_dangling), int(seed), _i32p(src), _i32p(dst))
    if rc != 0:
        raise ValueError("gg_er_edges: invalid arguments")
    return src, dst


def draws(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.gg_draws(lib.gg_key(seed, stream), start, count,
                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


# --------------------------------------------------------------------------
# numpy restatement of the same definitions (for pinning the C code)
# --------------------------------------------------------------------------

def numpy_mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def numpy_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = numpy_mix64(np.uint64(seed) + GAMMA)
        return numpy_mix64(k + np.uint64(stream + 1) * GAMMA)


def numpy_draw(key, i) -> np.ndarray:
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return numpy_mix64(np.uint64(key) + (i + np.uint64(1)) * GAMMA)


def numpy_unit(u: np.ndarray) -> np.ndarray:
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def numpy_scramble(v: np.ndarray, scale: int, seed: int) -> np.ndarray:
    mask = np.uint64((1 << scale) - 1)
    key = numpy_key(seed, S_PERM)
    sh = np.uint64((scale + 1) // 2)
    v = np.asarray(v, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for r in range(4):
            mul = numpy_draw(key, 2 * r) | np.uint64(1)
            add = numpy_draw(key, 2 * r + 1)
            v = (v * mul + add) & mask
            v = v ^ (v >> sh)
    return v & mask


def numpy_rmat_edges(scale: int, nedges: int, seed: int, abc=RMAT_ABC, permute: bool = True):
    a, b, c = abc
    key = numpy_key(seed, S_RMAT)
    e = np.arange(nedges, dtype=np.uint64)
    s = np.zeros(nedges, dtype=np.uint64)
    d = np.zeros(nedges, dtype=np.uint64)
    for level in range(scale):
        u = numpy_unit(numpy_draw(key, e * np.uint64(scale) + np.uint64(level)))
        sb = (u >= a + b).astype(np.uint64)
        db = (((u >= a) & (u < a + b)) | (u >= a + b + c)).astype(np.uint64)
        s = (s << np.uint64(1)) | sb
        d = (d << np.uint64(1)) | db
    if permute:
        s = numpy_scramble(s, scale, seed)
        d = numpy_scramble(d, scale, seed)
    return s.astype(np.int32), d.astype(np.int32)


# --------------------------------------------------------------------------
# other seeded workload pieces (no arithmetic of the method)
# --------------------------------------------------------------------------

def ppr_seed_sets(n: int, k: int, min_seeds: int = 1, max_seeds: int = 32, seed: int = 3,
                  log_uniform: bool = False):
    """k personalised-PageRank seed sets over n vertices; set sizes uniform
    (or log-uniform) in [min_seeds, max_seeds]; duplicate seeds collapsed."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    sets = []
    for _ in range(k):
        if log_uniform:
            cnt = int(np.floor(np.exp(rng.uniform(np.log(min_seeds), np.log(max_seeds + 1)))))
            cnt = min(max(cnt, min_seeds), max_seeds)
        else:
            cnt = int(rng.integers(min_seeds, max_seeds + 1))
        sets.append(np.unique(rng.integers(0, n, size=cnt).astype(np.int32)))
    return sets


def batch_graph_specs(count: int = 512, scale_lo: int = 8, scale_hi: int = 16,
                      ef_lo: int = 8, ef_hi: int = 32, seed: int = 3):
    """(scale, edge_factor, seed) for a batch of independent R-MAT graphs."""
    rng = np.random.Generator(np.random.Philox(key=seed + 1000))
    scales = rng.integers(scale_lo, scale_hi + 1, size=count)
    efs = rng.integers(ef_lo, ef_hi + 1, size=count)
    return [(int(s), int(e), int(seed * 100003 + g)) for g, (s, e) in enumerate(zip(scales, efs))]


def poisson_arrivals(rate_qps: float, count: int, seed: int = 4) -> np.ndarray:
    """Arrival times (seconds) of a Poisson request stream."""
    rng = np.random.Generator(np.random.Philox(key=seed + 2000))
    return np.cumsum(rng.exponential(1.0 / rate_qps, size=count))
