"""Pins for the CPU oracle against facts fixed by the paper and the mathematics.

None of these compares the oracle with itself: each expected value is a
closed form, an invariant, a dense linear solve built independently from the
raw edge list, a brute-force adjacency construction, or a hand-computed
GraphBLAS result (tests/golden/graphblas_semantics.json).
"""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle
from oracle import SparseVec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "graphblas_semantics.json")
D = 0.85


def _sv(n, d):
    items = sorted((int(k), float(v)) for k, v in d.items())
    return SparseVec(n, [k for k, _ in items], [v for _, v in items])


def _as_dict(v: SparseVec):
    return {int(i): float(x) for i, x in zip(v.idx, v.val)}


def _expect(v: SparseVec, d):
    assert _as_dict(v) == pytest.approx({int(k): float(x) for k, x in d.items()}, rel=1e-15, abs=0)
    assert set(_as_dict(v)) == {int(k) for k in d}


# ------------------------------------------------ GraphBLAS method semantics

@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_ewise_semantics(golden):
    n = golden["n"]
    u, v = _sv(n, golden["u"]), _sv(n, golden["v"])
    _expect(oracle.ewise_add("plus", u, v), golden["ewise_add_plus"])
    _expect(oracle.ewise_add("abs_diff", u, v), golden["ewise_add_abs_diff"])
    _expect(oracle.ewise_add(("max_div_by", 0.5), u, v), golden["ewise_add_max_div_by_0.5"])
    _expect(oracle.ewise_mult("times", u, v), golden["ewise_mult_times"])
    _expect(oracle.ewise_mult("div", u, v), golden["ewise_mult_div"])
    _expect(oracle.ewise_mult("first", u, v), golden["ewise_mult_first"])


def test_apply_reduce_semantics(golden):
    n = golden["n"]
    u = _sv(n, golden["u"])
    _expect(oracle.apply("abs", u), golden["apply_abs_u"])
    _expect(oracle.apply_bind2nd("times", u, 2.0), golden["apply_bind2nd_times_2_u"])
    assert oracle.reduce("plus", u) == golden["reduce_plus_u"]
    assert oracle.reduce("max", u) == golden["reduce_max_u"]
    assert oracle.reduce("plus", SparseVec(n, [], [])) == golden["reduce_plus_empty"]


def test_mxv_semantics(golden):
    g = golden["mxv"]
    u = _sv(g["ncols"], g["u"])
    _expect(oracle.mxv("plus", "times", g["ptr"], g["col"], u, aval=g["val"]), g["plus_times"])
    _expect(oracle.mxv("plus", "second", g["ptr"], g["col"], u, aval=g["val"]), g["plus_second"])


def test_mask_accum_replace_semantics(golden):
    g = golden["write"]
    n = g["n"]
    w, t, m = _sv(n, g["w_old"]), _sv(n, g["t"]), _sv(n, g["mask"])
    _expect(oracle.write(w, t, mask=m), g["value_mask"])
    _expect(oracle.write(w, t, mask=m, structural=True), g["structural_mask"])
    _expect(oracle.write(w, t, mask=m, replace=True), g["value_mask_replace"])
    _expect(oracle.write(w, t, accum="plus"), g["accum_plus_no_mask"])
    _expect(oracle.write(w, t, mask=m, complement=True), g["complement_value_mask"])


# ----------------------------------------------------- graph construction

def _brute_at(n, src, dst):
    """Set-based A^T: rows = destinations, sorted distinct non-self sources."""
    rows = [set() for _ in range(n)]
    for s, t in zip(src.tolist(), dst.tolist()):
        if s != t:
            rows[t].add(s)
    ptr = np.zeros(n + 1, dtype=np.int64)
    col = []
    for i in range(n):
        ptr[i + 1] = ptr[i] + len(rows[i])
        col.extend(sorted(rows[i]))
    return ptr, np.array(col, dtype=np.int64)


@pytest.mark.parametrize("seed", [0, 1, 7])
def test_build_at_matches_brute_force(seed):
    src, dst = graphgen.rmat_edges(7, 8, seed=seed)
    n = 1 << 7
    ptr, col = oracle.build_at(n, src, dst)
    bp, bc = _brute_at(n, src, dst)
    assert np.array_equal(ptr, bp) and np.array_equal(col, bc)
    od = oracle.out_degree(ptr, col)
    distinct = {(s, t) for s, t in zip(src.tolist(), dst.tolist()) if s != t}
    expect = np.zeros(n, dtype=np.int64)
    for s, _ in distinct:
        expect[s] += 1
    assert np.array_equal(od, expect)


def test_build_at_keeps_duplicates_and_self_loops_when_asked():
    src = np.array([0, 0, 1, 2, 2], dtype=np.int32)
    dst = np.array([1, 1, 1, 0, 2], dtype=np.int32)
    ptr, col = oracle.build_at(3, src, dst, drop_self=False, dedup=False)
    assert ptr.tolist() == [0, 1, 4, 5] and col.tolist() == [2, 0, 0, 1, 2]
    with pytest.raises(ValueError):
        oracle.build_at(3, np.array([0], np.int32), np.array([3], np.int32))


# ------------------------------------------------------ PageRank closed forms

def _pr(n, src, dst, **kw):
    src = np.asarray(src, dtype=np.int32)
    dst = np.asarray(dst, dtype=np.int32)
    return oracle.pagerank_edges(n, src, dst, **kw)


@pytest.mark.parametrize("mode", ["gap", "uniform"])
def test_cycle_and_complete_graph_stay_uniform(mode):
    n = 7
    src = np.arange(n); dst = (src + 1) % n
    r, k, hist = _pr(n, src, dst, tol=-1.0, itermax=6, mode=mode)
    assert k == 6
    assert np.max(np.abs(r - 1.0 / n)) < 1e-16
    m = 6
    s2, d2 = np.nonzero(~np.eye(m, dtype=bool))
    r, _, _ = _pr(m, s2, d2, tol=-1.0, itermax=5, mode=mode)
    assert np.max(np.abs(r - 1.0 / m)) < 1e-16


def test_bidirectional_star_closed_form():
    n = 9
    leaves = np.arange(1, n)
    src = np.concatenate([np.zeros(n - 1, int), leaves])
    dst = np.concatenate([leaves, np.zeros(n - 1, int)])
    r, k, hist = _pr(n, src, dst, tol=1e-15, itermax=1000, mode="uniform")
    rc = (1 + D * (n - 1)) / (n * (1 + D))
    rl = (1 - D) / n + D * rc / (n - 1)
    bound = D / (1 - D) * hist[-1] + 1e-15
    assert abs(r[0] - rc) <= bound
    assert np.max(np.abs(r[1:] - rl)) <= bound
    assert abs(rc + (n - 1) * rl - 1.0) < 1e-15


@pytest.mark.parametrize("n", [2, 5, 33])
def test_in_star_closed_forms(n):
    src = np.arange(1, n); dst = np.zeros(n - 1, int)
    r, _, hist = _pr(n, src, dst, tol=1e-15, itermax=1000, mode="uniform")
    rc = (1 - D) * (1 + D * (n - 1)) / (n - D - D * D * (n - 1))
    rl = (1 - D) / n + D * rc / n
    bound = D / (1 - D) * hist[-1] + 1e-15
    assert abs(r[0] - rc) <= bound and np.max(np.abs(r[1:] - rl)) <= bound
    if n == 2:
        assert abs(rc - (1 + D) / (2 + D)) < 1e-15
    r, _, hist = _pr(n, src, dst, tol=1e-15, itermax=1000, mode="gap")
    bound = D / (1 - D) * hist[-1] + 1e-15
    assert np.max(np.abs(r[1:] - (1 - D) / n)) <= bound
    assert abs(r[0] - (1 - D) / n * (1 + D * (n - 1))) <= bound


def test_empty_graph_and_zero_damping():
    n = 5
    e = np.zeros(0, np.int32)
    r, k, _ = _pr(n, e, e, tol=-1.0, itermax=3, mode="gap")
    assert k == 3 and np.allclose(r, (1 - D) / n, rtol=0, atol=1e-16)
    r, _, _ = _pr(n, e, e, tol=-1.0, itermax=3, mode="uniform")
    assert np.allclose(r, 1.0 / n, rtol=0, atol=1e-16)
    src, dst = graphgen.rmat_edges(6, 8, seed=3)
    r, _, _ = _pr(64, src, dst, damping=0.0, tol=-1.0, itermax=1)
    assert np.allclose(r, 1.0 / 64, rtol=0, atol=1e-16)


def test_iteration_count_convention():
    src, dst = graphgen.rmat_edges(6, 8, seed=4)
    r0, k0, _ = _pr(64, src, dst, tol=-1.0, itermax=0)
    assert k0 == 0 and np.all(r0 == 1.0 / 64)
    _, k5, h5 = _pr(64, src, dst, tol=-1.0, itermax=5)
    assert k5 == 5 and len(h5) == 5
    # the test precedes the body: a loose tolerance stops after the first
    # body whose change falls to or below it
    _, k, h = _pr(64, src, dst, tol=1e-3, itermax=100)
    assert h[-1] <= 1e-3 and np.all(h[:-1] > 1e-3) and k == len(h)


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", [0, 5])
def test_invariants_uniform_and_gap(seed):
    scale = 9
    n = 1 << scale
    src, dst = graphgen.rmat_edges(scale, 16, seed=seed)
    ptr, col = oracle.build_at(n, src, dst)
    od = oracle.out_degree(ptr, col)
    assert np.any(od == 0)   # R-MAT leaves some vertices without out-edges
    r, k, hist = oracle.pagerank(ptr, col, od, tol=-1.0, itermax=30, mode="uniform")
    assert np.all(r >= 0) and abs(r.sum() - 1.0) < n * np.finfo(float).eps
    assert np.all(hist[1:] <= D * hist[:-1] * (1 + 1e-12) + 1e-16)   # contraction <= d
    prev = None
    for it in range(1, 6):
        rg, _, _ = oracle.pagerank(ptr, col, od, tol=-1.0, itermax=it, mode="gap")
        if prev is not None:
            dang = prev[od == 0].sum()
            assert abs(rg.sum() - ((1 - D) + D * (prev.sum() - dang))) < 1e-13
        prev = rg


def _dense_system(n, src, dst, mode):
    A = np.zeros((n, n))
    for s, t in zip(src, dst):
        if s != t:
            A[s, t] = 1.0
    outdeg = A.sum(axis=1)
    M = A.T / np.maximum(outdeg, 1.0)[None, :]
    S = np.eye(n) - D * M
    if mode == "uniform":
        S -= (D / n) * np.outer(np.ones(n), (outdeg == 0).astype(float))
    return S


@pytest.mark.parametrize("mode", ["gap", "uniform"])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_matches_dense_solve(mode, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(8, 65))
    m = int(rng.integers(n, 4 * n))
    src = rng.integers(0, n, m); dst = rng.integers(0, n, m)
    src[: n // 5] = 0   # make a few repeated edges and hubs
    r, _, hist = _pr(n, src, dst, tol=1e-14, itermax=2000, mode=mode)
    rstar = np.linalg.solve(_dense_system(n, src, dst, mode), np.full(n, (1 - D) / n))
    assert np.max(np.abs(r - rstar)) <= D / (1 - D) * hist[-1] + 1e-13


def test_personalised_linearity():
    scale = 8
    n = 1 << scale
    src, dst = graphgen.rmat_edges(scale, 16, seed=9)
    ptr, col = oracle.build_at(n, src, dst)
    od = oracle.out_degree(ptr, col)
    seeds = np.array([3, 17, 200, 201], dtype=np.int64)
    for it in (1, 4, 12):
        full = SparseVec(n, seeds, np.full(len(seeds), 1.0 / len(seeds)))
        r, _, _ = oracle.pagerank(ptr, col, od, tol=-1.0, itermax=it, mode="uniform", personal=full)
        parts = [oracle.pagerank(ptr, col, od, tol=-1.0, itermax=it, mode="uniform",
                                 personal=SparseVec(n, [s], [1.0]))[0] for s in seeds]
        assert np.max(np.abs(r - np.mean(parts, axis=0))) < 1e-15
        assert abs(r.sum() - 1.0) < 1e-13


def test_personalised_matches_dense_solve():
    rng = np.random.default_rng(11)
    n = 40
    src = rng.integers(0, n, 120); dst = rng.integers(0, n, 120)
    v = np.zeros(n); v[[2, 9]] = 0.5
    r, _, hist = _pr(n, src, dst, tol=1e-14, itermax=2000, mode="uniform",
                     personal=SparseVec(n, [2, 9], [0.5, 0.5]))
    rstar = np.linalg.solve(_dense_system(n, src, dst, "uniform"), (1 - D) * v)
    assert np.max(np.abs(r - rstar)) <= D / (1 - D) * hist[-1] + 1e-13


# ------------------------------------------------------------ plants

def test_a_planted_mistake_is_caught():
    """Swapping the roles of A and A^T (a plausible transposition slip) gives a
    result that the dense solve rejects."""
    rng = np.random.default_rng(5)
    n = 30
    src = rng.integers(0, n, 90); dst = rng.integers(0, n, 90)
    r_wrong, _, _ = _pr(n, dst, src, tol=1e-14, itermax=2000, mode="uniform")
    rstar = np.linalg.solve(_dense_system(n, src, dst, "uniform"), np.full(n, (1 - D) / n))
    assert np.max(np.abs(r_wrong - rstar)) > 1e-6
