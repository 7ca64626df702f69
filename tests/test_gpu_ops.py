"""GPU methods through the C-ABI against the FP64 CPU oracle, element by
element: CSR build and degrees (bit-exact), element-wise methods with every
operator, the mask / accumulate / replace write step, apply, reduce, mxv
(general and merge-path kernels), scalars, and the API error model."""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle
from oracle import SparseVec

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "graphblas_semantics.json")
OPS = ["first", "second", "plus", "minus", "times", "div", "max", "min", "abs_diff"]


@pytest.fixture(scope="module")
def grb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2509_14211_gb300 as g

    g.load()
    return g


@pytest.fixture(params=["nonblocking", "blocking"])
def ctx(grb, request):
    mode = grb.GRB_NONBLOCKING if request.param == "nonblocking" else grb.GRB_BLOCKING
    c = grb.grb_context_new(mode)
    yield c
    grb.grb_free(c)


def _code(grb, name):
    return {"first": grb.GRB_FIRST, "second": grb.GRB_SECOND, "plus": grb.GRB_PLUS, "minus": grb.GRB_MINUS,
            "times": grb.GRB_TIMES, "div": grb.GRB_DIV, "max": grb.GRB_MAX, "min": grb.GRB_MIN,
            "abs_diff": grb.GRB_ABS_DIFF}[name]


def _rand_sparse(rng, n, density):
    idx = np.sort(rng.choice(n, size=max(1, int(n * density)), replace=False)).astype(np.int64)
    val = rng.standard_normal(len(idx)) + 0.5
    return SparseVec(n, idx, val)


def _upload(grb, ctx, sv, type_=None):
    t = type_ or grb.GRB_FP64
    v = grb.grb_vector_new(ctx, t, sv.n)
    grb.grb_vector_build(v, sv.idx.astype(np.int32), sv.val)
    return v


def _download(grb, v, type_=None):
    vals, pres = grb.grb_vector_extract_dense(v, type_ or grb.GRB_FP64)
    idx = np.nonzero(pres)[0]
    return SparseVec(len(vals), idx, vals[idx].astype(np.float64))


def _same(a: SparseVec, b: SparseVec, rtol=0.0):
    assert np.array_equal(a.idx, b.idx), "presence differs"
    if rtol == 0.0:
        assert np.array_equal(a.val, b.val), np.max(np.abs(a.val - b.val))
    else:
        np.testing.assert_allclose(a.val, b.val, rtol=rtol, atol=0)


# ------------------------------------------------------------------ CSR
@pytest.mark.parametrize("case", ["rmat12", "ragged", "edgeless", "hub"])
def test_csr_build_bit_exact(grb, ctx, case):
    if case == "rmat12":
        n = 1 << 12
        src, dst = graphgen.rmat_edges(12, 16, seed=5)
    elif case == "ragged":
        rng = np.random.default_rng(1)
        n = 3001
        src = rng.integers(0, n, 20000).astype(np.int32)
        dst = (rng.integers(0, n // 3, 20000) * 3).astype(np.int32)   # 2 of 3 rows empty
        src[:50] = dst[:50]                                              # self loops
        src[50:100], dst[50:100] = src[100:150], dst[100:150]            # duplicates
    elif case == "edgeless":
        n = 77
        src = dst = np.zeros(0, np.int32)
    else:
        n = 200000
        rng = np.random.default_rng(2)
        src = rng.integers(0, n, 150000).astype(np.int32)
        dst = np.zeros(150000, np.int32)                                 # one row spans ~70 tiles
        dst[::3] = rng.integers(0, n, 50000)
    A = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst)
    rp, ci = grb.grb_matrix_export_csr(A)
    op, oc = oracle.build_at(n, src, dst)
    assert np.array_equal(rp, op) and np.array_equal(ci, oc)
    deg = grb.grb_vector_new(ctx, grb.GRB_INT32, n)
    grb.grb_matrix_col_degree(deg, A)
    vals, pres = grb.grb_vector_extract_dense(deg, grb.GRB_INT32)
    od = oracle.out_degree(op, oc)
    assert np.array_equal(vals, od) and np.array_equal(pres.astype(bool), od > 0)
    assert grb.grb_vector_nvals(deg) == int(np.count_nonzero(od))
    grb.grb_free(deg)
    grb.grb_free(A)


def test_csr_build_keeps_duplicates_when_asked(grb, ctx):
    src = np.array([0, 0, 1, 2, 2], dtype=np.int32)
    dst = np.array([1, 1, 1, 0, 2], dtype=np.int32)
    A = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, 3, 3, src, dst, None, grb.GRB_BUILD_TRANSPOSE)
    rp, ci = grb.grb_matrix_export_csr(A)
    assert rp.tolist() == [0, 1, 4, 5] and ci.tolist() == [2, 0, 0, 1, 2]
    grb.grb_free(A)


def test_csr_build_rejects_bad_indices(grb, ctx):
    with pytest.raises(grb.GrbError) as e:
        grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, 3, 3, np.array([0], np.int32), np.array([3], np.int32))
    assert e.value.code == grb.GRB_INDEX_OUT_OF_BOUNDS


# ------------------------------------------------------- element-wise
@pytest.mark.parametrize("op", OPS + ["max_div_by"])
def test_ewise_add_mult_every_operator(grb, ctx, op):
    rng = np.random.default_rng((OPS + ["max_div_by"]).index(op))
    n = 5003
    u, v = _rand_sparse(rng, n, 0.3), _rand_sparse(rng, n, 0.6)
    gu, gv = _upload(grb, ctx, u), _upload(grb, ctx, v)
    w = grb.grb_vector_new(ctx, grb.GRB_FP64, n)
    if op == "max_div_by":
        bop, oop = grb.binop(grb.GRB_MAX_DIV_BY, 0.85), ("max_div_by", 0.85)
    else:
        bop, oop = grb.binop(_code(grb, op)), op
    grb.grb_ewise_add(w, None, None, bop, gu, gv)
    _same(_download(grb, w), oracle.ewise_add(oop, u, v))
    grb.grb_ewise_mult(w, None, None, bop, gu, gv)
    _same(_download(grb, w), oracle.ewise_mult(oop, u, v))
    for h in (gu, gv, w):
        grb.grb_free(h)


def test_apply_and_bind2nd(grb, ctx):
    rng = np.random.default_rng(3)
    n = 4099
    u = _rand_sparse(rng, n, 0.5)
    gu = _upload(grb, ctx, u)
    w = grb.grb_vector_new(ctx, grb.GRB_FP64, n)
    for name, code in (("identity", grb.GRB_IDENTITY), ("abs", grb.GRB_ABS), ("ainv", grb.GRB_AINV),
                       ("minv", grb.GRB_MINV)):
        grb.grb_apply(w, None, None, code, gu)
        _same(_download(grb, w), oracle.apply(name, u))
    grb.grb_apply_bind2nd(w, None, None, grb.binop(grb.GRB_TIMES), gu, 2.5)
    _same(_download(grb, w), oracle.apply_bind2nd("times", u, 2.5))
    s = grb.grb_scalar_new(ctx, grb.GRB_FP64)
    grb.grb_scalar_set(s, -1.25)
    grb.grb_apply_bind2nd_scalar(w, None, None, grb.binop(grb.GRB_MINUS), gu, s)
    _same(_download(grb, w), oracle.apply_bind2nd("minus", u, -1.25))
    for h in (gu, w, s):
        grb.grb_free(h)


def test_write_step_matches_golden_semantics(grb, ctx):
    with open(GOLDEN) as f:
        g = json.load(f)["write"]
    n = g["n"]

    def sv(d):
        items = sorted((int(k), float(x)) for k, x in d.items())
        return SparseVec(n, [k for k, _ in items], [x for _, x in items])

    w_old, t, m = sv(g["w_old"]), sv(g["t"]), sv(g["mask"])
    cases = [("value_mask", {}, 0), ("structural_mask", {}, grb.GRB_DESC_STRUCTURE),
             ("value_mask_replace", {}, grb.GRB_DESC_REPLACE), ("accum_plus_no_mask", {"accum": True}, 0),
             ("complement_value_mask", {}, grb.GRB_DESC_COMPLEMENT)]
    for key, kw, desc in cases:
        w = _upload(grb, ctx, w_old)
        gt = _upload(grb, ctx, t)
        gm = None if key == "accum_plus_no_mask" else _upload(grb, ctx, m)
        acc = grb.binop(grb.GRB_PLUS) if kw.get("accum") else None
        grb.grb_apply(w, gm, acc, grb.GRB_IDENTITY, gt, desc)
        got = _download(grb, w)
        want = {int(k): float(x) for k, x in g[key].items()}
        assert dict(zip(got.idx.tolist(), got.val.tolist())) == want, key
        for h in (w, gt, gm):
            grb.grb_free(h)


def test_reduce_monoids_and_scalars(grb, ctx):
    rng = np.random.default_rng(4)
    n = 100003
    u = _rand_sparse(rng, n, 0.4)
    gu = _upload(grb, ctx, u)
    s = grb.grb_scalar_new(ctx, grb.GRB_FP64)
    for mon, name in ((grb.GRB_MONOID_PLUS, "plus"), (grb.GRB_MONOID_MAX, "max"), (grb.GRB_MONOID_MIN, "min")):
        grb.grb_reduce(s, None, mon, gu)
        assert grb.grb_scalar_get(s) == pytest.approx(oracle.reduce(name, u), rel=1e-12, abs=1e-12)
    empty = grb.grb_vector_new(ctx, grb.GRB_FP64, 10)
    grb.grb_reduce(s, None, grb.GRB_MONOID_PLUS, empty)
    assert grb.grb_scalar_get(s) == 0.0
    s2 = grb.grb_scalar_new(ctx, grb.GRB_FP32)
    grb.grb_scalar_apply_bind2nd(s2, grb.binop(grb.GRB_TIMES), s, 3.0)
    assert grb.grb_scalar_get(s2) == 0.0
    e = grb.grb_scalar_new(ctx, grb.GRB_FP64)
    assert grb.grb_scalar_get(e) is None
    for h in (gu, s, s2, empty, e):
        grb.grb_free(h)


# ------------------------------------------------------------------ mxv
def _matrix(grb, ctx, n, seed, valued):
    src, dst = graphgen.rmat_edges(int(np.log2(n)), 8, seed=seed)
    A = grb.grb_matrix_build_csr(ctx, grb.GRB_FP64, n, n, src, dst)
    rp, ci = oracle.build_at(n, src, dst)
    return A, rp, ci


@pytest.mark.parametrize("sr,add,mul", [("PLUS_TIMES", "plus", "times"), ("PLUS_SECOND", "plus", "second"),
                                        ("MAX_SECOND", "max", "second"), ("MIN_PLUS", "min", "plus")])
@pytest.mark.parametrize("dense", [True, False])
def test_mxv_semirings(grb, ctx, sr, add, mul, dense):
    n = 1 << 13
    A, rp, ci = _matrix(grb, ctx, n, 7, False)
    rng = np.random.default_rng(5)
    u = SparseVec.full(rng.random(n)) if dense else _rand_sparse(rng, n, 0.3)
    gu = _upload(grb, ctx, u)
    w = grb.grb_vector_new(ctx, grb.GRB_FP64, n)
    grb.grb_mxv(w, None, None, getattr(grb, "GRB_" + sr), A, gu)
    got = _download(grb, w)
    want = oracle.mxv(add, mul, rp, ci, u)
    assert np.array_equal(got.idx, want.idx)
    np.testing.assert_allclose(got.val, want.val, rtol=1e-12, atol=1e-15)
    for h in (gu, w, A):
        grb.grb_free(h)


def test_mxv_accum_and_mask(grb, ctx):
    n = 1 << 12
    A, rp, ci = _matrix(grb, ctx, n, 8, False)
    rng = np.random.default_rng(6)
    u = SparseVec.full(rng.random(n))
    base = SparseVec.full(rng.random(n))
    m = _rand_sparse(rng, n, 0.5)
    gu, gm = _upload(grb, ctx, u), _upload(grb, ctx, m)
    w = _upload(grb, ctx, base)
    grb.grb_mxv(w, None, grb.binop(grb.GRB_PLUS), grb.GRB_PLUS_SECOND, A, gu)
    want = oracle.write(base, oracle.mxv("plus", "second", rp, ci, u), accum="plus")
    got = _download(grb, w)
    assert np.array_equal(got.idx, want.idx)
    np.testing.assert_allclose(got.val, want.val, rtol=1e-12)
    w2 = _upload(grb, ctx, base)
    grb.grb_mxv(w2, gm, None, grb.GRB_PLUS_TIMES, A, gu, grb.GRB_DESC_STRUCTURE)
    want = oracle.write(base, oracle.mxv("plus", "times", rp, ci, u), mask=m, structural=True)
    got = _download(grb, w2)
    assert np.array_equal(got.idx, want.idx)
    np.testing.assert_allclose(got.val, want.val, rtol=1e-12)
    for h in (gu, gm, w, w2, A):
        grb.grb_free(h)


# ------------------------------------------------------------ API errors
def test_extract_dense_into_caller_buffers(grb, ctx):
    """Values land in a caller's buffer: a CUDA tensor, a pinned or pageable
    host tensor, a numpy array -- the same values as the returned array;
    absent entries read 0; a wrong length or element size is refused."""
    import torch

    n = 1000
    sv = _rand_sparse(np.random.default_rng(11), n, 0.4)
    sv = SparseVec(n, sv.idx, sv.val.astype(np.float32))
    v = _upload(grb, ctx, sv, grb.GRB_FP32)
    want, pres = grb.grb_vector_extract_dense(v, grb.GRB_FP32)
    assert np.array_equal(np.nonzero(pres)[0], sv.idx) and np.all(want[pres == 0] == 0)
    outs = [torch.empty(n, dtype=torch.float32, device="cuda"), torch.empty(n, dtype=torch.float32).pin_memory(),
            torch.empty(n, dtype=torch.float32), np.empty(n, dtype=np.float32)]
    for out in outs:
        got, none = grb.grb_vector_extract_dense(v, grb.GRB_FP32, out=out, present=False)
        assert got is out and none is None
        host = out.cpu().numpy() if hasattr(out, "cpu") else out
        assert np.array_equal(host, want)
    with pytest.raises(ValueError):
        grb.grb_vector_extract_dense(v, grb.GRB_FP32, out=torch.empty(n - 1, dtype=torch.float32))
    with pytest.raises(ValueError):
        grb.grb_vector_extract_dense(v, grb.GRB_FP32, out=torch.empty(n, dtype=torch.float64))
    grb.grb_free(v)


def test_api_errors_are_immediate(grb, ctx):
    v = grb.grb_vector_new(ctx, grb.GRB_FP64, 10)
    u = grb.grb_vector_new(ctx, grb.GRB_FP64, 11)
    with pytest.raises(grb.GrbError) as e:
        grb.grb_ewise_add(v, None, None, grb.binop(grb.GRB_PLUS), v, u)
    assert e.value.code == grb.GRB_DIMENSION_MISMATCH
    with pytest.raises(grb.GrbError) as e:
        grb.grb_ewise_add(v, None, None, grb.binop(99), v, v)
    assert e.value.code == grb.GRB_INVALID_VALUE
    with pytest.raises(grb.GrbError) as e:
        grb.grb_vector_build(v, np.array([3, 3], np.int32), np.array([1.0, 2.0]))
    assert e.value.code == grb.GRB_INVALID_INDEX
    with pytest.raises(grb.GrbError) as e:
        grb.grb_vector_new(ctx, 99, 5)
    assert e.value.code == grb.GRB_INVALID_VALUE
    i = grb.grb_vector_new(ctx, grb.GRB_INT32, 10)
    with pytest.raises(grb.GrbError) as e:
        grb.grb_vector_copy(v, i)
    assert e.value.code == grb.GRB_DOMAIN_MISMATCH
    for h in (v, u, i):
        grb.grb_free(h)
    # the column counts are cached on the matrix: a vector of another
    # context is refused
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    A = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, 8, 8, np.array([0, 1, 2], np.int32),
                                 np.array([1, 2, 3], np.int32), None, BUILD_FLAGS)
    ctx2 = grb.grb_context_new(grb.GRB_NONBLOCKING)
    d2 = grb.grb_vector_new(ctx2, grb.GRB_INT32, 8)
    with pytest.raises(grb.GrbError) as e:
        grb.grb_matrix_col_degree(d2, A)
    assert e.value.code == grb.GRB_INVALID_VALUE
    grb.grb_free(d2)
    grb.grb_free(ctx2)
    grb.grb_free(A)
    for opt, bad in ((grb.GRB_OPT_HOT_BYTES, -1), (grb.GRB_OPT_HOT_BYTES, grb.GRB_HOT_BYTES_MAX + 1),
                     (grb.GRB_OPT_PERSISTENT, 4), (grb.GRB_OPT_SPIN_LIMIT, 0), (99, 1)):
        with pytest.raises(grb.GrbError) as e:
            grb.grb_context_set(ctx, opt, bad)
        assert e.value.code == grb.GRB_INVALID_VALUE


def test_device_wait_timeout_is_reported_not_hung(grb, ctx):
    rc = grb.grb_selftest_wait_timeout(ctx, 2000)
    assert rc == grb.GRB_DEVICE_TIMEOUT
    # the context stays usable
    v = grb.grb_vector_new(ctx, grb.GRB_FP64, 8)
    grb.grb_vector_fill(v, 2.0)
    s = grb.grb_scalar_new(ctx)
    grb.grb_reduce(s, None, grb.GRB_MONOID_PLUS, v)
    assert grb.grb_scalar_get(s) == 16.0
    grb.grb_free(v)
    grb.grb_free(s)


@pytest.mark.parametrize("tol", [-1.0, 1e-30])
def test_barrier_timeout_in_a_loop_leaves_the_next_solve_correct(grb, tol):
    """A grid barrier of the persistent PageRank loop that runs out of its
    (here tiny) spin budget returns GRB_DEVICE_TIMEOUT instead of waiting on;
    the barrier words it left mid-crossing are cleared with the status word,
    so the next solve on the same matrix and context is right.  A loop with a
    fixed body count (tol < 0) is only enqueued by grb_iterate_end, so its
    error comes back from the first call that waits (here the rank read); a
    loop that stops on its tolerance waits, and returns the error itself."""
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS, PageRankProblem

    n = 1 << 14   # ~43 CTAs: their arrivals at a barrier spread over far more than one poll
    src, dst = graphgen.rmat_edges(14, 16, seed=5)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    try:
        AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
        P = PageRankProblem(ctx, AT, n, 0.85, grb.GRB_FP32, grb.GRB_FP64, "uniform")
        grb.grb_context_set(ctx, grb.GRB_OPT_SPIN_LIMIT, 1)
        with pytest.raises(grb.GrbError) as e:
            P.run(tol, 30, "device")
            P.rank()
        assert e.value.code == grb.GRB_DEVICE_TIMEOUT
        if tol < 0:   # the error sticks to what the failing wait read
            with pytest.raises(grb.GrbError) as e:
                P.rank()
            assert e.value.code == grb.GRB_DEVICE_TIMEOUT
        grb.grb_context_set(ctx, grb.GRB_OPT_SPIN_LIMIT, 1 << 24)
        P.free()
        P = PageRankProblem(ctx, AT, n, 0.85, grb.GRB_FP32, grb.GRB_FP64, "uniform")
        assert P.run(-1.0, 30, "device") == 30
        ref, _, _ = oracle.pagerank_edges(n, src, dst, damping=0.85, tol=-1.0, itermax=30, mode="uniform")
        assert np.sum(np.abs(P.rank().astype(np.float64) - ref)) <= 1e-6
        P.free()
        grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)


def test_allocator_failure_is_reported_and_recoverable(grb):
    """Allocator-failure injection: with the allocator refusing every
    request, a method that needs new device memory fails with
    GRB_OUT_OF_MEMORY at its wait (execution error, sticky on the output)
    and the device loop fails the same way; once the allocator answers
    again the context computes correct results."""
    from paper_2509_14211_gb300.pagerank import PageRankProblem, build_graph

    gate = {"open": True}
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING, alloc_hook=lambda nbytes: gate["open"])
    try:
        n = 1 << 12
        src, dst = graphgen.rmat_edges(12, 8, seed=21)
        AT = build_graph(ctx, n, src, dst)
        u = grb.grb_vector_new(ctx, grb.GRB_FP64, 3 << 20)
        grb.grb_vector_fill(u, 2.0)
        gate["open"] = False
        w = grb.grb_vector_new(ctx, grb.GRB_FP64, 3 << 20)
        grb.grb_ewise_mult(w, None, None, grb.binop(grb.GRB_TIMES), u, u)   # recorded, not run
        with pytest.raises(grb.GrbError) as e:
            grb.grb_wait(w)
        assert e.value.code == grb.GRB_OUT_OF_MEMORY
        with pytest.raises(grb.GrbError) as e:
            P = PageRankProblem(ctx, AT, n, 0.85, grb.GRB_FP32)
            P.run(-1.0, 5)
        assert e.value.code == grb.GRB_OUT_OF_MEMORY
        gate["open"] = True
        w2 = grb.grb_vector_new(ctx, grb.GRB_FP64, 3 << 20)
        grb.grb_ewise_mult(w2, None, None, grb.binop(grb.GRB_TIMES), u, u)
        vals, _ = grb.grb_vector_extract_dense(w2, grb.GRB_FP64)
        assert np.all(vals == 4.0)
        P2 = PageRankProblem(ctx, AT, n, 0.85, grb.GRB_FP32)
        assert P2.run(-1.0, 5) == 5
        ref, _, _ = oracle.pagerank_edges(n, src, dst, damping=0.85, tol=-1.0, itermax=5, mode="uniform")
        assert np.sum(np.abs(P2.rank().astype(np.float64) - ref)) <= 1e-6
        for h in (w, w2, u):
            grb.grb_free(h)
        P2.free()
        grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)
