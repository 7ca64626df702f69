"""Serving loop (grb_ppr_serve): continuous batching of personalised-PageRank
queries.  Every answer must equal the query's answer alone (bit for bit:
slot arithmetic is independent of the other slots and of admission time)
and match the FP64 oracle at its body count (L1 <= 1e-6)."""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import SparseVec

pytestmark = pytest.mark.gpu
D = 0.85


@pytest.fixture(scope="module")
def grb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2509_14211_gb300 as g

    g.load()
    return g


@pytest.fixture(scope="module")
def setup(grb):
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    n = 1 << 12
    src, dst = graphgen.rmat_edges(12, 16, seed=4)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    yield n, src, dst, AT
    grb.grb_free(AT)
    grb.grb_free(ctx)


def _alone(grb, AT, n, seeds, tol, itermax):
    P = grb.grb_ppr_new(AT, D, 1)
    try:
        grb.grb_ppr_set(P, 0, seeds, tol, itermax)
        while True:
            grb.grb_ppr_run(P, 16)
            act, its, res = grb.grb_ppr_status(P)
            if not act[0]:
                break
        return grb.grb_ppr_get(P, 0, n), int(its[0])
    finally:
        grb.grb_free(P)


def test_burst_with_queueing_matches_alone(grb, setup):
    """80 queries -- 40 at once, then a Poisson stream at ~2000/s -- into 32
    slots: queries queue, are admitted while others are mid-flight, and
    still get their alone answer."""
    n, src, dst, AT = setup
    sets = graphgen.ppr_seed_sets(n, 80, 1, 64, seed=4, log_uniform=True)
    arr = np.concatenate([np.zeros(40), 0.001 + graphgen.poisson_arrivals(2000.0, 40, seed=4)])
    tol, itermax = 1e-7, 300
    out = grb.grb_ppr_serve(AT, arr, sets, damping=D, tol=tol, itermax=itermax, chunk=3, slots=32,
                            want_ranks=True)
    assert out["slots"] == 32 and out["max_in_flight"] == 32
    assert np.all(out["latency_s"] > 0) and np.all(out["resid"] <= tol) and np.all(out["iters"] < itermax)
    for q in range(80):
        r, it = _alone(grb, AT, n, sets[q], tol, itermax)
        assert it == out["iters"][q]
        assert np.array_equal(out["ranks"][q], r), q
    ptr, col = oracle.build_at(n, src, dst)
    od = oracle.out_degree(ptr, col)
    for q in (0, 41, 79):
        S = np.unique(sets[q])
        ref, _, _ = oracle.pagerank(ptr, col, od, damping=D, tol=-1.0, itermax=int(out["iters"][q]), mode="uniform",
                                    personal=SparseVec(n, S, np.full(len(S), 1.0 / len(S))))
        assert np.sum(np.abs(out["ranks"][q].astype(np.float64) - ref)) <= 1e-6


def test_sparse_arrivals_and_memory_admission(grb, setup):
    """Queries spread out in time are answered one or two at a time; with no
    slot limit the slot count comes from free memory (capped at 128)."""
    n, _, _, AT = setup
    sets = graphgen.ppr_seed_sets(n, 6, 1, 8, seed=9)
    arr = np.arange(6) * 0.05
    out = grb.grb_ppr_serve(AT, arr, sets, damping=D, tol=1e-6, itermax=200, chunk=4, slots=0)
    assert out["slots"] == grb.GRB_PPR_MAX_SLOTS
    assert out["max_in_flight"] <= 3
    assert out["wall_s"] >= arr[-1]
    assert np.all(out["iters"] > 0)


def test_single_vector_loop_matches_slots_and_oracle(grb, setup):
    """The single-vector loop (single_max): 12 queries arriving together with
    single_max = 100 all run alone on the fused persistent loop; the same
    queries through the slots (single_max = 0) take the same number of
    bodies (or one more or fewer: the residual is summed in another order)
    and agree within L1 1e-6, and both match the FP64 oracle at their body
    counts."""
    n, src, dst, AT = setup
    sets = graphgen.ppr_seed_sets(n, 12, 1, 64, seed=14, log_uniform=True)
    arr = np.zeros(12)
    tol, itermax = 1e-7, 300
    one = grb.grb_ppr_serve(AT, arr, sets, damping=D, tol=tol, itermax=itermax, chunk=4, slots=32,
                            want_ranks=True, single_max=100)
    slot = grb.grb_ppr_serve(AT, arr, sets, damping=D, tol=tol, itermax=itermax, chunk=4, slots=32,
                             want_ranks=True, single_max=0)
    assert one["single_queries"] == 12 and slot["single_queries"] == 0
    assert np.all(one["resid"] <= tol) and np.all(one["iters"] < itermax)
    assert np.all(np.abs(one["iters"] - slot["iters"]) <= 1)
    ptr, col = oracle.build_at(n, src, dst)
    od = oracle.out_degree(ptr, col)
    for q in range(12):
        S = np.unique(sets[q])
        pv = SparseVec(n, S, np.full(len(S), 1.0 / len(S)))
        ref, k, _ = oracle.pagerank(ptr, col, od, damping=D, tol=-1.0, itermax=int(one["iters"][q]),
                                    mode="uniform", personal=pv)
        assert np.sum(np.abs(one["ranks"][q].astype(np.float64) - ref)) <= 1e-6, q
        assert one["ranks"][q].min() >= 0.0
        if one["iters"][q] == slot["iters"][q]:
            assert np.sum(np.abs(one["ranks"][q].astype(np.float64) - slot["ranks"][q])) <= 1e-6, q


def test_single_vector_loop_on_the_input_vertex_order(grb):
    """The single-vector loop on a context without the degree-ordered copy
    (GRB_OPT_RELABEL 0: the personalised kernel without the hot copy) gives
    the oracle's ranks at its body count."""
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    n = 1 << 12
    src, dst = graphgen.rmat_edges(12, 16, seed=6)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 0)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    try:
        sets = graphgen.ppr_seed_sets(n, 3, 1, 16, seed=16)
        out = grb.grb_ppr_serve(AT, np.zeros(3), sets, damping=D, tol=1e-7, itermax=300, chunk=4, slots=32,
                                want_ranks=True, single_max=8)
        assert out["single_queries"] == 3
        ptr, col = oracle.build_at(n, src, dst)
        od = oracle.out_degree(ptr, col)
        for q in range(3):
            S = np.unique(sets[q])
            ref, _, _ = oracle.pagerank(ptr, col, od, damping=D, tol=-1.0, itermax=int(out["iters"][q]),
                                        mode="uniform", personal=SparseVec(n, S, np.full(len(S), 1.0 / len(S))))
            assert np.sum(np.abs(out["ranks"][q].astype(np.float64) - ref)) <= 1e-6, q
    finally:
        grb.grb_free(AT)
        grb.grb_free(ctx)


def test_low_load_runs_single_then_batches_a_burst(grb, setup):
    """single_max = 2: queries spread out in time are answered alone on the
    single-vector loop; a burst of 40 arrivals goes to the slots."""
    n, _, _, AT = setup
    sets = graphgen.ppr_seed_sets(n, 46, 1, 16, seed=15)
    arr = np.concatenate([np.arange(6) * 0.03, 0.2 + np.zeros(40)])
    out = grb.grb_ppr_serve(AT, arr, sets, damping=D, tol=1e-6, itermax=200, chunk=4, slots=64, single_max=2)
    assert out["single_queries"] >= 6 and out["single_queries"] < 46
    assert np.all(out["resid"] <= 1e-6) and np.all(out["iters"] > 0)
    assert out["max_in_flight"] > 2


def test_serve_argument_errors(grb, setup):
    n, _, _, AT = setup
    with pytest.raises(grb.GrbError) as e:
        grb.grb_ppr_serve(AT, [0.2, 0.1], [[1], [2]])
    assert e.value.code == grb.GRB_INVALID_VALUE
    with pytest.raises(grb.GrbError) as e:
        grb.grb_ppr_serve(AT, [0.0], [[]])
    assert e.value.code == grb.GRB_INVALID_VALUE
    with pytest.raises(grb.GrbError) as e:
        grb.grb_ppr_serve(AT, [0.0], [[n]])
    assert e.value.code == grb.GRB_INVALID_INDEX
    with pytest.raises(grb.GrbError) as e:
        grb.grb_ppr_serve(AT, [0.0], [[n]], single_max=4)     # checked on the single-vector path too
    assert e.value.code == grb.GRB_INVALID_INDEX
    with pytest.raises(grb.GrbError) as e:
        grb.grb_ppr_serve(AT, [0.0], [[1]], single_max=-1)
    assert e.value.code == grb.GRB_INVALID_VALUE


@pytest.mark.slow
def test_rmat24_full_size_properties(grb):
    """The serving workload at full size: R-MAT scale 24 (16.8 M vertices,
    268 M raw edges).  Two served queries are checked against the FP64 oracle
    at their body counts (L1 <= 1e-6; a few minutes of host CPU), and
    properties that hold at any size:
    - personalised PageRank is linear in its teleport vector (uniform
      dangling, r_0 = v): 15 bodies from seeds {a, b} equal the mean of those
      from {a} and from {b}, L1 <= 1e-5 (FP32 rounding over 16.8 M entries);
    - every result is non-negative with unit sum (|sum - 1| <= 1e-4);
    - served queries stop at an L1 change <= tol before itermax, and each
      equals the same query run alone, bit for bit."""
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    n = 1 << 24
    src, dst = graphgen.rmat_edges(24, 16, seed=4)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    ptr, col = oracle.build_at(n, src, dst)
    od = oracle.out_degree(ptr, col)
    del src, dst
    try:
        rng = np.random.default_rng(24)
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        P = grb.grb_ppr_new(AT, D, 3)
        try:
            for s, S in enumerate(([a], [b], [a, b])):
                grb.grb_ppr_set(P, s, np.array(S, np.int32), -1.0, 15)
            grb.grb_ppr_run(P, 15)
            r = [grb.grb_ppr_get(P, s, n).astype(np.float64) for s in range(3)]
        finally:
            grb.grb_free(P)
        for x in r:
            assert x.min() >= 0.0 and abs(x.sum() - 1.0) <= 1e-4
        assert np.sum(np.abs(r[2] - 0.5 * (r[0] + r[1]))) <= 1e-5
        del r
        sets = graphgen.ppr_seed_sets(n, 4, 1, 64, seed=4, log_uniform=True)
        out = grb.grb_ppr_serve(AT, np.zeros(4), sets, damping=D, tol=1e-6, itermax=200, chunk=4, n=n,
                                want_ranks=True)
        assert np.all(out["iters"] < 200) and np.all(out["resid"] <= 1e-6)
        for q in (0, 3):
            alone, its = _alone(grb, AT, n, sets[q], 1e-6, 200)
            assert its == out["iters"][q]
            assert np.array_equal(alone, out["ranks"][q])
            assert alone.min() >= 0.0 and abs(alone.astype(np.float64).sum() - 1.0) <= 1e-4
            S = np.unique(sets[q])
            ref, k, _ = oracle.pagerank(ptr, col, od, damping=D, tol=-1.0, itermax=its, mode="uniform",
                                        personal=SparseVec(n, S, np.full(len(S), 1.0 / len(S))))
            assert k == its
            assert np.sum(np.abs(out["ranks"][q].astype(np.float64) - ref)) <= 1e-6, q
            # the same query alone on the single-vector loop
            one = grb.grb_ppr_serve(AT, np.zeros(1), [sets[q]], damping=D, tol=1e-6, itermax=200, chunk=4, n=n,
                                    want_ranks=True, single_max=1)
            assert one["single_queries"] == 1 and abs(int(one["iters"][0]) - its) <= 1
            if int(one["iters"][0]) == its:
                assert np.sum(np.abs(one["ranks"][0].astype(np.float64) - ref)) <= 1e-6, q
    finally:
        grb.grb_free(AT)
        grb.grb_free(ctx)
