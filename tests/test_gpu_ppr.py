"""Batched personalised PageRank (grb_ppr_*) against the FP64 oracle.

Reading (the paper has no personalised variant): teleport v uniform over
the deduplicated seed set, r_0 = v, dangling mass spread uniformly over all
n vertices; slots are compared with the oracle run for the same number of
bodies as the slot reports.  FP32 ranks: L1 <= 1e-6 per slot."""
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
def graph12():
    n = 1 << 12
    src, dst = graphgen.rmat_edges(12, 16, seed=3)
    ptr, col = oracle.build_at(n, src, dst)
    return n, src, dst, ptr, col, oracle.out_degree(ptr, col)


def _oracle_ppr(g, seeds, iters):
    n, _, _, ptr, col, od = g
    S = np.unique(seeds)
    v = SparseVec(n, S, np.full(len(S), 1.0 / len(S)))
    return oracle.pagerank(ptr, col, od, damping=D, tol=-1.0, itermax=iters, mode="uniform", personal=v)


def _setup(grb, n, src, dst, slots):
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    P = grb.grb_ppr_new(AT, D, slots)
    return ctx, AT, P


def _teardown(grb, ctx, AT, P):
    grb.grb_free(P)
    grb.grb_free(AT)
    grb.grb_free(ctx)


def test_fixed_iterations_two_k_tiles_ragged(grb, graph12):
    """40 slots (a full k-tile of 32 and a partial one), 1-32 seeds each, 30
    bodies: every slot within L1 1e-6 of the oracle; empty slots stay
    inactive."""
    n, src, dst = graph12[:3]
    sets = graphgen.ppr_seed_sets(n, 40, 1, 32, seed=3)
    ctx, AT, P = _setup(grb, n, src, dst, 40)
    try:
        assert grb.grb_ppr_slots(P) == 64
        for s, S in enumerate(sets):
            grb.grb_ppr_set(P, s, S, -1.0, 30)
        grb.grb_ppr_run(P, 30)
        act, its, res = grb.grb_ppr_status(P)
        assert np.all(act[:40] == 0) and np.all(its[:40] == 30) and np.all(act[40:] == 0) and np.all(its[40:] == 0)
        for s, S in enumerate(sets):
            r = grb.grb_ppr_get(P, s, n).astype(np.float64)
            ref, k, hist = _oracle_ppr(graph12, S, 30)
            assert np.sum(np.abs(r - ref)) <= 1e-6, s
            assert abs(res[s] - hist[-1]) <= 1e-3 * hist[-1] + 1e-7
    finally:
        _teardown(grb, ctx, AT, P)


def test_tolerance_stop_per_slot(grb, graph12):
    """Each slot stops on its own loop test; ranks match the oracle at the
    slot's body count, and that count is the oracle's (+-1 near the threshold)."""
    n, src, dst = graph12[:3]
    sets = graphgen.ppr_seed_sets(n, 32, 1, 32, seed=5)
    tols = [10.0 ** -(3 + (s % 5)) for s in range(32)]
    ctx, AT, P = _setup(grb, n, src, dst, 32)
    try:
        for s, S in enumerate(sets):
            grb.grb_ppr_set(P, s, S, tols[s], 200)
        for _ in range(20):
            grb.grb_ppr_run(P, 10)
            act, its, res = grb.grb_ppr_status(P)
            if not act.any():
                break
        assert not act.any()
        for s, S in enumerate(sets):
            r = grb.grb_ppr_get(P, s, n).astype(np.float64)
            ref, _, _ = _oracle_ppr(graph12, S, int(its[s]))
            assert np.sum(np.abs(r - ref)) <= 1e-6, s
            assert res[s] <= tols[s]
            Sx = np.unique(S)
            v = SparseVec(n, Sx, np.full(len(Sx), 1.0 / len(Sx)))
            _, k_conv, _ = oracle.pagerank(*graph12[3:], damping=D, tol=tols[s], itermax=200, mode="uniform",
                                           personal=v)
            assert abs(k_conv - its[s]) <= 1, (s, k_conv, its[s])
    finally:
        _teardown(grb, ctx, AT, P)


def test_alone_equals_in_any_mix(grb, graph12):
    """A query alone, in a full batch, in another slot and k-tile, and
    admitted while other slots are mid-flight: bit-identical ranks."""
    n, src, dst = graph12[:3]
    sets = graphgen.ppr_seed_sets(n, 70, 1, 32, seed=7)
    q = sets[0]
    ctx, AT, P = _setup(grb, n, src, dst, 96)
    try:
        grb.grb_ppr_set(P, 0, q, -1.0, 25)
        grb.grb_ppr_run(P, 25)
        alone = grb.grb_ppr_get(P, 0, n)
        # in a full mix, at slot 0
        for s in range(70):
            grb.grb_ppr_set(P, s, sets[s], -1.0, 25)
        grb.grb_ppr_run(P, 25)
        assert np.array_equal(grb.grb_ppr_get(P, 0, n), alone)
        # at slot 77 (third k-tile, lane 13) while the others run on
        for s in range(1, 70):
            grb.grb_ppr_set(P, s, sets[s], -1.0, 40)
        grb.grb_ppr_run(P, 7)
        grb.grb_ppr_set(P, 77, q, -1.0, 25)
        grb.grb_ppr_run(P, 30)
        act, its, _ = grb.grb_ppr_status(P)
        assert its[77] == 25 and act[77] == 0
        assert np.array_equal(grb.grb_ppr_get(P, 77, n), alone)
        # slot reuse after clear
        grb.grb_ppr_clear(P, 77)
        grb.grb_ppr_set(P, 77, q, -1.0, 25)
        grb.grb_ppr_run(P, 25)
        assert np.array_equal(grb.grb_ppr_get(P, 77, n), alone)
    finally:
        _teardown(grb, ctx, AT, P)


def test_edge_seeds_and_errors(grb):
    """Seeds that are sinks or have no in-edges, duplicate seeds, an edgeless
    graph, and argument errors."""
    rng = np.random.default_rng(11)
    n = 5000
    src = rng.integers(0, n // 2, 20000).astype(np.int32)      # vertices >= n/2 are sinks
    dst = rng.integers(0, n, 20000).astype(np.int32)
    ptr, col = oracle.build_at(n, src, dst)
    g = (n, src, dst, ptr, col, oracle.out_degree(ptr, col))
    ctx, AT, P = _setup(grb, n, src, dst, 8)
    try:
        cases = [[n - 1], [0, 0, 0, 7], [n // 2 + 3, 1, 2], list(range(0, 64))]
        for s, S in enumerate(cases):
            grb.grb_ppr_set(P, s, np.array(S, np.int32), -1.0, 20)
        grb.grb_ppr_run(P, 20)
        for s, S in enumerate(cases):
            ref, _, _ = _oracle_ppr(g, np.array(S), 20)
            assert np.sum(np.abs(grb.grb_ppr_get(P, s, n).astype(np.float64) - ref)) <= 1e-6
        for bad in ([n], [-1]):
            with pytest.raises(grb.GrbError) as e:
                grb.grb_ppr_set(P, 0, np.array(bad, np.int32), -1.0, 5)
            assert e.value.code == grb.GRB_INVALID_INDEX
        with pytest.raises(grb.GrbError):
            grb.grb_ppr_set(P, 32, np.array([1], np.int32), -1.0, 5)
    finally:
        _teardown(grb, ctx, AT, P)
    with pytest.raises(grb.GrbError):
        ctx2 = grb.grb_context_new(grb.GRB_NONBLOCKING)
        try:
            A2 = grb.grb_matrix_build_csr(ctx2, grb.GRB_FP32, 10, 10, np.array([1], np.int32),
                                          np.array([2], np.int32), None, 7)
            try:
                grb.grb_ppr_new(A2, D, 129)
            finally:
                grb.grb_free(A2)
        finally:
            grb.grb_free(ctx2)
    # edgeless graph: every vertex a sink, r stays uniform-ish
    ctx, AT, P = _setup(grb, 100, np.zeros(0, np.int32), np.zeros(0, np.int32), 1)
    try:
        grb.grb_ppr_set(P, 0, np.array([3], np.int32), -1.0, 10)
        grb.grb_ppr_run(P, 10)
        e = np.zeros(0, np.int64)
        ref, _, _ = oracle.pagerank(np.zeros(101, np.int64), e, np.zeros(100, np.int64), damping=D, tol=-1.0,
                                    itermax=10, mode="uniform", personal=SparseVec(100, [3], [1.0]))
        assert np.sum(np.abs(grb.grb_ppr_get(P, 0, 100).astype(np.float64) - ref)) <= 1e-6
    finally:
        _teardown(grb, ctx, AT, P)


def test_rmat20_k64_full_size(grb):
    """The batched configuration: R-MAT scale 20, 64 slots with 1-32 seeds
    each, 20 bodies; four slots checked against the oracle, all slots for
    non-negativity and unit sum."""
    n = 1 << 20
    src, dst = graphgen.rmat_edges(20, 16, seed=3)
    sets = graphgen.ppr_seed_sets(n, 64, 1, 32, seed=3)
    ctx, AT, P = _setup(grb, n, src, dst, 64)
    try:
        for s, S in enumerate(sets):
            grb.grb_ppr_set(P, s, S, -1.0, 20)
        grb.grb_ppr_run(P, 20)
        ptr, col = oracle.build_at(n, src, dst)
        g = (n, src, dst, ptr, col, oracle.out_degree(ptr, col))
        for s in (0, 17, 40, 63):
            ref, _, _ = _oracle_ppr(g, sets[s], 20)
            assert np.sum(np.abs(grb.grb_ppr_get(P, s, n).astype(np.float64) - ref)) <= 1e-6
        for s in range(64):
            r = grb.grb_ppr_get(P, s, n).astype(np.float64)
            assert np.all(r >= 0) and abs(r.sum() - 1.0) < 1e-4
    finally:
        _teardown(grb, ctx, AT, P)


def test_vector_widths_give_identical_bits_and_tuner_picks_one(grb, graph12):
    """Each lane carrying 1, 2 or 4 slots is a layout choice only: the ranks
    are bit-identical; the autotuner times all three widths."""
    n, src, dst = graph12[:3]
    sets = graphgen.ppr_seed_sets(n, 40, 1, 32, seed=12)
    ctx, AT, P = _setup(grb, n, src, dst, 40)
    try:
        ms, vw = grb.grb_ppr_tune(P, 2)
        assert np.all(ms > 0) and vw in (1, 2, 4)
        results = {}
        for width in (1, 2, 4):
            grb.grb_ppr_layout(P, width)
            assert grb.grb_ppr_slots(P) == {1: 64, 2: 64, 4: 128}[width]
            for s, S in enumerate(sets):
                grb.grb_ppr_set(P, s, S, -1.0, 20)
            grb.grb_ppr_run(P, 20)
            results[width] = [grb.grb_ppr_get(P, s, n) for s in range(40)]
        for s in range(40):
            assert np.array_equal(results[1][s], results[2][s]) and np.array_equal(results[1][s], results[4][s]), s
        ref, _, _ = _oracle_ppr(graph12, sets[7], 20)
        assert np.sum(np.abs(results[4][7].astype(np.float64) - ref)) <= 1e-6
        with pytest.raises(grb.GrbError):
            grb.grb_ppr_layout(P, 3)
    finally:
        _teardown(grb, ctx, AT, P)
