"""PageRank on the GPU through the C-ABI against the FP64 CPU oracle.

Readings (the paper is silent on them): the FP64 and fixed-iteration cases
compare with the oracle run for the same number of iterations as the GPU
reports; FP64 must agree to max-abs 1e-12 per entry and FP32 to L1 1e-6.
Execution paths compared: persistent device loop, CUDA-graph device loop,
host loop with per-wait fusion, blocking mode (one kernel per method)."""
import numpy as np
import pytest

import graphgen
import oracle

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


def _run(grb, n, src, dst, rank_type, dangling, loop, tol, itermax, mode=None, persistent=0, fusion=True,
         mixed=False, relabel=True, hot_bytes=None, tma=0, bins=False):
    from paper_2509_14211_gb300.pagerank import pagerank

    ctx = grb.grb_context_new(mode if mode is not None else grb.GRB_NONBLOCKING)
    grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, persistent)
    grb.grb_context_set(ctx, grb.GRB_OPT_FUSION, 1 if fusion else 0)
    grb.grb_context_set(ctx, grb.GRB_OPT_MIXED, int(mixed))
    grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 1 if relabel else 0)
    if hot_bytes is not None:
        grb.grb_context_set(ctx, grb.GRB_OPT_HOT_BYTES, hot_bytes)
    grb.grb_context_set(ctx, grb.GRB_OPT_TMA_STAGES, tma)
    grb.grb_context_set(ctx, grb.GRB_OPT_ROW_BINS, 1 if bins else 0)
    try:
        r, it = pagerank(ctx, n, src, dst, damping=D, tol=tol, itermax=itermax, rank_type=rank_type,
                         dangling=dangling, loop=loop)
        stats = grb.grb_context_stats(ctx)
        hist = grb.grb_iterate_history(ctx)
    finally:
        grb.grb_free(ctx)
    return r, it, stats, hist


@pytest.fixture(scope="module")
def c0():
    """R-MAT scale 10, edge factor 16, seed 0 (the small FP64 configuration)."""
    n = 1 << 10
    src, dst = graphgen.rmat_edges(10, 16, seed=0)
    return n, src, dst


# (loop, persistent option, fusion, mode, degree-ordered copy for device loops)
PATHS = [("device", 1, True, "nb", True), ("device", 2, True, "nb", True), ("device", 1, True, "nb", False),
         ("device", 2, True, "nb", False), ("host", 0, True, "nb", True), ("host", 0, False, "nb", True),
         ("host", 0, True, "blocking", True)]


@pytest.mark.parametrize("loop,persistent,fusion,mode,relabel", PATHS)
@pytest.mark.parametrize("dangling", ["uniform", "gap"])
def test_fp64_rmat10_all_paths(grb, c0, loop, persistent, fusion, mode, relabel, dangling):
    n, src, dst = c0
    m = grb.GRB_BLOCKING if mode == "blocking" else grb.GRB_NONBLOCKING
    r, it, stats, _ = _run(grb, n, src, dst, grb.GRB_FP64, dangling, loop, 1e-10, 100, m, persistent, fusion,
                           relabel=relabel)
    ref_conv, k_conv, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=1e-10, itermax=100, mode=dangling)
    assert abs(it - k_conv) <= 1
    ref, k, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=-1.0, itermax=it, mode=dangling)
    assert np.max(np.abs(r - ref)) <= 1e-12
    if loop == "device":
        assert stats["persistent_loops"] == 1
    if mode == "blocking" or not fusion:
        assert stats["fused_groups"] == 0
    elif loop == "host":
        assert stats["fused_groups"] >= it and stats["elided_vectors"] > 0


@pytest.mark.parametrize("dangling", ["uniform", "gap"])
def test_fp32_fixed_iterations_scale16(grb, dangling):
    n = 1 << 16
    src, dst = graphgen.rmat_edges(16, 16, seed=1)
    ref, _, ref_hist = oracle.pagerank_edges(n, src, dst, damping=D, tol=-1.0, itermax=50, mode=dangling)
    # persistent kernel with the default, no, a partial-warp-sized and the
    # largest shared-memory hot copy (n = 65536: the largest covers 3/4 of
    # the vertices); the CUDA-graph loop; both on the input vertex order
    # and the tile arrays staged by bulk copies 2 and 3 tiles ahead
    # and the row-length-binned body with and without the hot copy
    for persistent, relabel, hot, tma, bins in ((1, True, None, 0, 0), (1, True, 0, 0, 0), (1, True, 1040, 0, 0),
                                                (1, True, grb.GRB_HOT_BYTES_MAX, 0, 0), (2, True, None, 0, 0),
                                                (1, False, None, 0, 0), (2, False, None, 0, 0), (1, True, None, 2, 0),
                                                (1, True, None, 3, 0), (1, True, 1040, 3, 0), (1, True, None, 0, 1),
                                                (1, True, 0, 0, 1), (1, False, None, 0, 1), (1, True, 1040, 0, 1)):
        r, it, _, (hist, _) = _run(grb, n, src, dst, grb.GRB_FP32, dangling, "device", -1.0, 50,
                                   persistent=persistent, relabel=relabel, hot_bytes=hot, tma=tma, bins=bins)
        assert it == 50
        assert np.sum(np.abs(r - ref)) <= 1e-6
        # FP32 ranks put a noise floor of ~n * eps32 * mean(r) ~ 1e-8 under
        # the L1 change between iterates
        np.testing.assert_allclose(hist, ref_hist, rtol=1e-3, atol=1e-7)
    r, it, _, _ = _run(grb, n, src, dst, grb.GRB_FP32, dangling, "host", -1.0, 50)
    assert it == 50 and np.sum(np.abs(r - ref)) <= 1e-6


def test_fp32_full_size_rmat22(grb):
    """R-MAT scale 22 (4.19M vertices, 67M raw edges), FP32 ranks, FP64
    residual, 50 fixed iterations: the benchmark configuration."""
    n = 1 << 22
    src, dst = graphgen.rmat_edges(22, 16, seed=1)
    ref, k, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=-1.0, itermax=50, mode="uniform")
    for tma, bins in ((0, False), (2, False), (0, True)):
        r, it, _, _ = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "device", -1.0, 50, persistent=1, tma=tma,
                           bins=bins)
        assert it == 50 == k
        assert np.sum(np.abs(r - ref)) <= 1e-6
    assert abs(np.sum(r) - 1.0) < 1e-4 and np.all(r >= 0)


# Mixed precision stops at an L1 change of 1e-6 (1-d)/d: by the L1
# contraction of the PageRank map, ||r - r*||_1 <= d/(1-d) * change <= 1e-6.
MIXED_TOL = 1e-6 * (1 - D) / D


def test_mixed_precision_er20_matches_converged_oracle(grb):
    """Erdos-Renyi, 2^20 vertices, out-degree 16, 2% sinks: BF16 gathers until
    the residual falls below 1e-3 (or stalls), then FP32; the result must be
    within L1 1e-6 of the FP64 oracle converged to 1e-13."""
    n = 1 << 20
    src, dst = graphgen.er_edges(n, 16, p_dangling=0.02, seed=2)
    r, it, _, (hist, phase) = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "device", MIXED_TOL, 500,
                                   persistent=1, mixed=2)
    assert phase == 1 and it < 500 and hist[-1] <= MIXED_TOL
    ref, _, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=1e-13, itermax=1000, mode="uniform")
    assert np.sum(np.abs(r - ref)) <= 1e-6


@pytest.mark.slow
def test_mixed_precision_er24_full_size_matches_converged_oracle(grb):
    """The full mixed-precision configuration (Erdos-Renyi, 2^24 vertices,
    ~268M edges, 2% sinks), BF16 gathers forced on: the switch happened, the
    stop rule was met, ranks are non-negative and sum to 1, the residual falls
    after the switch, and the result is within L1 1e-6 of the FP64 oracle
    converged to an L1 change of 1e-13 (a few minutes of host CPU)."""
    n = 1 << 24
    src, dst = graphgen.er_edges(n, 16, p_dangling=0.02, seed=2)
    r, it, _, (hist, phase) = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "device", MIXED_TOL, 500,
                                   persistent=1, mixed=2)
    assert phase == 1 and it < 500 and hist[-1] <= MIXED_TOL
    assert np.all(r >= 0) and abs(np.sum(r.astype(np.float64)) - 1.0) < 1e-4
    assert np.all(np.diff(hist[-10:]) < 0)
    ref, k, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=1e-13, itermax=1000, mode="uniform")
    assert k < 1000
    assert np.sum(np.abs(r - ref)) <= 1e-6


@pytest.mark.parametrize("log2n,expect_bf16", [(20, False), (24, False)])
def test_mixed_precision_planner_declines_while_w_fits_l2(grb, log2n, expect_bf16):
    """GRB_OPT_MIXED = 1 leaves the choice to the planner: BF16 gathers only
    once the FP32 gather vector (4n bytes) exceeds L2.  At 2^20 (4 MB) and
    2^24 (64 MB) it stays in L2 on a GB300, so the loop runs FP32 throughout
    (phase -1) and gives the FP32 loop's ranks bit for bit."""
    import torch

    n = 1 << log2n
    if 4 * n > torch.cuda.get_device_properties(0).L2_cache_size:
        pytest.skip("the vector does not fit this GPU's L2")
    src, dst = graphgen.er_edges(n, 16, p_dangling=0.02, seed=2)
    r1, it1, _, (_, phase) = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "device", MIXED_TOL, 500,
                                  persistent=1, mixed=1)
    r0, it0, _, _ = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "device", MIXED_TOL, 500,
                         persistent=1, mixed=0)
    assert phase == -1 and it1 == it0 and np.array_equal(r1, r0)


def test_mixed_precision_refines_to_fp32(grb):
    n = 1 << 15
    src, dst = graphgen.er_edges(n, 16, p_dangling=0.02, seed=2)
    r, it, _, (hist, phase) = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "device", 1e-7, 200,
                                   persistent=1, mixed=2)
    assert phase == 1                      # switched to the FP32 gather
    ref, _, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=1e-14, itermax=1000, mode="uniform")
    assert np.sum(np.abs(r - ref)) <= 1e-6


def test_deterministic_and_resumable(grb):
    from paper_2509_14211_gb300.pagerank import PageRankProblem, build_graph

    n = 1 << 14
    src, dst = graphgen.rmat_edges(14, 16, seed=3)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    try:
        AT = build_graph(ctx, n, src, dst)
        P = PageRankProblem(ctx, AT, n, D, grb.GRB_FP32)
        P.run(-1.0, 20)
        a = P.rank().copy()
        P.run(-1.0, 20)
        b = P.rank().copy()
        assert np.array_equal(a, b)                       # bit-reproducible
        # checkpoint after 12 bodies, resume for 8 more
        P.run(-1.0, 12)
        ck = P.rank().copy()
        grb.grb_vector_build(P.r, np.arange(n, dtype=np.int32), ck.astype(np.float64))
        grb.grb_scalar_set(P.rdiff, 1.0)
        grb.grb_iterate_begin(ctx)
        P.body()
        assert grb.grb_iterate_end(ctx, P.rdiff, -1.0, 8) == 8
        # bit for bit: the resumed loop's prologue sums the dangling mass of
        # the checkpoint in another order than body 12's epilogue did, but both
        # sums are FP64-accurate (~1e-14 relative) and the teleport is rounded
        # to FP32 from them, so the two agree unless the sum sits within 1e-14
        # of an FP32 rounding boundary
        assert np.array_equal(P.rank(), a)
        P.free()
        grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)


def test_fixed_count_loops_are_enqueued_back_to_back(grb):
    """Fixed-count device loops return without waiting: three loops enqueued
    back to back (the rank vector rebuilt between them) end with the same
    ranks and history as one loop run alone, and the device times of all
    three are reported."""
    from paper_2509_14211_gb300.pagerank import PageRankProblem, build_graph

    n = 1 << 14
    src, dst = graphgen.rmat_edges(14, 16, seed=8)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    try:
        AT = build_graph(ctx, n, src, dst)
        P = PageRankProblem(ctx, AT, n, D, grb.GRB_FP32)
        assert P.run(-1.0, 20) == 20
        alone = P.rank().copy()
        hist_alone, _ = grb.grb_iterate_history(ctx)
        for _ in range(3):
            assert P.run(-1.0, 20) == 20
        assert np.array_equal(P.rank(), alone)
        hist, _ = grb.grb_iterate_history(ctx)
        assert np.array_equal(hist, hist_alone) and len(hist) == 20
        times = grb.grb_context_loop_times(ctx, 3)
        assert len(times) == 3 and np.all(times > 0)
        ref, _, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=-1.0, itermax=20, mode="uniform")
        assert np.sum(np.abs(alone.astype(np.float64) - ref)) <= 1e-6
        P.free()
        grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)


@pytest.mark.parametrize("case", ["single_vertex", "edgeless", "hub", "ragged"])
def test_edge_graphs(grb, case):
    if case == "single_vertex":
        n, src, dst = 1, np.zeros(0, np.int32), np.zeros(0, np.int32)
    elif case == "edgeless":
        n, src, dst = 1000, np.zeros(0, np.int32), np.zeros(0, np.int32)
    elif case == "hub":      # one row of ~100k in-edges spans ~50 tiles
        rng = np.random.default_rng(9)
        n = 150000
        src = rng.integers(0, n, 120000).astype(np.int32)
        dst = np.where(rng.random(120000) < 0.8, 7, rng.integers(0, n, 120000)).astype(np.int32)
    else:
        rng = np.random.default_rng(10)
        n = 12345
        src = rng.integers(0, n, 40000).astype(np.int32)
        dst = (rng.integers(0, n // 7, 40000) * 7).astype(np.int32)
    for rank_type, tol_ok in ((grb.GRB_FP64, 1e-12), (grb.GRB_FP32, 1e-6)):
        ref, _, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=-1.0, itermax=15, mode="uniform")
        for loop, relabel, bins in (("device", True, False), ("device", False, False), ("host", True, False),
                                    ("device", True, True), ("device", False, True)):
            r, it, _, _ = _run(grb, n, src, dst, rank_type, "uniform", loop, -1.0, 15, relabel=relabel,
                               persistent=1 if loop == "device" else 0, bins=bins)
            assert it == 15
            err = np.max(np.abs(r - ref)) if rank_type == grb.GRB_FP64 else np.sum(np.abs(r - ref))
            assert err <= tol_ok, (case, loop, err)


def test_loop_kernel_counts(grb, c0):
    """Fusion shows in the launch counts: the device loop launches one kernel
    per loop, the host loop a few per iteration, blocking mode one per
    method."""
    n, src, dst = c0
    _, it_d, sd, _ = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "device", -1.0, 30, persistent=1)
    _, it_h, sh, _ = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "host", -1.0, 30)
    _, it_b, sb, _ = _run(grb, n, src, dst, grb.GRB_FP32, "uniform", "host", -1.0, 30, mode=grb.GRB_BLOCKING)
    assert it_d == it_h == it_b == 30
    assert sh["kernel_launches"] - sd["kernel_launches"] >= 2 * 30
    assert sb["kernel_launches"] > sh["kernel_launches"]
    assert sb["fused_groups"] == 0 and sh["fused_groups"] >= 30


def _sink_free(case):
    """Graphs in which every vertex has an out-edge: no dangling mass, the
    sink vector of the program is empty."""
    if case == "cycle":                      # one directed cycle: r stays 1/n
        n = 7
        src = np.arange(n, dtype=np.int32)
        return n, src, ((src + 1) % n).astype(np.int32)
    rng = np.random.default_rng(21)
    n = 3000
    # 3 distinct out-edges per vertex, none to itself; in-degrees vary (some
    # vertices have none: rows without nonzeros)
    offs = np.stack([1 + rng.choice(n - 1, 3, replace=False) for _ in range(n)])
    src = np.repeat(np.arange(n), 3).astype(np.int32)
    dst = ((src + offs.reshape(-1)) % n).astype(np.int32)
    return n, src, dst


@pytest.mark.parametrize("case", ["cycle", "out3"])
@pytest.mark.parametrize("loop,persistent,fusion,mode,relabel", PATHS)
def test_sink_free_graphs_all_paths(grb, case, loop, persistent, fusion, mode, relabel):
    """A degenerate case of the method: no vertex without out-edges, so the
    dangling-mass sum runs over an empty set.  FP64 ranks after 15 bodies
    match the oracle within 1e-12 on every path, in both dangling modes (which
    agree here); the cycle stays at 1/n exactly in exact arithmetic."""
    n, src, dst = _sink_free(case)
    for dangling in ("uniform", "gap"):
        ref, _, _ = oracle.pagerank_edges(n, src, dst, damping=D, tol=-1.0, itermax=15, mode=dangling)
        r, it, _, _ = _run(grb, n, src, dst, grb.GRB_FP64, dangling, loop, -1.0, 15,
                           mode=grb.GRB_BLOCKING if mode == "blocking" else None, persistent=persistent,
                           fusion=fusion, relabel=relabel)
        assert it == 15
        assert np.max(np.abs(r - ref)) <= 1e-12, (case, loop, persistent, dangling)
        if case == "cycle":
            assert np.max(np.abs(r - 1.0 / n)) <= 1e-15
