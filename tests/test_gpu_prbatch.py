"""Batch of independent graphs (grb_prbatch_*): every graph of a
block-diagonal A^T against the FP64 oracle run on that graph alone (uniform
dangling; same body count; FP32 ranks: L1 <= 1e-6 per graph)."""
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


def _graphs(count, lo, hi, seed):
    out = []
    for scale, ef, s in graphgen.batch_graph_specs(count, lo, hi, 4, 16, seed=seed):
        src, dst = graphgen.rmat_edges(scale, ef, seed=s)
        out.append((1 << scale, src, dst))
    return out


def _build(grb, graphs):
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    n, src, dst, vptr = grb.block_diagonal_edges(graphs)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    B = grb.grb_prbatch_new(AT, vptr, D)
    return ctx, AT, B, n, vptr


def _free(grb, ctx, AT, B):
    grb.grb_free(B)
    grb.grb_free(AT)
    grb.grb_free(ctx)


def test_fixed_iterations_match_oracle_per_graph(grb):
    graphs = _graphs(40, 3, 10, seed=3)
    ctx, AT, B, n, vptr = _build(grb, graphs)
    try:
        ms, chosen = grb.grb_prbatch_tune(B, 2)
        assert len(ms) >= 1 and 1 <= chosen <= len(ms)
        grb.grb_prbatch_run(B, -1.0, 20, 7)
        r, its, res = grb.grb_prbatch_result(B, n, len(graphs))
        assert np.all(its == 20)
        for g, (ng, src, dst) in enumerate(graphs):
            ref, k, hist = oracle.pagerank_edges(ng, src, dst, damping=D, tol=-1.0, itermax=20, mode="uniform")
            rg = r[vptr[g]:vptr[g + 1]].astype(np.float64)
            assert np.sum(np.abs(rg - ref)) <= 1e-6, g
            assert abs(res[g] - hist[-1]) <= 1e-3 * hist[-1] + 1e-7
        # the launch shape does not change the results
        grb.grb_prbatch_tune(B, 1)
        grb.grb_prbatch_run(B, -1.0, 20, 20)
        r2, _, _ = grb.grb_prbatch_result(B, n, len(graphs))
        assert np.array_equal(r, r2)
    finally:
        _free(grb, ctx, AT, B)


def test_per_graph_stopping(grb):
    """Each graph stops on its own test; body counts are the oracle's (+-1
    near the threshold) and the ranks match the oracle at that count."""
    graphs = _graphs(24, 4, 11, seed=8)
    ctx, AT, B, n, vptr = _build(grb, graphs)
    try:
        grb.grb_prbatch_run(B, 1e-6, 300, 8)
        r, its, res = grb.grb_prbatch_result(B, n, len(graphs))
        assert np.all(res <= 1e-6) and np.all(its < 300)
        assert len(set(its.tolist())) > 1            # graphs finished at different bodies
        for g, (ng, src, dst) in enumerate(graphs):
            _, k_conv, _ = oracle.pagerank_edges(ng, src, dst, damping=D, tol=1e-6, itermax=300, mode="uniform")
            assert abs(k_conv - its[g]) <= 1, (g, k_conv, its[g])
            ref, _, _ = oracle.pagerank_edges(ng, src, dst, damping=D, tol=-1.0, itermax=int(its[g]), mode="uniform")
            assert np.sum(np.abs(r[vptr[g]:vptr[g + 1]].astype(np.float64) - ref)) <= 1e-6, g
    finally:
        _free(grb, ctx, AT, B)


def test_tiny_and_edgeless_members_and_errors(grb):
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    graphs = [(1, np.zeros(0, np.int32), np.zeros(0, np.int32)),
              (5, np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32)),
              (300, np.zeros(0, np.int32), np.zeros(0, np.int32))] + _graphs(3, 8, 9, seed=2)
    ctx, AT, B, n, vptr = _build(grb, graphs)
    try:
        grb.grb_prbatch_run(B, -1.0, 12, 5)
        r, its, _ = grb.grb_prbatch_result(B, n, len(graphs))
        for g, (ng, src, dst) in enumerate(graphs):
            ref, _, _ = oracle.pagerank_edges(ng, src, dst, damping=D, tol=-1.0, itermax=12, mode="uniform")
            assert np.sum(np.abs(r[vptr[g]:vptr[g + 1]].astype(np.float64) - ref)) <= 1e-6, g
    finally:
        _free(grb, ctx, AT, B)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    try:
        AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, 10, 10, np.array([1, 6], np.int32),
                                      np.array([2, 3], np.int32), None, BUILD_FLAGS)
        try:
            for vptr in ([0, 5, 10], [0, 10, 10], [0, 4]):
                with pytest.raises(grb.GrbError) as e:
                    grb.grb_prbatch_new(AT, vptr, D)
                assert e.value.code == grb.GRB_INVALID_VALUE
        finally:
            grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)


def test_512_graphs_scale_8_to_16_sampled(grb):
    """The batch configuration: 512 R-MAT graphs, scale 8-16, edge factor
    8-32 (seed 3), 30 bodies in one CUDA-graph launch; 12 graphs checked
    against the oracle, all for non-negativity and unit sum."""
    specs = graphgen.batch_graph_specs(512, 8, 16, 8, 32, seed=3)
    graphs = []
    for scale, ef, s in specs:
        src, dst = graphgen.rmat_edges(scale, ef, seed=s)
        graphs.append((1 << scale, src, dst))
    ctx, AT, B, n, vptr = _build(grb, graphs)
    try:
        grb.grb_prbatch_run(B, -1.0, 30, 30)
        r, its, _ = grb.grb_prbatch_result(B, n, len(graphs))
        assert np.all(its == 30)
        for g in range(0, 512, 43):
            ng, src, dst = graphs[g]
            ref, _, _ = oracle.pagerank_edges(ng, src, dst, damping=D, tol=-1.0, itermax=30, mode="uniform")
            assert np.sum(np.abs(r[vptr[g]:vptr[g + 1]].astype(np.float64) - ref)) <= 1e-6, g
        sums = np.add.reduceat(r.astype(np.float64), vptr[:-1])
        assert np.all(r >= 0) and np.all(np.abs(sums - 1.0) < 1e-4)
    finally:
        _free(grb, ctx, AT, B)
