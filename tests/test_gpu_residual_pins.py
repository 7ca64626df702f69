"""The FP64 reductions of the FP32 PageRank loops, pinned exactly.

In the §IV listing the loop test is rdiff = reduce(+, t) with t = |t - r|, an
element-wise vector of the rank's type (here FP32), and, with the dangling
rank spread uniformly, the teleport of the next body is
(1 - damping)/n + damping * D / n with D the rank summed over the vertices
without out-edges.  Both sums run in FP64 (the scalars are FP64).  These tests
check what the GPU reports against exactly rounded sums (math.fsum) of the
GPU's OWN FP32 iterates r_{k-1} and r_k -- not against the oracle, whose
iterates differ from the GPU's by FP32 rounding -- so they pin the
reductions themselves:

  rdiff_k  = sum_i fl32(|r_{k-1,i} - r_{k,i}|)     relative error <= 1e-12
  D_k      = sum_{i sink} r_{k,i}                   relative error <= 1e-12
  r_{k,i}  = fl32((1-d)/n + (d/n) * D_{k-1})        bit for bit, for every i
                                                    without in-edges

Runs of k-1 and k bodies from r_0 = 1/n give r_{k-1} and r_k: every GPU
reduction has a fixed order, so the trajectories are identical.
"""
import math

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu
D = 0.85
REL = 1e-12


@pytest.fixture(scope="module")
def grb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2509_14211_gb300 as g

    g.load()
    return g


def _degrees(n, src, dst):
    """Out- and in-degree after the CSR build's dedup and self-loop removal."""
    keep = src != dst
    key = np.unique(src[keep].astype(np.int64) * n + dst[keep].astype(np.int64))
    s, d = key // n, key % n
    return np.bincount(s, minlength=n), np.bincount(d, minlength=n)


def _teleport(n, dmass):
    # the listing's scalar chain: D * (damping / n) + (1 - damping) / n in
    # FP64, then assigned to the FP32 rank vector
    return np.float32(np.float64(np.float64(dmass * (D / n)) + (1.0 - D) / n))


def _pin(grb, n, src, dst, ks, persistent, relabel, loop="device", bins=False):
    from paper_2509_14211_gb300.pagerank import PageRankProblem, build_graph

    outdeg, indeg = _degrees(n, src, dst)
    sinks = outdeg == 0
    roots = indeg == 0
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    try:
        grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, persistent)
        grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 1 if relabel else 0)
        grb.grb_context_set(ctx, grb.GRB_OPT_ROW_BINS, 1 if bins else 0)
        AT = build_graph(ctx, n, src, dst)
        P = PageRankProblem(ctx, AT, n, D, grb.GRB_FP32, grb.GRB_FP64, "uniform")
        for k in ks:
            assert P.run(-1.0, k - 1, loop) == k - 1
            r_prev = P.rank().copy()
            assert P.run(-1.0, k, loop) == k
            r_k = P.rank().copy()
            rdiff = P.residual()
            diff32 = np.abs(r_prev - r_k)                 # FP32, as the vector t holds it
            ref_rdiff = math.fsum(diff32.astype(np.float64))
            assert abs(rdiff - ref_rdiff) <= REL * ref_rdiff, (k, rdiff, ref_rdiff)
            if loop == "device":
                hist, dang, _ = grb.grb_iterate_history(ctx, with_dang=True)
                assert len(hist) == k and hist[-1] == rdiff
                ref_d = math.fsum(r_k[sinks].astype(np.float64))
                ref_dprev = math.fsum(r_prev[sinks].astype(np.float64))
                assert abs(dang[-1] - ref_d) <= REL * ref_d, (k, dang[-1], ref_d)
                assert abs(dang[-2] - ref_dprev) <= REL * ref_dprev, (k, dang[-2], ref_dprev)
                # the next body's teleport is built from the reported mass
                if roots.any():
                    assert np.all(r_k[roots] == _teleport(n, dang[-2])), k
        P.free()
        grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)


# (persistent option, degree-ordered copy, row-length bins): the persistent
# kernel with the shared-memory hot copy, the persistent kernel on the input
# vertex order, the CUDA-graph loop of one fused kernel per body, the binned
# body
PATHS = [(1, True, False), (1, False, False), (2, True, False), (1, True, True)]


@pytest.mark.parametrize("persistent,relabel,bins", PATHS)
def test_residual_and_dangling_mass_rmat16(grb, persistent, relabel, bins):
    n = 1 << 16
    src, dst = graphgen.rmat_edges(16, 16, seed=1)
    _pin(grb, n, src, dst, (2, 5, 30), persistent, relabel, bins=bins)


def test_residual_host_loop_rmat16(grb):
    """The host loop with per-wait fusion (the reduction kernels of the
    planner): the residual scalar after k bodies."""
    n = 1 << 16
    src, dst = graphgen.rmat_edges(16, 16, seed=1)
    _pin(grb, n, src, dst, (2, 7), 0, True, loop="host")


def test_residual_and_dangling_mass_rmat22(grb):
    """The benchmark configuration: R-MAT scale 22, bodies 49 and 50."""
    n = 1 << 22
    src, dst = graphgen.rmat_edges(22, 16, seed=1)
    _pin(grb, n, src, dst, (2, 50), 1, True)
