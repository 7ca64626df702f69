"""PageRank at the largest sizes the library takes.

Row offsets and column indices are int32, so a CSR holds fewer than 2^31
nonzeros.  The fused kernels (the device loop, the per-wait fused mxv) take
a matrix while nrows + nnz stays below 2^31 - 2^24, their int32 indexing
headroom; past it the planner runs the loop body on the general kernels,
which index with int64.  Both regimes are run at their largest size.

The oracle cannot run at these sizes, so the checks are properties that hold
at any size:

  - a 16-regular digraph (every vertex has 16 out-edges and 16 in-edges):
    the uniform vector is the fixed point (every column of the
    column-stochastic matrix sums to 1, every row of A^T has 16 entries of
    d/16), so from r_0 = 1/n every body returns 1/n in every entry up to FP32
    rounding -- including the rows of the last tiles, at the largest nonzero
    offsets the path holds.  Fused: n = 125,000,000, nnz = 2,000,000,000;
    general: n = 2^27 - 1, nnz = 2^31 - 16;
  - R-MAT scale 27 with 2^31 - 1 edges (duplicates and self loops dropped):
    the degree-ordered copy and the shared-memory hot copy at full size;
    ranks non-negative and summing to 1, and the reported residual equal to
    the L1 distance of the GPU's own two last iterates summed exactly.
Inputs are generated on the device with seeded torch generators (the host
would need 17 GB for an edge list).
"""
import math

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
D = 0.85
OFFSETS = [1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 377, 610, 987]


@pytest.fixture(scope="module")
def grb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    free, _ = torch.cuda.mem_get_info()
    if free < 120 * 2**30:
        pytest.skip("needs ~120 GB of free device memory")
    import paper_2509_14211_gb300 as g

    g.load()
    return g


def _regular_edges(n, offsets):
    """Edges i -> (i + c) mod n for every offset c: in- and out-degree 16."""
    import torch

    m = len(offsets) * n
    src = torch.empty(m, dtype=torch.int32, device="cuda")
    dst = torch.empty(m, dtype=torch.int32, device="cuda")
    i = torch.arange(n, dtype=torch.int64, device="cuda")
    for k, c in enumerate(offsets):
        src[k * n:(k + 1) * n] = i.to(torch.int32)
        dst[k * n:(k + 1) * n] = ((i + c) % n).to(torch.int32)
    return src, dst


def _rmat_edges(scale, m, seed, a=0.57, b=0.19, c=0.19):
    """R-MAT edge list on the device: at each of `scale` levels a quadrant
    (a, b, c, 1-a-b-c) picks one bit of source and destination."""
    import torch

    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    src = torch.zeros(m, dtype=torch.int32, device="cuda")
    dst = torch.zeros(m, dtype=torch.int32, device="cuda")
    for lvl in range(scale):
        u = torch.rand(m, generator=gen, device="cuda")
        bit = 1 << (scale - 1 - lvl)
        right = (u >= a) & (u < a + b) | (u >= a + b + c)   # quadrants b and d: destination bit
        down = u >= a + b                                    # quadrants c and d: source bit
        del u
        dst.add_(right.to(torch.int32).mul_(bit))
        src.add_(down.to(torch.int32).mul_(bit))
        del right, down
    return src, dst


def _solve(grb, n, make_edges, bodies):
    """Build A^T from the edges make_edges() returns (freed once the CSR is
    built), then run `bodies` fixed-count device loops from r_0 = 1/n."""
    import torch

    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS, PageRankProblem

    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    try:
        src, dst = make_edges()
        m = src.numel()
        AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
        torch.cuda.synchronize()
        del src, dst
        torch.cuda.empty_cache()
        nnz = grb.grb_matrix_nvals(AT)
        P = PageRankProblem(ctx, AT, n, D, grb.GRB_FP32, grb.GRB_FP64, "uniform")
        out = []
        for k in bodies:
            assert P.run(-1.0, k, "device") == k
            out.append((P.rank().copy(), P.residual()))
        stats = grb.grb_context_stats(ctx)
        P.free()
        grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)
    return m, nnz, out, stats


def _check_uniform(n, out):
    for r, rdiff in out:
        dev = np.abs(r.astype(np.float64) * n - 1.0)
        assert dev.max() <= 4e-6, (dev.max(), int(dev.argmax()))
        assert abs(np.sum(r.astype(np.float64)) - 1.0) <= 1e-5
        assert rdiff <= 8e-6


def test_regular_digraph_largest_fused(grb):
    """nrows + nnz = 2,125,000,000, just under the fused kernels' limit: the
    persistent loop runs every body."""
    n = 125_000_000
    _, nnz, out, stats = _solve(grb, n, lambda: _regular_edges(n, OFFSETS + [n // 2]), (1, 4))
    assert nnz == 16 * n
    assert stats["persistent_loops"] == 2
    _check_uniform(n, out)


def test_regular_digraph_at_the_int32_nonzero_limit(grb):
    """nnz = 2^31 - 16, the most a CSR holds: past the fused kernels' limit,
    the loop body runs on the general (int64-indexed) kernels."""
    n = (1 << 27) - 1
    m, nnz, out, stats = _solve(grb, n, lambda: _regular_edges(n, OFFSETS + [1 << 26]), (1, 4))
    assert m == (1 << 31) - 16
    assert nnz == (1 << 31) - 16                  # no duplicates, no self loops
    assert stats["persistent_loops"] == 0
    _check_uniform(n, out)


def test_rmat27_near_the_edge_limit(grb):
    scale, m = 27, (1 << 31) - 1
    n = 1 << scale
    _, nnz, out, _ = _solve(grb, n, lambda: _rmat_edges(scale, m, seed=7), (9, 10))
    assert 0 < nnz <= m
    (r9, _), (r10, rdiff) = out
    for r in (r9, r10):
        assert np.all(r >= 0.0) and np.all(np.isfinite(r))
        assert abs(np.sum(r.astype(np.float64)) - 1.0) <= 1e-4
    ref = math.fsum(np.abs(r9 - r10).astype(np.float64))   # |t - r| in FP32, summed exactly
    assert abs(rdiff - ref) <= 1e-12 * ref, (rdiff, ref)
