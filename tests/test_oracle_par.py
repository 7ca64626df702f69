"""The multi-core timing variant of the oracle (oracle_par.c) against the
pinned single-core oracle: same iteration counts, ranks within 1e-12 (only
the reductions' summation order differs), on a skewed R-MAT graph and on a
graph with many vertices without in- or out-edges, in both dangling modes."""
import numpy as np
import pytest

import graphgen
import oracle


@pytest.mark.parametrize("mode", ["uniform", "gap"])
@pytest.mark.parametrize("tol,itermax", [(1e-10, 100), (-1.0, 25)])
def test_par_matches_serial_rmat(mode, tol, itermax):
    n = 1 << 13
    src, dst = graphgen.rmat_edges(13, 16, seed=7)
    ptr, col = oracle.build_at(n, src, dst)
    od = oracle.out_degree(ptr, col)
    r, k, h = oracle.pagerank(ptr, col, od, damping=0.85, tol=tol, itermax=itermax, mode=mode)
    rp, kp, hp = oracle.pagerank_par(ptr, col, od, damping=0.85, tol=tol, itermax=itermax, mode=mode)
    assert k == kp
    assert np.max(np.abs(r - rp)) <= 1e-12
    # rank entries differ by FP64 rounding, so the late, tiny residuals agree
    # to n * eps absolutely
    np.testing.assert_allclose(hp, h, rtol=1e-11, atol=1e-13)


def test_par_matches_serial_sparse_graph():
    rng = np.random.default_rng(11)
    n = 5000
    src = rng.integers(0, n // 3, 6000).astype(np.int32)
    dst = (rng.integers(0, n // 5, 6000) * 5).astype(np.int32)
    ptr, col = oracle.build_at(n, src, dst)
    od = oracle.out_degree(ptr, col)
    r, k, _ = oracle.pagerank(ptr, col, od, damping=0.85, tol=-1.0, itermax=20, mode="uniform")
    rp, kp, _ = oracle.pagerank_par(ptr, col, od, damping=0.85, tol=-1.0, itermax=20, mode="uniform")
    assert k == kp == 20
    assert np.max(np.abs(r - rp)) <= 1e-12
    assert oracle.par_threads() >= 1
