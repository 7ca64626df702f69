"""The bounds-checked debug build (libgrb_checked.so, include/grb_debug.h).

A child process loads the checked build (GRB_CHECK_BOUNDS=1) and runs
tests/checked_worker.py; this process runs the same problems on the release
library.  Checked:
  - clean runs give the release build's ranks bit for bit (the checks change
    no arithmetic), on the persistent loop, the CUDA-graph loop, the host
    loop, the blocking path and batched personalised PageRank;
  - the device structure check reports each planted failure (a column index
    outside [0, ncols), a row_ptr entry out of order or outside [0, nnz],
    row_ptr[0] != 0, row_ptr[n] != nnz) with what failed and where;
  - a column index overwritten after validation (n, then -1) is caught by
    the in-kernel checks of every loop and reported as
    GRB_INDEX_OUT_OF_BOUNDS naming the index; the context stays usable and
    the repaired matrix gives the clean ranks again;
  - a column index planted before the matrix's first use is caught by the
    structure check before any kernel walks the matrix.
No fault reaches the GPU: the checked build never addresses memory with an
unchecked index (every gathered column index is tested before use).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
OOB = -102   # GRB_INDEX_OUT_OF_BOUNDS
D = 0.85
ITERS = 12


@pytest.fixture(scope="module")
def grb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2509_14211_gb300 as g

    g.load()
    return g


@pytest.fixture(scope="module")
def checked_run(grb, tmp_path_factory):
    from paper_2509_14211_gb300 import _build

    if not os.path.exists(_build.LIB_CHECKED):
        pytest.fail("libgrb_checked.so was not built (__graft_entry__.build() builds it)")
    out = tmp_path_factory.mktemp("checked")
    env = dict(os.environ, GRB_CHECK_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_worker.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    with open(out / "report.json") as f:
        return out, json.load(f)


def _release_ranks(grb, mode, persistent, loop):
    from paper_2509_14211_gb300.pagerank import PageRankProblem, build_graph

    n = 1 << 12
    src, dst = graphgen.rmat_edges(12, 16, seed=5)
    ctx = grb.grb_context_new(grb.GRB_BLOCKING if mode == "blocking" else grb.GRB_NONBLOCKING)
    try:
        grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, persistent)
        grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 0)
        AT = build_graph(ctx, n, src, dst)
        P = PageRankProblem(ctx, AT, n, D, grb.GRB_FP32, grb.GRB_FP64, "uniform")
        P.run(-1.0, ITERS, loop)
        r = P.rank().copy()
        P.free()
        grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)
    return r


PATHS = [("persistent", "nonblocking", 1, "device"), ("graph", "nonblocking", 2, "device"),
         ("host", "nonblocking", 0, "host"), ("blocking", "blocking", 0, "host")]


def test_structure_check_reports_each_planted_failure(checked_run):
    _, rep = checked_run
    c = rep["check_csr"]
    assert c["valid"] == [0, 0, 0]
    assert c["col_high"] == [OOB, 1, 5]            # column 5 of a 5-column matrix
    assert c["col_negative"] == [OOB, 1, -1]
    assert c["row_ptr_decreasing"] == [OOB, 2, 2]  # row_ptr[3] < row_ptr[2]
    assert c["row_ptr_end"] == [OOB, 2, 5]         # row_ptr[n] != nnz
    assert c["row_ptr_start"] == [OOB, 2, 0]       # row_ptr[0] != 0
    assert c["row_ptr_above_nnz"] == [OOB, 2, 2]   # row_ptr[2] = 9 > nnz


@pytest.mark.parametrize("name,mode,persistent,loop", PATHS)
def test_checked_build_clean_run_is_bit_identical(grb, checked_run, name, mode, persistent, loop):
    out, _ = checked_run
    checked = np.load(out / f"clean_{name}.npy")
    assert np.array_equal(checked, _release_ranks(grb, mode, persistent, loop)), name


@pytest.mark.parametrize("name", [p[0] for p in PATHS])
def test_in_kernel_checks_catch_a_bad_column(checked_run, name):
    _, rep = checked_run
    r = rep[name]
    n = 1 << 12
    for bad in (n, -1):
        code, msg = r[f"bad_{bad}"]
        assert code == OOB, (name, bad, code, msg)
    # the context's error text names the index
    assert f"column index {n} outside" in r[f"bad_{n}"][1], r
    assert "column index -1 outside" in r["bad_-1"][1], r
    assert r["repaired_code"] is None and r["repaired_equal"], r
    code, msg = r["before_first_use"]
    assert code == OOB and f"column index {n + 3} outside" in msg, (name, code, msg)


def test_ppr_tiles_check_their_columns(grb, checked_run):
    out, rep = checked_run
    r = rep["ppr"]
    assert r["bad_code"] == OOB and r["repaired_code"] is None and r["repaired_equal"], r
    # the clean batched run matches the release build bit for bit
    from paper_2509_14211_gb300.pagerank import build_graph

    n = 1 << 12
    src, dst = graphgen.rmat_edges(12, 16, seed=5)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    try:
        AT = build_graph(ctx, n, src, dst)
        P = grb.grb_ppr_new(AT, D, 4)
        for s, sd in enumerate([[1, 2], [100], [7, 8, 9], [4000]]):
            grb.grb_ppr_set(P, s, np.array(sd, np.int32), -1.0, ITERS)
        grb.grb_ppr_run(P, ITERS)
        grb.grb_ppr_status(P)
        rel = np.stack([grb.grb_ppr_get(P, s, n) for s in range(4)])
        grb.grb_free(P)
        grb.grb_free(AT)
    finally:
        grb.grb_free(ctx)
    assert np.array_equal(np.load(out / "clean_ppr.npy"), rel)
