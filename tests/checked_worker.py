"""Runs in a child process with GRB_CHECK_BOUNDS=1, so that the package
loads the bounds-checked build (libgrb_checked.so); the parent test compares
what it writes with the release library.  Usage:

    python checked_worker.py OUTDIR

Writes OUTDIR/clean_<path>.npy (ranks of clean runs) and OUTDIR/report.json
(what every planted fault reported).  Faults are planted only through the
structure check's host-array entry and by overwriting a column index with a
value just outside [0, n) after the structure was validated -- a case the
in-kernel checks of the bounds-checked library turn into GRB_INDEX_OUT_OF_BOUNDS.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import graphgen  # noqa: E402

# (name, context mode, persistent option, loop): the device paths that walk
# the column indices on every body
PATHS = [("persistent", "nonblocking", 1, "device"), ("graph", "nonblocking", 2, "device"),
         ("host", "nonblocking", 0, "host"), ("blocking", "blocking", 0, "host")]
D = 0.85
ITERS = 12


def _ctx(grb, mode, persistent):
    ctx = grb.grb_context_new(grb.GRB_BLOCKING if mode == "blocking" else grb.GRB_NONBLOCKING)
    grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, persistent)
    grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 0)   # the loops walk this matrix's own columns
    return ctx


def _solve(P, loop):
    """ITERS bodies and the ranks: (ranks, None, "") or (None, grb_info code,
    the context's error text)."""
    import paper_2509_14211_gb300 as grb

    try:
        P.run(-1.0, ITERS, loop)
        return P.rank(), None, ""
    except grb.GrbError as e:
        return None, e.code, grb.grb_error(P.ctx)


def main(out):
    import torch

    import paper_2509_14211_gb300 as grb
    from paper_2509_14211_gb300.pagerank import PageRankProblem, build_graph

    assert grb.CHECKED and grb.LIB_PATH.endswith("libgrb_checked.so")
    grb.load()
    torch.cuda.set_device(0)
    n = 1 << 12
    src, dst = graphgen.rmat_edges(12, 16, seed=5)
    rep = {}

    # the structure check on host arrays: one planted failure per case
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    rp = np.array([0, 2, 4, 5, 5, 7], np.int32)
    ci = np.array([1, 3, 0, 2, 4, 0, 1], np.int32)
    cases = {"valid": (rp, ci), "col_high": (rp, np.where(np.arange(7) == 3, 5, ci)),
             "col_negative": (rp, np.where(np.arange(7) == 6, -1, ci)),
             "row_ptr_decreasing": (np.array([0, 2, 4, 3, 5, 7], np.int32), ci),
             "row_ptr_end": (np.array([0, 2, 4, 5, 5, 6], np.int32), ci),
             "row_ptr_start": (np.array([1, 2, 4, 5, 5, 7], np.int32), ci),
             "row_ptr_above_nnz": (np.array([0, 2, 9, 5, 5, 7], np.int32), ci)}
    rep["check_csr"] = {k: list(grb.grb_debug_check_csr(ctx, a, b, 5)) for k, (a, b) in cases.items()}
    grb.grb_free(ctx)

    for name, mode, persistent, loop in PATHS:
        r = {}
        ctx = _ctx(grb, mode, persistent)
        AT = build_graph(ctx, n, src, dst)
        _, col = grb.grb_matrix_export_csr(AT)
        k = len(col) // 3
        P = PageRankProblem(ctx, AT, n, D, grb.GRB_FP32, grb.GRB_FP64, "uniform")
        clean, code, _ = _solve(P, loop)
        assert code is None, (name, code)
        np.save(os.path.join(out, f"clean_{name}.npy"), clean)
        # a column index just outside [0, n), then -1, after validation
        for bad in (n, -1):
            grb.grb_debug_set_col(AT, k, bad)
            res, code, msg = _solve(P, loop)
            r[f"bad_{bad}"] = [code, msg]
            grb.grb_debug_set_col(AT, k, int(col[k]))
        # the context stays usable: the repaired matrix gives the clean ranks
        again, code, _ = _solve(P, loop)
        r["repaired_code"] = code
        r["repaired_equal"] = bool(again is not None and np.array_equal(again, clean))
        P.free()
        grb.grb_free(AT)
        # a fault planted before the matrix's first use: the structure check
        # runs before any kernel walks it
        AT = build_graph(ctx, n, src, dst)
        grb.grb_debug_set_col(AT, 7, n + 3)
        try:
            P = PageRankProblem(ctx, AT, n, D, grb.GRB_FP32, grb.GRB_FP64, "uniform")
            res, code, msg = _solve(P, loop)
            P.free()
        except grb.GrbError as e:
            code, msg = e.code, grb.grb_error(ctx)
        r["before_first_use"] = [code, msg]
        grb.grb_free(AT)
        grb.grb_free(ctx)
        rep[name] = r

    # batched personalised PageRank: the tile kernel's column checks
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = build_graph(ctx, n, src, dst)
    _, col = grb.grb_matrix_export_csr(AT)
    Pp = grb.grb_ppr_new(AT, D, 4)
    seeds = [[1, 2], [100], [7, 8, 9], [4000]]

    def ppr_round():
        for s, sd in enumerate(seeds):
            grb.grb_ppr_set(Pp, s, np.array(sd, np.int32), -1.0, ITERS)
        try:
            grb.grb_ppr_run(Pp, ITERS)
            grb.grb_ppr_status(Pp)
            return np.stack([grb.grb_ppr_get(Pp, s, n) for s in range(len(seeds))]), None
        except grb.GrbError as e:
            return None, e.code

    clean, code = ppr_round()
    assert code is None, code
    np.save(os.path.join(out, "clean_ppr.npy"), clean)
    grb.grb_debug_set_col(AT, len(col) // 2, n)
    _, rep_code = ppr_round()
    grb.grb_debug_set_col(AT, len(col) // 2, int(col[len(col) // 2]))
    again, code2 = ppr_round()
    rep["ppr"] = {"bad_code": rep_code, "repaired_code": code2,
                  "repaired_equal": bool(again is not None and np.array_equal(again, clean))}
    grb.grb_free(Pp)
    grb.grb_free(AT)
    grb.grb_free(ctx)

    with open(os.path.join(out, "report.json"), "w") as f:
        json.dump(rep, f)


if __name__ == "__main__":
    main(sys.argv[1])
