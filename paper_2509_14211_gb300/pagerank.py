"""PageRank written against the grb_* calls, as the §IV listing
(`pagerank_gap`) writes it against AppGrB.

This module is user code of the library: it only issues GraphBLAS calls.
Every vector operation runs in libgrb.so's CUDA kernels; the host computes
nothing but the two scalar constants the listing itself computes on the host
((1 - damping)/n and, for uniform dangling, damping/n).

Dangling modes:
  "gap"      the listing as printed: rank held by vertices without
             out-edges is dropped (sum(r) < 1).
  "uniform"  that rank D is spread evenly, r = (1-d)/n + d*D/n + A^T (r./d),
             written with GraphBLAS calls the way LAGraph does it
             (reduce over the sinks, assign the scalar, mxv with accum +).
Loop modes:
  "device"   grb_iterate_begin/end: the planner runs the whole loop on the
             GPU (one persistent kernel or a CUDA graph of fused kernels).
  "host"     the listing's while loop on the host, wait(r) and a scalar read
             per iteration (per-wait fusion).
"""
from __future__ import annotations

import numpy as np

from . import (GRB_ABS_DIFF, GRB_BUILD_DEDUP, GRB_BUILD_DROP_SELF, GRB_BUILD_TRANSPOSE, GRB_DESC_COMPLEMENT,
               GRB_DESC_STRUCTURE, GRB_DIV, GRB_FIRST, GRB_FP32, GRB_FP64, GRB_INT32, GRB_MAX_DIV_BY,
               GRB_MONOID_PLUS, GRB_PLUS, GRB_PLUS_SECOND, GRB_TIMES, binop, grb_apply_bind2nd, grb_assign_scalar,
               grb_ewise_add, grb_ewise_mult, grb_free, grb_iterate_begin, grb_iterate_end,
               grb_matrix_build_csr, grb_matrix_col_degree, grb_mxv, grb_reduce, grb_scalar_apply_bind2nd,
               grb_scalar_get, grb_scalar_new, grb_scalar_set, grb_vector_copy, grb_vector_extract_dense,
               grb_vector_fill, grb_vector_new, grb_wait)

BUILD_FLAGS = GRB_BUILD_TRANSPOSE | GRB_BUILD_DROP_SELF | GRB_BUILD_DEDUP


def build_graph(ctx, n, src, dst):
    """A^T (pattern only, iso 1) from a COO edge list: row i holds the
    sources of the edges j -> i (duplicates and self loops dropped)."""
    return grb_matrix_build_csr(ctx, GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)


class PageRankProblem:
    """The setup part of the listing (everything before the loop), kept so
    that the loop can be run several times (benchmarks)."""

    def __init__(self, ctx, AT, n, damping=0.85, rank_type=GRB_FP32, resid_type=GRB_FP64,
                 dangling="uniform"):
        self.ctx, self.AT, self.n = ctx, AT, int(n)
        self.damping, self.T, self.dangling = float(damping), rank_type, dangling
        T = rank_type
        # out_degree and d = ewise_add(max(x/damping, y), conv(out_degree), full(1/damping))
        self.deg = grb_vector_new(ctx, GRB_INT32, n)
        grb_matrix_col_degree(self.deg, AT)
        self.d = grb_vector_new(ctx, T, n)
        grb_vector_fill(self.d, 1.0 / damping)
        grb_ewise_add(self.d, None, None, binop(GRB_MAX_DIV_BY, damping), self.deg, self.d)
        grb_wait(self.d)
        self.teleport = (1.0 - damping) / n
        self.rt = grb_vector_new(ctx, T, n)
        grb_vector_fill(self.rt, self.teleport)
        # sinks: vertices with no out-degree entry (structural complement mask)
        self.sinks = grb_vector_new(ctx, T, n)
        self.one = grb_scalar_new(ctx, T)
        grb_scalar_set(self.one, 1.0)
        grb_assign_scalar(self.sinks, self.deg, None, self.one, GRB_DESC_STRUCTURE | GRB_DESC_COMPLEMENT)
        grb_wait(self.sinks)
        self.r = grb_vector_new(ctx, T, n)
        self.t = grb_vector_new(ctx, T, n)
        self.w = grb_vector_new(ctx, T, n)
        self.z = grb_vector_new(ctx, T, n)
        self.D = grb_scalar_new(ctx, resid_type)
        self.rdiff = grb_scalar_new(ctx, resid_type)

    def reset(self):
        grb_vector_fill(self.r, 1.0 / self.n)
        grb_scalar_set(self.rdiff, 1.0)

    def body(self, wait_r=True):
        """One iteration of the listing's loop body."""
        r, t = self.r, self.t
        grb_vector_copy(t, r)                                                   # t = r
        if self.dangling == "gap":
            grb_ewise_mult(r, None, None, binop(GRB_DIV), t, self.d)            # r = t ./ d
            grb_mxv(r, None, None, GRB_PLUS_SECOND, self.AT, r)                 # r = A^T (+.second) r
            grb_ewise_add(r, None, None, binop(GRB_PLUS), self.rt, r)           # r = rt + r
        else:
            grb_ewise_mult(self.w, None, None, binop(GRB_DIV), t, self.d)       # w = t ./ d
            grb_ewise_mult(self.z, None, None, binop(GRB_FIRST), t, self.sinks) # z = t restricted to sinks
            grb_reduce(self.D, None, GRB_MONOID_PLUS, self.z)                   # D = dangling mass
            grb_scalar_apply_bind2nd(self.D, binop(GRB_TIMES), self.D, self.damping / self.n)
            grb_scalar_apply_bind2nd(self.D, binop(GRB_PLUS), self.D, self.teleport)
            grb_assign_scalar(r, None, None, self.D)                            # r = (1-d)/n + d*D/n
            grb_mxv(r, None, binop(GRB_PLUS), GRB_PLUS_SECOND, self.AT, self.w)  # r += A^T w
        if wait_r:
            grb_wait(r)
        grb_ewise_add(t, None, None, binop(GRB_ABS_DIFF), t, r)                 # t = |t - r|
        grb_reduce(self.rdiff, None, GRB_MONOID_PLUS, t)                        # rdiff = sum(t)

    def run(self, tol=1e-10, itermax=100, loop="device"):
        """Run the loop from r = 1/n; returns the number of bodies executed."""
        self.reset()
        if loop == "device":
            grb_iterate_begin(self.ctx)
            self.body()
            return grb_iterate_end(self.ctx, self.rdiff, tol, itermax)
        it = 0
        while it < itermax and grb_scalar_get(self.rdiff) > tol:
            self.body()
            it += 1
        return it

    def rank(self):
        vals, _ = grb_vector_extract_dense(self.r, self.T)
        return vals

    def residual(self):
        return grb_scalar_get(self.rdiff)

    def free(self):
        for h in (self.deg, self.d, self.rt, self.sinks, self.r, self.t, self.w, self.z, self.one, self.D,
                  self.rdiff):
            grb_free(h)


def pagerank(ctx, n, src, dst, damping=0.85, tol=1e-10, itermax=100, rank_type=GRB_FP32, dangling="uniform",
             loop="device", resid_type=GRB_FP64):
    """Build A^T, run PageRank, return (ranks as float64 numpy, iterations)."""
    AT = build_graph(ctx, n, src, dst)
    P = PageRankProblem(ctx, AT, n, damping, rank_type, resid_type, dangling)
    iters = P.run(tol, itermax, loop)
    r = P.rank().astype(np.float64)
    P.free()
    grb_free(AT)
    return r, iters
