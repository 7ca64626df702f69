"""The allocation-free reduction (grb_reduce_dense_noalloc), for callers that
cannot allocate device memory when they reduce -- code inside a host
framework that owns the whole memory budget, code under a hard memory cap, or
a path that cannot pay for cudaMalloc's synchronisation.  Its scratch is a
fixed device array shared by every call, so each case runs two calls in a
row on it and checks both against the allocating entry point (grb_reduce on
a vector, same tolerance as the other reduction tests) and against a fold on
the host that shares nothing with the GPU path (math.fsum for PLUS, numpy
for MAX / MIN / TIMES).  Collected last so that a run stopping at the first
failure has run everything else first."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2509_14211_gb300 as grb

    grb.load()
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    yield grb, torch, ctx
    grb.grb_free(ctx)


def _allocating(grb, ctx, data, monoid):
    """The same fold through the allocating entry point (grb_reduce)."""
    v = grb.grb_vector_new(ctx, grb.GRB_FP64, max(len(data), 1))
    if len(data):
        grb.grb_vector_build(v, np.arange(len(data), dtype=np.int32), data.astype(np.float64))
    s = grb.grb_scalar_new(ctx, grb.GRB_FP64)
    grb.grb_reduce(s, None, monoid, v)
    val = grb.grb_scalar_get(s)
    grb.grb_free(v)
    grb.grb_free(s)
    return val


def _host(grb, data, monoid):
    """Exactly rounded sum, or numpy's max / min / product, in FP64."""
    x = data.astype(np.float64)
    if monoid == grb.GRB_MONOID_PLUS:
        return math.fsum(x)
    if monoid == grb.GRB_MONOID_MAX:
        return float(np.max(x)) if len(x) else -math.inf
    if monoid == grb.GRB_MONOID_MIN:
        return float(np.min(x)) if len(x) else math.inf
    return float(np.prod(x)) if len(x) else 1.0


def _close(got, want, scale):
    if math.isinf(want):
        return got == want
    return abs(got - want) <= 1e-12 * max(1.0, scale)


def test_noalloc_matches_grb_reduce_and_host_fold_on_consecutive_calls(env):
    grb, torch, ctx = env
    rng = np.random.default_rng(42)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    P, X, N, T = grb.GRB_MONOID_PLUS, grb.GRB_MONOID_MAX, grb.GRB_MONOID_MIN, grb.GRB_MONOID_TIMES
    F64, F32, I32 = grb.GRB_FP64, grb.GRB_FP32, grb.GRB_INT32
    cases = [(3_000_017, F64, P, "normal"), (77, F64, P, "normal"), (1_000_000, F32, X, "normal"),
             (grb.GRB_NOALLOC_MAX_N, F32, P, "normal"),      # the largest size the scratch holds
             (4096 * 37, F64, P, "normal"),                   # a whole number of 4096-element chunks
             (4096, F32, N, "normal"), (250_001, I32, P, "int"), (99_999, I32, N, "int"),
             (5_000, F64, T, "near1"), (0, F64, P, "normal"), (0, F32, X, "normal"), (0, I32, N, "int"),
             (0, F64, T, "near1")]
    dts = {F64: torch.float64, F32: torch.float32, I32: torch.int32}
    for n, type_, monoid, dist in cases:
        if dist == "int":
            data = rng.integers(-1000, 1000, n)
        elif dist == "near1":
            data = 1.0 + 1e-3 * rng.standard_normal(n)
        else:
            data = rng.standard_normal(n)
        x = torch.tensor(data, dtype=dts[type_], device="cuda")
        exact = x.double().cpu().numpy()          # the values as the GPU reads them
        want_gpu = _allocating(grb, ctx, exact, monoid)
        want_host = _host(grb, exact, monoid)
        scale = float(np.sum(np.abs(exact))) if monoid == P else abs(want_host) if math.isfinite(want_host) else 1.0
        for _ in range(2):                     # two calls in a row on the shared scratch
            out.fill_(np.nan)
            rc = grb.grb_reduce_dense_noalloc(x, type_, n, monoid, out)
            assert rc == grb.GRB_SUCCESS
            torch.cuda.synchronize()
            got = float(out.item())
            assert _close(got, want_gpu, scale), (n, type_, monoid, got, want_gpu)
            assert _close(got, want_host, scale), (n, type_, monoid, got, want_host)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    grb, torch, _ = env
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = grb.grb_reduce_dense_noalloc(x, grb.GRB_FP64, grb.GRB_NOALLOC_MAX_N + 1, grb.GRB_MONOID_PLUS, out)
    assert rc == grb.GRB_INVALID_VALUE
    assert grb.grb_reduce_dense_noalloc(x, grb.GRB_BF16, 16, grb.GRB_MONOID_PLUS, out) == grb.GRB_INVALID_VALUE
    # still usable afterwards
    assert grb.grb_reduce_dense_noalloc(x, grb.GRB_FP64, 16, grb.GRB_MONOID_PLUS, out) == grb.GRB_SUCCESS
    torch.cuda.synchronize()
    assert out.item() == 0.0
