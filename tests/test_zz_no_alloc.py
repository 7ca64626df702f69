"""The allocation-free reduction (grb_reduce_dense_noalloc), for callers that
cannot allocate device memory when they reduce -- inside a stream capture,
under a host framework that owns the memory budget, or on a path that cannot
pay for cudaMalloc's synchronisation.  Its scratch is a fixed device array,
so this file checks it against the allocating entry point (grb_reduce on a
vector) on consecutive calls that reuse that array.  Collected last so that a
run stopping at the first failure has run everything else first."""
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


def _reference(grb, ctx, data, monoid):
    v = grb.grb_vector_new(ctx, grb.GRB_FP64, len(data))
    grb.grb_vector_build(v, np.arange(len(data), dtype=np.int32), data.astype(np.float64))
    s = grb.grb_scalar_new(ctx, grb.GRB_FP64)
    grb.grb_reduce(s, None, monoid, v)
    val = grb.grb_scalar_get(s)
    grb.grb_free(v)
    grb.grb_free(s)
    return val


def test_noalloc_matches_grb_reduce_on_consecutive_calls(env):
    grb, torch, ctx = env
    rng = np.random.default_rng(42)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cases = [(3_000_017, grb.GRB_FP64, grb.GRB_MONOID_PLUS), (77, grb.GRB_FP64, grb.GRB_MONOID_PLUS),
             (1_000_000, grb.GRB_FP32, grb.GRB_MONOID_MAX), (grb.GRB_NOALLOC_MAX_N, grb.GRB_FP32, grb.GRB_MONOID_PLUS)]
    for n, type_, monoid in cases:
        data = rng.standard_normal(n)
        dt = torch.float64 if type_ == grb.GRB_FP64 else torch.float32
        x = torch.tensor(data, dtype=dt, device="cuda")
        for _ in range(2):                     # two calls in a row on the shared scratch
            out.fill_(np.nan)
            rc = grb.grb_reduce_dense_noalloc(x, type_, n, monoid, out)
            assert rc == grb.GRB_SUCCESS
            torch.cuda.synchronize()
            got = float(out.item())
            want = _reference(grb, ctx, x.double().cpu().numpy(), monoid)
            assert abs(got - want) <= 1e-12 * max(1.0, float(np.sum(np.abs(data)))), (n, got, want)


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
