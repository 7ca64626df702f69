"""The shared input generator against its numpy restatement and its
published definitions (SplitMix64; R-MAT quadrant probabilities)."""
import numpy as np
import pytest

import graphgen


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0 (state advanced by GAMMA before mixing) yields
    # 0xE220A8397B1DCDAF as its first output (Steele, Lea, Flood 2014;
    # the same value is the first output of Java's SplittableRandom(0)).
    z = graphgen.numpy_mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("scale,seed,permute", [(5, 0, True), (9, 3, True), (8, 1, False)])
def test_rmat_c_matches_numpy(scale, seed, permute):
    m = (1 << scale) * 8
    s, d = graphgen.rmat_edges(scale, 8, seed=seed, permute=permute)
    s2, d2 = graphgen.numpy_rmat_edges(scale, m, seed, permute=permute)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)


def test_draws_match():
    k = graphgen.numpy_key(11, 4)
    assert np.array_equal(graphgen.draws(11, 4, 100, 50), graphgen.numpy_draw(k, np.arange(100, 150)))


def test_scramble_is_a_permutation():
    for scale in (1, 2, 7, 12):
        v = np.arange(1 << scale, dtype=np.uint64)
        p = graphgen.numpy_scramble(v, scale, seed=5)
        assert np.array_equal(np.sort(p), v)


def test_rmat_quadrant_frequencies():
    # unpermuted, the top bit of (src, dst) is the first level's quadrant
    scale = 10
    s, d = graphgen.rmat_edges(scale, 16, seed=2, permute=False)
    top_s, top_d = s >> (scale - 1), d >> (scale - 1)
    m = len(s)
    freq = [np.mean((top_s == a) & (top_d == b)) for a, b in ((0, 0), (0, 1), (1, 0), (1, 1))]
    for f, p in zip(freq, (0.57, 0.19, 0.19, 0.05)):
        assert abs(f - p) < 5 * np.sqrt(p * (1 - p) / m)


def test_er_dangling_vertices_have_no_out_edges():
    n = 1 << 12
    s, d = graphgen.er_edges(n, 16, p_dangling=0.02, seed=2)
    lib = graphgen._load()
    dang = np.array([lib.gg_er_is_dangling(2, v, 0.02) for v in range(n)], dtype=bool)
    assert 0.01 < dang.mean() < 0.03
    ok = s != d
    assert not np.any(dang[s[ok]])
    assert s.min() >= 0 and s.max() < n and d.min() >= 0 and d.max() < n
