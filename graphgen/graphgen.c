/*
 * Seeded synthetic graph inputs: R-MAT and Erdos-Renyi edge lists.
 *
 * This module holds no PageRank or GraphBLAS arithmetic.  It turns a seed
 * into COO edge lists (int32 src/dst pairs) that both the CPU oracle and the
 * GPU library consume, so that the two sides see identical inputs.
 *
 * Random numbers come from a counter-based SplitMix64 stream: the 64-bit
 * finaliser of Steele, Lea and Flood ("Fast splittable pseudorandom number
 * generators", OOPSLA 2014) applied to key + (i+1)*GAMMA.  Every draw is a
 * pure function of (seed, stream, counter), so the edge list does not depend
 * on the number of threads and a numpy restatement gives bit-identical output.
 *
 * R-MAT follows Chakrabarti, Zhan and Faloutsos (SDM 2004): each of the
 * `scale` levels picks one quadrant with probabilities (a, b, c, 1-a-b-c);
 * quadrant (0,1) sets the destination bit, (1,0) the source bit.  Vertex
 * labels are then scrambled by a seeded bijection of [0, 2^scale), as the
 * Graph500 generator does, so that hubs are not clustered at low ids.
 */
#include <stdint.h>
#include <stddef.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of stream `stream` under `seed`. */
uint64_t gg_key(uint64_t seed, uint64_t stream) {
    return gg_mix64(gg_mix64(seed + GG_GAMMA) + (stream + 1) * GG_GAMMA);
}

/* Counter-based draw i of the stream with key `key`. */
uint64_t gg_draw(uint64_t key, uint64_t i) {
    return gg_mix64(key + (i + 1) * GG_GAMMA);
}

static inline double gg_unit(uint64_t u) {          /* [0, 1), 53 bits */
    return (double)(u >> 11) * (1.0 / 9007199254740992.0);
}

static inline uint64_t gg_below(uint64_t u, uint64_t n) { /* [0, n), n <= 2^32 */
    return ((u >> 32) * n) >> 32;
}

/* Streams used by the generators (fixed, documented constants). */
enum { GG_S_RMAT = 1, GG_S_PERM = 2, GG_S_ER_DANG = 3, GG_S_ER_SRC = 4, GG_S_ER_DST = 5 };

/* Seeded bijection of [0, 2^scale): four rounds of (odd multiply + add)
 * followed by a right xorshift, all modulo 2^scale.  Each step is invertible
 * on scale-bit words, so the composition is a permutation. */
uint64_t gg_scramble(uint64_t v, int scale, uint64_t seed) {
    if (scale <= 0) return 0;
    const uint64_t mask = (scale >= 64) ? ~0ULL : ((1ULL << scale) - 1ULL);
    const uint64_t key = gg_key(seed, GG_S_PERM);
    const int sh = (scale + 1) / 2;
    for (int r = 0; r < 4; ++r) {
        const uint64_t mul = gg_draw(key, 2 * (uint64_t)r) | 1ULL;
        const uint64_t add = gg_draw(key, 2 * (uint64_t)r + 1);
        v = (v * mul + add) & mask;
        v ^= v >> sh;
    }
    return v & mask;
}

/* R-MAT edge list: nedges directed pairs over 2^scale vertices. */
int gg_rmat_edges(int scale, int64_t nedges, double a, double b, double c,
                  uint64_t seed, int permute, int32_t* src, int32_t* dst) {
    if (scale < 1 || scale > 30 || nedges < 0 || !src || !dst) return -1;
    const uint64_t key = gg_key(seed, GG_S_RMAT);
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        uint64_t s = 0, d = 0;
        for (int l = 0; l < scale; ++l) {
            const double u = gg_unit(gg_draw(key, (uint64_t)e * (uint64_t)scale + (uint64_t)l));
            uint64_t sb, db;
            if (u < a)        { sb = 0; db = 0; }
            else if (u < ab)  { sb = 0; db = 1; }
            else if (u < abc) { sb = 1; db = 0; }
            else              { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        if (permute) { s = gg_scramble(s, scale, seed); d = gg_scramble(d, scale, seed); }
        src[e] = (int32_t)s;
        dst[e] = (int32_t)d;
    }
    return 0;
}

/* Dangling marker of the Erdos-Renyi generator: vertex v is forced to have
 * no out-edges with probability p_dangling. */
int gg_er_is_dangling(uint64_t seed, int64_t v, double p_dangling) {
    return gg_unit(gg_draw(gg_key(seed, GG_S_ER_DANG), (uint64_t)v)) < p_dangling;
}

/* Erdos-Renyi style directed edge list: nedges draws, source uniform over
 * non-dangling vertices (rejection, at most 64 tries, then a self loop that
 * the CSR build drops), destination uniform over all vertices. */
int gg_er_edges(int64_t n, int64_t nedges, double p_dangling, uint64_t seed,
                int32_t* src, int32_t* dst) {
    if (n < 1 || n > 2147483647LL || nedges < 0 || !src || !dst) return -1;
    const uint64_t kd = gg_key(seed, GG_S_ER_DANG);
    const uint64_t ks = gg_key(seed, GG_S_ER_SRC);
    const uint64_t kt = gg_key(seed, GG_S_ER_DST);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        const uint64_t t = gg_below(gg_draw(kt, (uint64_t)e), (uint64_t)n);
        uint64_t s = t;                       /* fallback: self loop */
        for (int tr = 0; tr < 64; ++tr) {
            const uint64_t cand = gg_below(gg_draw(ks, (uint64_t)e * 64ULL + (uint64_t)tr), (uint64_t)n);
            if (!(gg_unit(gg_draw(kd, cand)) < p_dangling)) { s = cand; break; }
        }
        src[e] = (int32_t)s;
        dst[e] = (int32_t)t;
    }
    return 0;
}

/* Raw 64-bit draws (used to check the numpy restatement). */
void gg_draws(uint64_t key, uint64_t start, int64_t count, uint64_t* out) {
    for (int64_t i = 0; i < count; ++i) out[i] = gg_draw(key, start + (uint64_t)i);
}
