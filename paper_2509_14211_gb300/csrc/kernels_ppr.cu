// Batched personalised PageRank: k queries iterate together as one sparse x
// dense product over A^T.  The paper's method runs one rank vector; here the
// same fused body (division folded into the previous epilogue, row sums,
// teleport, residual and dangling mass in the row epilogue) runs for many
// slots at once:
//
//   r_s' = (1 - d) v_s + d D_s / n + A^T w_s,   w_s = r_s ./ dvec,
//   D_s  = sum of r_s over vertices without out-edges,  res_s = |r_s - r_s'|_1
//
// with v_s uniform over slot s's seed set (dangling mass spread over all n
// vertices, so r_s is linear in v_s).
//
// Layout: r and w are [k-tile][n][32 V] FP32 -- lane l of a warp owns the V
// consecutive slots l V .. l V + V - 1 of its k-tile (V = 1, 2, 4: the vector
// width), and the values of one source vertex for a k-tile are 128 V
// contiguous bytes, so every gather is fully used cache lines and one warp
// instruction moves V slots per lane.  A warp walks the nonzeros of a
// 256-nonzero tile (the same tile plan as the single-vector kernels) one by
// one, all lanes adding their slots' values; row ends come from the row-end
// bitmap.  Rows split across tiles are finished by ppr_fixups_kernel from
// per-tile carries (it also takes the rows without nonzeros), and
// ppr_finish_kernel folds the per-CTA partials of every slot in a fixed
// order.  The three kernels of an iteration are separated by
// kernel boundaries (the caller captures iterations in a CUDA graph), so
// there are no device-side waits.
//
// Every slot's arithmetic (row sums in tile order, carries in tile order,
// fixed-order folds over a grid that depends neither on k nor on the vector
// width) is independent of the other slots, of its position and of the
// width: a query gives the same bits alone, in any batch and at any width.
#include "grb_device.cuh"

namespace grb {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int NW = PPR_BLOCK / 32;

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// per-warp partials of every slot: [warp][slot]
struct PprSmem {
    double res[NW][PPR_MAX_SLOTS];
    double dang[NW][PPR_MAX_SLOTS];
};

template <int V>
struct Vec;
template <>
struct Vec<1> {
    float x[1];
    __device__ __forceinline__ void ld(const float* p) { x[0] = __ldg(p); }
    __device__ __forceinline__ void ld_cs(const float* p) { x[0] = __ldcs(p); }
    __device__ __forceinline__ void ld_cg(const float* p) { x[0] = __ldcg(p); }
    __device__ __forceinline__ void st(float* p) const { *p = x[0]; }
    __device__ __forceinline__ void st_cs(float* p) const { __stcs(p, x[0]); }
};
template <>
struct Vec<2> {
    float x[2];
    __device__ __forceinline__ void set(float2 a) { x[0] = a.x; x[1] = a.y; }
    __device__ __forceinline__ void ld(const float* p) { set(__ldg(reinterpret_cast<const float2*>(p))); }
    __device__ __forceinline__ void ld_cs(const float* p) { set(__ldcs(reinterpret_cast<const float2*>(p))); }
    __device__ __forceinline__ void ld_cg(const float* p) { set(__ldcg(reinterpret_cast<const float2*>(p))); }
    __device__ __forceinline__ void st(float* p) const { *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]); }
    __device__ __forceinline__ void st_cs(float* p) const {
        __stcs(reinterpret_cast<float2*>(p), make_float2(x[0], x[1]));
    }
};
template <>
struct Vec<4> {
    float x[4];
    __device__ __forceinline__ void set(float4 a) {
        x[0] = a.x;
        x[1] = a.y;
        x[2] = a.z;
        x[3] = a.w;
    }
    __device__ __forceinline__ void ld(const float* p) { set(__ldg(reinterpret_cast<const float4*>(p))); }
    __device__ __forceinline__ void ld_cs(const float* p) { set(__ldcs(reinterpret_cast<const float4*>(p))); }
    __device__ __forceinline__ void ld_cg(const float* p) { set(__ldcg(reinterpret_cast<const float4*>(p))); }
    __device__ __forceinline__ void st(float* p) const {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
    __device__ __forceinline__ void st_cs(float* p) const {
        __stcs(reinterpret_cast<float4*>(p), make_float4(x[0], x[1], x[2], x[3]));
    }
};

// Per-lane state of the lane's V slots in the current k-tile.  It is read
// or updated only at row ends, so it lives in shared memory (one column per
// thread: conflict-free) and leaves the registers to the tile loop; only
// `any` (some slot of the lane is live) stays in a register.  The
// compensated sums run the same operations as in registers.
template <int V>
struct LaneStore {
    float tb[V][PPR_BLOCK];
    float rs[V][PPR_BLOCK], rc[V][PPR_BLOCK];   // residual: Kahan sum and compensation
    float ds[V][PPR_BLOCK], dc[V][PPR_BLOCK];   // dangling mass
    uint8_t act[V][PPR_BLOCK];
};

template <int V>
__device__ __forceinline__ LaneStore<V>& lane_store() {
    __shared__ LaneStore<V> st;
    return st;
}

template <int V>
struct Lane {
    bool any;
    __device__ __forceinline__ bool act(int v) const { return lane_store<V>().act[v][threadIdx.x] != 0; }
    __device__ __forceinline__ float tb(int v) const { return lane_store<V>().tb[v][threadIdx.x]; }
    __device__ __forceinline__ static void kahan(float& s_, float& c_, float x) {
        float s = s_, c = c_;
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
        s_ = s;
        c_ = c;
    }
    __device__ __forceinline__ void res_add(int v, float x) {
        LaneStore<V>& st = lane_store<V>();
        kahan(st.rs[v][threadIdx.x], st.rc[v][threadIdx.x], x);
    }
    __device__ __forceinline__ void dang_add(int v, float x) {
        LaneStore<V>& st = lane_store<V>();
        kahan(st.ds[v][threadIdx.x], st.dc[v][threadIdx.x], x);
    }
    __device__ __forceinline__ double res_value(int v) const {
        const LaneStore<V>& st = lane_store<V>();
        return (double)st.rs[v][threadIdx.x] - (double)st.rc[v][threadIdx.x];
    }
    __device__ __forceinline__ double dang_value(int v) const {
        const LaneStore<V>& st = lane_store<V>();
        return (double)st.ds[v][threadIdx.x] - (double)st.dc[v][threadIdx.x];
    }
};

__device__ __forceinline__ bool bit_of(const uint32_t* b, int i) { return (__ldg(b + (i >> 5)) >> (i & 31)) & 1u; }

// (1 - d) v_s[i] for this lane's slots.  The seed bitmap filters almost
// every row; on a hit the k-tile's seed rows (sorted) are binary-searched.
// The row is the same for the whole warp, so the control flow is uniform.
template <int V>
__device__ __forceinline__ void seed_terms_hit(const PprParams& p, int kt, int i, int lane, float (&sv)[V]) {
#pragma unroll
    for (int v = 0; v < V; ++v) sv[v] = 0.f;
    int lo = __ldg(p.seed_ptr + kt), hi = __ldg(p.seed_ptr + kt + 1);
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(p.seed_row + mid) < i) lo = mid + 1;
        else hi = mid;
    }
    for (int e = lo; e < end && __ldg(p.seed_row + e) == i; ++e) {
        const int s = __ldg(p.seed_lane + e);   // slot within the k-tile
        if (s / V == lane) {
            const float val = __ldg(p.seed_val + e);
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (s % V == v) sv[v] = val;
        }
    }
}

template <int V>
__device__ __forceinline__ void seed_terms(const PprParams& p, int kt, int i, int lane, float (&sv)[V]) {
    if (!bit_of(p.seedbits, i)) {
#pragma unroll
        for (int v = 0; v < V; ++v) sv[v] = 0.f;
        return;
    }
    seed_terms_hit<V>(p, kt, i, lane, sv);
}

// Epilogue of row i for this lane's slots: r' = (seed + d D / n) + sum, the
// next gather value, and the residual / dangling-mass terms.  A finished
// (inactive) slot writes nothing: its last iterate stays in the buffer the
// finish kernel recorded.
template <int V>
__device__ __forceinline__ void ppr_row(const PprParams& p, int kt, int i, const float (&sum)[V], int lane,
                                        Lane<V>& L) {
    float sv[V];
    seed_terms<V>(p, kt, i, lane, sv);   // uniform across the warp
    if (!L.any) return;
    const size_t o = ((size_t)kt * (size_t)p.nrows + (size_t)i) * (PPR_LANES * V) + (size_t)lane * V;
    Vec<V> rold, rn, wn;
    rold.ld_cs(p.r_old + o);
    const float dd = __ldg(p.dd + i);
    const bool sink = bit_of(p.sinkbits, i);
    bool all = true;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        rn.x[v] = (sv[v] + L.tb(v)) + sum[v];
        wn.x[v] = rn.x[v] / dd;
        all = all && L.act(v);
        if (L.act(v)) {
            L.res_add(v, fabsf(rold.x[v] - rn.x[v]));
            if (sink) L.dang_add(v, rn.x[v]);
        }
    }
    if (all) {
        rn.st_cs(p.r_new + o);
        wn.st(p.w_new + o);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (L.act(v)) {
                p.r_new[o + v] = rn.x[v];
                p.w_new[o + v] = wn.x[v];
            }
    }
}

// A row without nonzeros (r' = seed + teleport term): its memory inputs,
// loaded ahead so that several rows' loads are in flight together, and the
// epilogue itself -- the same arithmetic as ppr_row with a zero sum.
template <int V>
struct EmptyIn {
    Vec<V> rold;
    float dd;
    bool sink, seed;
};

template <int V>
__device__ __forceinline__ EmptyIn<V> empty_row_inputs(const PprParams& p, int kt, int i, int lane, const Lane<V>& L) {
    EmptyIn<V> a;
    a.seed = bit_of(p.seedbits, i);
    a.dd = 1.f;
    a.sink = false;
#pragma unroll
    for (int v = 0; v < V; ++v) a.rold.x[v] = 0.f;
    if (L.any) {
        const size_t o = ((size_t)kt * (size_t)p.nrows + (size_t)i) * (PPR_LANES * V) + (size_t)lane * V;
        a.rold.ld_cs(p.r_old + o);
        a.dd = __ldg(p.dd + i);
        a.sink = bit_of(p.sinkbits, i);
    }
    return a;
}

template <int V>
__device__ __forceinline__ void empty_row(const PprParams& p, int kt, int i, int lane, Lane<V>& L,
                                          const EmptyIn<V>& a) {
    float sv[V];
    if (a.seed) seed_terms_hit<V>(p, kt, i, lane, sv);   // uniform across the warp
    else {
#pragma unroll
        for (int v = 0; v < V; ++v) sv[v] = 0.f;
    }
    if (!L.any) return;
    const size_t o = ((size_t)kt * (size_t)p.nrows + (size_t)i) * (PPR_LANES * V) + (size_t)lane * V;
    Vec<V> rn, wn;
    bool all = true;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        rn.x[v] = (sv[v] + L.tb(v)) + 0.f;
        wn.x[v] = rn.x[v] / a.dd;
        all = all && L.act(v);
        if (L.act(v)) {
            L.res_add(v, fabsf(a.rold.x[v] - rn.x[v]));
            if (a.sink) L.dang_add(v, rn.x[v]);
        }
    }
    if (all) {
        rn.st_cs(p.r_new + o);
        wn.st(p.w_new + o);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (L.act(v)) {
                p.r_new[o + v] = rn.x[v];
                p.w_new[o + v] = wn.x[v];
            }
    }
}

template <int V>
__device__ __forceinline__ void lane_begin(const PprParams& p, int kt, int lane, Lane<V>& L) {
    const int base = kt * PPR_LANES * V + lane * V;
    L.any = false;
    LaneStore<V>& st = lane_store<V>();
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const bool a = __ldg(p.active + base + v) != 0;
        st.act[v][threadIdx.x] = a ? 1 : 0;
        st.tb[v][threadIdx.x] = __ldg(p.tele_base + base + v);
        st.rs[v][threadIdx.x] = 0.f;
        st.rc[v][threadIdx.x] = 0.f;
        st.ds[v][threadIdx.x] = 0.f;
        st.dc[v][threadIdx.x] = 0.f;
        L.any = L.any || a;
    }
}

template <int V>
__device__ __forceinline__ void lane_end(int kt, int lane, int warp, const Lane<V>& L, PprSmem& sm) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int s = kt * PPR_LANES * V + lane * V + v;
        sm.res[warp][s] = L.res_value(v);
        sm.dang[warp][s] = L.dang_value(v);
    }
}

// Per-CTA partials of every slot: the warps' accumulators folded in warp
// order.
__device__ __forceinline__ void flush_slot_partials(const PprParams& p, PprSmem& sm) {
    __syncthreads();
    const int S = p.kt * PPR_LANES * p.vw;
    for (int s = threadIdx.x; s < S; s += PPR_BLOCK) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < NW; ++w) {
            a += sm.res[w][s];
            b += sm.dang[w][s];
        }
        p.part[((size_t)blockIdx.x * S + s) * 2] = a;
        p.part[((size_t)blockIdx.x * S + s) * 2 + 1] = b;
    }
}

__device__ __forceinline__ void zero_smem(PprSmem& sm) {
    for (int q = threadIdx.x; q < NW * PPR_MAX_SLOTS; q += PPR_BLOCK) {
        (&sm.res[0][0])[q] = 0.0;
        (&sm.dang[0][0])[q] = 0.0;
    }
    __syncthreads();
}

// Phase A for one tile: the warp walks the tile's nonzeros; the lane adds its
// slots' values of each source vertex.  Loads are issued U nonzeros at a
// time (U V floats per lane in flight).
template <int V>
__device__ __forceinline__ void ppr_tile(const PprParams& p, int kt, int t, int lane, Lane<V>& L, bool all_live) {
    constexpr int U = V == 4 ? 4 : 8;
    constexpr int W = PPR_LANES * V;
    const uint32_t meta = __ldg(p.tile_meta + t);
    const int rfirst = (int)(meta & 0x7fffffffu);
    const int x_lo = (int)(meta >> 31);
    const int kl = t * PR_NZTILE + lane * PR_NZLANE;
    const int4* cp = reinterpret_cast<const int4*>(p.col_idx + kl);
    const int4 ca = __ldcs(cp), cb = __ldcs(cp + 1);
    const uint32_t myf = (__ldcs(p.rowend_bits + (kl >> 5)) >> (kl & 31)) & 0xffu;
    const int nvalid = min(max(p.nnz - t * PR_NZTILE, 0), PR_NZTILE);
    const int pre_i = rfirst + lane < p.n_ne ? __ldg(p.ne_rows + rfirst + lane) : 0;
    const float* Wb = p.w_old + (size_t)kt * (size_t)p.nrows * W + (size_t)lane * V;
    const size_t tslot = ((size_t)kt * p.ntiles + t) * W + (size_t)lane * V;
    const bool dense = all_live && nvalid == PR_NZTILE;
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    int r = 0;   // rows of the tile finished so far (the same in every lane)
    for (int src = 0; src < 32; ++src) {
        if (src * PR_NZLANE >= nvalid) break;
        // the 8 column indices lane `src` loaded, in every lane
        int c[PR_NZLANE];
        c[0] = __shfl_sync(FULL, ca.x, src);
        c[1] = __shfl_sync(FULL, ca.y, src);
        c[2] = __shfl_sync(FULL, ca.z, src);
        c[3] = __shfl_sync(FULL, ca.w, src);
        c[4] = __shfl_sync(FULL, cb.x, src);
        c[5] = __shfl_sync(FULL, cb.y, src);
        c[6] = __shfl_sync(FULL, cb.z, src);
        c[7] = __shfl_sync(FULL, cb.w, src);
#ifdef GRB_CHECK_BOUNDS
#pragma unroll
        for (int q = 0; q < PR_NZLANE; ++q) c[q] = GRB_CHECKED(c[q], p.nrows, p.status, BOUNDS_COLUMN);
#endif
        const uint32_t f = __shfl_sync(FULL, myf, src);
#pragma unroll
        for (int q0 = 0; q0 < PR_NZLANE; q0 += U) {
            Vec<V> g[U];
            if (dense) {
                // a whole tile and every lane with a live slot: no per-load test
#pragma unroll
                for (int q = 0; q < U; ++q) g[q].ld(Wb + (size_t)c[q0 + q] * W);
            } else {
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    // lanes whose slots are all finished or empty load nothing
                    // (in a partly filled k-tile the line traffic shrinks)
                    if (L.any && src * PR_NZLANE + q0 + q < nvalid) {
                        g[q].ld(Wb + (size_t)c[q0 + q] * W);
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) g[q].x[v] = 0.f;
                    }
                }
            }
            const uint32_t fq = (f >> q0) & ((1u << U) - 1u);
            if (fq == 0u) {
                // no row ends among these U nonzeros (the same in every lane)
#pragma unroll
                for (int q = 0; q < U; ++q)
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] += g[q].x[v];
                continue;
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] += g[q].x[v];
                if ((fq >> q) & 1u) {
                    if (r == 0 && x_lo) {
                        Vec<V> a;
#pragma unroll
                        for (int v = 0; v < V; ++v) a.x[v] = acc[v];
                        a.st(p.first + tslot);   // a row begun in an earlier tile: phase B
                    } else {
                        const int i = r < 32 ? __shfl_sync(FULL, pre_i, r) : __ldg(p.ne_rows + rfirst + r);
                        ppr_row<V>(p, kt, i, acc, lane, L);
                    }
                    ++r;
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] = 0.f;
                }
            }
        }
    }
    Vec<V> a;
#pragma unroll
    for (int v = 0; v < V; ++v) a.x[v] = acc[v];
    a.st(p.agg + tslot);   // the row still open at the tile's end
}

// Phase A: the warp tiles, k-tile by k-tile (so the warps of the GPU share
// one k-tile of w in L2 at a time); the rows without nonzeros go to phase B.
// Tile t goes to the same warp in every k-tile, so every slot sees the same
// summation order.
// The V = 4 tile loop keeps 16 gathered floats, 4 sums and 8 compensated
// accumulators per lane: it gets the registers of one CTA per SM.
template <int V>
__global__ void __launch_bounds__(PPR_BLOCK, (V == 4 ? 1 : 2)) ppr_tiles_kernel(const __grid_constant__ PprParams p) {
    __shared__ PprSmem sm;
    zero_smem(sm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * NW;
    const int w0 = blockIdx.x * NW + warp;
    for (int kt = 0; kt < p.kt; ++kt) {
        Lane<V> L;
        lane_begin<V>(p, kt, lane, L);
        // a k-tile without an active slot is skipped (the same decision in
        // every warp: all read the same flags)
        if (!__any_sync(FULL, L.any)) continue;
        const bool all_live = __all_sync(FULL, L.any);   // every lane has a live slot
        for (int t = w0; t < p.ntiles; t += nwarps) ppr_tile<V>(p, kt, t, lane, L, all_live);
        lane_end<V>(kt, lane, warp, L, sm);
    }
    flush_slot_partials(p, sm);
}

// Phase B: rows split across tiles, one warp per (k-tile, tile) with a
// fixup: the carries of the earlier tiles in tile order, then this tile's
// part; then the rows without nonzeros.
template <int V>
__global__ void __launch_bounds__(PPR_BLOCK, (V == 4 ? 1 : 2)) ppr_fixups_kernel(const __grid_constant__ PprParams p) {
    __shared__ PprSmem sm;
    zero_smem(sm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * NW;
    constexpr int W = PPR_LANES * V;
    for (int kt = 0; kt < p.kt; ++kt) {
        Lane<V> L;
        lane_begin<V>(p, kt, lane, L);
        if (!__any_sync(FULL, L.any)) continue;
        for (int t = blockIdx.x * NW + warp; t < p.ntiles; t += nwarps) {
            const FixDesc f = p.fix[t];
            if (f.row < 0) continue;
            const size_t base = (size_t)kt * p.ntiles * W + (size_t)lane * V;
            float sum[V];
#pragma unroll
            for (int v = 0; v < V; ++v) sum[v] = 0.f;
            for (int tt = f.ts; tt < t; ++tt) {
                Vec<V> a;
                a.ld_cg(p.agg + base + (size_t)tt * W);
#pragma unroll
                for (int v = 0; v < V; ++v) sum[v] += a.x[v];
            }
            Vec<V> a;
            a.ld_cg(p.first + base + (size_t)t * W);
#pragma unroll
            for (int v = 0; v < V; ++v) sum[v] += a.x[v];
            ppr_row<V>(p, kt, f.row, sum, lane, L);
        }
        // rows without nonzeros: the epilogue with an empty sum, four rows
        // per warp per step -- their index loads, then their input loads,
        // issued together (the tile kernel's registers stay with its loop)
        const int w0 = blockIdx.x * NW + warp;
        for (int e0 = w0; e0 < p.n_empty; e0 += 4 * nwarps) {
            int i[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * nwarps;
                i[u] = e < p.n_empty ? __ldg(p.empty_rows + e) : -1;
            }
            EmptyIn<V> in[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i[u] >= 0) in[u] = empty_row_inputs<V>(p, kt, i[u], lane, L);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i[u] >= 0) empty_row<V>(p, kt, i[u], lane, L, in[u]);
        }
        lane_end<V>(kt, lane, warp, L, sm);
    }
    flush_slot_partials(p, sm);
}

// One warp per slot: fold the partials of both phases in a fixed order
// (lane l takes CTAs l, l+32, ...; then a fixed shuffle tree), count the
// body, test the slot's loop condition and set its next teleport term.
__global__ void ppr_finish_kernel(const __grid_constant__ PprFinish f) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (s >= f.slots) return;
    if (!f.active[s]) return;   // uniform across the warp
    double R = 0.0, D = 0.0;
    for (int c = lane; c < f.grid_a; c += 32) {
        R += f.part_a[((size_t)c * f.slots + s) * 2];
        D += f.part_a[((size_t)c * f.slots + s) * 2 + 1];
    }
    for (int c = lane; c < f.grid_b; c += 32) {
        R += f.part_b[((size_t)c * f.slots + s) * 2];
        D += f.part_b[((size_t)c * f.slots + s) * 2 + 1];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        R += __shfl_xor_sync(FULL, R, off);
        D += __shfl_xor_sync(FULL, D, off);
    }
    if (lane == 0) {
        const int32_t k = f.iters[s] + 1;
        f.iters[s] = k;
        f.resid[s] = R;
        f.tele_base[s] = (float)(f.damping * D / (double)f.n);
        if (!(R > f.tol[s]) || k >= f.itermax[s]) {
            f.active[s] = 0;
            f.final_buf[s] = f.out_buf;   // where this body left the slot's rank
        }
    }
}

// Zero the queued slots' columns of the current rank / gather buffers.  A
// block covers rows in groups of 2^lg threads (2^lg >= np, the queued slots,
// at most PPR_MAX_SLOTS): thread t takes slot t mod 2^lg of row t >> lg, so
// the queued slots of one row are adjacent threads (their writes share the
// row's cache lines) and no thread divides by np.
__global__ void ppr_init_zero_kernel(const __grid_constant__ PprInitBatch a, int lg) {
    __shared__ long long col[PPR_MAX_SLOTS];   // queued slot k: its k-tile's base + its lane
    for (int k = threadIdx.x; k < a.np; k += blockDim.x) {
        const int s = a.slots[k];
        col[k] = (long long)(s / a.width) * a.nrows * a.width + (s % a.width);
    }
    __syncthreads();
    const int k = threadIdx.x & ((1 << lg) - 1);
    if (k >= a.np) return;
    const int rows_per_pass = blockDim.x >> lg;
    const long long c = col[k];
    for (long long i = (long long)blockIdx.x * rows_per_pass + (threadIdx.x >> lg); i < a.nrows;
         i += (long long)gridDim.x * rows_per_pass) {
        const size_t o = (size_t)(c + i * a.width);
        a.r[o] = 0.f;
        a.w[o] = 0.f;
    }
}

// One CTA per queued slot: its seeds, its first teleport term and its state.
__global__ void ppr_init_seed_kernel(const __grid_constant__ PprInitBatch a) {
    const int k = blockIdx.x;
    const int s = a.slots[k];
    const int kt = s / a.width, l = s % a.width;
    const int b = a.seed_off[k], e = a.seed_off[k + 1];
    const float r0 = a.r0[k];
    for (int q = b + threadIdx.x; q < e; q += blockDim.x) {
        const int i = a.seeds[q];
        const size_t o = ((size_t)kt * a.nrows + i) * a.width + l;
        a.r[o] = r0;
        a.w[o] = r0 / a.dd[i];
    }
    if (threadIdx.x == 0) {
        // dangling mass of the start vector, in seed order
        double D = 0.0;
        for (int q = b; q < e; ++q)
            if ((a.sinkbits[a.seeds[q] >> 5] >> (a.seeds[q] & 31)) & 1u) D += (double)r0;
        a.tele_base[s] = (float)(a.damping * D / (double)a.nrows);
        a.active[s] = a.act[k];
        a.iters[s] = 0;
        a.itermax_out[s] = a.itermax[k];
        a.tol_out[s] = a.tol[k];
        a.resid[s] = 1.0;
        a.final_buf[s] = a.cur;
    }
}

__global__ void ppr_seedbits_kernel(int32_t nseeds, const int32_t* rows, uint32_t* bits) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nseeds; q += gridDim.x * blockDim.x)
        atomicOr(bits + (rows[q] >> 5), 1u << (rows[q] & 31));
}

__global__ void ppr_extract_kernel(int32_t n, const float* r, int32_t width, int32_t slot, float* out) {
    const int kt = slot / width, l = slot % width;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = r[((size_t)kt * n + i) * width + l];
}

__global__ void ppr_divisor_kernel(int32_t n, const int32_t* deg, double damping, float* dd, uint32_t* sinkbits) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double a = (double)deg[i] / damping, b = 1.0 / damping;
        dd[i] = (float)(a > b ? a : b);
    }
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < (n + 31) / 32; w += gridDim.x * blockDim.x) {
        uint32_t b = 0;
        for (int q = 0; q < 32; ++q) {
            const int i = w * 32 + q;
            if (i < n && deg[i] == 0) b |= 1u << q;
        }
        sinkbits[w] = b;
    }
}

inline int grid_1d(int64_t n, int block = 256) {
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

bool valid_vw(int32_t vw) { return vw == 1 || vw == 2 || vw == 4; }

}  // namespace

cudaError_t launch_ppr_tiles(cudaStream_t st, const PprParams& p, int grid) {
    if (!valid_vw(p.vw) || p.kt < 1 || p.kt * PPR_LANES * p.vw > PPR_MAX_SLOTS) return cudaErrorInvalidValue;
    switch (p.vw) {
        case 1: ppr_tiles_kernel<1><<<grid, PPR_BLOCK, 0, st>>>(p); break;
        case 2: ppr_tiles_kernel<2><<<grid, PPR_BLOCK, 0, st>>>(p); break;
        default: ppr_tiles_kernel<4><<<grid, PPR_BLOCK, 0, st>>>(p); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ppr_fixups(cudaStream_t st, const PprParams& p, int grid) {
    if (!valid_vw(p.vw) || p.kt < 1 || p.kt * PPR_LANES * p.vw > PPR_MAX_SLOTS) return cudaErrorInvalidValue;
    switch (p.vw) {
        case 1: ppr_fixups_kernel<1><<<grid, PPR_BLOCK, 0, st>>>(p); break;
        case 2: ppr_fixups_kernel<2><<<grid, PPR_BLOCK, 0, st>>>(p); break;
        default: ppr_fixups_kernel<4><<<grid, PPR_BLOCK, 0, st>>>(p); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ppr_finish(cudaStream_t st, const PprFinish& f) {
    const int per_block = 8;
    ppr_finish_kernel<<<(f.slots + per_block - 1) / per_block, 32 * per_block, 0, st>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_ppr_init_batch(cudaStream_t st, const PprInitBatch& a) {
    if (a.np <= 0) return cudaSuccess;
    if (a.np > PPR_MAX_SLOTS) return cudaErrorInvalidValue;   // queued entries are distinct slots
    int lg = 0;
    while ((1 << lg) < a.np) ++lg;
    ppr_init_zero_kernel<<<grid_1d((int64_t)a.nrows << lg), 256, 0, st>>>(a, lg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ppr_init_seed_kernel<<<a.np, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ppr_seedbits(cudaStream_t st, int32_t nseeds, const int32_t* rows, uint32_t* bits, int64_t nwords) {
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (size_t)nwords, st);
    if (e != cudaSuccess || nseeds <= 0) return e;
    ppr_seedbits_kernel<<<grid_1d(nseeds), 256, 0, st>>>(nseeds, rows, bits);
    return cudaGetLastError();
}

cudaError_t launch_ppr_extract(cudaStream_t st, int32_t n, const float* r, int32_t width, int32_t slot, float* out) {
    ppr_extract_kernel<<<grid_1d(n), 256, 0, st>>>(n, r, width, slot, out);
    return cudaGetLastError();
}

cudaError_t launch_ppr_divisor(cudaStream_t st, int32_t n, const int32_t* deg, double damping, float* dd,
                               uint32_t* sinkbits) {
    ppr_divisor_kernel<<<grid_1d(n), 256, 0, st>>>(n, deg, damping, dd, sinkbits);
    return cudaGetLastError();
}

}  // namespace grb
