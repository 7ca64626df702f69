// Fused PageRank iteration over the rows of A^T (§IV pagerank_gap body):
//
//     w = t ./ d ;  s = A^T (+.second) w ;  r = rt + s ;  rdiff = sum |t - r|
//
// as ONE pass over the CSR arrays: the element-wise division is folded into
// the gather (or into the previous iteration's epilogue, which writes
// w_next = r / d beside r), the mxv row sums, the teleport add, the residual
// and the dangling-mass reductions all happen in the row epilogue.  This is
// the GPU form of the single fused loop the paper generates at `wait`
// (§III-B, Fig. "materialize"), extended across the SpMV.
//
// Work decomposition: the nonzeros are cut into warp tiles of PR_NZTILE
// consecutive entries (PR_NZLANE per lane, loaded as two 16-byte pieces), so
// every warp gets the same gather work whatever the row lengths (R-MAT
// in-degrees range from 0 to ~10^5).  A bitmap marks the last nonzero of
// every row, so a lane finds its row boundaries with a popc and a shift;
// rows are numbered in the compressed list of non-empty rows, and the empty
// rows (~40% of an R-MAT graph) get their epilogue in a separate streaming
// loop.  Warps are independent: per-lane segmented sums go to the warp's
// shared-memory slice, and a warp-wide segmented scan joins rows split across
// lanes (ballots number the rows and mark where segments start; only the
// carried values are shuffled).  Rows split across tiles are finished from
// per-tile carries (phase A writes them, phase B adds them up in a fixed
// order): after a grid barrier, or -- in the pipelined persistent loop --
// by look-back over carries the other warps published, each tagged with the
// body, so that a body has a single grid barrier.  Every wait is bounded.
// All reductions have a fixed order, so results are bit-reproducible.
//
// Three epilogue flavours, compiled separately so that the loop's per-row
// code carries no run-time configuration checks: LEAN (the PageRank loop:
// scalar teleport base, residual and next gather value always produced, no
// presence array), MG (a batch of independent graphs: per-graph teleport
// and loop state, per-row residual and dangling terms) and the general one
// the planner uses for other fused groups and for the unfused mxv.
#include <climits>

#include "grb_device.cuh"

namespace grb {

namespace {

constexpr int NWARP = PR_BLOCK / 32;
constexpr uint32_t FULLMASK = 0xffffffffu;

// Minimum resident CTAs per SM requested from the register allocator.
#ifndef PR_MINBLOCKS
#define PR_MINBLOCKS 4
#endif
// 1: load the use-once matrix arrays with evict-first (streaming) hints.
#ifndef PR_STREAM_HINTS
#define PR_STREAM_HINTS 1
#endif
// 1: ask for the largest L1 / smallest shared-memory carveout.
#ifndef PR_MAX_L1
#define PR_MAX_L1 0
#endif

template <class X>
__device__ __forceinline__ X ld_stream(const X* p) {
#if PR_STREAM_HINTS
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

template <class T>
struct WarpSmem {
    T rowsum[PR_NZTILE];   // sums of the rows ending in the warp's current tile
};

template <class T, int NW = NWARP>
struct Smem {
    WarpSmem<T> w[NW];
    double red[NW];
    double red2[NW];
    double bc[2];
    int ok;
};

// Loads of vectors that a kernel also writes.  NC: the data was written by
// an earlier launch, so the read-only path is safe.  Otherwise (persistent
// kernel) the data was written by other CTAs before a grid barrier; a plain
// L1-cached load is still correct because the barrier's gpu-scope acquire
// (ld.acquire + fence) orders it after those writes, and the hardware
// invalidates the SM's L1 on such an acquire.
template <class G, bool NC>
__device__ __forceinline__ float gload_f(const G* p, int j);

template <>
__device__ __forceinline__ float gload_f<float, true>(const float* p, int j) { return __ldg(p + j); }
template <>
__device__ __forceinline__ float gload_f<float, false>(const float* p, int j) { return __ldca(p + j); }
template <>
__device__ __forceinline__ float gload_f<__nv_bfloat16, true>(const __nv_bfloat16* p, int j) {
    const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + j);
    return __uint_as_float(((uint32_t)b) << 16);
}
template <>
__device__ __forceinline__ float gload_f<__nv_bfloat16, false>(const __nv_bfloat16* p, int j) {
    const unsigned short b = __ldca(reinterpret_cast<const unsigned short*>(p) + j);
    return __uint_as_float(((uint32_t)b) << 16);
}

template <class T, bool NC>
__device__ __forceinline__ T tload(const T* p, int j) {
    if (NC) return __ldg(p + j);
    return __ldca(p + j);
}

template <class G>
__device__ __forceinline__ void gstore(G* p, int i, float x);
template <>
__device__ __forceinline__ void gstore<float>(float* p, int i, float x) { p[i] = x; }
template <>
__device__ __forceinline__ void gstore<__nv_bfloat16>(__nv_bfloat16* p, int i, float x) { p[i] = __float2bfloat16_rn(x); }

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

// Bounded grid-wide barrier (all CTAs of a cooperative launch).  Returns
// false when a wait ran out (status set); callers then leave the kernel.
__device__ bool grid_sync(SyncWords* s, int32_t* status, int64_t spin_limit, uint32_t expected, int* ok_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t gen = ld_acquire_u32(&s->bar_gen);
        __threadfence();
        const uint32_t arrived = atomicAdd(&s->bar_count, 1u);
        if (arrived == expected - 1) {
            atomicExch(&s->bar_count, 0u);
            __threadfence();
            st_release_u32(&s->bar_gen, gen + 1);
        } else {
            int64_t spins = 0;
            while (ld_acquire_u32(&s->bar_gen) == gen) {
                if (++spins > spin_limit || ((spins & 255) == 0 && status && *(volatile int32_t*)status != 0)) {
                    set_status(status, (int32_t)GRB_DEVICE_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (ok && status && *(volatile int32_t*)status != 0) ok = 0;
        *ok_sh = ok;
    }
    __syncthreads();
    return *ok_sh != 0;
}

// Deterministic fold of the per-CTA partials part[0..n) (pairs of doubles).
template <class T, int BLK = PR_BLOCK>
__device__ __forceinline__ void reduce_parts(const double* part, int n, double& a, double& b, Smem<T, BLK / 32>& sm) {
    double x = 0.0, y = 0.0;
    for (int c = threadIdx.x; c < n; c += BLK) {
        x += ld_relaxed_f64(part + 2 * c);
        y += ld_relaxed_f64(part + 2 * c + 1);
    }
    x = block_sum_d<BLK>(x, sm.red);
    y = block_sum_d<BLK>(y, sm.red2);
    if (threadIdx.x == 0) { sm.bc[0] = x; sm.bc[1] = y; }
    __syncthreads();
    a = sm.bc[0];
    b = sm.bc[1];
    __syncthreads();
}

// Per-lane running sums of the residual and the dangling mass (nonnegative
// terms).  GB300's FP64 pipe is narrow, so for FP32 ranks each lane keeps its
// sum as an unevaluated pair hi + lo of FP32 numbers ("double-float"): every
// addition takes its exact rounding error from Knuth's TwoSum and folds it,
// with the old low part, back in through Dekker's FastTwoSum (|s| >= |e|
// holds for nonnegative terms).  That carries about 48 significant bits, so a
// lane's sum of n terms is off by at most ~n * 2^-47 relative -- FP64-grade,
// independent of the magnitude spread -- and hi + lo goes to the FP64
// cross-thread reduction once per body.  FP64 ranks sum in FP64.
template <class T>
struct Acc {
    double s = 0.0;
    __device__ __forceinline__ void add(T x) { s += (double)x; }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bv = s - hi;
        const float e = ((hi - (s - bv)) + (x - bv)) + lo;
        hi = s + e;
        lo = e - (hi - s);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Per-launch view of the gather / epilogue buffers.
template <class T, class G>
struct TileIO {
    const G* w;        // G_W gather source
    const float* w32;  // FP32 gather source after the mixed-precision switch
    const T* t;        // G_TD numerator
    const T* d;        // G_TD divisor
    const T* r_old;    // residual reference
    T* out;
    uint8_t* out_present;
    G* w_next;
    float* w32_next;
    T tele;            // base value when it comes from a scalar
    int tele_scalar;   // 1: base = tele, 0: base from p.base
    int phase32;       // mixed precision: gather from w32
    const G* hot;      // shared-memory copy of w[0, hot_n) (HOT kernels)
    int hot_n;
    uint32_t epoch;    // single-pass bodies: the body's tag on published tile carries
};

// Epilogue kinds: the general one (any fused group), the PageRank loop body
// (scalar teleport, residual and next gather value always produced), the
// loop body of a batch of independent graphs (per-graph teleport and loop
// state, per-row residual / dangling terms folded per graph later), and the
// PageRank loop body of one personalised query (the loop body plus the
// query's teleport term (1-d)/|S| on its seed rows).
enum : int { EPI_GEN = 0, EPI_LEAN = 1, EPI_MG = 2, EPI_PERS = 3 };

// Epilogue inputs of one row, loaded ahead of use.
template <class T, int EPI>
struct RowIn {
    T rold;
    T dd;
    uint32_t sinkword;
};
template <class T>
struct RowIn<T, EPI_PERS> {
    T rold;
    T dd;
    uint32_t sinkword;
    uint32_t seedword;
};

template <class T, class G, bool NC, int EPI>
__device__ __forceinline__ RowIn<T, EPI> row_inputs(const PrParams& p, const TileIO<T, G>& io, int i) {
    constexpr bool LEAN = EPI != EPI_GEN;
    RowIn<T, EPI> in;
    in.rold = (T)0;
    in.dd = (T)1;
    in.sinkword = 0;
    if (LEAN || p.want_resid) in.rold = tload<T, NC>(io.r_old, i);
    if (LEAN || io.w_next || io.w32_next) in.dd = __ldg(reinterpret_cast<const T*>(p.dd) + i);
    if (p.want_dang) in.sinkword = __ldg(p.sinkbits + (i >> 5));
    if constexpr (EPI == EPI_PERS) in.seedword = __ldg(p.pers_bits + (i >> 5));
    return in;
}

// Everything a finished row produces: the output value, its presence, the
// next gather value, and its residual / dangling-mass contributions.
template <class T, class G, int EPI>
__device__ __forceinline__ void row_epilogue(const PrParams& p, const TileIO<T, G>& io, int i, T s, bool nonempty,
                                             const RowIn<T, EPI>& in, Acc<T>& resid, Acc<T>& dang) {
    T v;
    if constexpr (EPI == EPI_MG) {
        // row i of graph g: nothing once g's loop has ended (its rank stays
        // in the buffer its last body wrote)
        const int g = __ldg(p.graph_of + i);
        if (!__ldg(p.g_active + g)) return;
        const T tg = (T)__ldg(p.g_tele + g);
        v = nonempty ? tg + s : tg;
        io.out[i] = v;
        gstore<G>(io.w_next, i, (float)(v / in.dd));
        p.row_res[i] = (float)abs_c<T>(in.rold - v);
        p.row_dang[i] = ((in.sinkword >> (i & 31)) & 1u) ? (float)v : 0.f;
        return;
    }
    if constexpr (EPI == EPI_PERS) {
        // r_i = ((1-d)/|S| [i in S] + d D / n) + s_i
        const T base = ((in.seedword >> (i & 31)) & 1u) ? (T)p.pers_val + io.tele : io.tele;
        v = nonempty ? base + s : base;
        io.out[i] = v;
        resid.add(abs_c<T>(in.rold - v));
        if ((in.sinkword >> (i & 31)) & 1u) dang.add(v);
        gstore<G>(io.w_next, i, (float)(v / in.dd));
        return;
    }
    if (EPI == EPI_LEAN) {
        v = nonempty ? io.tele + s : io.tele;
        io.out[i] = v;
        resid.add(abs_c<T>(in.rold - v));
        if (p.want_dang && ((in.sinkword >> (i & 31)) & 1u)) dang.add(v);
        const T q = v / in.dd;
        if (sizeof(G) == 2 && io.phase32) io.w32_next[i] = (float)q;   // only BF16 gathers switch
        else if constexpr (sizeof(T) == 8) reinterpret_cast<double*>(io.w_next)[i] = (double)q;
        else gstore<G>(io.w_next, i, (float)q);
        return;
    }
    bool has;
    if (p.has_base) {
        T b = (T)0;
        bool bh = true;
        if (io.tele_scalar) b = io.tele;
        else bh = vin_get<T>(p.base, i, b);
        if (nonempty) { v = bh ? b + s : s; has = true; }
        else { v = b; has = bh; }
    } else {
        v = s;
        has = nonempty;
    }
    if (!has) v = (T)0;
    io.out[i] = v;
    if (io.out_present) io.out_present[i] = has ? 1 : 0;
    if (p.want_resid) resid.add(abs_c<T>(in.rold - v));
    if (p.want_dang && ((in.sinkword >> (i & 31)) & 1u)) dang.add(v);
    if (io.w_next || io.w32_next) {
        const T q = v / in.dd;
        if (io.w32_next) io.w32_next[i] = (float)q;
        else if constexpr (sizeof(T) == 8) reinterpret_cast<double*>(io.w_next)[i] = (double)q;
        else gstore<G>(io.w_next, i, (float)q);
    }
}

template <class T, class G, int GMODE, bool NC, bool HOT = false>
__device__ __forceinline__ T gather(const PrParams& p, const TileIO<T, G>& io, int j) {
    j = GRB_CHECKED(j, p.ncols, p.status, BOUNDS_COLUMN);
    if constexpr (HOT) {
        // the hot copy in shared memory, or L2 (bypassing L1: the columns
        // past the copy are rarely reused soon enough for L1 to help); two
        // predicated loads, no branch
        float a = 0.f, b = 0.f;
        if (j < io.hot_n) a = (float)io.hot[j];
        else b = (float)__ldcg(io.w + j);
        return (T)(a + b);
    }
    if (GMODE == G_W) {
        if (sizeof(G) == 2 && io.phase32) return (T)gload_f<float, NC>(io.w32, j);
        if constexpr (sizeof(T) == 8) return tload<T, NC>(reinterpret_cast<const T*>(io.w), j);
        else return (T)gload_f<G, NC>(io.w, j);
    } else if (GMODE == G_TD) {
        return tload<T, NC>(io.t, j) / tload<T, NC>(io.d, j);
    }
    return (T)p.g_iso;
}

// Phase A for one warp tile (nonzeros [t*PR_NZTILE, (t+1)*PR_NZTILE), lane l
// owning PR_NZLANE consecutive ones).  Each lane gathers its values into
// registers and finds its row boundaries in the row-end bitmap (a popc and a
// shift, no search); rows ending in the tile are numbered in the compressed
// list of non-empty rows from the tile's first row.  Per-lane segmented sums
// go to shared memory, a warp scan joins rows split across lanes.  Rows that
// start and end in the tile go through the epilogue; the tile's part of a
// first row that began earlier goes to first[t]; the part of the row still
// open at the end goes to agg[t].
// The loads that start a tile: its column indices, row-end bits and the
// first row a lane finishes.  They depend only on the tile index (and the
// tile's metadata), so a warp issues them ahead of use (one tile ahead, two
// in the pipelined phase A) and their memory latency overlaps the gathers.
struct TilePre {
    uint32_t meta;
    int4 ca, cb;
    uint32_t bits;
    int pre_i;   // -1: the lane finishes no row numbered rfirst + lane
};

__device__ __forceinline__ TilePre tile_pre(const PrParams& p, int t, uint32_t meta) {
    // The matrix arrays are read once per body: streaming loads (evict-first)
    // keep them from pushing the gathered vector out of L2.
    const int lane = threadIdx.x & 31;
    const int kl = t * PR_NZTILE + lane * PR_NZLANE;
    TilePre f;
    f.meta = meta;
    const int4* cp = reinterpret_cast<const int4*>(p.col_idx + kl);
    f.ca = ld_stream(cp);
    f.cb = ld_stream(cp + 1);
    f.bits = ld_stream(p.rowend_bits + (kl >> 5));
    const int rfirst = (int)(meta & 0x7fffffffu);
    f.pre_i = rfirst + lane < p.n_ne ? ld_stream(p.ne_rows + rfirst + lane) : -1;
    return f;
}

// What a tile's loads deliver: the gathered values of the lane's nonzeros
// and the epilogue inputs of the first row the lane finishes.
template <class T, int EPI>
struct TileVals {
    T v[PR_NZLANE];
    RowIn<T, EPI> pre;
};

// First half of a tile: issue its gathers and the epilogue loads of the
// lane's first row.  Nothing waits for them here.
template <class T, class G, int GMODE, bool NC, int EPI, bool HOT = false>
__device__ __forceinline__ TileVals<T, EPI> tile_issue(const PrParams& p, int t, const TilePre& f,
                                                       const TileIO<T, G>& io) {
    static_assert(PR_NZLANE == 8, "two 16-byte column loads per lane");
    TileVals<T, EPI> tv;
    tv.pre.rold = (T)0;
    tv.pre.dd = (T)1;
    tv.pre.sinkword = 0;
    if (f.pre_i >= 0) tv.pre = row_inputs<T, G, NC, EPI>(p, io, f.pre_i);
    const int cols[PR_NZLANE] = {f.ca.x, f.ca.y, f.ca.z, f.ca.w, f.cb.x, f.cb.y, f.cb.z, f.cb.w};
    // padding entries of the last tile hold column 0: the load is in bounds,
    // and tile_finish discards its value
#pragma unroll
    for (int q = 0; q < PR_NZLANE; ++q) tv.v[q] = gather<T, G, GMODE, NC, HOT>(p, io, cols[q]);
    return tv;
}

// A tile's carry (the part of the row open at its end).  In single-pass
// bodies (LB) it is published as one 64-bit word {value, body tag}, so a
// reader that sees the tag sees the value: no fence, no separate flag.
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* a, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* a) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}

template <bool LB, class T, class G>
__device__ __forceinline__ void store_carry(const PrParams& p, const TileIO<T, G>& io, int t, T val) {
    if constexpr (LB && sizeof(T) == 4) {
        st_relaxed_u64(reinterpret_cast<unsigned long long*>(p.agg) + t,
                       ((unsigned long long)io.epoch << 32) | (unsigned long long)__float_as_uint((float)val));
    } else {
        reinterpret_cast<T*>(p.agg)[t] = val;
    }
}

// Second half: row numbering, segmented sums, carries and the epilogue.
template <class T, class G, bool NC, int EPI, bool LB = false>
__device__ __forceinline__ void tile_finish(const PrParams& p, int t, const TilePre& f, const TileVals<T, EPI>& tv,
                                            const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang,
                                            WarpSmem<T>& ws) {
    const int lane = threadIdx.x & 31;
    const uint32_t meta = f.meta;
    const int rfirst = (int)(meta & 0x7fffffffu);
    const int x_lo = (int)(meta >> 31);
    const int kl = t * PR_NZTILE + lane * PR_NZLANE;
    const uint32_t myf = (f.bits >> (kl & 31)) & 0xffu;
    const int pre_i = f.pre_i >= 0 ? f.pre_i : 0;
    const RowIn<T, EPI>& pre = tv.pre;
    T v[PR_NZLANE];
#pragma unroll
    for (int q = 0; q < PR_NZLANE; ++q) v[q] = tv.v[q];
    if (t == p.ntiles - 1) {   // the last tile: drop the padding's values
        const int nvalid = min(max(p.nnz - kl, 0), PR_NZLANE);
#pragma unroll
        for (int q = 0; q < PR_NZLANE; ++q)
            if (q >= nvalid) v[q] = (T)0;
    }

    // ---- a tile in which no row ends (inside a long row: ~40% of the tiles
    // of an R-MAT graph) is all carry: the lane sums and the warp scan only,
    // the same additions in the same order as below when no lane ends a row
    if (__all_sync(FULLMASK, myf == 0u)) {
        T val = (T)0;
#pragma unroll
        for (int q = 0; q < PR_NZLANE; ++q) val += v[q];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T v2 = __shfl_up_sync(FULLMASK, val, off);
            if (lane >= off) val = v2 + val;
        }
        if (lane == 31) store_carry<LB>(p, io, t, val);
        return;
    }

    // ---- row numbering: rows ending before this lane's nonzeros and in the
    // whole tile, from the four bit planes of the per-lane counts (0..8)
    const int cnt = __popc(myf);
    const uint32_t below = (1u << lane) - 1u;
    int before = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t plane = __ballot_sync(FULLMASK, (cnt >> b) & 1);
        before += __popc(plane & below) << b;
    }
    const int nrows = (int)__reduce_add_sync(FULLMASK, (unsigned)cnt);

    // ---- per-lane segmented sums (row sums in ascending column order)
    T acc = (T)0;
    int idx = before;
#pragma unroll
    for (int q = 0; q < PR_NZLANE; ++q) {
        acc += v[q];
        if ((myf >> q) & 1u) {
            ws.rowsum[idx] = acc;
            ++idx;
            acc = (T)0;
        }
    }

    // ---- warp segmented (reduce-by-key) scan of the lane carries: lane
    // l - off carries into lane l's open row when no lane in (l - off, l]
    // ends a row.  With h the highest lane <= l that ends one (-1 if none),
    // that is off <= l - h (and off <= l for the lane to exist).
    const uint32_t heads = __ballot_sync(FULLMASK, cnt > 0) & (0xffffffffu >> (31 - lane));
    const int h = heads ? 31 - __clz(heads) : -1;
    const int lim = min(lane - h, lane);
    T val = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T v2 = __shfl_up_sync(FULLMASK, val, off);
        if (off <= lim) val = v2 + val;
    }
    // the carry of lanes below ends this lane's first row (row `before`)
    const T exv = __shfl_up_sync(FULLMASK, val, 1);
    if (lane > 0 && cnt > 0) ws.rowsum[before] = exv + ws.rowsum[before];
    if (lane == 31) store_carry<LB>(p, io, t, val);
    __syncwarp();

    // ---- epilogue of the rows finished here (row x on lane x % 32)
    if (x_lo == 1 && nrows > 0 && lane == 0) reinterpret_cast<T*>(p.first)[t] = ws.rowsum[0];
    if (lane >= x_lo && lane < nrows) row_epilogue<T, G, EPI>(p, io, pre_i, ws.rowsum[lane], true, pre, resid, dang);
    for (int x = 32 + lane; x < nrows; x += 32) {
        const int i = ld_stream(p.ne_rows + rfirst + x);
        const RowIn<T, EPI> in = row_inputs<T, G, NC, EPI>(p, io, i);
        row_epilogue<T, G, EPI>(p, io, i, ws.rowsum[x], true, in, resid, dang);
    }
    __syncwarp();
}

template <class T, class G, int GMODE, bool NC, int EPI, bool HOT = false>
__device__ __forceinline__ void warp_tile(const PrParams& p, int t, const TilePre& f, const TileIO<T, G>& io,
                                          Acc<T>& resid, Acc<T>& dang, WarpSmem<T>& ws) {
    const TileVals<T, EPI> tv = tile_issue<T, G, GMODE, NC, EPI, HOT>(p, t, f, io);
    tile_finish<T, G, NC, EPI>(p, t, f, tv, io, resid, dang, ws);
}

// Rows without nonzeros: the epilogue with an empty sum.
// U rows per step: their index loads, then their input loads, are issued
// together (one round trip each instead of one per row); a thread still
// takes its rows in grid-stride order, so U does not change the sums.
template <class T, class G, bool NC, int EPI, int U = 1>
__device__ __forceinline__ void empty_rows(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang) {
    const int nthreads = gridDim.x * blockDim.x;
    if constexpr (U == 1) {
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.n_empty; e += nthreads) {
            const int i = ld_stream(p.empty_rows + e);
            const RowIn<T, EPI> in = row_inputs<T, G, NC, EPI>(p, io, i);
            row_epilogue<T, G, EPI>(p, io, i, (T)0, false, in, resid, dang);
        }
        return;
    }
    for (int e0 = blockIdx.x * blockDim.x + threadIdx.x; e0 < p.n_empty; e0 += U * nthreads) {
        int i[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nthreads;
            i[u] = e < p.n_empty ? ld_stream(p.empty_rows + e) : -1;
        }
        RowIn<T, EPI> in[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i[u] >= 0) in[u] = row_inputs<T, G, NC, EPI>(p, io, i[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i[u] >= 0) row_epilogue<T, G, EPI>(p, io, i[u], (T)0, false, in[u], resid, dang);
    }
}

// Phase B: rows split across tiles.  Each thread takes tiles with a short
// fixup (at most PR_LONG carries to add); each warp takes a long one.
template <class T, class G, bool NC, int EPI>
__device__ __forceinline__ void fixups(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang) {
    const T* agg = reinterpret_cast<const T*>(p.agg);
    const T* first = reinterpret_cast<const T*>(p.first);
    const int nthreads = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < p.ntiles; t += nthreads) {
        const FixDesc f = p.fix[t];
        if (f.row < 0 || t - f.ts > PR_LONG) continue;
        const RowIn<T, EPI> in = row_inputs<T, G, NC, EPI>(p, io, f.row);
        T sum = (T)0;
        for (int tt = f.ts; tt < t; ++tt) sum += __ldcg(agg + tt);
        sum += __ldcg(first + t);
        row_epilogue<T, G, EPI>(p, io, f.row, sum, true, in, resid, dang);
    }
    // rows spanning many tiles (hubs): one warp each, FP64 partial sums
    const int lane = threadIdx.x & 31;
    const int bw = blockDim.x >> 5;
    const int nwarps = gridDim.x * bw;
    for (int q = blockIdx.x * bw + (threadIdx.x >> 5); q < p.nlong; q += nwarps) {
        const int32_t t = p.longfix[q];
        const FixDesc f = p.fix[t];
        double sum = 0.0;
        for (int tt = f.ts + lane; tt < t; tt += 32) sum += (double)__ldcg(agg + tt);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(FULLMASK, sum, off);
        if (lane == 0) {
            sum += (double)__ldcg(first + t);
            const RowIn<T, EPI> in = row_inputs<T, G, NC, EPI>(p, io, f.row);
            row_epilogue<T, G, EPI>(p, io, f.row, (T)sum, true, in, resid, dang);
        }
    }
}

// Single-pass bodies: the rows split across tiles are finished by the warp
// that finished the tile they end in, after its tile loop (by then the
// carries of the tiles before them, finished by other warps, have almost
// always been published), from the carries tagged with this body.  Each
// lane takes one of the warp's tiles (short fixups, at most PR_LONG
// carries, summed by the lane); fixups of longer rows take the whole warp.
// The sums are those of phase B, in the same order: the same bits.  Every
// wait is for a lower tile index, so the waits cannot form a cycle; each is
// bounded.
template <class T>
__device__ __forceinline__ T carry_of(const PrParams& p, const unsigned long long* agg, int tt, uint32_t epoch,
                                      bool& ok) {
    for (int64_t spins = 0; ok; ++spins) {
        const unsigned long long x = ld_relaxed_u64(agg + tt);
        if ((uint32_t)(x >> 32) == epoch) return (T)__uint_as_float((uint32_t)x);
        if (spins > p.spin_limit) ok = false;
    }
    return (T)0;
}

template <class T, class G, int EPI, int NW>
__device__ __forceinline__ void lookback_fixups(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid,
                                                Acc<T>& dang) {
    static_assert(sizeof(T) == 4, "single-pass bodies publish FP32 carries");
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * NW + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * NW;
    const unsigned long long* agg = reinterpret_cast<const unsigned long long*>(p.agg);
    const T* first = reinterpret_cast<const T*>(p.first);
    bool ok = true;
    __syncwarp();   // first[] of this warp's tiles, written by lane 0, read by any lane
    for (int64_t k0 = 0; w0 + k0 * nw < p.ntiles; k0 += 32) {
        const int64_t tl = w0 + (k0 + lane) * nw;
        int longt = -1;
        if (tl < p.ntiles && (__ldg(p.tile_meta + tl) >> 31)) {
            const int t = (int)tl;
            const FixDesc f = p.fix[t];
            if (f.row >= 0) {
                if (t - f.ts <= PR_LONG) {
                    const RowIn<T, EPI> in = row_inputs<T, G, false, EPI>(p, io, f.row);
                    T sum = (T)0;
                    for (int tt = f.ts; tt < t; ++tt) sum += carry_of<T>(p, agg, tt, io.epoch, ok);
                    sum += first[t];
                    row_epilogue<T, G, EPI>(p, io, f.row, sum, true, in, resid, dang);
                } else {
                    longt = t;
                }
            }
        }
        for (uint32_t m = __ballot_sync(FULLMASK, longt >= 0); m; m &= m - 1) {
            const int t = __shfl_sync(FULLMASK, longt, __ffs(m) - 1);
            const FixDesc f = p.fix[t];
            double sum = 0.0;
            for (int tt = f.ts + lane; tt < t; tt += 32) sum += (double)carry_of<T>(p, agg, tt, io.epoch, ok);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(FULLMASK, sum, off);
            if (lane == 0) {
                sum += (double)first[t];
                const RowIn<T, EPI> in = row_inputs<T, G, false, EPI>(p, io, f.row);
                row_epilogue<T, G, EPI>(p, io, f.row, (T)sum, true, in, resid, dang);
            }
        }
    }
    if (!ok) set_status(p.status, (int32_t)GRB_DEVICE_TIMEOUT);
}

// Phase A over the tiles of this warp (static assignment, next tile's
// coordinates prefetched), then the rows without nonzeros (EU per thread per
// step, their loads batched).
template <class T, class G, int GMODE, bool NC, int EPI, bool HOT = false, int NW = NWARP, int EU = 1>
__device__ __forceinline__ void phase_a(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang,
                                        Smem<T, NW>& sm) {
    const int warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * NW;
    int t = blockIdx.x * NW + warp;
    // software pipeline: the metadata two tiles ahead, the tile-start loads
    // one tile ahead
    uint32_t meta2 = t + nwarps < p.ntiles ? __ldg(p.tile_meta + t + nwarps) : 0u;
    TilePre f;
    if (t < p.ntiles) f = tile_pre(p, t, __ldg(p.tile_meta + t));
    for (; t < p.ntiles; t += nwarps) {
        const TilePre cur = f;
        const int t1 = t + nwarps;
        if (t1 < p.ntiles) {
            const uint32_t m1 = meta2;
            meta2 = t1 + nwarps < p.ntiles ? __ldg(p.tile_meta + t1 + nwarps) : 0u;
            f = tile_pre(p, t1, m1);
        }
        warp_tile<T, G, GMODE, NC, EPI, HOT>(p, t, cur, io, resid, dang, sm.w[warp]);
    }
    empty_rows<T, G, NC, EPI, EU>(p, io, resid, dang);
}

// Phase A with the gathers one tile deep: tile t+nwarps's gathers are issued
// before tile t's scans and epilogue, so every warp keeps two tiles' loads in
// flight; tile-start loads run two tiles ahead and the metadata three.
template <class T, class G, int GMODE, int EPI, bool HOT, int NW, bool LB = false>
__device__ __forceinline__ void phase_a_pipe(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang,
                                             Smem<T, NW>& sm) {
    const int warp = threadIdx.x >> 5;
    const int nw = gridDim.x * NW;
    int t = blockIdx.x * NW + warp;
    if (t < p.ntiles) {
        TilePre f0 = tile_pre(p, t, __ldg(p.tile_meta + t));
        TilePre f1;
        f1.pre_i = -1;
        f1.meta = 0u;
        if (t + nw < p.ntiles) f1 = tile_pre(p, t + nw, __ldg(p.tile_meta + t + nw));
        uint32_t meta2 = t + 2 * nw < p.ntiles ? __ldg(p.tile_meta + t + 2 * nw) : 0u;
        TileVals<T, EPI> v0 = tile_issue<T, G, GMODE, false, EPI, HOT>(p, t, f0, io);
        for (; t < p.ntiles; t += nw) {
            const int t1 = t + nw, t2 = t + 2 * nw, t3 = t + 3 * nw;
            TileVals<T, EPI> v1;
            if (t1 < p.ntiles) v1 = tile_issue<T, G, GMODE, false, EPI, HOT>(p, t1, f1, io);
            TilePre f2;
            f2.pre_i = -1;
            f2.meta = 0u;
            if (t2 < p.ntiles) {
                f2 = tile_pre(p, t2, meta2);
                meta2 = t3 < p.ntiles ? __ldg(p.tile_meta + t3) : 0u;
            }
            tile_finish<T, G, false, EPI, LB>(p, t, f0, v0, io, resid, dang, sm.w[warp]);
            f0 = f1;
            f1 = f2;
            v0 = v1;
        }
        if constexpr (LB) lookback_fixups<T, G, EPI, NW>(p, io, resid, dang);
    }
    empty_rows<T, G, false, EPI, 4>(p, io, resid, dang);
}

// ------------------------------------------------ row-length-binned body
// The alternative work decomposition (GRB_OPT_ROW_BINS): every non-empty row
// is summed by one group of threads sized by the row's length -- a thread
// (1-4 nonzeros), 4, 8 or 16 lanes (5-256), a warp (257-8192) or a whole
// CTA (longer: the hub rows, whose per-warp sums meet in shared memory) --
// so there are no split rows, no carries and no fixup phase, one grid
// barrier per body instead of two.  The lanes of a group take the row's
// nonzeros round-robin (the group's column loads are coalesced), gather from
// the hot copy or L2, and fold their sums with a fixed butterfly.  Rows come
// from per-bin lists (PR_BINS bins plus the empty rows); within a bin, the
// groups of the grid take the rows round-robin.
template <int GS, class T, class G, int EPI, bool HOT>
__device__ __forceinline__ void bin_groups(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang,
                                           int lo_b, int hi_b) {
    constexpr int NG = 32 / GS;   // groups per warp
    const int lane = threadIdx.x & 31, sub = lane % GS, grp = lane / GS;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    // every warp makes the same number of rounds (the butterfly needs all lanes)
    for (int base = lo_b + gw * NG; base < hi_b; base += nwarps * NG) {
        const int k = base + grp;
        const bool have = k < hi_b;
        int i = 0, lo = 0, hi = 0;
        if (have) {
            i = ld_stream(p.bin_rows + k);
            lo = __ldg(p.row_ptr + i);
            hi = __ldg(p.row_ptr + i + 1);
        }
        RowIn<T, EPI> in{};
        if (have && sub == 0) in = row_inputs<T, G, false, EPI>(p, io, i);
        // four running sums per lane (shorter rounding chains, loads in flight)
        T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
        int e = lo + sub;
        for (; e + 3 * GS < hi; e += 4 * GS) {
            const int c0 = ld_stream(p.col_idx + e), c1 = ld_stream(p.col_idx + e + GS);
            const int c2 = ld_stream(p.col_idx + e + 2 * GS), c3 = ld_stream(p.col_idx + e + 3 * GS);
            a0 += gather<T, G, G_W, false, HOT>(p, io, c0);
            a1 += gather<T, G, G_W, false, HOT>(p, io, c1);
            a2 += gather<T, G, G_W, false, HOT>(p, io, c2);
            a3 += gather<T, G, G_W, false, HOT>(p, io, c3);
        }
        for (; e < hi; e += GS) a0 += gather<T, G, G_W, false, HOT>(p, io, ld_stream(p.col_idx + e));
        T acc = (a0 + a1) + (a2 + a3);
        __syncwarp();
#pragma unroll
        for (int off = GS / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(FULLMASK, acc, off);
        if (have && sub == 0) row_epilogue<T, G, EPI>(p, io, i, acc, true, in, resid, dang);
    }
}

template <class T, class G, int EPI, bool HOT, int NW>
__device__ __forceinline__ void bin_cta_rows(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang,
                                             int lo_b, int hi_b, T* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = lo_b + blockIdx.x; k < hi_b; k += gridDim.x) {   // the same in the whole CTA
        const int i = __ldg(p.bin_rows + k);
        const int lo = __ldg(p.row_ptr + i), hi = __ldg(p.row_ptr + i + 1);
        RowIn<T, EPI> in{};
        if (threadIdx.x == 0) in = row_inputs<T, G, false, EPI>(p, io, i);
        T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
        const int step = NW * 32;
        int e = lo + (int)threadIdx.x;
        for (; e + 3 * step < hi; e += 4 * step) {
            const int c0 = ld_stream(p.col_idx + e), c1 = ld_stream(p.col_idx + e + step);
            const int c2 = ld_stream(p.col_idx + e + 2 * step), c3 = ld_stream(p.col_idx + e + 3 * step);
            a0 += gather<T, G, G_W, false, HOT>(p, io, c0);
            a1 += gather<T, G, G_W, false, HOT>(p, io, c1);
            a2 += gather<T, G, G_W, false, HOT>(p, io, c2);
            a3 += gather<T, G, G_W, false, HOT>(p, io, c3);
        }
        for (; e < hi; e += step) a0 += gather<T, G, G_W, false, HOT>(p, io, ld_stream(p.col_idx + e));
        T acc = (a0 + a1) + (a2 + a3);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULLMASK, acc, off);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            T sum = red[0];
            for (int w = 1; w < NW; ++w) sum += red[w];
            row_epilogue<T, G, EPI>(p, io, i, sum, true, in, resid, dang);
        }
        __syncthreads();
    }
}

template <class T, class G, int EPI, bool HOT, int NW>
__device__ __forceinline__ void phase_bins(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang,
                                           Smem<T, NW>& sm) {
    bin_cta_rows<T, G, EPI, HOT, NW>(p, io, resid, dang, p.bin_off[5], p.bin_off[6], sm.w[0].rowsum);
    bin_groups<32, T, G, EPI, HOT>(p, io, resid, dang, p.bin_off[4], p.bin_off[5]);
    bin_groups<16, T, G, EPI, HOT>(p, io, resid, dang, p.bin_off[3], p.bin_off[4]);
    bin_groups<8, T, G, EPI, HOT>(p, io, resid, dang, p.bin_off[2], p.bin_off[3]);
    bin_groups<4, T, G, EPI, HOT>(p, io, resid, dang, p.bin_off[1], p.bin_off[2]);
    bin_groups<1, T, G, EPI, HOT>(p, io, resid, dang, p.bin_off[0], p.bin_off[1]);
    empty_rows<T, G, false, EPI, 4>(p, io, resid, dang);
}

// ------------------------------------------------ bulk-copy staging of tiles
// The persistent loop can stream the per-tile arrays (256 column indices and
// the 8 row-end words of a tile, 1056 bytes) into shared memory with
// cp.async.bulk, PR_TMA_STAGES tiles ahead of the warp that will use them;
// each stage has an mbarrier that the copy completes.  The warp's lane 0
// issues the copies; every wait is bounded.
struct alignas(16) TmaStage {
    int32_t cols[PR_NZTILE];
    uint32_t bits[PR_NZTILE / 32];
};
constexpr uint32_t TMA_STAGE_BYTES = sizeof(TmaStage);
static_assert(TMA_STAGE_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}

// Bounded wait for phase `parity` of a stage's barrier.
__device__ __forceinline__ bool stage_wait(uint64_t* b, uint32_t parity, int64_t limit) {
    for (int64_t spins = 0; !mbar_try_wait(b, parity); ++spins)
        if (spins > limit) return false;
    return true;
}

__device__ __forceinline__ void stage_issue(const PrParams& p, int t, TmaStage* st, uint64_t* b) {
    mbar_expect_tx(b, TMA_STAGE_BYTES);
    bulk_to_smem(st->cols, p.col_idx + (size_t)t * PR_NZTILE, PR_NZTILE * sizeof(int32_t), b);
    bulk_to_smem(st->bits, p.rowend_bits + (size_t)t * (PR_NZTILE / 32), (PR_NZTILE / 32) * sizeof(uint32_t), b);
}

// Phase A with the tile arrays staged by bulk copies.  `seq` counts the
// tiles this warp has consumed in the launch (it selects the stage and the
// barrier phase) and carries over from body to body.
template <class T, class G, int GMODE, int EPI, bool HOT, int NW, int NST>
__device__ __forceinline__ void phase_a_tma(const PrParams& p, const TileIO<T, G>& io, Acc<T>& resid, Acc<T>& dang,
                                            Smem<T, NW>& sm, TmaStage* stages, uint64_t* bars, uint32_t& seq) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * NW;
    const int w0 = blockIdx.x * NW + warp;
    const int count = w0 < p.ntiles ? (p.ntiles - w0 + nwarps - 1) / nwarps : 0;
    TmaStage* S = stages + warp * NST;
    uint64_t* B = bars + warp * NST;
    if (lane == 0)
        for (int k = 0; k < count && k < NST; ++k) stage_issue(p, w0 + k * nwarps, S + (seq + k) % NST, B + (seq + k) % NST);
    __syncwarp();
    auto first_row = [&](uint32_t meta) {
        const int rfirst = (int)(meta & 0x7fffffffu);
        return rfirst + lane < p.n_ne ? ld_stream(p.ne_rows + rfirst + lane) : -1;
    };
    uint32_t meta_cur = count > 0 ? __ldg(p.tile_meta + w0) : 0u;
    uint32_t meta_next = count > 1 ? __ldg(p.tile_meta + w0 + nwarps) : 0u;
    int pre_cur = count > 0 ? first_row(meta_cur) : -1;
    int k = 0;
    for (; k < count; ++k) {
        const int t = w0 + k * nwarps;
        const uint32_t u = seq + (uint32_t)k;
        const int s = (int)(u % NST);
        if (!stage_wait(B + s, (u / NST) & 1u, p.spin_limit)) {
            set_status(p.status, (int32_t)GRB_DEVICE_TIMEOUT);
            break;
        }
        TilePre f;
        f.meta = meta_cur;
        f.pre_i = pre_cur;
        f.ca = *reinterpret_cast<const int4*>(S[s].cols + lane * PR_NZLANE);
        f.cb = *reinterpret_cast<const int4*>(S[s].cols + lane * PR_NZLANE + 4);
        f.bits = S[s].bits[lane >> 2];
        __syncwarp();
        if (lane == 0 && k + NST < count) {
            // the warp's reads of this stage come before the copy's writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            stage_issue(p, t + NST * nwarps, S + s, B + s);
        }
        if (k + 1 < count) {
            meta_cur = meta_next;
            meta_next = k + 2 < count ? __ldg(p.tile_meta + t + 2 * nwarps) : 0u;
            pre_cur = first_row(meta_cur);
        }
        warp_tile<T, G, GMODE, false, EPI, HOT>(p, t, f, io, resid, dang, sm.w[warp]);
    }
    if (k < count) {
        // a wait ran out: let this warp's copies still in flight land (again
        // bounded) before the kernel leaves at the next grid barrier
        for (int q = k; q < count && q < k + NST; ++q) {
            const uint32_t u = seq + (uint32_t)q;
            stage_wait(B + u % NST, (u / NST) & 1u, p.spin_limit);
        }
    }
    seq += (uint32_t)count;
    empty_rows<T, G, false, EPI>(p, io, resid, dang);
}

template <class T>
__device__ __forceinline__ T tele_value(const PrParams& p) {
    return p.tele_from_slot ? (T)round_to(p.out.type, *p.tele_slot) : (T)p.tele_const;
}

// One fused body per launch (also the fast unfused mxv): phase A, grid
// barrier, phase B, then the last CTA folds the per-CTA partials.  LEAN
// launches are bodies of an iterated sequence (a CUDA graph): each first
// checks the loop condition left by the previous launch and does nothing
// once it fails.
template <class T, class G, int GMODE, bool LEAN>
__global__ void __launch_bounds__(PR_BLOCK, PR_MINBLOCKS) pr_iter_kernel(const __grid_constant__ PrParams p) {
    __shared__ Smem<T> sm;
    __shared__ bool last;
    const int it = p.iter_index;
    if (LEAN) {
        const double rd = it == 0 ? p.rdiff0 : *(volatile double*)p.resid_slot;
        const int64_t done_so_far = *(volatile int64_t*)p.iters_done;
        if (!(rd > p.tol) || done_so_far != it) return;
    }
    TileIO<T, G> io{};
    io.tele_scalar = p.tele_from_slot;
    io.tele = tele_value<T>(p);
    if (LEAN) {
        io.r_old = reinterpret_cast<const T*>(it == 0 ? p.r0 : p.rbuf[(it - 1) & 1]);
        io.out = reinterpret_cast<T*>(p.rbuf[it & 1]);
        io.w = reinterpret_cast<const G*>(p.wbuf[it & 1]);
        io.w_next = reinterpret_cast<G*>(p.wbuf[(it + 1) & 1]);
        io.out_present = nullptr;
    } else {
        io.w = reinterpret_cast<const G*>(p.w);
        io.t = reinterpret_cast<const T*>(p.t);
        io.d = reinterpret_cast<const T*>(p.d);
        io.r_old = reinterpret_cast<const T*>(p.r_old);
        io.out = reinterpret_cast<T*>(p.out.vals);
        io.out_present = p.out.full ? nullptr : p.out.present;
        io.w_next = reinterpret_cast<G*>(p.w_next);
    }
    io.w32 = nullptr;
    io.w32_next = nullptr;
    io.phase32 = 0;
    Acc<T> racc, dacc;
    phase_a<T, G, GMODE, true, LEAN ? EPI_LEAN : EPI_GEN>(p, io, racc, dacc, sm);
    if (!grid_sync(p.sync, p.status, p.spin_limit, gridDim.x, &sm.ok)) return;
    fixups<T, G, true, LEAN ? EPI_LEAN : EPI_GEN>(p, io, racc, dacc);
    const double resid = block_sum_d<PR_BLOCK>(racc.value(), sm.red);
    const double dang = block_sum_d<PR_BLOCK>(dacc.value(), sm.red2);
    if (threadIdx.x == 0) {
        p.part[2 * blockIdx.x] = resid;
        p.part[2 * blockIdx.x + 1] = dang;
        __threadfence();
        last = atomicAdd(&p.sync->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double R, D;
    reduce_parts<T>(p.part, gridDim.x, R, D, sm);
    if (threadIdx.x == 0) {
        R = round_to(p.resid_type, R);
        if (p.resid_slot && (LEAN || p.want_resid)) *p.resid_slot = R;
        if (p.dang_slot && p.want_dang) *p.dang_slot = D;
        if (p.tele_slot && p.want_dang) *p.tele_slot = schain_apply(p.chain, D);
        if (LEAN) {
            if (p.hist) p.hist[it] = R;
            if (p.dhist) p.dhist[it] = D;
            *p.iters_done = it + 1;
        }
        p.sync->done = 0;
        p.sync->launch += 1;
    }
}

// Whole loop in one launch: prologue (w_0 = r_0 ./ d and the dangling mass of
// r_0), then bodies while the condition holds; each body is phase A,
// barrier, phase B, barrier (single pass, LB: phase A with the look-back
// fixups, barrier), and every CTA folds the same partials in the same
// order, so all CTAs take the same loop decision.
//
// HOT (one CTA of BLK = PR_HOT_BLOCK threads per SM): at the start of each body the
// CTA copies w[0, hot_n) into shared memory and serves gathers of those
// columns from there.  With vertices numbered by descending out-degree these
// are the most-gathered entries (for R-MAT, the first 32K of 4M vertices
// take about half of all gathers), so half of the random gathers never reach
// L1/L2; the copy costs hot_n words per CTA per body from L2.
static_assert(sizeof(Smem<float, PR_HOT_BLOCK / 32>) <= PR_HOT_STATIC_SMEM, "static shared memory bound");

template <class T, class G, int BLK, bool HOT, int NST = 0, bool PERS = false, bool BINS = false>
__global__ void __launch_bounds__(BLK, ((HOT || BLK >= 1024) ? 1 : PR_MINBLOCKS))
    pr_persistent_kernel(const __grid_constant__ PrParams p) {
    constexpr int EPI = PERS ? EPI_PERS : EPI_LEAN;
    // single pass per body: split rows finished by look-back inside phase A,
    // one grid barrier per body instead of two (the pipelined hot path)
    constexpr bool LB = HOT && NST == 0 && !BINS && sizeof(T) == 4;
    __shared__ Smem<T, BLK / 32> sm;
    extern __shared__ int4 hot_raw[];
    // dynamic shared memory: [hot copy (hot_n words)][NST tile stages per
    // warp][NST barriers per warp]
    TmaStage* stages = reinterpret_cast<TmaStage*>(reinterpret_cast<char*>(hot_raw) + (size_t)p.hot_n * sizeof(G));
    uint64_t* bars = reinterpret_cast<uint64_t*>(stages + (BLK / 32) * (NST > 0 ? NST : 1));
    uint32_t seq = 0;
    if constexpr (NST > 0) {
        if ((threadIdx.x & 31) == 0)
            for (int q = 0; q < NST; ++q) mbar_init(bars + (threadIdx.x >> 5) * NST + q, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        __syncwarp();
    }
    const int G_ = gridDim.x;
    const T* dd = reinterpret_cast<const T*>(p.dd);
    const T* r0 = reinterpret_cast<const T*>(p.r0);
    int phase32 = 0;

    // prologue
    double dang = 0.0;
    for (int i = blockIdx.x * BLK + threadIdx.x; i < p.nrows; i += G_ * BLK) {
        const T rv = r0[i];
        const T q = rv / dd[i];
        if constexpr (sizeof(T) == 8) reinterpret_cast<double*>(p.wbuf[0])[i] = (double)q;
        else gstore<G>(reinterpret_cast<G*>(p.wbuf[0]), i, (float)q);
        if (p.want_dang && ((p.sinkbits[i >> 5] >> (i & 31)) & 1u)) dang += (double)rv;
    }
    if constexpr (LB) {
        // no carry of this launch is published yet
        unsigned long long* a64 = reinterpret_cast<unsigned long long*>(p.agg);
        for (int k = blockIdx.x * BLK + threadIdx.x; k < p.ntiles; k += G_ * BLK) a64[k] = 0ull;
    }
    dang = block_sum_d<BLK>(dang, sm.red2);
    if (threadIdx.x == 0) {
        p.part[2 * blockIdx.x] = 0.0;
        p.part[2 * blockIdx.x + 1] = dang;
    }
    if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
    double R, D;
    reduce_parts<T, BLK>(p.part, G_, R, D, sm);
    T tele = p.tele_from_slot ? (T)round_to(p.out.type, schain_apply(p.chain, D)) : (T)p.tele_const;
    double rd = p.rdiff0;
    double rd_prev = rd;
    int it = 0;
    while (it < p.iters && rd > p.tol) {
        TileIO<T, G> io{};
        io.r_old = it == 0 ? r0 : reinterpret_cast<const T*>(p.rbuf[(it - 1) & 1]);
        io.out = reinterpret_cast<T*>(p.rbuf[it & 1]);
        io.out_present = nullptr;
        io.w = reinterpret_cast<const G*>(p.wbuf[it & 1]);
        io.w_next = reinterpret_cast<G*>(p.wbuf[(it + 1) & 1]);
        io.w32 = reinterpret_cast<const float*>(p.wbuf32[it & 1]);
        io.w32_next = reinterpret_cast<float*>(p.wbuf32[(it + 1) & 1]);
        io.phase32 = phase32;
        io.tele = tele;
        io.tele_scalar = 1;
        io.hot = reinterpret_cast<const G*>(hot_raw);
        io.hot_n = HOT ? p.hot_n : 0;
        io.epoch = (uint32_t)it + 1u;
        if constexpr (HOT) {
            // w of this body was written before the last grid barrier
            const int4* src = reinterpret_cast<const int4*>(io.w);
            const int nvec = (int)(((int64_t)p.hot_n * (int64_t)sizeof(G)) / 16);
            for (int k = threadIdx.x; k < nvec; k += BLK) hot_raw[k] = __ldcg(src + k);
            __syncthreads();
        }
        Acc<T> racc, dacc;
        if constexpr (BINS) {
            phase_bins<T, G, EPI, HOT, BLK / 32>(p, io, racc, dacc, sm);   // no split rows: no phase B
        } else {
            if constexpr (NST > 0)
                phase_a_tma<T, G, G_W, EPI, HOT, BLK / 32, NST>(p, io, racc, dacc, sm, stages, bars, seq);
            else if constexpr (HOT)
                phase_a_pipe<T, G, G_W, EPI, HOT, BLK / 32, LB>(p, io, racc, dacc, sm);
            else
                phase_a<T, G, G_W, false, EPI, HOT, BLK / 32>(p, io, racc, dacc, sm);
            if constexpr (!LB) {
                if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
                fixups<T, G, false, EPI>(p, io, racc, dacc);
            }
        }
        const double resid = block_sum_d<BLK>(racc.value(), sm.red);
        dang = block_sum_d<BLK>(dacc.value(), sm.red2);
        double* part = p.part + 2 * G_ * ((it + 1) & 1);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = resid;
            part[2 * blockIdx.x + 1] = dang;
        }
        if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
        reduce_parts<T, BLK>(part, G_, R, D, sm);
        rd = round_to(p.resid_type, R);
        if (p.tele_from_slot) tele = (T)round_to(p.out.type, schain_apply(p.chain, D));
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (p.hist) p.hist[it] = rd;
            if (p.dhist) p.dhist[it] = D;
        }
        ++it;
        // mixed precision: once the residual is small -- or has stopped
        // falling, i.e. the BF16 rounding floor is reached (one body whose
        // residual fell by less than 5%; in exact arithmetic the L1 change
        // contracts at least by the damping factor each body) -- rebuild w in
        // FP32 from the rank just written and gather FP32 from the next body
        // on.  Every CTA sees the same residuals, so all take the same decision.
        const bool stalled = it > 1 && rd > 0.95 * rd_prev;
        rd_prev = rd;
        if (sizeof(G) == 2 && p.mixed && !phase32 && (rd < p.mixed_switch || stalled) && it < p.iters && rd > p.tol) {
            T* rcur = reinterpret_cast<T*>(p.rbuf[(it - 1) & 1]);
            float* w32 = reinterpret_cast<float*>(p.wbuf32[it & 1]);
            // With uniform dangling the rank sum is invariant (1) in exact
            // arithmetic, but BF16 rounding of nearly equal ranks is
            // correlated and shifts it; a mass error only decays by the
            // damping factor per body, so the FP32 phase would crawl.  The
            // rank is renormalised to unit sum once, at the switch (the fixed
            // point is unchanged).  Each CTA scales only its own entries.
            double scale = 1.0;
            if (p.tele_from_slot) {
                double ms = 0.0;
                for (int i = blockIdx.x * BLK + threadIdx.x; i < p.nrows; i += G_ * BLK) ms += (double)__ldcg(rcur + i);
                ms = block_sum_d<BLK>(ms, sm.red);
                // the partial buffer the body just read stays untouched; the
                // other one is next written after two more grid barriers
                double* part2 = p.part + 2 * G_ * ((it + 1) & 1);
                if (threadIdx.x == 0) {
                    part2[2 * blockIdx.x] = ms;
                    part2[2 * blockIdx.x + 1] = 0.0;
                }
                if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
                double M, Z;
                reduce_parts<T, BLK>(part2, G_, M, Z, sm);
                if (M > 0.0) scale = 1.0 / M;
                D *= scale;
                tele = (T)round_to(p.out.type, schain_apply(p.chain, D));
            }
            for (int i = blockIdx.x * BLK + threadIdx.x; i < p.nrows; i += G_ * BLK) {
                T rv = __ldcg(rcur + i);
                if (scale != 1.0) {
                    rv = (T)((double)rv * scale);
                    rcur[i] = rv;
                }
                w32[i] = (float)(rv / dd[i]);
            }
            phase32 = 1;
            if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (it > 0 && p.resid_slot) *p.resid_slot = rd;
        if (p.dang_slot) *p.dang_slot = D;
        if (p.tele_slot) *p.tele_slot = (double)tele;
        *p.iters_done = it;
        if (p.expect_iters > 0 && it != p.expect_iters) set_status(p.status, (int32_t)GRB_PANIC);
        if (p.mixed_phase) *p.mixed_phase = phase32;
        p.sync->launch += 1;
    }
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(FULLMASK, x, off);
    return x;
}

// One body of a batch of independent graphs (block-diagonal A^T): the same
// tiles, barrier and fixups as a PageRank body, with the per-graph epilogue
// (per-row residual and dangling terms), then -- after a grid barrier -- the
// per-graph folds: chunk sums by warps over all CTAs, another barrier, a
// warp per graph over its chunks.  Every sum has a fixed order whatever the
// grid, so the results do not depend on the launch shape.
__global__ void __launch_bounds__(PR_BLOCK, PR_MINBLOCKS) pr_batch_kernel(const __grid_constant__ PrParams p) {
    __shared__ Smem<float> sm;
    const int from = p.iter_index & 1;
    TileIO<float, float> io{};
    io.r_old = reinterpret_cast<const float*>(p.rbuf[from]);
    io.out = reinterpret_cast<float*>(p.rbuf[from ^ 1]);
    io.w = reinterpret_cast<const float*>(p.wbuf[from]);
    io.w_next = reinterpret_cast<float*>(p.wbuf[from ^ 1]);
    Acc<float> racc, dacc;
    // per-row residual and dangling terms (folded per graph below): the
    // order of the rows does not matter, so the empty ones go four at a time
    phase_a<float, float, G_W, true, EPI_MG, false, NWARP, 4>(p, io, racc, dacc, sm);
    if (!grid_sync(p.sync, p.status, p.spin_limit, gridDim.x, &sm.ok)) return;
    fixups<float, float, true, EPI_MG>(p, io, racc, dacc);
    if (!grid_sync(p.sync, p.status, p.spin_limit, gridDim.x, &sm.ok)) return;

    const MgFinish& f = p.mg;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * NWARP + (threadIdx.x >> 5);
    const int nw = gridDim.x * NWARP;
    // chunk sums: lane-strided double-float sums of the rows' FP32 terms,
    // then a fixed FP64 warp tree (chunks of finished graphs are skipped)
    for (int c = gw; c < f.nchunks; c += nw) {
        if (!__ldcg(f.active + __ldg(f.chunk_graph + c))) continue;   // the same in the warp
        const int lo = __ldg(f.chunk_lo + c), hi = __ldg(f.chunk_lo + c + 1);
        Acc<float> R, D;
        for (int i = lo + lane; i < hi; i += 32) {
            R.add(__ldcg(f.row_res + i));
            D.add(__ldcg(f.row_dang + i));
        }
        const double r = warp_sum_d(R.value()), d = warp_sum_d(D.value());
        if (lane == 0) {
            f.chunk_part[2 * c] = r;
            f.chunk_part[2 * c + 1] = d;
        }
    }
    if (!grid_sync(p.sync, p.status, p.spin_limit, gridDim.x, &sm.ok)) return;
    for (int g = gw; g < f.ngraphs; g += nw) {
        if (!__ldcg(f.active + g)) continue;
        const int c0 = __ldg(f.g_chunk + g), c1 = __ldg(f.g_chunk + g + 1);
        double R = 0.0, D = 0.0;
        for (int c = c0 + lane; c < c1; c += 32) {
            R += __ldcg(f.chunk_part + 2 * c);
            D += __ldcg(f.chunk_part + 2 * c + 1);
        }
        R = warp_sum_d(R);
        D = warp_sum_d(D);
        if (lane == 0) {
            const int32_t k = f.iters[g] + 1;
            const double ng = (double)(__ldg(f.vptr + g + 1) - __ldg(f.vptr + g));
            f.iters[g] = k;
            f.resid[g] = R;
            f.tele[g] = (float)((1.0 - f.damping) / ng + f.damping * D / ng);
            if (!(R > f.tol) || k >= f.itermax) {
                f.active[g] = 0;
                f.final_buf[g] = from ^ 1;
            }
        }
    }
}

constexpr int MG_BLOCK = 256;

__global__ void __launch_bounds__(MG_BLOCK) mg_init_kernel(const __grid_constant__ MgInit a) {
    __shared__ double red[MG_BLOCK / 32];
    const int g = blockIdx.x;
    const int64_t lo = a.vptr[g], hi = a.vptr[g + 1];
    const double ng = (double)(hi - lo);
    const float r0 = (float)(1.0 / ng);
    double D = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += MG_BLOCK) {
        a.r[i] = r0;
        a.w[i] = r0 / a.dd[i];
        if ((a.sinkbits[i >> 5] >> (i & 31)) & 1u) D += (double)r0;
    }
    D = block_sum_d<MG_BLOCK>(D, red);
    if (threadIdx.x == 0) {
        a.active[g] = a.start_active;
        a.iters[g] = 0;
        a.resid[g] = 1.0;
        a.final_buf[g] = 0;
        a.tele[g] = (float)((1.0 - a.damping) / ng + a.damping * D / ng);
    }
}

__global__ void mg_graph_of_kernel(int32_t ngraphs, const int64_t* vptr, int32_t n, const int32_t* row_ptr,
                                   const int32_t* col_idx, int32_t* graph_of, unsigned long long* bad) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = ngraphs;   // last g with vptr[g] <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (vptr[mid] <= i) lo = mid;
            else hi = mid;
        }
        graph_of[i] = lo;
        const int64_t b = vptr[lo], e = vptr[lo + 1];
        bool out = false;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) out |= col_idx[k] < b || col_idx[k] >= e;
        if (out) atomicAdd(bad, 1ull);
    }
}

// A barrier that expects one arrival more than there are CTAs: every CTA's
// wait runs out after spin_limit polls and the kernel returns with
// GRB_DEVICE_TIMEOUT in *status.  Exercises the bounded-wait path.
__global__ void barrier_selftest_kernel(SyncWords* sync, int32_t* status, int64_t spin_limit) {
    __shared__ int ok;
    grid_sync(sync, status, spin_limit, gridDim.x + 1, &ok);
}

// Start vector and seed bitmap of one personalised query: r0[i] = val and
// bit i set for every seed i (after renumbering by old2new when given).
// r0 and bits are cleared beforehand; duplicate seeds write the same value.
__global__ void pr_seed_scatter_kernel(int32_t nseeds, const int32_t* seeds, const int32_t* old2new, float val,
                                       float* r0, uint32_t* bits) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nseeds; k += gridDim.x * blockDim.x) {
        int i = seeds[k];
        if (old2new) i = old2new[i];
        r0[i] = val;
        atomicOr(bits + (i >> 5), 1u << (i & 31));
    }
}

template <class K>
cudaError_t coop_launch(K kernel, int grid, cudaStream_t st, const PrParams& p) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(PR_BLOCK);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, p);
}

template <class K>
int occupancy(K kernel) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, PR_BLOCK, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

// Kernel table: rank type x gather type x gather mode x (one body | whole
// loop | body of an iterated sequence).
template <class T, class G>
struct Table {
    static void* pick(int32_t gmode, int persistent, int lean) {
        if (persistent) return (void*)pr_persistent_kernel<T, G, PR_BLOCK, false>;
        if (lean) return (void*)pr_iter_kernel<T, G, G_W, true>;
        if (gmode == G_TD) return (void*)pr_iter_kernel<T, G, G_TD, false>;
        if (gmode == G_ISO) return (void*)pr_iter_kernel<T, G, G_ISO, false>;
        return (void*)pr_iter_kernel<T, G, G_W, false>;
    }
};

void* pick_kernel_raw(int32_t rank_type, int32_t gather_type, int32_t gmode, int persistent, int lean) {
    if (rank_type == GRB_FP64) return Table<double, double>::pick(gmode, persistent, lean);
    if (rank_type != GRB_FP32) return nullptr;
    if (gather_type == GRB_BF16) {
        if (!persistent && !lean) return nullptr;   // BF16 gathers only in PageRank loops
        return Table<float, __nv_bfloat16>::pick(gmode, persistent, lean);
    }
    return Table<float, float>::pick(gmode, persistent, lean);
}

void* pick_kernel(int32_t rank_type, int32_t gather_type, int32_t gmode, int persistent, int lean) {
    void* k = pick_kernel_raw(rank_type, gather_type, gmode, persistent, lean);
    // these kernels use little shared memory: give the rest to L1, which
    // caches the gathered vector (a per-function hint, set before the
    // occupancy query so that both see the same configuration)
#if PR_MAX_L1
    if (k) cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxL1);
#endif
    return k;
}

// The persistent loop with the shared-memory copy of the hottest gathered
// entries: FP32 ranks and gathers only (the FP64 kernel's row-sum slices for
// PR_HOT_BLOCK / 32 warps would exceed the static shared-memory limit).
void* pick_hot(int32_t rank_type, int32_t gather_type, size_t dyn, int32_t nst, bool bins = false) {
    if (rank_type != GRB_FP32 || gather_type != GRB_FP32) return nullptr;
    void* k = nullptr;
    if (bins) nst = -1;
    switch (nst) {
        case -1: k = (void*)pr_persistent_kernel<float, float, PR_HOT_BLOCK, true, 0, false, true>; break;
        case 0: k = (void*)pr_persistent_kernel<float, float, PR_HOT_BLOCK, true, 0>; break;
        case 2: k = (void*)pr_persistent_kernel<float, float, PR_HOT_BLOCK, true, 2>; break;
        case 3: k = (void*)pr_persistent_kernel<float, float, PR_HOT_BLOCK, true, 3>; break;
        default: return nullptr;
    }
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) return nullptr;
    return k;
}

}  // namespace

int pr_batch_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pr_batch_kernel, PR_BLOCK, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_pr_batch(cudaStream_t st, const PrParams& p0, int from, int grid) {
    PrParams p = p0;
    p.iter_index = from;
    return coop_launch(pr_batch_kernel, grid, st, p);
}

cudaError_t launch_mg_init(cudaStream_t st, const MgInit& a) {
    if (a.ngraphs <= 0) return cudaSuccess;
    mg_init_kernel<<<a.ngraphs, MG_BLOCK, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mg_graph_of(cudaStream_t st, int32_t ngraphs, const int64_t* vptr, int32_t n,
                               const int32_t* row_ptr, const int32_t* col_idx, int32_t* graph_of,
                               unsigned long long* bad) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || n <= 0) return e;
    int grid = (n + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    mg_graph_of_kernel<<<grid, 256, 0, st>>>(ngraphs, vptr, n, row_ptr, col_idx, graph_of, bad);
    return cudaGetLastError();
}

// The persistent loop of one personalised query (FP32): with the hot copy
// (degree-ordered matrix) or without.
void* pick_pers(int32_t hot_n, size_t dyn) {
    if (hot_n > 0) {
        void* k = (void*)pr_persistent_kernel<float, float, PR_HOT_BLOCK, true, 0, true>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) return nullptr;
        return k;
    }
    return (void*)pr_persistent_kernel<float, float, PR_BLOCK, false, 0, true>;
}

int pr_pers_blocks_per_sm(int32_t hot_n) {
    const size_t dyn = hot_n > 0 ? pr_hot_dynamic_smem(hot_n, 0) : 0;
    void* k = pick_pers(hot_n, dyn);
    int nb = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, hot_n > 0 ? PR_HOT_BLOCK : PR_BLOCK, dyn) !=
                  cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_pr_pers(cudaStream_t st, const PrParams& p, int grid) {
    if (p.hot_n % 4 != 0 || p.hot_n > p.nrows || p.mixed || !p.pers_bits) return cudaErrorInvalidValue;
    const size_t dyn = p.hot_n > 0 ? pr_hot_dynamic_smem(p.hot_n, 0) : 0;
    void* k = pick_pers(p.hot_n, dyn);
    if (!k) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(p.hot_n > 0 ? PR_HOT_BLOCK : PR_BLOCK);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {(void*)&p};
    return cudaLaunchKernelExC(&cfg, k, args);
}

cudaError_t launch_pr_seed_scatter(cudaStream_t st, int32_t nseeds, const int32_t* seeds, const int32_t* old2new,
                                   float val, float* r0, uint32_t* bits) {
    if (nseeds <= 0) return cudaSuccess;
    pr_seed_scatter_kernel<<<(nseeds + 255) / 256, 256, 0, st>>>(nseeds, seeds, old2new, val, r0, bits);
    return cudaGetLastError();
}

size_t pr_hot_dynamic_smem(int32_t hot_n, int32_t tma_stages) {
    return (size_t)hot_n * sizeof(float) + (size_t)(PR_HOT_BLOCK / 32) * tma_stages * (TMA_STAGE_BYTES + 8);
}

int pr_blocks_per_sm(int32_t rank_type, int32_t gather_type, int32_t gmode, int persistent, int32_t hot_n,
                     int32_t tma_stages, bool bins) {
    int block = PR_BLOCK;
    size_t dyn = 0;
    void* k = nullptr;
    if (persistent == 1 && hot_n > 0) {
        dyn = pr_hot_dynamic_smem(hot_n, bins ? 0 : tma_stages);
        block = PR_HOT_BLOCK;
        k = pick_hot(rank_type, gather_type, dyn, tma_stages, bins);
    } else if (persistent == 1 && bins) {
        k = rank_type == GRB_FP32 && gather_type == GRB_FP32
                ? (void*)pr_persistent_kernel<float, float, PR_BLOCK, false, 0, false, true>
                : nullptr;
    } else {
        k = pick_kernel(rank_type, gather_type, gmode, persistent == 1, persistent == 2);
    }
    if (!k) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, dyn) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_pr(cudaStream_t st, const PrParams& p, int32_t rank_type, int32_t gather_type, int grid,
                      int persistent) {
    // persistent: 0 = one body (planner), 1 = whole loop, 2 = body of an
    // iterated sequence
    const bool hot = persistent == 1 && p.hot_n > 0;
    const bool bins = persistent == 1 && p.bin_rows;
    if (hot && (p.hot_n % 4 != 0 || p.hot_n > p.nrows || p.mixed)) return cudaErrorInvalidValue;
    if (bins && (p.mixed || p.tma_stages || rank_type != GRB_FP32 || gather_type != GRB_FP32))
        return cudaErrorInvalidValue;
    const size_t dyn = hot ? pr_hot_dynamic_smem(p.hot_n, bins ? 0 : p.tma_stages) : 0;
    void* k = hot ? pick_hot(rank_type, gather_type, dyn, p.tma_stages, bins)
            : bins ? (void*)pr_persistent_kernel<float, float, PR_BLOCK, false, 0, false, true>
                   : pick_kernel(rank_type, gather_type, p.gmode, persistent == 1, persistent == 2);
    if (!k) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(hot ? PR_HOT_BLOCK : PR_BLOCK);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {(void*)&p};
    return cudaLaunchKernelExC(&cfg, k, args);
}

cudaError_t launch_barrier_selftest(cudaStream_t st, SyncWords* sync, int32_t* status, int64_t spin_limit, int grid) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, sync, status, spin_limit);
}

}  // namespace grb
