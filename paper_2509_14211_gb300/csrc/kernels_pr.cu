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
// Work decomposition (merge path): the merge of the row-end offsets
// row_ptr[1..n] with the nonzero indices 0..nnz-1 is cut into warp tiles of
// PR_WTILE items, so every warp gets the same work whatever the row lengths
// (R-MAT in-degrees range from 0 to ~10^5).  Warps are independent: a warp
// stages its tile's row ends and gathered values in its own shared-memory
// slice, each lane walks PR_WITEMS merge items, and a warp-wide segmented
// scan (shuffles) joins rows split across lanes.  Rows split across tiles
// are finished in a second phase after a grid barrier, from per-tile carries
// (phase A writes them, phase B adds them up in a fixed order); there are no
// cross-warp waits inside a phase, and every barrier wait is bounded.  All
// reductions have a fixed order, so results are bit-reproducible.
#include <climits>

#include "grb_device.cuh"

namespace grb {

namespace {

constexpr int NWARP = PR_BLOCK / 32;
constexpr uint32_t FULLMASK = 0xffffffffu;

template <class T>
struct WarpSmem {
    int32_t rowend[PR_WTILE];
    T val[PR_WTILE];
    T rowsum[PR_WTILE];
};

template <class T>
struct Smem {
    WarpSmem<T> w[NWARP];
    double red[NWARP];
    double red2[NWARP];
    double bc[2];
    int ok;
};

template <class G, bool NC>
__device__ __forceinline__ float gload_f(const G* p, int64_t j);

template <>
__device__ __forceinline__ float gload_f<float, true>(const float* p, int64_t j) { return __ldg(p + j); }
template <>
__device__ __forceinline__ float gload_f<float, false>(const float* p, int64_t j) { return __ldcg(p + j); }
template <>
__device__ __forceinline__ float gload_f<__nv_bfloat16, true>(const __nv_bfloat16* p, int64_t j) {
    const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + j);
    return __uint_as_float(((uint32_t)b) << 16);
}
template <>
__device__ __forceinline__ float gload_f<__nv_bfloat16, false>(const __nv_bfloat16* p, int64_t j) {
    const unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p) + j);
    return __uint_as_float(((uint32_t)b) << 16);
}

template <class T, bool NC>
__device__ __forceinline__ T tload(const T* p, int64_t j) {
    if (NC) return __ldg(p + j);
    return __ldcg(p + j);
}

template <class G>
__device__ __forceinline__ void gstore(G* p, int64_t i, float x);
template <>
__device__ __forceinline__ void gstore<float>(float* p, int64_t i, float x) { p[i] = x; }
template <>
__device__ __forceinline__ void gstore<__nv_bfloat16>(__nv_bfloat16* p, int64_t i, float x) { p[i] = __float2bfloat16_rn(x); }

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
template <class T>
__device__ __forceinline__ void reduce_parts(const double* part, int n, double& a, double& b, Smem<T>& sm) {
    double x = 0.0, y = 0.0;
    for (int c = threadIdx.x; c < n; c += PR_BLOCK) {
        x += ld_relaxed_f64(part + 2 * c);
        y += ld_relaxed_f64(part + 2 * c + 1);
    }
    x = block_sum_d<PR_BLOCK>(x, sm.red);
    y = block_sum_d<PR_BLOCK>(y, sm.red2);
    if (threadIdx.x == 0) { sm.bc[0] = x; sm.bc[1] = y; }
    __syncthreads();
    a = sm.bc[0];
    b = sm.bc[1];
    __syncthreads();
}

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
};

// Everything a finished row produces: the output value, its presence, the
// next gather value, and its residual / dangling-mass contributions.
template <class T, class G, bool NC>
__device__ __forceinline__ void row_epilogue(const PrParams& p, const TileIO<T, G>& io, int64_t i, T s, bool nonempty,
                                             double& resid, double& dang) {
    T v;
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
    if (p.want_resid) resid += (double)abs_c<T>(tload<T, NC>(io.r_old, i) - v);
    if (p.want_dang && ((__ldg(p.sinkbits + (i >> 5)) >> (i & 31)) & 1u)) dang += (double)v;
    if (io.w_next || io.w32_next) {
        const T q = v / __ldg(reinterpret_cast<const T*>(p.dd) + i);
        if (io.w32_next) io.w32_next[i] = (float)q;
        else if constexpr (sizeof(T) == 8) reinterpret_cast<double*>(io.w_next)[i] = (double)q;
        else gstore<G>(io.w_next, i, (float)q);
    }
}

template <class T, class G, int GMODE, bool NC>
__device__ __forceinline__ T gather(const PrParams& p, const TileIO<T, G>& io, int32_t j) {
    if (GMODE == G_W) {
        if (io.phase32) return (T)gload_f<float, NC>(io.w32, j);
        if constexpr (sizeof(T) == 8) return tload<T, NC>(reinterpret_cast<const T*>(io.w), j);
        else return (T)gload_f<G, NC>(io.w, j);
    } else if (GMODE == G_TD) {
        return tload<T, NC>(io.t, j) / tload<T, NC>(io.d, j);
    }
    return (T)p.g_iso;
}

// Phase A for one warp tile: row sums of the rows that start and end in the
// tile go through the epilogue; the tile's part of a first row that began
// earlier goes to first[t]; the part of the row still open at the end goes
// to agg[t].
template <class T, class G, int GMODE, bool NC>
__device__ __forceinline__ void warp_tile(const PrParams& p, int t, const TileIO<T, G>& io, double& resid,
                                          double& dang, WarpSmem<T>& ws) {
    const int lane = threadIdx.x & 31;
    const int32_t i0 = __ldg(p.tile_i + t), k0 = __ldg(p.tile_k + t);
    const int32_t i1 = __ldg(p.tile_i + t + 1), k1 = __ldg(p.tile_k + t + 1);
    const int nA = i1 - i0, nB = k1 - k0;
    const int32_t row0start = __ldg(p.row_ptr + i0);

    // ---- stage: column indices, then the gathers; row ends
    int32_t cols[PR_WITEMS];
#pragma unroll
    for (int q = 0; q < PR_WITEMS; ++q) {
        const int y = lane + 32 * q;
        cols[q] = y < nB ? __ldg(p.col_idx + k0 + y) : 0;
    }
#pragma unroll
    for (int q = 0; q < PR_WITEMS; ++q) {
        const int x = lane + 32 * q;
        if (x < nA) ws.rowend[x] = __ldg(p.row_ptr + i0 + 1 + x);
    }
#pragma unroll
    for (int q = 0; q < PR_WITEMS; ++q) {
        const int y = lane + 32 * q;
        if (y < nB) ws.val[y] = gather<T, G, GMODE, NC>(p, io, cols[q]);
    }
    __syncwarp();

    // ---- per-lane merge walk over PR_WITEMS items
    const int total = nA + nB;
    int d0 = lane * PR_WITEMS;
    if (d0 > total) d0 = total;
    int d1 = d0 + PR_WITEMS;
    if (d1 > total) d1 = total;
    int lo = d0 - nB > 0 ? d0 - nB : 0;
    int hi = d0 < nA ? d0 : nA;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ws.rowend[mid] <= k0 + (d0 - mid - 1)) lo = mid + 1;
        else hi = mid;
    }
    int x = lo, y = d0 - lo;
    const int x_start = x;
    T acc = (T)0;
    for (int dd = d0; dd < d1; ++dd) {
        if (x < nA && (y >= nB || ws.rowend[x] <= k0 + y)) {
            ws.rowsum[x] = acc;
            acc = (T)0;
            ++x;
        } else {
            acc += ws.val[y];
            ++y;
        }
    }

    // ---- warp segmented (reduce-by-key) scan of the lane carries
    const int key = x;
    T val = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int k2 = __shfl_up_sync(FULLMASK, key, off);
        const T v2 = __shfl_up_sync(FULLMASK, val, off);
        if (lane >= off && k2 == key) val = v2 + val;
    }
    const int exk = __shfl_up_sync(FULLMASK, key, 1);
    const T exv = __shfl_up_sync(FULLMASK, val, 1);
    if (lane > 0 && x > x_start && exk == x_start) ws.rowsum[x_start] = exv + ws.rowsum[x_start];
    if (lane == 31) p.agg[t] = (double)val;
    __syncwarp();

    // ---- epilogue of the rows finished here
    const int x_lo = (k0 > row0start) ? 1 : 0;
    if (x_lo == 1 && nA > 0 && lane == 0) p.first[t] = (double)ws.rowsum[0];
    for (int xr = x_lo + lane; xr < nA; xr += 32) {
        const int32_t rs = xr == 0 ? row0start : ws.rowend[xr - 1];
        row_epilogue<T, G, NC>(p, io, (int64_t)i0 + xr, ws.rowsum[xr], ws.rowend[xr] > rs, resid, dang);
    }
    __syncwarp();
}

// Phase B: rows split across tiles.  Each thread takes tiles with a short
// fixup (at most PR_LONG carries to add); each warp takes a long one.
template <class T, class G, bool NC>
__device__ __forceinline__ void fixups(const PrParams& p, const TileIO<T, G>& io, double& resid, double& dang) {
    const int64_t nthreads = (int64_t)gridDim.x * PR_BLOCK;
    for (int64_t t = (int64_t)blockIdx.x * PR_BLOCK + threadIdx.x; t < p.ntiles; t += nthreads) {
        const FixDesc f = p.fix[t];
        if (f.row < 0 || t - f.ts > PR_LONG) continue;
        double sum = 0.0;
        for (int64_t tt = f.ts; tt < t; ++tt) sum += __ldcg(p.agg + tt);
        sum += __ldcg(p.first + t);
        row_epilogue<T, G, NC>(p, io, f.row, (T)sum, true, resid, dang);
    }
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * NWARP;
    for (int64_t q = (int64_t)blockIdx.x * NWARP + (threadIdx.x >> 5); q < p.nlong; q += nwarps) {
        const int32_t t = p.longfix[q];
        const FixDesc f = p.fix[t];
        double sum = 0.0;
        for (int64_t tt = f.ts + lane; tt < t; tt += 32) sum += __ldcg(p.agg + tt);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(FULLMASK, sum, off);
        if (lane == 0) {
            sum += __ldcg(p.first + t);
            row_epilogue<T, G, NC>(p, io, f.row, (T)sum, true, resid, dang);
        }
    }
}

template <class T>
__device__ __forceinline__ T tele_value(const PrParams& p) {
    return p.tele_from_slot ? (T)round_to(p.out.type, *p.tele_slot) : (T)0;
}

// One fused body per launch (also the fast unfused mxv): phase A, grid
// barrier, phase B, then the last CTA folds the per-CTA partials.  In an
// iterated sequence (p.iters_done != null) the launch first checks the loop
// condition left by the previous launch and does nothing once it fails.
template <class T, class G, int GMODE>
__global__ void __launch_bounds__(PR_BLOCK) pr_iter_kernel(const __grid_constant__ PrParams p) {
    __shared__ Smem<T> sm;
    __shared__ bool last;
    const bool iterated = p.iters_done != nullptr;
    const int it = p.iter_index;
    if (iterated) {
        const double rd = it == 0 ? p.rdiff0 : *(volatile double*)p.resid_slot;
        const int64_t done_so_far = *(volatile int64_t*)p.iters_done;
        if (!(rd > p.tol) || done_so_far != it) return;
    }
    TileIO<T, G> io{};
    io.tele_scalar = p.tele_from_slot;
    io.tele = tele_value<T>(p);
    if (iterated) {
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
    double resid = 0.0, dang = 0.0;
    const int warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * NWARP;
    for (int t = blockIdx.x * NWARP + warp; t < p.ntiles; t += nwarps)
        warp_tile<T, G, GMODE, true>(p, t, io, resid, dang, sm.w[warp]);
    if (!grid_sync(p.sync, p.status, p.spin_limit, gridDim.x, &sm.ok)) return;
    fixups<T, G, true>(p, io, resid, dang);
    resid = block_sum_d<PR_BLOCK>(resid, sm.red);
    dang = block_sum_d<PR_BLOCK>(dang, sm.red2);
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
        if (p.resid_slot && p.want_resid) *p.resid_slot = R;
        if (p.dang_slot && p.want_dang) *p.dang_slot = D;
        if (p.tele_slot && p.want_dang) *p.tele_slot = schain_apply(p.chain, D);
        if (iterated) {
            if (p.hist) p.hist[it] = R;
            *p.iters_done = it + 1;
        }
        p.sync->done = 0;
        p.sync->launch += 1;
    }
}

// Whole loop in one launch: prologue (w_0 = r_0 ./ d and the dangling mass of
// r_0), then bodies while the condition holds; each body is phase A,
// barrier, phase B, barrier, and every CTA folds the same partials in the
// same order, so all CTAs take the same loop decision.
template <class T, class G>
__global__ void __launch_bounds__(PR_BLOCK) pr_persistent_kernel(const __grid_constant__ PrParams p) {
    __shared__ Smem<T> sm;
    const int G_ = gridDim.x;
    const T* dd = reinterpret_cast<const T*>(p.dd);
    const T* r0 = reinterpret_cast<const T*>(p.r0);
    int phase32 = 0;
    const int warp = threadIdx.x >> 5;
    const int nwarps = G_ * NWARP;

    // prologue
    double dang = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * PR_BLOCK + threadIdx.x; i < p.nrows; i += (int64_t)G_ * PR_BLOCK) {
        const T rv = r0[i];
        const T q = rv / dd[i];
        if constexpr (sizeof(T) == 8) reinterpret_cast<double*>(p.wbuf[0])[i] = (double)q;
        else gstore<G>(reinterpret_cast<G*>(p.wbuf[0]), i, (float)q);
        if (p.want_dang && ((p.sinkbits[i >> 5] >> (i & 31)) & 1u)) dang += (double)rv;
    }
    dang = block_sum_d<PR_BLOCK>(dang, sm.red2);
    if (threadIdx.x == 0) {
        p.part[2 * blockIdx.x] = 0.0;
        p.part[2 * blockIdx.x + 1] = dang;
    }
    if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
    double R, D;
    reduce_parts<T>(p.part, G_, R, D, sm);
    T tele = p.tele_from_slot ? (T)round_to(p.out.type, schain_apply(p.chain, D)) : (T)0;
    double rd = p.rdiff0;
    int it = 0;
    while (it < p.iters && rd > p.tol) {
        TileIO<T, G> io{};
        io.r_old = it == 0 ? r0 : reinterpret_cast<const T*>(p.rbuf[(it - 1) & 1]);
        io.out = reinterpret_cast<T*>(p.rbuf[it & 1]);
        io.out_present = nullptr;
        io.w = reinterpret_cast<const G*>(p.wbuf[it & 1]);
        io.w_next = reinterpret_cast<G*>(p.wbuf[(it + 1) & 1]);
        io.w32 = reinterpret_cast<const float*>(p.wbuf32[it & 1]);
        io.w32_next = phase32 ? reinterpret_cast<float*>(p.wbuf32[(it + 1) & 1]) : nullptr;
        io.phase32 = phase32;
        io.tele = tele;
        io.tele_scalar = p.tele_from_slot;
        double resid = 0.0;
        dang = 0.0;
        for (int t = blockIdx.x * NWARP + warp; t < p.ntiles; t += nwarps)
            warp_tile<T, G, G_W, false>(p, t, io, resid, dang, sm.w[warp]);
        if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
        fixups<T, G, false>(p, io, resid, dang);
        resid = block_sum_d<PR_BLOCK>(resid, sm.red);
        dang = block_sum_d<PR_BLOCK>(dang, sm.red2);
        double* part = p.part + 2 * G_ * ((it + 1) & 1);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = resid;
            part[2 * blockIdx.x + 1] = dang;
        }
        if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
        reduce_parts<T>(part, G_, R, D, sm);
        rd = round_to(p.resid_type, R);
        if (p.tele_from_slot) tele = (T)round_to(p.out.type, schain_apply(p.chain, D));
        if (blockIdx.x == 0 && threadIdx.x == 0 && p.hist) p.hist[it] = rd;
        ++it;
        // mixed precision: once the residual is small, rebuild w in FP32 from
        // the rank just written and gather FP32 from the next body on
        if (p.mixed && !phase32 && rd < p.mixed_switch && it < p.iters && rd > p.tol) {
            const T* rcur = reinterpret_cast<const T*>(p.rbuf[(it - 1) & 1]);
            float* w32 = reinterpret_cast<float*>(p.wbuf32[it & 1]);
            for (int64_t i = (int64_t)blockIdx.x * PR_BLOCK + threadIdx.x; i < p.nrows; i += (int64_t)G_ * PR_BLOCK)
                w32[i] = (float)(__ldcg(rcur + i) / dd[i]);
            phase32 = 1;
            if (!grid_sync(p.sync, p.status, p.spin_limit, G_, &sm.ok)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (it > 0 && p.resid_slot) *p.resid_slot = rd;
        if (p.dang_slot) *p.dang_slot = D;
        if (p.tele_slot) *p.tele_slot = (double)tele;
        *p.iters_done = it;
        if (p.mixed_phase) *p.mixed_phase = phase32;
        p.sync->launch += 1;
    }
}

// A barrier that expects one arrival more than there are CTAs: every CTA's
// wait runs out after spin_limit polls and the kernel returns with
// GRB_DEVICE_TIMEOUT in *status.  Exercises the bounded-wait path.
__global__ void barrier_selftest_kernel(SyncWords* sync, int32_t* status, int64_t spin_limit) {
    __shared__ int ok;
    grid_sync(sync, status, spin_limit, gridDim.x + 1, &ok);
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

}  // namespace

int pr_blocks_per_sm(int32_t rank_type, int32_t gather_type, int32_t gmode, int persistent) {
    if (rank_type == GRB_FP64) {
        if (persistent) return occupancy(pr_persistent_kernel<double, double>);
        if (gmode == G_TD) return occupancy(pr_iter_kernel<double, double, G_TD>);
        if (gmode == G_ISO) return occupancy(pr_iter_kernel<double, double, G_ISO>);
        return occupancy(pr_iter_kernel<double, double, G_W>);
    }
    if (gather_type == GRB_BF16) {
        if (persistent) return occupancy(pr_persistent_kernel<float, __nv_bfloat16>);
        return occupancy(pr_iter_kernel<float, __nv_bfloat16, G_W>);
    }
    if (persistent) return occupancy(pr_persistent_kernel<float, float>);
    if (gmode == G_TD) return occupancy(pr_iter_kernel<float, float, G_TD>);
    if (gmode == G_ISO) return occupancy(pr_iter_kernel<float, float, G_ISO>);
    return occupancy(pr_iter_kernel<float, float, G_W>);
}

cudaError_t launch_pr(cudaStream_t st, const PrParams& p, int32_t rank_type, int32_t gather_type, int grid,
                      int persistent) {
    if (rank_type == GRB_FP64) {
        if (persistent) return coop_launch(pr_persistent_kernel<double, double>, grid, st, p);
        if (p.gmode == G_TD) return coop_launch(pr_iter_kernel<double, double, G_TD>, grid, st, p);
        if (p.gmode == G_ISO) return coop_launch(pr_iter_kernel<double, double, G_ISO>, grid, st, p);
        return coop_launch(pr_iter_kernel<double, double, G_W>, grid, st, p);
    }
    if (rank_type != GRB_FP32) return cudaErrorInvalidValue;
    if (gather_type == GRB_BF16) {
        if (persistent) return coop_launch(pr_persistent_kernel<float, __nv_bfloat16>, grid, st, p);
        if (p.gmode != G_W) return cudaErrorInvalidValue;
        return coop_launch(pr_iter_kernel<float, __nv_bfloat16, G_W>, grid, st, p);
    }
    if (persistent) return coop_launch(pr_persistent_kernel<float, float>, grid, st, p);
    if (p.gmode == G_TD) return coop_launch(pr_iter_kernel<float, float, G_TD>, grid, st, p);
    if (p.gmode == G_ISO) return coop_launch(pr_iter_kernel<float, float, G_ISO>, grid, st, p);
    return coop_launch(pr_iter_kernel<float, float, G_W>, grid, st, p);
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
