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
// Work decomposition: merge-path tiles.  The merge of the row-end offsets
// row_ptr[1..n] with the nonzero indices 0..nnz-1 is cut into tiles of
// PR_TILE items, so every CTA gets the same amount of work whatever the row
// lengths (R-MAT in-degrees range from 0 to ~10^5).  A tile stages its row
// ends and its gathered values in shared memory (coalesced col_idx loads),
// each thread walks PR_ITEMS merge items, a block-wide segmented scan joins
// rows split across threads, and rows split across tiles are joined by a
// look-back on published per-tile carries (tiles only ever wait on lower
// tiles, which are owned by co-resident CTAs of a cooperative launch, so the
// waits always end; every wait is bounded anyway and reports a timeout
// instead of hanging).  All reductions are fixed-order: results are
// bit-reproducible run to run.
#include <climits>

#include "grb_device.cuh"

namespace grb {

namespace {

constexpr int NW = PR_BLOCK / 32;
constexpr uint32_t FULLMASK = 0xffffffffu;

template <class T>
struct Smem {
    int32_t rowend[PR_TILE];
    T val[PR_TILE];
    T rowsum[PR_TILE];
    int32_t row0start;
    int32_t wkey[NW], wpk[NW];
    T wval[NW], wpv[NW];
    double red[NW];
    double red2[NW];
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

__device__ __forceinline__ void gstore_d(double* p, int64_t i, double x) { p[i] = x; }

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

// Bounded grid-wide barrier (all CTAs of a cooperative launch).  Returns
// false when a wait ran out (status set); callers then leave the kernel.
__device__ bool grid_sync(SyncWords* s, int32_t* status, int64_t spin_limit, uint32_t expected) {
    __shared__ int ok_sh;
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
                __nanosleep(64);
            }
        }
        __threadfence();
        if (ok && status && *(volatile int32_t*)status != 0) ok = 0;
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Deterministic fold of the per-CTA partials part[0..n) (pairs of doubles).
__device__ __forceinline__ void reduce_parts(const double* part, int n, double& a, double& b, double* sh, double* sh2) {
    double x = 0.0, y = 0.0;
    for (int c = threadIdx.x; c < n; c += PR_BLOCK) {
        x += ld_relaxed_f64(part + 2 * c);
        y += ld_relaxed_f64(part + 2 * c + 1);
    }
    x = block_sum_d<PR_BLOCK>(x, sh);
    y = block_sum_d<PR_BLOCK>(y, sh2);
    __shared__ double bc[2];
    if (threadIdx.x == 0) { bc[0] = x; bc[1] = y; }
    __syncthreads();
    a = bc[0];
    b = bc[1];
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

template <class T, class G, int GMODE, bool NC>
__device__ __forceinline__ void process_tile(const PrParams& p, int t, uint32_t epoch, const TileIO<T, G>& io,
                                             double& resid, double& dang, Smem<T>& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t i0 = __ldg(p.tile_i + t), k0 = __ldg(p.tile_k + t);
    const int32_t i1 = __ldg(p.tile_i + t + 1), k1 = __ldg(p.tile_k + t + 1);
    const int nA = i1 - i0, nB = k1 - k0;

    // ---- stage row ends and gathered values
    if (tid == 0) sm.row0start = __ldg(p.row_ptr + i0);
    for (int x = tid; x < nA; x += PR_BLOCK) sm.rowend[x] = __ldg(p.row_ptr + i0 + 1 + x);
    int32_t cols[PR_ITEMS];
#pragma unroll
    for (int q = 0; q < PR_ITEMS; ++q) {
        const int y = tid + q * PR_BLOCK;
        cols[q] = y < nB ? __ldg(p.col_idx + k0 + y) : 0;
    }
#pragma unroll
    for (int q = 0; q < PR_ITEMS; ++q) {
        const int y = tid + q * PR_BLOCK;
        if (y < nB) {
            T g;
            if (GMODE == G_W) {
                if (io.phase32) g = (T)gload_f<float, NC>(io.w32, cols[q]);
                else if constexpr (sizeof(T) == 8) g = tload<T, NC>(reinterpret_cast<const T*>(io.w), cols[q]);
                else g = (T)gload_f<G, NC>(io.w, cols[q]);
            } else if (GMODE == G_TD) {
                g = tload<T, NC>(io.t, cols[q]) / tload<T, NC>(io.d, cols[q]);
            } else {
                g = (T)p.g_iso;
            }
            sm.val[y] = g;
        }
    }
    __syncthreads();

    // ---- per-thread merge walk
    const int total = nA + nB;
    int d0 = tid * PR_ITEMS;
    if (d0 > total) d0 = total;
    int d1 = d0 + PR_ITEMS;
    if (d1 > total) d1 = total;
    int lo = d0 - nB > 0 ? d0 - nB : 0;
    int hi = d0 < nA ? d0 : nA;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sm.rowend[mid] <= k0 + (d0 - mid - 1)) lo = mid + 1;
        else hi = mid;
    }
    int x = lo, y = d0 - lo;
    const int x_start = x;
    T acc = (T)0;
    for (int dd = d0; dd < d1; ++dd) {
        if (x < nA && (y >= nB || sm.rowend[x] <= k0 + y)) {
            sm.rowsum[x] = acc;
            acc = (T)0;
            ++x;
        } else {
            acc += sm.val[y];
            ++y;
        }
    }

    // ---- block-wide segmented (reduce-by-key) scan of the thread carries
    int key = x;
    T val = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int k2 = __shfl_up_sync(FULLMASK, key, off);
        const T v2 = __shfl_up_sync(FULLMASK, val, off);
        if (lane >= off && k2 == key) val = v2 + val;
    }
    if (lane == 31) { sm.wkey[warp] = key; sm.wval[warp] = val; }
    __syncthreads();
    if (warp == 0) {
        int wk = lane < NW ? sm.wkey[lane] : INT_MAX;
        T wv = lane < NW ? sm.wval[lane] : (T)0;
#pragma unroll
        for (int off = 1; off < NW; off <<= 1) {
            const int k2 = __shfl_up_sync(FULLMASK, wk, off);
            const T v2 = __shfl_up_sync(FULLMASK, wv, off);
            if (lane >= off && k2 == wk) wv = v2 + wv;
        }
        const int ek = __shfl_up_sync(FULLMASK, wk, 1);
        const T ev = __shfl_up_sync(FULLMASK, wv, 1);
        if (lane < NW) {
            sm.wpk[lane] = lane == 0 ? -1 : ek;
            sm.wpv[lane] = lane == 0 ? (T)0 : ev;
        }
    }
    __syncthreads();
    const int pk = sm.wpk[warp];
    const T pv = sm.wpv[warp];
    const T incl = (pk == key) ? pv + val : val;
    int exk = __shfl_up_sync(FULLMASK, key, 1);
    T exv = __shfl_up_sync(FULLMASK, incl, 1);
    if (lane == 0) { exk = pk; exv = pv; }
    if (x > x_start && exk == x_start) sm.rowsum[x_start] = exv + sm.rowsum[x_start];
    __syncthreads();  // the look-back below updates rowsum[0] too

    // ---- publish the carry of the row still open at the tile end
    if (tid == PR_BLOCK - 1) {
        p.agg[t] = (double)incl;
        st_release_u32(p.flag + t, epoch);
    }

    // ---- look-back: the first row began in earlier tiles
    if (warp == 0 && nA > 0 && k0 > sm.row0start) {
        const int32_t rstart = sm.row0start;
        double P = 0.0;
        int base = t - 1;
        bool done = false;
        while (!done) {
            const int tt = base - lane;
            double v = 0.0;
            bool stop_here = true;
            if (tt >= 0 && __ldg(p.tile_k + tt + 1) > rstart) {
                stop_here = __ldg(p.tile_k + tt) <= rstart;
                int64_t spins = 0;
                while (ld_acquire_u32(p.flag + tt) != epoch) {
                    // give up after spin_limit polls, or at once when another
                    // wait of this launch already gave up
                    if (++spins > p.spin_limit || ((spins & 255) == 0 && *(volatile int32_t*)p.status != 0)) {
                        set_status(p.status, (int32_t)GRB_DEVICE_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                }
                v = ld_relaxed_f64(p.agg + tt);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(FULLMASK, v, off);
            P += __shfl_sync(FULLMASK, v, 0);
            done = __any_sync(FULLMASK, stop_here);
            base -= 32;
        }
        if (lane == 0) sm.rowsum[0] = (T)P + sm.rowsum[0];
    }
    __syncthreads();

    // ---- row epilogue (coalesced over the tile's rows)
    for (int xr = tid; xr < nA; xr += PR_BLOCK) {
        const int64_t i = (int64_t)i0 + xr;
        const int32_t rs = xr == 0 ? sm.row0start : sm.rowend[xr - 1];
        const bool nonempty = sm.rowend[xr] > rs;
        const T s = sm.rowsum[xr];
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
        if (p.want_resid) {
            const T ro = tload<T, NC>(io.r_old, i);
            resid += (double)abs_c<T>(ro - v);
        }
        if (p.want_dang && ((__ldg(p.sinkbits + (i >> 5)) >> (i & 31)) & 1u)) dang += (double)v;
        if (io.w_next || io.w32_next) {
            const T q = v / __ldg(reinterpret_cast<const T*>(p.dd) + i);
            if (io.w32_next) io.w32_next[i] = (float)q;
            else if constexpr (sizeof(T) == 8) gstore_d(reinterpret_cast<double*>(io.w_next), i, (double)q);
            else gstore<G>(io.w_next, i, (float)q);
        }
    }
    __syncthreads();
}

template <class T>
__device__ __forceinline__ T tele_value(const PrParams& p) {
    return p.tele_from_slot ? (T)round_to(p.out.type, *p.tele_slot) : (T)0;
}

// One fused body per launch (also the fast unfused mxv).  In an iterated
// sequence (p.iters_done != null) the launch first checks the loop
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
    const uint32_t epoch = *(volatile uint32_t*)&p.sync->launch + 1u;
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
    for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x)
        process_tile<T, G, GMODE, true>(p, t, epoch, io, resid, dang, sm);
    if (!p.want_resid && !p.want_dang && !iterated) {
        // no reductions: only the epoch counter needs the last block
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(&p.sync->done, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            p.sync->done = 0;
            p.sync->launch = epoch;
        }
        return;
    }
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
    reduce_parts(p.part, gridDim.x, R, D, sm.red, sm.red2);
    if (threadIdx.x == 0) {
        R = round_to(p.resid_type, R);
        if (p.resid_slot) *p.resid_slot = R;
        if (p.dang_slot) *p.dang_slot = D;
        if (p.tele_slot && p.want_dang) *p.tele_slot = schain_apply(p.chain, D);
        if (iterated) {
            if (p.hist) p.hist[it] = R;
            *p.iters_done = it + 1;
        }
        p.sync->done = 0;
        p.sync->launch = epoch;
    }
}

// Whole loop in one launch: prologue (w_0 = r_0 ./ d and the dangling mass of
// r_0), then bodies separated by grid barriers while the condition holds.
template <class T, class G>
__global__ void __launch_bounds__(PR_BLOCK) pr_persistent_kernel(const __grid_constant__ PrParams p) {
    __shared__ Smem<T> sm;
    const uint32_t base_epoch = *(volatile uint32_t*)&p.sync->launch;
    const int G_ = gridDim.x;
    const T* dd = reinterpret_cast<const T*>(p.dd);
    const T* r0 = reinterpret_cast<const T*>(p.r0);
    int phase32 = 0;

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
    if (!grid_sync(p.sync, p.status, p.spin_limit, G_)) return;
    double R, D;
    reduce_parts(p.part, G_, R, D, sm.red, sm.red2);
    T tele = p.tele_from_slot ? (T)round_to(p.out.type, schain_apply(p.chain, D)) : (T)0;
    double rd = p.rdiff0;
    int it = 0;
    while (it < p.iters && rd > p.tol) {
        const uint32_t epoch = base_epoch + 1u + (uint32_t)it;
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
        for (int t = blockIdx.x; t < p.ntiles; t += G_)
            process_tile<T, G, G_W, false>(p, t, epoch, io, resid, dang, sm);
        resid = block_sum_d<PR_BLOCK>(resid, sm.red);
        dang = block_sum_d<PR_BLOCK>(dang, sm.red2);
        double* part = p.part + 2 * G_ * ((it + 1) & 1);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = resid;
            part[2 * blockIdx.x + 1] = dang;
        }
        if (!grid_sync(p.sync, p.status, p.spin_limit, G_)) return;
        reduce_parts(part, G_, R, D, sm.red, sm.red2);
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
            if (!grid_sync(p.sync, p.status, p.spin_limit, G_)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (it > 0 && p.resid_slot) *p.resid_slot = rd;
        if (p.dang_slot) *p.dang_slot = D;
        if (p.tele_slot) *p.tele_slot = (double)tele;
        *p.iters_done = it;
        if (p.mixed_phase) *p.mixed_phase = phase32;
        p.sync->launch = base_epoch + (uint32_t)it;
    }
}

// A barrier that expects one arrival more than there are CTAs: every CTA's
// wait runs out after spin_limit polls and the kernel returns with
// GRB_DEVICE_TIMEOUT in *status.  Exercises the bounded-wait path.
__global__ void barrier_selftest_kernel(SyncWords* sync, int32_t* status, int64_t spin_limit) {
    grid_sync(sync, status, spin_limit, gridDim.x + 1);
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
