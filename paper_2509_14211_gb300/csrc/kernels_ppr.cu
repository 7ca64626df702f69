// Batched personalised PageRank: k queries iterate together as one sparse x
// dense product over A^T.  The paper's method runs one rank vector; here the
// same fused body (division folded into the previous epilogue, row sums,
// teleport, residual and dangling mass in the row epilogue) runs for
// PPR_LANES slots per warp:
//
//   r_s' = (1 - d) v_s + d D_s / n + A^T w_s,   w_s = r_s ./ dvec,
//   D_s  = sum of r_s over vertices without out-edges,  res_s = |r_s - r_s'|_1
//
// with v_s uniform over slot s's seed set (dangling mass spread over all n
// vertices, so r_s is linear in v_s).
//
// Layout: r and w are [k-tile][n][32] FP32 -- lane l of a warp owns slot
// 32*kt + l, and the values of one source vertex for a k-tile are one
// contiguous 128-byte line, so every gather is a fully used cache line.
// A warp walks the nonzeros of a 256-nonzero tile (the same tile plan as the
// single-vector kernels) one by one, all lanes adding their slot's value;
// row ends come from the row-end bitmap.  Rows split across tiles are
// finished by ppr_fixups_kernel from per-tile carries, and
// ppr_finish_kernel folds the per-CTA partials of every slot in a fixed
// order.  The three kernels of an iteration are separated by kernel
// boundaries (the caller captures iterations in a CUDA graph), so there are
// no device-side waits.
//
// Every slot's arithmetic (row sums in tile order, carries in tile order,
// fixed-order folds over a grid that does not depend on k) is independent of
// the other slots: a query gives the same bits alone and in any batch.
#include "grb_device.cuh"

namespace grb {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int NW = PPR_BLOCK / 32;
constexpr int KT_MAX = PPR_MAX_SLOTS / PPR_LANES;

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

struct PprSmem {
    double res[KT_MAX][NW][32];
    double dang[KT_MAX][NW][32];
};

__device__ __forceinline__ bool bit_of(const uint32_t* b, int i) { return (__ldg(b + (i >> 5)) >> (i & 31)) & 1u; }

// (1 - d) v_s[i] for this lane's slot.  The seed bitmap filters almost every
// row; on a hit the k-tile's seed rows (sorted) are binary-searched.  The row
// is the same for the whole warp, so the control flow is uniform.
__device__ __forceinline__ float seed_term(const PprParams& p, int kt, int i, int lane) {
    if (!bit_of(p.seedbits, i)) return 0.f;
    int lo = __ldg(p.seed_ptr + kt), hi = __ldg(p.seed_ptr + kt + 1);
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(p.seed_row + mid) < i) lo = mid + 1;
        else hi = mid;
    }
    float v = 0.f;
    for (int e = lo; e < end && __ldg(p.seed_row + e) == i; ++e)
        if (__ldg(p.seed_lane + e) == lane) v = __ldg(p.seed_val + e);
    return v;
}

// Epilogue of row i for this lane's slot: r' = (seed + d D / n) + sum, the
// next gather value, and the residual / dangling-mass terms.  A finished
// (inactive) slot writes nothing: its last iterate stays in the buffer the
// finish kernel recorded.
__device__ __forceinline__ void ppr_row(const PprParams& p, int kt, int i, float sum, int lane, bool act, float tb,
                                        Kahan& res, Kahan& dang) {
    const float sv = seed_term(p, kt, i, lane);   // uniform across the warp
    if (!act) return;
    const size_t o = ((size_t)kt * (size_t)p.nrows + (size_t)i) * PPR_LANES + (size_t)lane;
    const float rold = __ldcs(p.r_old + o);
    const float dd = __ldg(p.dd + i);
    const float rn = (sv + tb) + sum;
    __stcs(p.r_new + o, rn);
    p.w_new[o] = rn / dd;
    res.add(fabsf(rold - rn));
    if (bit_of(p.sinkbits, i)) dang.add(rn);
}

// Per-CTA partials of every slot: the warps' accumulators folded in warp
// order.
__device__ __forceinline__ void flush_slot_partials(const PprParams& p, PprSmem& sm) {
    __syncthreads();
    const int S = p.kt * PPR_LANES;
    for (int s = threadIdx.x; s < S; s += PPR_BLOCK) {
        const int kt = s / PPR_LANES, l = s % PPR_LANES;
        double a = 0.0, b = 0.0;
        for (int w = 0; w < NW; ++w) {
            a += sm.res[kt][w][l];
            b += sm.dang[kt][w][l];
        }
        p.part[((size_t)blockIdx.x * S + s) * 2] = a;
        p.part[((size_t)blockIdx.x * S + s) * 2 + 1] = b;
    }
}

__device__ __forceinline__ void zero_smem(PprSmem& sm, int kts) {
    for (int q = threadIdx.x; q < kts * NW * 32; q += PPR_BLOCK) {
        (&sm.res[0][0][0])[q] = 0.0;
        (&sm.dang[0][0][0])[q] = 0.0;
    }
    __syncthreads();
}

// Phase A: the warp tiles, k-tile by k-tile (so the warps of the GPU share
// one k-tile of w in L2 at a time), then the empty rows.  Tile t goes to the
// same warp in every k-tile, so every slot sees the same summation order.
__device__ __forceinline__ void ppr_tile(const PprParams& p, int kt, int t, int lane, bool act, float tb, Kahan& res,
                                         Kahan& dang) {
    const uint32_t meta = __ldg(p.tile_meta + t);
    const int rfirst = (int)(meta & 0x7fffffffu);
    const int x_lo = (int)(meta >> 31);
    const int kl = t * PR_NZTILE + lane * PR_NZLANE;
    const int4* cp = reinterpret_cast<const int4*>(p.col_idx + kl);
    const int4 ca = __ldcs(cp), cb = __ldcs(cp + 1);
    const uint32_t myf = (__ldcs(p.rowend_bits + (kl >> 5)) >> (kl & 31)) & 0xffu;
    const int nvalid = min(max(p.nnz - t * PR_NZTILE, 0), PR_NZTILE);
    const int pre_i = rfirst + lane < p.n_ne ? __ldg(p.ne_rows + rfirst + lane) : 0;
    const float* W = p.w_old + (size_t)kt * (size_t)p.nrows * PPR_LANES + lane;
    const size_t tslot = ((size_t)kt * p.ntiles + t) * PPR_LANES + lane;
    float acc = 0.f;
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
        const uint32_t f = __shfl_sync(FULL, myf, src);
        float v[PR_NZLANE];
#pragma unroll
        for (int q = 0; q < PR_NZLANE; ++q)
            v[q] = src * PR_NZLANE + q < nvalid ? __ldg(W + (size_t)c[q] * PPR_LANES) : 0.f;
#pragma unroll
        for (int q = 0; q < PR_NZLANE; ++q) {
            acc += v[q];
            if ((f >> q) & 1u) {
                if (r == 0 && x_lo) {
                    p.first[tslot] = acc;   // a row begun in an earlier tile: phase B
                } else {
                    const int i = r < 32 ? __shfl_sync(FULL, pre_i, r) : __ldg(p.ne_rows + rfirst + r);
                    ppr_row(p, kt, i, acc, lane, act, tb, res, dang);
                }
                ++r;
                acc = 0.f;
            }
        }
    }
    p.agg[tslot] = acc;   // the row still open at the tile's end
}

__global__ void __launch_bounds__(PPR_BLOCK, 2) ppr_tiles_kernel(const __grid_constant__ PprParams p) {
    __shared__ PprSmem sm;
    zero_smem(sm, p.kt);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * NW;
    const int w0 = blockIdx.x * NW + warp;
    for (int kt = 0; kt < p.kt; ++kt) {
        Kahan res, dang;
        const bool act = __ldg(p.active + kt * PPR_LANES + lane) != 0;
        const float tb = __ldg(p.tele_base + kt * PPR_LANES + lane);
        // a k-tile without an active slot is skipped (the same decision in
        // every warp: all read the same flags)
        if (!__any_sync(FULL, act)) {
            sm.res[kt][warp][lane] = 0.0;
            sm.dang[kt][warp][lane] = 0.0;
            continue;
        }
        for (int t = w0; t < p.ntiles; t += nwarps) ppr_tile(p, kt, t, lane, act, tb, res, dang);
        // rows without nonzeros: the epilogue with an empty sum
        for (int e = w0; e < p.n_empty; e += nwarps)
            ppr_row(p, kt, __ldg(p.empty_rows + e), 0.f, lane, act, tb, res, dang);
        sm.res[kt][warp][lane] = res.value();
        sm.dang[kt][warp][lane] = dang.value();
    }
    flush_slot_partials(p, sm);
}

// Phase B: rows split across tiles, one warp per (k-tile, tile) with a
// fixup: the carries of the earlier tiles in tile order, then this tile's
// part.
__global__ void __launch_bounds__(PPR_BLOCK, 2) ppr_fixups_kernel(const __grid_constant__ PprParams p) {
    __shared__ PprSmem sm;
    zero_smem(sm, p.kt);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * NW;
    for (int kt = 0; kt < p.kt; ++kt) {
        Kahan res, dang;
        const bool act = __ldg(p.active + kt * PPR_LANES + lane) != 0;
        const float tb = __ldg(p.tele_base + kt * PPR_LANES + lane);
        if (!__any_sync(FULL, act)) {
            sm.res[kt][warp][lane] = 0.0;
            sm.dang[kt][warp][lane] = 0.0;
            continue;
        }
        for (int t = blockIdx.x * NW + warp; t < p.ntiles; t += nwarps) {
            const FixDesc f = p.fix[t];
            if (f.row < 0) continue;
            const size_t base = (size_t)kt * p.ntiles * PPR_LANES + lane;
            float sum = 0.f;
            for (int tt = f.ts; tt < t; ++tt) sum += __ldcg(p.agg + base + (size_t)tt * PPR_LANES);
            sum += __ldcg(p.first + base + (size_t)t * PPR_LANES);
            ppr_row(p, kt, f.row, sum, lane, act, tb, res, dang);
        }
        sm.res[kt][warp][lane] = res.value();
        sm.dang[kt][warp][lane] = dang.value();
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

__global__ void ppr_init_zero_kernel(PprInit a) {
    const int kt = a.slot / PPR_LANES, l = a.slot % PPR_LANES;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nrows; i += gridDim.x * blockDim.x) {
        const size_t o = ((size_t)kt * a.nrows + i) * PPR_LANES + l;
        a.r[o] = 0.f;
        a.w[o] = 0.f;
    }
}

__global__ void ppr_init_seed_kernel(PprInit a) {
    const int kt = a.slot / PPR_LANES, l = a.slot % PPR_LANES;
    double D = 0.0;
    for (int q = threadIdx.x; q < a.nseeds; q += blockDim.x) {
        const int i = a.seeds[q];
        const size_t o = ((size_t)kt * a.nrows + i) * PPR_LANES + l;
        a.r[o] = a.r0;
        a.w[o] = a.r0 / a.dd[i];
    }
    // dangling mass of the start vector (one thread, in seed order)
    if (threadIdx.x == 0) {
        for (int q = 0; q < a.nseeds; ++q)
            if ((a.sinkbits[a.seeds[q] >> 5] >> (a.seeds[q] & 31)) & 1u) D += (double)a.r0;
        a.tele_base[a.slot] = (float)(a.damping * D / (double)a.nrows);
    }
}

__global__ void ppr_seedbits_kernel(int32_t nseeds, const int32_t* rows, uint32_t* bits) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nseeds; q += gridDim.x * blockDim.x)
        atomicOr(bits + (rows[q] >> 5), 1u << (rows[q] & 31));
}

__global__ void ppr_extract_kernel(int32_t n, const float* r, int32_t slot, float* out) {
    const int kt = slot / PPR_LANES, l = slot % PPR_LANES;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = r[((size_t)kt * n + i) * PPR_LANES + l];
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

}  // namespace

int ppr_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ppr_tiles_kernel, PPR_BLOCK, 0) != cudaSuccess) return 1;
    int nb2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, ppr_fixups_kernel, PPR_BLOCK, 0) != cudaSuccess) return 1;
    nb = nb < nb2 ? nb : nb2;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_ppr_tiles(cudaStream_t st, const PprParams& p, int grid) {
    if (p.kt < 1 || p.kt > KT_MAX) return cudaErrorInvalidValue;
    ppr_tiles_kernel<<<grid, PPR_BLOCK, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_ppr_fixups(cudaStream_t st, const PprParams& p, int grid) {
    if (p.kt < 1 || p.kt > KT_MAX) return cudaErrorInvalidValue;
    ppr_fixups_kernel<<<grid, PPR_BLOCK, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_ppr_finish(cudaStream_t st, const PprFinish& f) {
    const int per_block = 8;
    ppr_finish_kernel<<<(f.slots + per_block - 1) / per_block, 32 * per_block, 0, st>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_ppr_init_slot(cudaStream_t st, const PprInit& a) {
    ppr_init_zero_kernel<<<grid_1d(a.nrows), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ppr_init_seed_kernel<<<1, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ppr_seedbits(cudaStream_t st, int32_t nseeds, const int32_t* rows, uint32_t* bits, int64_t nwords) {
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (size_t)nwords, st);
    if (e != cudaSuccess || nseeds <= 0) return e;
    ppr_seedbits_kernel<<<grid_1d(nseeds), 256, 0, st>>>(nseeds, rows, bits);
    return cudaGetLastError();
}

cudaError_t launch_ppr_extract(cudaStream_t st, int32_t n, const float* r, int32_t slot, float* out) {
    ppr_extract_kernel<<<grid_1d(n), 256, 0, st>>>(n, r, slot, out);
    return cudaGetLastError();
}

cudaError_t launch_ppr_divisor(cudaStream_t st, int32_t n, const int32_t* deg, double damping, float* dd,
                               uint32_t* sinkbits) {
    ppr_divisor_kernel<<<grid_1d(n), 256, 0, st>>>(n, deg, damping, dd, sinkbits);
    return cudaGetLastError();
}

}  // namespace grb
