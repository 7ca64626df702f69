// CSR construction from a COO edge list on the GPU (integer, bit-exact), the
// per-column degree (the out-degree of §IV's PageRank when the stored matrix
// is A^T), and the merge-path tile plan used by the row-gather kernels.
//
// Build: pack each edge into one 64-bit key (row << cbits | col), sort the
// keys with a device radix sort over exactly the bits in use, drop duplicate
// keys (GRB_BUILD_DEDUP) and self loops (GRB_BUILD_DROP_SELF; they are given
// the out-of-range row `nrows` so that they sort last and are cut off), then
// split the keys into col_idx and derive row_ptr from the row boundaries.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

#include <climits>
#include <vector>

#include "grb_device.cuh"

namespace grb {

namespace {

__global__ void make_keys_kernel(int64_t m, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                 int64_t nrows, int64_t ncols, int transpose, int drop_self, int cbits,
                                 uint64_t* __restrict__ keys, int32_t* __restrict__ perm, int32_t* bad) {
    const uint64_t invalid = (uint64_t)nrows << cbits;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = transpose ? dst[e] : src[e];
        const int64_t c = transpose ? src[e] : dst[e];
        uint64_t key;
        if (r < 0 || r >= nrows || c < 0 || c >= ncols) {
            atomicMin(bad, (int32_t)e);
            key = invalid;
        } else if (drop_self && src[e] == dst[e]) {
            key = invalid;
        } else {
            key = ((uint64_t)r << cbits) | (uint64_t)c;
        }
        keys[e] = key;
        if (perm) perm[e] = (int32_t)e;
    }
}

// Number of keys below `invalid` in a sorted array (one thread).
__global__ void count_valid_kernel(const uint64_t* keys, const int64_t* nkeys_dev, int64_t nkeys_host,
                                   uint64_t invalid, int64_t* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t lo = 0, hi = nkeys_dev ? *nkeys_dev : nkeys_host;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < invalid) lo = mid + 1;
        else hi = mid;
    }
    *out = lo;
}

__global__ void split_keys_kernel(int64_t nv, const uint64_t* __restrict__ keys, int cbits, int64_t nrows,
                                  int32_t* __restrict__ row_ptr, int32_t* __restrict__ col_idx) {
    const uint64_t cmask = (cbits >= 64) ? ~0ull : ((1ull << cbits) - 1ull);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[e];
        const int64_t r = (int64_t)(key >> cbits);
        col_idx[e] = (int32_t)(key & cmask);
        const int64_t prev = (e == 0) ? -1 : (int64_t)(keys[e - 1] >> cbits);
        for (int64_t rr = prev + 1; rr <= r; ++rr) row_ptr[rr] = (int32_t)e;
        if (e == nv - 1)
            for (int64_t rr = r + 1; rr <= nrows; ++rr) row_ptr[rr] = (int32_t)nv;
    }
}

__global__ void gather_vals_kernel(int64_t nv, const int32_t* __restrict__ perm, const void* vin, void* vout,
                                   int32_t esize) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = perm[e];
        if (esize == 8) static_cast<uint64_t*>(vout)[e] = static_cast<const uint64_t*>(vin)[s];
        else if (esize == 4) static_cast<uint32_t*>(vout)[e] = static_cast<const uint32_t*>(vin)[s];
        else static_cast<uint16_t*>(vout)[e] = static_cast<const uint16_t*>(vin)[s];
    }
}

__global__ void col_count_kernel(int64_t nnz, const int32_t* __restrict__ col_idx, int32_t* deg) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[col_idx[p]], 1);
}

__global__ void deg_present_kernel(int64_t n, const int32_t* deg, uint8_t* present) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        present[i] = deg[i] > 0 ? 1 : 0;
}

__global__ void nonempty_kernel(int64_t nrows, const int32_t* row_ptr, unsigned long long* out) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x)
        c += row_ptr[i + 1] > row_ptr[i] ? 1 : 0;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

// Merge-path coordinates (rows consumed, nonzeros consumed) of the start of
// every tile: the merge of the row-end offsets row_ptr[1..n] with the
// nonzero indices 0..nnz-1, a row end taken first on ties.
__global__ void tile_plan_kernel(const int32_t* __restrict__ row_ptr, int32_t nrows, int32_t nnz, int64_t ntiles,
                                 int32_t* tile_i, int32_t* tile_k) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t total = (int64_t)nrows + nnz;
        const int64_t diag = t * PR_WTILE < total ? t * PR_WTILE : total;
        int64_t lo = diag - nnz > 0 ? diag - nnz : 0;
        int64_t hi = diag < nrows ? diag : nrows;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)row_ptr[mid + 1] <= diag - mid - 1) lo = mid + 1;
            else hi = mid;
        }
        tile_i[t] = (int32_t)lo;
        tile_k[t] = (int32_t)(diag - lo);
    }
}

// A tile whose first row i0 began before the tile (tile_k > row_ptr[i0]) and
// ends inside it (tile_i[t+1] > i0) gets a fixup: the row and the first tile
// ts holding its nonzeros (the last tile whose start is at or before the
// row's first nonzero).  Rows spanning more than PR_LONG tiles are listed
// separately for a warp-wide sum.
__global__ void fix_plan_kernel(const int32_t* __restrict__ row_ptr, int64_t ntiles, const int32_t* __restrict__ tile_i,
                                const int32_t* __restrict__ tile_k, FixDesc* fix, int32_t* longfix, int32_t* nlong) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i0 = tile_i[t];
        const int32_t start = row_ptr[i0];
        FixDesc f;
        f.row = -1;
        f.ts = 0;
        if (tile_k[t] > start && tile_i[t + 1] > i0) {
            int64_t lo = 0, hi = ntiles + 1;   // first index with tile_k > start
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (tile_k[mid] <= start) lo = mid + 1;
                else hi = mid;
            }
            f.row = i0;
            f.ts = (int32_t)(lo - 1);
            if (t - f.ts > PR_LONG) longfix[atomicAdd(nlong, 1)] = (int32_t)t;
        }
        fix[t] = f;
    }
}

inline int grid_for(int64_t n, int block = 256, int cap = 152 * 32) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

inline int bits_for(uint64_t x) {  // bits needed to represent values 0..x
    int b = 1;
    while (b < 63 && (x >> b) != 0) ++b;
    return b;
}

struct Scratch {
    AllocFn af;
    FreeFn ff;
    void* actx;
    std::vector<std::pair<void*, size_t>> held;
    void* get(size_t bytes) {
        void* p = af(actx, bytes ? bytes : 16);
        if (p) held.emplace_back(p, bytes ? bytes : 16);
        return p;
    }
    ~Scratch() {
        for (auto& h : held) ff(actx, h.first, h.second);
    }
};

}  // namespace

cudaError_t csr_build(cudaStream_t st, const CsrBuildArgs& a, AllocFn af, FreeFn ff, void* actx, int32_t** row_ptr_out,
                      int32_t** col_idx_out, void** vals_out, int64_t* nnz_out, int32_t* bad_index) {
    Scratch S{af, ff, actx, {}};
    const int64_t m = a.nedges;
    const int cbits = bits_for(a.ncols > 0 ? (uint64_t)(a.ncols - 1) : 0);
    const int rbits = bits_for((uint64_t)a.nrows);
    const int end_bit = cbits + rbits;
    const uint64_t invalid = (uint64_t)a.nrows << cbits;
    const int32_t esize = a.val_type == GRB_FP64 ? 8 : (a.val_type == GRB_BF16 ? 2 : 4);
    cudaError_t err;
    *bad_index = INT_MAX;

    uint64_t* keys = (uint64_t*)S.get(sizeof(uint64_t) * (m > 0 ? m : 1));
    uint64_t* keys2 = (uint64_t*)S.get(sizeof(uint64_t) * (m > 0 ? m : 1));
    int32_t* perm = a.vals ? (int32_t*)S.get(sizeof(int32_t) * (m > 0 ? m : 1)) : nullptr;
    int32_t* perm2 = a.vals ? (int32_t*)S.get(sizeof(int32_t) * (m > 0 ? m : 1)) : nullptr;
    int32_t* bad = (int32_t*)S.get(sizeof(int32_t));
    int64_t* counts = (int64_t*)S.get(2 * sizeof(int64_t));
    if (!keys || !keys2 || !bad || !counts || (a.vals && (!perm || !perm2))) return cudaErrorMemoryAllocation;
    const int32_t big = INT_MAX;
    if ((err = cudaMemcpyAsync(bad, &big, sizeof(int32_t), cudaMemcpyHostToDevice, st)) != cudaSuccess) return err;
    if (m > 0) {
        make_keys_kernel<<<grid_for(m), 256, 0, st>>>(m, a.src, a.dst, a.nrows, a.ncols, a.transpose, a.drop_self,
                                                      cbits, keys, perm, bad);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    int32_t bad_h = INT_MAX;
    if ((err = cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return err;
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
    if (bad_h != INT_MAX) {
        *bad_index = bad_h;
        return cudaSuccess;
    }

    // sort by (row, col); stable, so among duplicates the first edge comes first
    uint64_t* sorted = keys;
    int32_t* sperm = perm;
    if (m > 1) {
        size_t tbytes = 0;
        if (a.vals) err = cub::DeviceRadixSort::SortPairs(nullptr, tbytes, keys, keys2, perm, perm2, (int)m, 0, end_bit, st);
        else err = cub::DeviceRadixSort::SortKeys(nullptr, tbytes, keys, keys2, (int)m, 0, end_bit, st);
        if (err != cudaSuccess) return err;
        void* tmp = S.get(tbytes);
        if (!tmp) return cudaErrorMemoryAllocation;
        if (a.vals) err = cub::DeviceRadixSort::SortPairs(tmp, tbytes, keys, keys2, perm, perm2, (int)m, 0, end_bit, st);
        else err = cub::DeviceRadixSort::SortKeys(tmp, tbytes, keys, keys2, (int)m, 0, end_bit, st);
        if (err != cudaSuccess) return err;
        sorted = keys2;
        sperm = perm2;
    }
    const int64_t* nuniq_dev = nullptr;
    uint64_t* final_keys = sorted;
    int32_t* final_perm = sperm;
    if (a.dedup && m > 1) {
        uint64_t* ukeys = (sorted == keys) ? keys2 : keys;
        int32_t* uperm = (sperm == perm) ? perm2 : perm;
        size_t tbytes = 0;
        if (a.vals)
            err = cub::DeviceSelect::UniqueByKey(nullptr, tbytes, sorted, sperm, ukeys, uperm, counts, (int64_t)m, st);
        else
            err = cub::DeviceSelect::Unique(nullptr, tbytes, sorted, ukeys, counts, (int64_t)m, st);
        if (err != cudaSuccess) return err;
        void* tmp = S.get(tbytes);
        if (!tmp) return cudaErrorMemoryAllocation;
        if (a.vals)
            err = cub::DeviceSelect::UniqueByKey(tmp, tbytes, sorted, sperm, ukeys, uperm, counts, (int64_t)m, st);
        else
            err = cub::DeviceSelect::Unique(tmp, tbytes, sorted, ukeys, counts, (int64_t)m, st);
        if (err != cudaSuccess) return err;
        final_keys = ukeys;
        final_perm = uperm;
        nuniq_dev = counts;
    }
    count_valid_kernel<<<1, 32, 0, st>>>(final_keys, nuniq_dev, m, invalid, counts + 1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    int64_t nv = 0;
    if ((err = cudaMemcpyAsync(&nv, counts + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return err;
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;

    int32_t* row_ptr = (int32_t*)af(actx, sizeof(int32_t) * (a.nrows + 1));
    int32_t* col_idx = (int32_t*)af(actx, sizeof(int32_t) * (nv > 0 ? nv : 1));
    void* vals = a.vals ? af(actx, (size_t)esize * (nv > 0 ? nv : 1)) : nullptr;
    if (!row_ptr || !col_idx || (a.vals && !vals)) {
        if (row_ptr) ff(actx, row_ptr, sizeof(int32_t) * (a.nrows + 1));
        if (col_idx) ff(actx, col_idx, sizeof(int32_t) * (nv > 0 ? nv : 1));
        if (vals) ff(actx, vals, (size_t)esize * (nv > 0 ? nv : 1));
        return cudaErrorMemoryAllocation;
    }
    if (nv == 0) {
        if ((err = cudaMemsetAsync(row_ptr, 0, sizeof(int32_t) * (a.nrows + 1), st)) != cudaSuccess) return err;
    } else {
        split_keys_kernel<<<grid_for(nv), 256, 0, st>>>(nv, final_keys, cbits, a.nrows, row_ptr, col_idx);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if (a.vals) {
            gather_vals_kernel<<<grid_for(nv), 256, 0, st>>>(nv, final_perm, a.vals, vals, esize);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
        }
    }
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
    *row_ptr_out = row_ptr;
    *col_idx_out = col_idx;
    *vals_out = vals;
    *nnz_out = nv;
    return cudaSuccess;
}

cudaError_t launch_col_degree(cudaStream_t st, int64_t ncols, int64_t nnz, const int32_t* col_idx, int32_t* deg,
                              uint8_t* present) {
    cudaError_t e = cudaMemsetAsync(deg, 0, sizeof(int32_t) * (ncols > 0 ? ncols : 1), st);
    if (e != cudaSuccess) return e;
    if (nnz > 0) col_count_kernel<<<grid_for(nnz), 256, 0, st>>>(nnz, col_idx, deg);
    if (ncols > 0) deg_present_kernel<<<grid_for(ncols), 256, 0, st>>>(ncols, deg, present);
    return cudaGetLastError();
}

cudaError_t launch_nonempty_rows(cudaStream_t st, int64_t nrows, const int32_t* row_ptr, unsigned long long* out) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || nrows <= 0) return e;
    nonempty_kernel<<<grid_for(nrows, 256, 152 * 8), 256, 0, st>>>(nrows, row_ptr, out);
    return cudaGetLastError();
}

cudaError_t launch_tile_plan(cudaStream_t st, const int32_t* row_ptr, int32_t nrows, int32_t nnz, int64_t ntiles,
                             int32_t* tile_i, int32_t* tile_k) {
    tile_plan_kernel<<<grid_for(ntiles + 1), 256, 0, st>>>(row_ptr, nrows, nnz, ntiles, tile_i, tile_k);
    return cudaGetLastError();
}

cudaError_t launch_fix_plan(cudaStream_t st, const int32_t* row_ptr, int64_t ntiles, const int32_t* tile_i,
                            const int32_t* tile_k, FixDesc* fix, int32_t* longfix, int32_t* nlong_dev) {
    cudaError_t e = cudaMemsetAsync(nlong_dev, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    fix_plan_kernel<<<grid_for(ntiles), 256, 0, st>>>(row_ptr, ntiles, tile_i, tile_k, fix, longfix, nlong_dev);
    return cudaGetLastError();
}

}  // namespace grb
