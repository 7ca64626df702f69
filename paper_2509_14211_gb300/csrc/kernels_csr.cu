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
#include <cub/device/device_scan.cuh>
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

// Structure check of a CSR matrix: row_ptr starts at 0, ends at nnz and
// never decreases; every column index lies in [0, ncols).  Reads only
// row_ptr[0..nrows] and col_idx[0..nnz) -- no value read is used as an
// address -- and records the first failure in the status words.
__global__ void csr_check_kernel(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col_idx, int32_t* status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i <= nrows; i += stride) {
        const int64_t a = row_ptr[i];
        bool bad = a < 0 || a > nnz || (i == 0 && a != 0) || (i == nrows && a != nnz);
        if (i < nrows && (int64_t)row_ptr[i + 1] < a) bad = true;
        if (bad) bounds_record(status, BOUNDS_ROW_PTR, (long long)i);
    }
    for (int64_t k = t0; k < nnz; k += stride) {
        const int64_t j = col_idx[k];
        if (j < 0 || j >= ncols) bounds_record(status, BOUNDS_COLUMN, (long long)j);
    }
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

// ---------------------------------------------------------- row plan
// Ordered split of the rows into non-empty and empty ones: block b covers
// rows [256b, 256b+256); pass 1 counts its non-empty rows, an exclusive scan
// gives offsets, pass 2 writes both lists in ascending order.
__global__ void row_count_kernel(int32_t nrows, const int32_t* __restrict__ row_ptr, int32_t* block_counts) {
    const int32_t i = blockIdx.x * 256 + threadIdx.x;
    const bool ne = i < nrows && row_ptr[i + 1] > row_ptr[i];
    const int c = __syncthreads_count(ne);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = c;
}

__global__ void row_split_kernel(int32_t nrows, const int32_t* __restrict__ row_ptr, const int32_t* block_off,
                                 int32_t* ne_rows, int32_t* empty_rows) {
    __shared__ int warp_ne[8];
    const int32_t i = blockIdx.x * 256 + threadIdx.x;
    const bool valid = i < nrows;
    const bool ne = valid && row_ptr[i + 1] > row_ptr[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ball = __ballot_sync(0xffffffffu, ne);
    if (lane == 0) warp_ne[warp] = __popc(ball);
    __syncthreads();
    int before_ne = 0;
    for (int w = 0; w < warp; ++w) before_ne += warp_ne[w];
    before_ne += __popc(ball & ((1u << lane) - 1u));
    const int32_t ne_off = block_off[blockIdx.x] + before_ne;
    if (ne) ne_rows[ne_off] = i;
    else if (valid) empty_rows[(blockIdx.x * 256 - block_off[blockIdx.x]) + (threadIdx.x - before_ne)] = i;
}

// Bit (end-1) of every non-empty row: its last nonzero.
__global__ void rowend_bits_kernel(int32_t n_ne, const int32_t* __restrict__ ne_rows,
                                   const int32_t* __restrict__ row_ptr, uint32_t* bits) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_ne; r += gridDim.x * blockDim.x) {
        const int32_t k = row_ptr[ne_rows[r] + 1] - 1;
        atomicOr(&bits[k >> 5], 1u << (k & 31));
    }
}

// Tile t covers nonzeros [t*PR_NZTILE, (t+1)*PR_NZTILE).  Its first row is the
// non-empty row holding nonzero t*PR_NZTILE; bit 31 marks that this row began
// in an earlier tile.  Such a row that also ends in tile t gets a fixup: the
// row and the tile ts holding its first nonzero.  Rows spanning more than
// PR_LONG tiles are listed separately for a warp-wide sum.
__global__ void tile_meta_kernel(int64_t ntiles, int32_t n_ne, const int32_t* __restrict__ ne_rows,
                                 const int32_t* __restrict__ row_ptr, uint32_t* meta, FixDesc* fix, int32_t* longfix,
                                 int32_t* nlong) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = t * PR_NZTILE;
        int32_t lo = 0, hi = n_ne;    // first non-empty row whose end is past k0
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if ((int64_t)row_ptr[ne_rows[mid] + 1] <= k0) lo = mid + 1;
            else hi = mid;
        }
        FixDesc f;
        f.row = -1;
        f.ts = 0;
        uint32_t cont = 0;
        if (lo < n_ne) {
            const int32_t i = ne_rows[lo];
            const int64_t start = row_ptr[i], end = row_ptr[i + 1];
            if (start < k0) {
                cont = 1;
                if (end <= k0 + PR_NZTILE) {
                    f.row = i;
                    f.ts = (int32_t)(start / PR_NZTILE);
                    if (t - f.ts > PR_LONG) longfix[atomicAdd(nlong, 1)] = (int32_t)t;
                }
            }
        }
        meta[t] = (uint32_t)lo | (cont << 31);
        fix[t] = f;
    }
}

// ------------------------------------------------------- relabelling
__global__ void iota_kernel(int32_t n, int32_t* v) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}

__global__ void invert_perm_kernel(int32_t n, const int32_t* __restrict__ new2old, int32_t* old2new) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) old2new[new2old[k]] = k;
}

// Row lengths of the relabelled A^T: new row k is old row new2old[k]
// (len[n] = 0 so that an exclusive scan gives row_ptr[n] = nnz).
__global__ void relabel_rowlen_kernel(int32_t n, const int32_t* __restrict__ row_ptr,
                                      const int32_t* __restrict__ new2old, int32_t* len) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x) {
        if (k == n) {
            len[k] = 0;
        } else {
            const int32_t o = new2old[k];
            len[k] = row_ptr[o + 1] - row_ptr[o];
        }
    }
}

// Columns of the relabelled A^T: each new row holds the old row's entries in
// their old order, each column renamed by old2new.
//
// Row starts of the renumbered matrix: rid[new_ptr[k]] = k for every
// non-empty row k (a max-scan then gives every nonzero its row).
__global__ void row_start_kernel(int32_t n, const int32_t* __restrict__ new_ptr, int32_t* rid) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int32_t b = new_ptr[k];
        if (new_ptr[k + 1] > b) rid[b] = k;
    }
}

// One thread per nonzero of the renumbered matrix: nonzero p of new row k
// is entry p - new_ptr[k] of old row new2old[k], its column renumbered.
__global__ void relabel_cols_flat_kernel(int64_t nnz, const int32_t* __restrict__ rid,
                                         const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                         const int32_t* __restrict__ new2old, const int32_t* __restrict__ old2new,
                                         const int32_t* __restrict__ new_ptr, int32_t* new_col) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = rid[p];
        const int32_t o = new2old[k];
        new_col[p] = old2new[col_idx[row_ptr[o] + (int32_t)(p - new_ptr[k])]];
    }
}

struct MaxI32 {
    __device__ __forceinline__ int32_t operator()(int32_t a, int32_t b) const { return a > b ? a : b; }
};

__global__ void permute_gather_kernel(int32_t n, const int32_t* __restrict__ perm, const void* in, void* out,
                                      int32_t esize) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int32_t s = perm[k];
        if (esize == 8) static_cast<uint64_t*>(out)[k] = static_cast<const uint64_t*>(in)[s];
        else static_cast<uint32_t*>(out)[k] = static_cast<const uint32_t*>(in)[s];
    }
}

__global__ void permute_bits_kernel(int32_t n, const int32_t* __restrict__ new2old, const uint32_t* in_bits,
                                    uint32_t* out_bits) {
    const int32_t nw = (n + 31) / 32;
    for (int32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        uint32_t b = 0;
        for (int q = 0; q < 32; ++q) {
            const int32_t k = w * 32 + q;
            if (k >= n) break;
            const int32_t o = new2old[k];
            b |= ((in_bits[o >> 5] >> (o & 31)) & 1u) << q;
        }
        out_bits[w] = b;
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

    // col_idx is padded with column 0 to a whole number of nonzero tiles so
    // that the row-gather kernels can load it in aligned 16-byte pieces
    const int64_t npad = padded_nnz(nv);
    int32_t* row_ptr = (int32_t*)af(actx, sizeof(int32_t) * (a.nrows + 1));
    int32_t* col_idx = (int32_t*)af(actx, sizeof(int32_t) * npad);
    void* vals = a.vals ? af(actx, (size_t)esize * (nv > 0 ? nv : 1)) : nullptr;
    if (!row_ptr || !col_idx || (a.vals && !vals)) {
        if (row_ptr) ff(actx, row_ptr, sizeof(int32_t) * (a.nrows + 1));
        if (col_idx) ff(actx, col_idx, sizeof(int32_t) * npad);
        if (vals) ff(actx, vals, (size_t)esize * (nv > 0 ? nv : 1));
        return cudaErrorMemoryAllocation;
    }
    if ((err = cudaMemsetAsync(col_idx + nv, 0, sizeof(int32_t) * (npad - nv), st)) != cudaSuccess) return err;
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

cudaError_t launch_col_count(cudaStream_t st, int64_t ncols, int64_t nnz, const int32_t* col_idx, int32_t* deg) {
    cudaError_t e = cudaMemsetAsync(deg, 0, sizeof(int32_t) * (ncols > 0 ? ncols : 1), st);
    if (e != cudaSuccess) return e;
    if (nnz > 0) col_count_kernel<<<grid_for(nnz), 256, 0, st>>>(nnz, col_idx, deg);
    return cudaGetLastError();
}

cudaError_t launch_csr_check(cudaStream_t st, int64_t nrows, int64_t ncols, int64_t nnz, const int32_t* row_ptr,
                             const int32_t* col_idx, int32_t* status) {
    const int64_t work = nrows + 1 > nnz ? nrows + 1 : nnz;
    csr_check_kernel<<<grid_for(work), 256, 0, st>>>(nrows, ncols, nnz, row_ptr, col_idx, status);
    return cudaGetLastError();
}

cudaError_t launch_deg_present(cudaStream_t st, int64_t ncols, const int32_t* deg, uint8_t* present) {
    if (ncols > 0) deg_present_kernel<<<grid_for(ncols), 256, 0, st>>>(ncols, deg, present);
    return cudaGetLastError();
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

__global__ void sum_prefix_kernel(int32_t h, const int32_t* __restrict__ v, unsigned long long* out) {
    unsigned long long c = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < h; i += gridDim.x * blockDim.x) c += (unsigned)v[i];
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

cudaError_t degree_order(cudaStream_t st, int32_t n, const int32_t* deg, int32_t* new2old, int32_t* old2new,
                         AllocFn af, FreeFn ff, void* actx, int32_t top_h, unsigned long long* top_sum) {
    Scratch S{af, ff, actx, {}};
    cudaError_t e;
    int32_t* ids = (int32_t*)S.get(sizeof(int32_t) * n);
    int32_t* keys_out = (int32_t*)S.get(sizeof(int32_t) * n);
    if (!ids || !keys_out) return cudaErrorMemoryAllocation;
    iota_kernel<<<grid_for(n), 256, 0, st>>>(n, ids);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // stable descending sort by degree: ties keep ascending ids
    size_t tb = 0;
    if ((e = cub::DeviceRadixSort::SortPairsDescending(nullptr, tb, deg, keys_out, ids, new2old, n, 0, 32, st)) !=
        cudaSuccess)
        return e;
    void* tmp = S.get(tb);
    if (!tmp) return cudaErrorMemoryAllocation;
    if ((e = cub::DeviceRadixSort::SortPairsDescending(tmp, tb, deg, keys_out, ids, new2old, n, 0, 32, st)) !=
        cudaSuccess)
        return e;
    invert_perm_kernel<<<grid_for(n), 256, 0, st>>>(n, new2old, old2new);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (top_sum) {
        // edges whose source is among the top_h vertices (keys_out is sorted)
        unsigned long long* d = (unsigned long long*)S.get(sizeof(unsigned long long));
        if (!d) return cudaErrorMemoryAllocation;
        if ((e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        const int32_t h = top_h < n ? top_h : n;
        if (h > 0) sum_prefix_kernel<<<grid_for(h), 256, 0, st>>>(h, keys_out, d);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(top_sum, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return e;
    }
    return cudaStreamSynchronize(st);
}

__global__ void block_degree_keys_kernel(int32_t n, const int32_t* __restrict__ deg, const int32_t* __restrict__ block,
                                         unsigned long long* keys, int32_t* ids) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // ascending key: block first, then descending degree; ties keep the id order
        keys[i] = ((unsigned long long)(uint32_t)block[i] << 32) | (unsigned long long)(uint32_t)(0x7fffffff - deg[i]);
        ids[i] = i;
    }
}

cudaError_t block_degree_order(cudaStream_t st, int32_t n, const int32_t* col_idx, int64_t nnz, const int32_t* block,
                               int32_t* new2old, int32_t* old2new, AllocFn af, FreeFn ff, void* actx) {
    Scratch S{af, ff, actx, {}};
    cudaError_t e;
    int32_t* deg = (int32_t*)S.get(sizeof(int32_t) * n);
    unsigned long long* keys = (unsigned long long*)S.get(sizeof(unsigned long long) * n);
    unsigned long long* keys_out = (unsigned long long*)S.get(sizeof(unsigned long long) * n);
    int32_t* ids = (int32_t*)S.get(sizeof(int32_t) * n);
    if (!deg || !keys || !keys_out || !ids) return cudaErrorMemoryAllocation;
    if ((e = cudaMemsetAsync(deg, 0, sizeof(int32_t) * n, st)) != cudaSuccess) return e;
    if (nnz > 0) col_count_kernel<<<grid_for(nnz), 256, 0, st>>>(nnz, col_idx, deg);
    block_degree_keys_kernel<<<grid_for(n), 256, 0, st>>>(n, deg, block, keys, ids);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    size_t tb = 0;
    if ((e = cub::DeviceRadixSort::SortPairs(nullptr, tb, keys, keys_out, ids, new2old, n, 0, 64, st)) != cudaSuccess)
        return e;
    void* tmp = S.get(tb);
    if (!tmp) return cudaErrorMemoryAllocation;
    if ((e = cub::DeviceRadixSort::SortPairs(tmp, tb, keys, keys_out, ids, new2old, n, 0, 64, st)) != cudaSuccess)
        return e;
    invert_perm_kernel<<<grid_for(n), 256, 0, st>>>(n, new2old, old2new);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t relabel_order(cudaStream_t st, const RelabelArgs& a, unsigned long long* top_sum, AllocFn af, FreeFn ff,
                          void* actx) {
    return degree_order(st, a.n, a.coldeg, a.new2old, a.old2new, af, ff, actx, a.top_h, top_sum);
}

cudaError_t relabel_build(cudaStream_t st, const RelabelArgs& a, AllocFn af, FreeFn ff, void* actx) {
    Scratch S{af, ff, actx, {}};
    cudaError_t e;
    const int32_t n = a.n;
    int32_t* deg = (int32_t*)S.get(sizeof(int32_t) * (n + 1));
    if (!deg) return cudaErrorMemoryAllocation;
    relabel_rowlen_kernel<<<grid_for(n + 1), 256, 0, st>>>(n, a.row_ptr, a.new2old, deg);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    size_t tb = 0;
    if ((e = cub::DeviceScan::ExclusiveSum(nullptr, tb, deg, a.new_row_ptr, n + 1, st)) != cudaSuccess) return e;
    void* tmp = S.get(tb);
    if (!tmp) return cudaErrorMemoryAllocation;
    if ((e = cub::DeviceScan::ExclusiveSum(tmp, tb, deg, a.new_row_ptr, n + 1, st)) != cudaSuccess) return e;
    // padding of the last tile: column 0, as in the CSR build
    if ((e = cudaMemsetAsync(a.new_col_idx, 0, sizeof(int32_t) * padded_nnz(a.nnz), st)) != cudaSuccess) return e;
    if (a.nnz > 0) {
        // every nonzero's new row (row starts, then a max-scan), then one
        // thread per nonzero: all lanes busy whatever the row lengths
        int32_t* rid = (int32_t*)S.get(sizeof(int32_t) * (size_t)a.nnz);
        if (!rid) return cudaErrorMemoryAllocation;
        if ((e = cudaMemsetAsync(rid, 0, sizeof(int32_t) * (size_t)a.nnz, st)) != cudaSuccess) return e;
        row_start_kernel<<<grid_for(n), 256, 0, st>>>(n, a.new_row_ptr, rid);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        size_t sb = 0;
        if ((e = cub::DeviceScan::InclusiveScan(nullptr, sb, rid, rid, MaxI32(), a.nnz, st)) != cudaSuccess) return e;
        void* stmp = S.get(sb);
        if (!stmp) return cudaErrorMemoryAllocation;
        if ((e = cub::DeviceScan::InclusiveScan(stmp, sb, rid, rid, MaxI32(), a.nnz, st)) != cudaSuccess) return e;
        relabel_cols_flat_kernel<<<grid_for(a.nnz), 256, 0, st>>>(a.nnz, rid, a.row_ptr, a.col_idx, a.new2old,
                                                                  a.old2new, a.new_row_ptr, a.new_col_idx);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(st);
}

cudaError_t launch_permute(cudaStream_t st, int32_t n, const int32_t* perm, const void* in, void* out, int32_t esize) {
    if (n <= 0) return cudaSuccess;
    permute_gather_kernel<<<grid_for(n), 256, 0, st>>>(n, perm, in, out, esize);
    return cudaGetLastError();
}

cudaError_t launch_permute_bits(cudaStream_t st, int32_t n, const int32_t* new2old, const uint32_t* in_bits,
                                uint32_t* out_bits) {
    if (n <= 0) return cudaSuccess;
    permute_bits_kernel<<<grid_for((n + 31) / 32), 256, 0, st>>>(n, new2old, in_bits, out_bits);
    return cudaGetLastError();
}

cudaError_t build_row_plan(cudaStream_t st, const PlanArgs& a, AllocFn af, FreeFn ff, void* actx) {
    Scratch S{af, ff, actx, {}};
    cudaError_t e;
    const int32_t nblk = (a.nrows + 255) / 256;
    int32_t* bc = (int32_t*)S.get(sizeof(int32_t) * (nblk + 1));
    int32_t* bo = (int32_t*)S.get(sizeof(int32_t) * (nblk + 1));
    if (!bc || !bo) return cudaErrorMemoryAllocation;
    row_count_kernel<<<nblk, 256, 0, st>>>(a.nrows, a.row_ptr, bc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    size_t tb = 0;
    if ((e = cub::DeviceScan::ExclusiveSum(nullptr, tb, bc, bo, nblk + 1, st)) != cudaSuccess) return e;
    void* tmp = S.get(tb);
    if (!tmp) return cudaErrorMemoryAllocation;
    // bc[nblk] must be 0 so that bo[nblk] is the total
    if ((e = cudaMemsetAsync(bc + nblk, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = cub::DeviceScan::ExclusiveSum(tmp, tb, bc, bo, nblk + 1, st)) != cudaSuccess) return e;
    row_split_kernel<<<nblk, 256, 0, st>>>(a.nrows, a.row_ptr, bo, a.ne_rows, a.empty_rows);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int32_t n_ne = 0;
    if ((e = cudaMemcpyAsync(&n_ne, bo + nblk, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    const size_t nbits_words = (size_t)a.ntiles * PR_NZTILE / 32;
    if ((e = cudaMemsetAsync(a.rowend_bits, 0, sizeof(uint32_t) * nbits_words, st)) != cudaSuccess) return e;
    if (n_ne > 0) {
        rowend_bits_kernel<<<grid_for(n_ne), 256, 0, st>>>(n_ne, a.ne_rows, a.row_ptr, a.rowend_bits);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(a.counts + 2, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    tile_meta_kernel<<<grid_for(a.ntiles), 256, 0, st>>>(a.ntiles, n_ne, a.ne_rows, a.row_ptr, a.tile_meta, a.fix,
                                                          a.longfix, a.counts + 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int32_t counts01[2] = {n_ne, a.nrows - n_ne};
    if ((e = cudaMemcpyAsync(a.counts, counts01, sizeof(counts01), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);
}

}  // namespace grb
