// Element-wise methods, the GraphBLAS write step, reductions, scalar chains
// and format conversions.  These are the one-kernel-per-method building
// blocks of blocking mode (§II) and the fallback of the planner; the fused
// element-wise + reduce kernel below is what the planner emits for
// reduce(ewise(...)) chains such as the residual and the dangling mass.
#include "grb_device.cuh"

namespace grb {

namespace {

constexpr int EW_BLOCK = 256;

template <class C>
__device__ __forceinline__ bool ew_eval(const EwSpec& e, int64_t i, C& out) {
    C xu, xv;
    switch (e.kind) {
        case EW_COPY: return vin_get<C>(e.u, i, out);
        case EW_APPLY:
            if (!vin_get<C>(e.u, i, xu)) return false;
            out = unop<C>(e.unop, xu);
            return true;
        case EW_APPLY_B2:
            if (!vin_get<C>(e.u, i, xu)) return false;
            out = binop<C>(e.op.code, e.op.k, xu, (C)round_to(e.ctype, sin_get(e.s)));
            return true;
        case EW_ASSIGN:
            out = (C)round_to(e.ctype, sin_get(e.s));
            return true;
        case EW_EADD: {
            const bool hu = vin_get<C>(e.u, i, xu), hv = vin_get<C>(e.v, i, xv);
            if (hu && hv) out = binop<C>(e.op.code, e.op.k, xu, xv);
            else if (hu) out = xu;
            else if (hv) out = xv;
            return hu || hv;
        }
        case EW_EMULT: {
            if (!vin_get<C>(e.u, i, xu) || !vin_get<C>(e.v, i, xv)) return false;
            out = binop<C>(e.op.code, e.op.k, xu, xv);
            return true;
        }
    }
    return false;
}

// Round an intermediate to the element type it is stored in.
template <class C>
__device__ __forceinline__ C round_c(int32_t type, C x) {
    if (type == GRB_INT32) return (C)(int32_t)x;
    if (type == GRB_BF16) return (C)__bfloat162float(__float2bfloat16_rn((float)x));
    return x;
}

template <class C>
__global__ void __launch_bounds__(EW_BLOCK) ewise_kernel(int64_t n, EwSpec e, WriteSpec w, VOut out) {
    for (int64_t i = (int64_t)blockIdx.x * EW_BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * EW_BLOCK) {
        C tv = (C)0;
        const bool th = ew_eval<C>(e, i, tv);
        if (th) tv = round_c<C>(e.ctype, tv);
        bool zh = th;
        C zv = tv;
        if (w.has_accum) {
            C wv;
            const bool wh = vin_get<C>(w.w_old, i, wv);
            if (wh && th) zv = round_c<C>(e.ctype, binop<C>(w.accum.code, w.accum.k, wv, tv));
            else if (wh) zv = wv;
            zh = wh || th;
        }
        bool m = true;
        if (w.use_mask) {
            double mv = 0.0;
            const bool mh = vin_get<double>(w.mask, i, mv);
            m = w.structural ? mh : (mh && mv != 0.0);
            if (w.complement) m = !m;
        }
        bool oh;
        C ov = (C)0;
        if (m) { oh = zh; ov = zv; }
        else if (w.replace) oh = false;
        else oh = vin_get<C>(w.w_old, i, ov);
        if (!oh) ov = (C)0;
        store_as<C>(out.vals, out.type, i, ov);
        if (!out.full) out.present[i] = oh ? 1 : 0;
    }
}

// Deterministic reduce(monoid, ewise(...)): block b folds a fixed contiguous
// chunk, the last block to finish folds the per-block results in order.
template <class C>
__global__ void __launch_bounds__(EW_BLOCK) ew_reduce_kernel(int64_t n, EwSpec e, int32_t mon, int32_t has_accum,
                                                             OpSpec accum, SIn s_old, SChain chain, int32_t out_type,
                                                             double* out_slot, double* scratch, uint32_t* counter) {
    __shared__ double sh[EW_BLOCK / 32];
    __shared__ bool last;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    double acc = monoid_identity(mon);
    for (int64_t i = lo + threadIdx.x; i < hi; i += EW_BLOCK) {
        C x;
        if (ew_eval<C>(e, i, x)) acc = monoid_apply<double>(mon, acc, (double)round_c<C>(e.ctype, x));
    }
    const double bsum = block_monoid_d<EW_BLOCK>(mon, acc, sh);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = bsum;
        __threadfence();
        const uint32_t prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double r = monoid_identity(mon);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += EW_BLOCK)
        r = monoid_apply<double>(mon, r, ld_relaxed_f64(scratch + b));
    r = block_monoid_d<EW_BLOCK>(mon, r, sh);
    if (threadIdx.x == 0) {
        r = round_to(out_type, r);
        if (has_accum) r = round_to(out_type, binop<double>(accum.code, accum.k, sin_get(s_old), r));
        *out_slot = schain_apply(chain, r);
        *counter = 0;
    }
}

__global__ void scalar_chain_kernel(SIn in, SChain chain, int32_t out_type, double* out_slot) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out_slot = schain_apply(chain, sin_get(in));
}

__global__ void count_present_kernel(int64_t n, const uint8_t* present, unsigned long long* out) {
    __shared__ unsigned long long sh;
    if (threadIdx.x == 0) sh = 0;
    __syncthreads();
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += present[i] ? 1 : 0;
    atomicAdd(&sh, c);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(out, sh);
}

__global__ void to_dense_kernel(int64_t n, VIn v, void* out_vals, uint8_t* out_present) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = 0.0;
        const bool h = vin_get<double>(v, i, x);
        if (v.type == GRB_FP64) static_cast<double*>(out_vals)[i] = h ? x : 0.0;
        else store_as<double>(out_vals, v.type, i, h ? x : 0.0);
        if (out_present) out_present[i] = h ? 1 : 0;
    }
}

__global__ void build_sparse_kernel(int64_t n, const int32_t* idx, const double* vals, int64_t nvals, int32_t type,
                                    void* out_vals, uint8_t* out_present, int32_t* status) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nvals; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = idx[k];
        if (i < 0 || i >= n || (k > 0 && idx[k - 1] >= i)) {   // out of range, unsorted or duplicate
            atomicCAS(status, 0, (int32_t)GRB_INVALID_INDEX);
            continue;
        }
        store_as<double>(out_vals, type, i, vals[k]);
        out_present[i] = 1;
    }
}

__global__ void sinkbits_kernel(int64_t n, VIn v, uint32_t* bits) {
    const int64_t nw = (n + 31) / 32;
    for (int64_t wd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wd < nw; wd += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = 0;
        for (int q = 0; q < 32; ++q) {
            const int64_t i = wd * 32 + q;
            double x;
            if (i < n && vin_get<double>(v, i, x)) b |= 1u << q;
        }
        bits[wd] = b;
    }
}

// Warp-per-row semiring mxv for the general case (valued A, bitmap u, any
// semiring): lane-strided terms, fixed shuffle tree.
template <class C>
__global__ void mxv_generic_kernel(int64_t nrows, const int32_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ col_idx, const void* avals, int32_t a_type,
                                   double a_iso, VIn u, int32_t add_mon, int32_t mul_op, VOut out,
                                   int64_t ncols, int32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); row < nrows; row += warps) {
        const int32_t b = row_ptr[row], e = row_ptr[row + 1];
        C acc = (C)monoid_identity(add_mon);
        bool found = false;
        // 64-bit: on a matrix with close to 2^31 nonzeros p + 32 passes INT32_MAX
        for (int64_t p = (int64_t)b + lane; p < e; p += 32) {
            C x;
            const int32_t j = col_idx[p];
            if (!vin_get<C>(u, GRB_CHECKED(j, ncols, status, BOUNDS_COLUMN), x)) continue;
            const C a = avals ? load_as<C>(avals, a_type, p) : (C)a_iso;
            acc = monoid_apply<C>(add_mon, acc, binop<C>(mul_op, 0.0, a, x));
            found = true;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc = monoid_apply<C>(add_mon, acc, __shfl_down_sync(0xffffffffu, acc, off));
        found = __any_sync(0xffffffffu, found);
        if (lane == 0) {
            store_as<C>(out.vals, out.type, row, found ? acc : (C)0);
            if (!out.full) out.present[row] = found ? 1 : 0;
        }
    }
}

inline int grid_for(int64_t n, int block, int cap = 152 * 32) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

inline bool is_f32(int32_t t) { return t == GRB_FP32 || t == GRB_BF16; }

}  // namespace

cudaError_t launch_ewise(cudaStream_t st, int64_t n, const EwSpec& e, const WriteSpec& w, VOut out) {
    if (n <= 0) return cudaSuccess;
    if (is_f32(e.ctype)) ewise_kernel<float><<<grid_for(n, EW_BLOCK), EW_BLOCK, 0, st>>>(n, e, w, out);
    else ewise_kernel<double><<<grid_for(n, EW_BLOCK), EW_BLOCK, 0, st>>>(n, e, w, out);
    return cudaGetLastError();
}

cudaError_t launch_ew_reduce(cudaStream_t st, int64_t n, const EwSpec& e, int32_t monoid, int32_t has_accum,
                             OpSpec accum, SIn s_old, const SChain& chain, int32_t out_type, double* out_slot,
                             double* scratch, uint32_t* counter, int grid) {
    if (is_f32(e.ctype))
        ew_reduce_kernel<float><<<grid, EW_BLOCK, 0, st>>>(n, e, monoid, has_accum, accum, s_old, chain, out_type,
                                                           out_slot, scratch, counter);
    else
        ew_reduce_kernel<double><<<grid, EW_BLOCK, 0, st>>>(n, e, monoid, has_accum, accum, s_old, chain, out_type,
                                                            out_slot, scratch, counter);
    return cudaGetLastError();
}

cudaError_t launch_scalar_chain(cudaStream_t st, SIn in, const SChain& chain, int32_t out_type, double* out_slot) {
    scalar_chain_kernel<<<1, 32, 0, st>>>(in, chain, out_type, out_slot);
    return cudaGetLastError();
}

cudaError_t launch_count_present(cudaStream_t st, int64_t n, const uint8_t* present, unsigned long long* out) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || n <= 0) return e;
    count_present_kernel<<<grid_for(n, 256, 152 * 4), 256, 0, st>>>(n, present, out);
    return cudaGetLastError();
}

cudaError_t launch_to_dense(cudaStream_t st, int64_t n, VIn v, void* out_vals, uint8_t* out_present) {
    if (n <= 0) return cudaSuccess;
    to_dense_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, v, out_vals, out_present);
    return cudaGetLastError();
}

cudaError_t launch_build_sparse(cudaStream_t st, int64_t n, const int32_t* idx, const double* vals, int64_t nvals,
                                int32_t type, void* out_vals, uint8_t* out_present, int32_t* status) {
    if (nvals <= 0) return cudaSuccess;
    build_sparse_kernel<<<grid_for(nvals, 256), 256, 0, st>>>(n, idx, vals, nvals, type, out_vals, out_present, status);
    return cudaGetLastError();
}

cudaError_t launch_sinkbits(cudaStream_t st, int64_t n, VIn v, uint32_t* bits) {
    const int64_t nw = (n + 31) / 32;
    if (nw <= 0) return cudaSuccess;
    sinkbits_kernel<<<grid_for(nw, 256), 256, 0, st>>>(n, v, bits);
    return cudaGetLastError();
}

cudaError_t launch_mxv_generic(cudaStream_t st, int64_t nrows, const int32_t* row_ptr, const int32_t* col_idx,
                               const void* avals, int32_t a_type, double a_iso, VIn u, int32_t add_monoid,
                               int32_t mul_op, VOut out, int64_t ncols, int32_t* status) {
    if (nrows <= 0) return cudaSuccess;
    const int grid = grid_for(nrows * 32, 256);
    if (is_f32(out.type))
        mxv_generic_kernel<float><<<grid, 256, 0, st>>>(nrows, row_ptr, col_idx, avals, a_type, a_iso, u, add_monoid,
                                                        mul_op, out, ncols, status);
    else
        mxv_generic_kernel<double><<<grid, 256, 0, st>>>(nrows, row_ptr, col_idx, avals, a_type, a_iso, u, add_monoid,
                                                         mul_op, out, ncols, status);
    return cudaGetLastError();
}

}  // namespace grb
