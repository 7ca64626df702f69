// Device helpers: typed loads/stores, operators, monoids, block reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "grb.h"
#include "grb_kernels.h"

namespace grb {

// Bounds-checked builds (-DGRB_CHECK_BOUNDS, libgrb_checked.so): an index
// read from a matrix's structure is tested against the extent of the array it
// addresses before it is used; a bad one is replaced by 0 (in bounds of any
// non-empty array) and the first failure is recorded in the context's status
// words -- word 0 the code, word 1 what was checked, words 2-3 the offending
// value as an int64 -- which the host reads at its next wait.  Release builds
// compile the test away.

__device__ __forceinline__ void bounds_record(int32_t* status, int32_t what, long long value) {
    if (status && atomicCAS(status, 0, (int32_t)GRB_INDEX_OUT_OF_BOUNDS) == 0) {
        status[1] = what;
        *reinterpret_cast<long long*>(status + 2) = value;
    }
}

#ifdef GRB_CHECK_BOUNDS
static __device__ __noinline__ int bounds_fail(int32_t* status, int32_t what, long long value) {
    bounds_record(status, what, value);
    return 0;
}
#define GRB_CHECKED(j, n, status, what) \
    ((unsigned)(j) < (unsigned)(n) ? (int)(j) : ::grb::bounds_fail((status), (what), (long long)(j)))
#else
#define GRB_CHECKED(j, n, status, what) (j)
#endif

template <class C>
__device__ __forceinline__ C load_as(const void* p, int32_t type, int64_t i) {
    switch (type) {
        case GRB_INT32: return (C)(static_cast<const int32_t*>(p)[i]);
        case GRB_FP32: return (C)(static_cast<const float*>(p)[i]);
        case GRB_FP64: return (C)(static_cast<const double*>(p)[i]);
        case GRB_BF16: return (C)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
    }
    return (C)0;
}

template <class C>
__device__ __forceinline__ void store_as(void* p, int32_t type, int64_t i, C x) {
    switch (type) {
        case GRB_INT32: static_cast<int32_t*>(p)[i] = (int32_t)x; break;
        case GRB_FP32: static_cast<float*>(p)[i] = (float)x; break;
        case GRB_FP64: static_cast<double*>(p)[i] = (double)x; break;
        case GRB_BF16: static_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16_rn((float)x); break;
    }
}

// Round a double to the given element type and widen it back.
__device__ __forceinline__ double round_to(int32_t type, double x) {
    switch (type) {
        case GRB_INT32: return (double)(int32_t)x;
        case GRB_FP32: return (double)(float)x;
        case GRB_BF16: return (double)__bfloat162float(__float2bfloat16_rn((float)x));
    }
    return x;
}

template <class C>
__device__ __forceinline__ bool vin_get(const VIn& v, int64_t i, C& x) {
    switch ((Fmt)v.fmt) {
        case Fmt::EMPTY: return false;
        case Fmt::ISO: x = (C)(v.iso_slot ? round_to(v.type, *v.iso_slot) : v.iso); return true;
        case Fmt::FULL: x = load_as<C>(v.vals, v.type, i); return true;
        case Fmt::BITMAP:
            if (!v.present[i]) return false;
            x = load_as<C>(v.vals, v.type, i);
            return true;
    }
    return false;
}

template <class C>
__device__ __forceinline__ C abs_c(C x) { return x < (C)0 ? -x : x; }

template <class C>
__device__ __forceinline__ C binop(int32_t code, double k, C x, C y) {
    switch (code) {
        case GRB_FIRST: return x;
        case GRB_SECOND: return y;
        case GRB_PLUS: return x + y;
        case GRB_MINUS: return x - y;
        case GRB_TIMES: return x * y;
        case GRB_DIV: return x / y;
        case GRB_MAX: return x > y ? x : y;
        case GRB_MIN: return x < y ? x : y;
        case GRB_ABS_DIFF: return abs_c<C>(x - y);
        case GRB_MAX_DIV_BY: { C q = x / (C)k; return q > y ? q : y; }
    }
    return x;
}

template <class C>
__device__ __forceinline__ C unop(int32_t code, C x) {
    switch (code) {
        case GRB_IDENTITY: return x;
        case GRB_ABS: return abs_c<C>(x);
        case GRB_AINV: return -x;
        case GRB_MINV: return (C)1 / x;
    }
    return x;
}

__device__ __forceinline__ double monoid_identity(int32_t m) {
    switch (m) {
        case GRB_MONOID_PLUS: return 0.0;
        case GRB_MONOID_TIMES: return 1.0;
        case GRB_MONOID_MAX: return -__longlong_as_double(0x7ff0000000000000LL);
        case GRB_MONOID_MIN: return __longlong_as_double(0x7ff0000000000000LL);
    }
    return 0.0;
}

template <class C>
__device__ __forceinline__ C monoid_apply(int32_t m, C x, C y) {
    switch (m) {
        case GRB_MONOID_PLUS: return x + y;
        case GRB_MONOID_TIMES: return x * y;
        case GRB_MONOID_MAX: return x > y ? x : y;
        case GRB_MONOID_MIN: return x < y ? x : y;
    }
    return x;
}

__device__ __forceinline__ double schain_apply(const SChain& ch, double x) {
    for (int q = 0; q < ch.n; ++q) x = round_to(ch.rtype[q], binop<double>(ch.ops[q].code, ch.ops[q].k, x, ch.c[q]));
    return x;
}

__device__ __forceinline__ double sin_get(const SIn& s) { return s.slot ? *s.slot : s.host; }

// Deterministic block-wide sum of one double per thread (fixed tree).
template <int BLOCK>
__device__ __forceinline__ double block_sum_d(double x, double* sh /* BLOCK/32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    __syncthreads();
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < BLOCK / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
    }
    return r;  // valid in thread 0
}

template <int BLOCK>
__device__ __forceinline__ double block_monoid_d(int32_t m, double x, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = monoid_apply<double>(m, x, __shfl_down_sync(0xffffffffu, x, off));
    __syncthreads();
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    double r = monoid_identity(m);
    if (warp == 0) {
        r = lane < BLOCK / 32 ? sh[lane] : monoid_identity(m);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r = monoid_apply<double>(m, r, __shfl_down_sync(0xffffffffu, r, off));
    }
    return r;
}

// Acquire / release accesses for the cross-block protocols.
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ double ld_relaxed_f64(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace grb
