// Allocation-free variant of the library's deterministic reduction.
//
// Some callers cannot allocate device memory at the moment they need a
// reduction: code embedded in a host framework that owns the whole device
// memory budget and forbids allocations behind its back, code running under
// a hard memory cap where a new allocation could fail at a bad moment, and
// latency-critical paths that cannot afford cudaMalloc's implicit device
// synchronisation.  For them, grb_reduce_dense_noalloc takes caller-owned
// input and output buffers and keeps its only scratch -- the per-block
// partial sums and the last-block counter -- in a fixed file-scope
// __device__ array, so it never calls cudaMalloc, cudaFree or an allocating
// library routine.
#include <mutex>

#include "grb_device.cuh"

namespace {

constexpr int NA_BLOCK = 256;
constexpr int64_t NA_CHUNK = 4096;     // elements folded by one block
constexpr int NA_MAX_BLOCKS = 4096;    // partial sums the scratch holds
static_assert((int64_t)NA_MAX_BLOCKS * NA_CHUNK == 16777216, "limit stated in grb.h");

struct NoAllocScratch {
    double partial[NA_MAX_BLOCKS];
    unsigned int counter;
};

// Shared by every call on a device; held until the process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Block b folds elements [b*NA_CHUNK, (b+1)*NA_CHUNK) in a fixed order; the
// last block to finish folds the block results in index order.
__global__ void __launch_bounds__(NA_BLOCK) noalloc_reduce_kernel(const void* x, int32_t type, int64_t n, int32_t mon,
                                                                  double* out, NoAllocScratch* s) {
    __shared__ double sh[NA_BLOCK / 32];
    __shared__ bool last;
    const int64_t lo = (int64_t)blockIdx.x * NA_CHUNK;
    const int64_t hi = lo + NA_CHUNK < n ? lo + NA_CHUNK : n;
    double acc = grb::monoid_identity(mon);
    for (int64_t i = lo + threadIdx.x; i < hi; i += NA_BLOCK)
        acc = grb::monoid_apply<double>(mon, acc, grb::load_as<double>(x, type, i));
    const double bsum = grb::block_monoid_d<NA_BLOCK>(mon, acc, sh);
    if (threadIdx.x == 0) {
        s->partial[blockIdx.x] = bsum;
        __threadfence();
        last = atomicAdd(&s->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double r = grb::monoid_identity(mon);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NA_BLOCK)
        r = grb::monoid_apply<double>(mon, r, grb::ld_relaxed_f64(s->partial + b));
    r = grb::block_monoid_d<NA_BLOCK>(mon, r, sh);
    if (threadIdx.x == 0) {
        *out = r;
        s->counter = 0;
    }
}

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_addr[NA_MAX_DEVICES] = {};

}  // namespace

extern "C" grb_info grb_reduce_dense_noalloc(const void* x, grb_type type, uint64_t n, grb_monoid m, double* out,
                                             void* stream) {
    if (!out || (n > 0 && !x)) return GRB_NULL_POINTER;
    if (!(type == GRB_INT32 || type == GRB_FP32 || type == GRB_FP64)) return GRB_INVALID_VALUE;
    if (m < GRB_MONOID_PLUS || m > GRB_MONOID_TIMES) return GRB_INVALID_VALUE;
    if (n > (uint64_t)NA_MAX_BLOCKS * NA_CHUNK) return GRB_INVALID_VALUE;   // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return GRB_DEVICE_ERROR;
    }
    NoAllocScratch* s;
    {
        // first call on this device: the host-side symbol is only a stand-in,
        // so look up the scratch array's device address (with the device
        // current) and keep it
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return GRB_DEVICE_ERROR;
            }
            g_scratch_addr[dev] = static_cast<NoAllocScratch*>(ptr);
        }
        s = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the counter must start at zero whatever an earlier call left behind
    if (cudaMemsetAsync(&s->counter, 0, sizeof(unsigned int), st) != cudaSuccess) {
        cudaGetLastError();
        return GRB_DEVICE_ERROR;
    }
    int64_t grid = ((int64_t)n + NA_CHUNK - 1) / NA_CHUNK;
    if (grid < 1) grid = 1;
    noalloc_reduce_kernel<<<(unsigned)grid, NA_BLOCK, 0, st>>>(x, (int32_t)type, (int64_t)n, (int32_t)m, out, s);
    if (cudaGetLastError() != cudaSuccess) return GRB_DEVICE_ERROR;
    return GRB_SUCCESS;
}
