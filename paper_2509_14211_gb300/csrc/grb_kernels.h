// Host-callable launchers of the CUDA kernels and the plain-data structs they
// take.  Nothing here knows about handles or the DAG; grb_core.h builds these
// descriptors from materialised versions.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "grb.h"

namespace grb {

enum class Fmt : int32_t { EMPTY = 0, ISO = 1, FULL = 2, BITMAP = 3 };

// Read-only vector operand.  ISO: every entry equals `iso`; FULL: `vals`
// holds n values; BITMAP: `vals` + `present` (uint8 per entry).
struct VIn {
    const void* vals = nullptr;
    const uint8_t* present = nullptr;
    double iso = 0.0;
    const double* iso_slot = nullptr;  // ISO value held in device memory (pending scalar)
    int32_t type = 2;                  // grb_type
    int32_t fmt = 0;                   // Fmt
};

// Output vector: values of `type`; `present` written unless `full`.
struct VOut {
    void* vals = nullptr;
    uint8_t* present = nullptr;
    int32_t type = 2;
    int32_t full = 1;
};

// Scalar operand: device slot (a double) when non-null, else the host value.
struct SIn {
    const double* slot = nullptr;
    double host = 0.0;
};

struct OpSpec {
    int32_t code = 0;  // grb_opcode
    double k = 0.0;
};

// Scalar post-processing chain: x = op_i(x, c_i), applied in order.
struct SChain {
    int32_t n = 0;
    OpSpec ops[6];
    double c[6] = {0, 0, 0, 0, 0, 0};
    int32_t rtype[6] = {3, 3, 3, 3, 3, 3};  // type each step rounds to
};

enum EwKind : int32_t { EW_APPLY = 1, EW_APPLY_B2 = 2, EW_ASSIGN = 3, EW_EADD = 4, EW_EMULT = 5, EW_COPY = 6 };

// Element-wise method T(i) (before the write step).
struct EwSpec {
    int32_t kind = EW_COPY;
    OpSpec op;
    int32_t unop = 0;
    int32_t ctype = 2;   // type the op computes and rounds in (output's type)
    VIn u, v;
    SIn s;
};

// GraphBLAS write step: w<mask> accum= T.
struct WriteSpec {
    VIn mask;
    int32_t use_mask = 0, structural = 0, complement = 0, replace = 0;
    int32_t has_accum = 0;
    OpSpec accum;
    VIn w_old;
};

// Row-gather plan of a CSR matrix: every warp takes tiles of PR_NZTILE
// consecutive nonzeros, PR_NZLANE per lane.
constexpr int PR_BLOCK = 256;
constexpr int PR_NZLANE = 8;
constexpr int PR_NZTILE = 32 * PR_NZLANE;
constexpr int PR_LONG = 8;   // split rows spanning more tiles are joined by a whole warp

// The fused row-gather kernels (the PageRank, batched PPR and graph-batch
// bodies and their row plan) index rows and nonzeros with int32, including
// grid-stride steps (below 2^24) and row offsets within a tile; they take a
// matrix only when nrows + nnz stays below this limit.  Larger matrices (up
// to the CSR limit of 2^31 - 1 rows and nonzeros) run on the general kernels,
// which index with int64.
constexpr int64_t PR_INDEX_LIMIT = (int64_t(1) << 31) - (int64_t(1) << 24);
static_assert(PR_INDEX_LIMIT == GRB_FUSED_INDEX_LIMIT, "the header states the same limit");

// col_idx arrays are allocated to a whole number of tiles (padding = col 0).
inline int64_t padded_nnz(int64_t nnz) {
    const int64_t t = (nnz > 0 ? nnz : 1) + PR_NZTILE - 1;
    return t / PR_NZTILE * PR_NZTILE;
}

struct SyncWords {
    uint32_t launch;     // launches so far (diagnostics)
    uint32_t bar_count;  // grid barrier arrivals
    uint32_t bar_gen;    // grid barrier generation
    uint32_t done;       // last-block-done counter
    uint32_t stop;       // unused
    uint32_t pad[3];
};

// Fixup descriptor of a tile whose first row began in an earlier tile and
// ends in this one: the row and the first tile holding its nonzeros.
struct FixDesc {
    int32_t row;   // -1: no fixup
    int32_t ts;
};

enum GatherMode : int32_t { G_W = 0, G_TD = 1, G_ISO = 2 };

// Per-graph fold of a batch body, run inside the body's cooperative launch
// after a grid barrier: the rows' residual and dangling terms are summed per
// chunk (at most MG_CHUNK consecutive rows of one graph, a warp each), then
// per graph over its chunks (a warp each), all in fixed orders; then the
// body is counted, the graph's loop test applied and its next teleport
// (1-d)/n_g + d D_g / n_g set.
constexpr int MG_CHUNK = 1024;
struct MgFinish {
    int32_t ngraphs = 0;
    const int64_t* vptr = nullptr;     // ngraphs + 1 row offsets
    const float* row_res = nullptr;
    const float* row_dang = nullptr;
    int32_t nchunks = 0;
    const int32_t* chunk_lo = nullptr;    // nchunks + 1 row offsets
    const int32_t* chunk_graph = nullptr; // graph of each chunk
    const int32_t* g_chunk = nullptr;     // ngraphs + 1 chunk offsets
    double* chunk_part = nullptr;         // per chunk: residual, dangling mass
    int32_t* active = nullptr;
    int32_t* iters = nullptr;
    int32_t itermax = 0;
    double tol = 0.0;
    double* resid = nullptr;
    float* tele = nullptr;
    int32_t* final_buf = nullptr;
    double damping = 0.85;
};

// Fused row-gather kernel over the rows of a CSR matrix (merge-path tiles):
//   s_i   = sum over j in row i of g(j),  g = w[j] | t[j]/d[j] | g_iso
//   out_i = base_i + s_i (row non-empty) | base_i (row empty)   when has_base
//         = s_i, present iff row non-empty                        otherwise
// plus optional epilogue outputs: w_next_i = out_i / dd_i, the residual
// sum |r_old_i - out_i| and the dangling mass sum over sink rows of out_i.
// The context's status words: int32 0 the code (a bounded wait that ran out,
// a failed bounds check), int32 1 what a bounds check tested, int32 2-3 the
// offending value as an int64.
constexpr size_t STATUS_BYTES = 16;
enum BoundsWhat : int32_t { BOUNDS_COLUMN = 1, BOUNDS_ROW_PTR = 2 };

struct PrParams {
    // matrix and plan
    const int32_t* row_ptr = nullptr;
    const int32_t* col_idx = nullptr;   // padded to ntiles * PR_NZTILE
    int32_t nrows = 0, nnz = 0;
    int32_t ncols = 0;                  // entries of the gathered vector (bounds-checked builds)
    int32_t ntiles = 0;
    const uint32_t* tile_meta = nullptr;  // first non-empty row of the tile | (continues a row) << 31
    const uint32_t* rowend_bits = nullptr;  // bit k: nonzero k is the last of its row
    const int32_t* ne_rows = nullptr;     // the non-empty rows, ascending
    int32_t n_ne = 0;
    const int32_t* empty_rows = nullptr;  // the empty rows, ascending
    int32_t n_empty = 0;
    double* agg = nullptr;       // carry of the row open at each tile's end
    double* first = nullptr;     // this tile's part of a split first row
    const FixDesc* fix = nullptr;
    const int32_t* longfix = nullptr;
    int32_t nlong = 0;
    double* part = nullptr;      // [2][grid][2]
    SyncWords* sync = nullptr;
    int32_t* status = nullptr;
    int64_t spin_limit = 1 << 24;
    // gather
    int32_t gmode = G_W;
    const void* w = nullptr;     // G_W gather vector (gather type)
    const void* t = nullptr;     // G_TD numerator (rank type)
    const void* d = nullptr;     // G_TD divisor (rank type)
    double g_iso = 0.0;
    // base (accumulated output / teleport)
    int32_t has_base = 0;
    VIn base;
    // outputs
    VOut out;
    void* w_next = nullptr;      // gather type
    const void* dd = nullptr;    // divisor of w_next (rank type, full)
    const uint32_t* sinkbits = nullptr;
    const void* r_old = nullptr; // residual reference (rank type, full)
    int32_t want_resid = 0, want_dang = 0;
    double* resid_slot = nullptr;
    int32_t resid_type = 3;
    double* dang_slot = nullptr;
    double* tele_slot = nullptr; // chain(dangling mass)
    SChain chain;
    // persistent / iterated execution
    int32_t iters = 1;           // persistent: maximum number of bodies
    int32_t iter_index = 0;      // per-iteration launch: index of this body
    double tol = -1.0;
    double* hist = nullptr;      // residual history (itermax doubles)
    double* dhist = nullptr;     // dangling-mass history (itermax doubles; uniform dangling)
    int32_t expect_iters = 0;    // persistent: > 0 when the host assumed this body count
                                 // (fixed-count loop); any other count sets GRB_PANIC
    int64_t* iters_done = nullptr;
    const void* r0 = nullptr;    // persistent: input of body 0
    void* rbuf[2] = {nullptr, nullptr};
    void* wbuf[2] = {nullptr, nullptr};
    double rdiff0 = 1.0;         // value of the loop condition before body 0
    int32_t tele_from_slot = 0;  // base is the scalar tele_slot (uniform dangling)
    double tele_const = 0.0;     // PageRank loops without it: the iso teleport value
    // mixed precision (BF16 gather until the residual drops below mixed_switch)
    int32_t mixed = 0;
    double mixed_switch = 1e-3;
    void* wbuf32[2] = {nullptr, nullptr};
    int32_t* mixed_phase = nullptr;  // 0 = BF16 gather, 1 = FP32 gather
    // persistent loop: gathers of columns < hot_n are served from a copy of
    // w[0, hot_n) in shared memory (multiple of 4; 0 = off; FP32 only)
    int32_t hot_n = 0;
    // hot persistent loop: tile arrays staged by bulk copies this many tiles
    // ahead (0 = register prefetch one tile ahead; 2 or 3)
    int32_t tma_stages = 0;
    // batch of independent graphs (block-diagonal A^T): per-row graph id,
    // per-graph loop state and teleport, per-row residual / dangling terms
    const int32_t* graph_of = nullptr;
    const int32_t* g_active = nullptr;
    const float* g_tele = nullptr;
    float* row_res = nullptr;
    float* row_dang = nullptr;
    MgFinish mg;                 // the per-graph folds at the end of each body
    // one personalised query (EPI_PERS loops): its seed rows (bitmap in the
    // loop's vertex order) get the teleport term pers_val = (1-d)/|S|
    const uint32_t* pers_bits = nullptr;
    float pers_val = 0.f;
    // row-length-binned body (persistent FP32 loop): the non-empty rows by
    // group size, bins [bin_off[b], bin_off[b+1]) of bin_rows for b = thread,
    // 4, 8, 16 lanes, warp, CTA (null: the nonzero-split tiles)
    const int32_t* bin_rows = nullptr;
    int32_t bin_off[7] = {0, 0, 0, 0, 0, 0, 0};
};
// Row-length bins of the binned body: rows of at most PR_BIN_MAX[b] nonzeros
// go to bin b (groups of 1, 4, 8, 16, 32 lanes), longer ones to the CTA bin.
constexpr int PR_BIN_MAX[5] = {4, 16, 64, 256, 8192};

// Start state of every graph of a batch: r = 1/n_g, w = r ./ d, the first
// teleport from the dangling mass of r, active = (itermax > 0 && 1 > tol).
struct MgInit {
    int32_t ngraphs = 0;
    const int64_t* vptr = nullptr;
    const float* dd = nullptr;
    const uint32_t* sinkbits = nullptr;
    float* r = nullptr;
    float* w = nullptr;
    int32_t* active = nullptr;
    int32_t* iters = nullptr;
    double* resid = nullptr;
    float* tele = nullptr;
    int32_t* final_buf = nullptr;
    int32_t start_active = 1;
    double damping = 0.85;
};

// --------------------------------------------------------------- launchers
cudaError_t launch_ewise(cudaStream_t st, int64_t n, const EwSpec& e, const WriteSpec& w, VOut out);
cudaError_t launch_ew_reduce(cudaStream_t st, int64_t n, const EwSpec& e, int32_t monoid, int32_t has_accum,
                             OpSpec accum, SIn s_old, const SChain& chain, int32_t out_type, double* out_slot,
                             double* scratch, uint32_t* counter, int grid);
cudaError_t launch_scalar_chain(cudaStream_t st, SIn in, const SChain& chain, int32_t out_type, double* out_slot);
cudaError_t launch_count_present(cudaStream_t st, int64_t n, const uint8_t* present, unsigned long long* out);
cudaError_t launch_to_dense(cudaStream_t st, int64_t n, VIn v, void* out_vals, uint8_t* out_present);
cudaError_t launch_build_sparse(cudaStream_t st, int64_t n, const int32_t* idx, const double* vals, int64_t nvals,
                                int32_t type, void* out_vals, uint8_t* out_present, int32_t* status);
cudaError_t launch_sinkbits(cudaStream_t st, int64_t n, VIn v, uint32_t* bits);
cudaError_t launch_mxv_generic(cudaStream_t st, int64_t nrows, const int32_t* row_ptr, const int32_t* col_idx,
                               const void* avals, int32_t a_type, double a_iso, VIn u, int32_t add_monoid,
                               int32_t mul_op, VOut out, int64_t ncols, int32_t* status);

// CSR build: returns the deduplicated nnz through *nnz_out (synchronises).
struct CsrBuildArgs {
    int64_t nrows, ncols, nedges;
    const int32_t* src;   // device
    const int32_t* dst;   // device
    const void* vals;     // device or null
    int32_t val_type;
    int32_t transpose, drop_self, dedup;
};
using AllocFn = void* (*)(void* ctx, size_t bytes);
using FreeFn = void (*)(void* ctx, void* p, size_t bytes);
cudaError_t csr_build(cudaStream_t st, const CsrBuildArgs& a, AllocFn af, FreeFn ff, void* actx,
                      int32_t** row_ptr, int32_t** col_idx, void** vals_out, int64_t* nnz_out, int32_t* bad_index);
// deg[j] = entries in column j
cudaError_t launch_col_count(cudaStream_t st, int64_t ncols, int64_t nnz, const int32_t* col_idx, int32_t* deg);
// Structure check (bounds-checked builds, before a matrix's first use): the
// first row_ptr entry out of order or outside [0, nnz], or column index
// outside [0, ncols), goes to status (GRB_INDEX_OUT_OF_BOUNDS, what, value).
cudaError_t launch_csr_check(cudaStream_t st, int64_t nrows, int64_t ncols, int64_t nnz, const int32_t* row_ptr,
                             const int32_t* col_idx, int32_t* status);
// present[j] = deg[j] > 0
cudaError_t launch_deg_present(cudaStream_t st, int64_t ncols, const int32_t* deg, uint8_t* present);
cudaError_t launch_col_degree(cudaStream_t st, int64_t ncols, int64_t nnz, const int32_t* col_idx,
                              int32_t* deg, uint8_t* present);
cudaError_t launch_nonempty_rows(cudaStream_t st, int64_t nrows, const int32_t* row_ptr, unsigned long long* out);

// Merge-path plan and the fused kernels.
// Row-gather plan: the non-empty / empty row lists, the row-end bitmap, the
// per-tile metadata and fixup table.  Device outputs are preallocated by
// the caller (ne_rows/empty_rows: nrows each, bits: ntiles*PR_NZTILE/32,
// meta/fix: ntiles, longfix: ntiles); counts[0..2] = n_ne, n_empty, nlong.
struct PlanArgs {
    const int32_t* row_ptr;
    int32_t nrows, nnz;
    int64_t ntiles;
    int32_t* ne_rows;
    int32_t* empty_rows;
    uint32_t* rowend_bits;
    uint32_t* tile_meta;
    FixDesc* fix;
    int32_t* longfix;
    int32_t* counts;
};
cudaError_t build_row_plan(cudaStream_t st, const PlanArgs& a, AllocFn af, FreeFn ff, void* actx);

// Vertex relabelling by descending degree (stable): new2old[k] = vertex
// with the k-th largest degree, old2new its inverse (synchronises).
// *top_sum (host, optional) = sum of the top_h largest degrees.
cudaError_t degree_order(cudaStream_t st, int32_t n, const int32_t* deg, int32_t* new2old, int32_t* old2new,
                         AllocFn af, FreeFn ff, void* actx, int32_t top_h = 0, unsigned long long* top_sum = nullptr);
// Symmetric relabelling of a square pattern CSR matrix (A^T) by descending
// column count (the out-degree of the graph): new row k = old row new2old[k]
// with every column j renamed old2new[j], entries kept in their old order.
// relabel_order computes new2old / old2new and *top_sum (host) = the number
// of nonzeros in the top_h columns of largest count; relabel_build then
// writes new_row_ptr[n+1] and new_col_idx[padded_nnz(nnz)].  Both
// synchronise; outputs are preallocated by the caller.
struct RelabelArgs {
    int32_t n;
    int64_t nnz;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    int32_t* new_row_ptr;
    int32_t* new_col_idx;
    int32_t* new2old;
    int32_t* old2new;
    int32_t top_h;
    const int32_t* coldeg = nullptr;   // entries per column (relabel_order), computed by the caller
};
cudaError_t relabel_order(cudaStream_t st, const RelabelArgs& a, unsigned long long* top_sum, AllocFn af, FreeFn ff,
                          void* actx);
cudaError_t relabel_build(cudaStream_t st, const RelabelArgs& a, AllocFn af, FreeFn ff, void* actx);
// Renumbering inside blocks: vertices sorted by (block[i], descending column
// count of A^T, id), so every block keeps its index range (synchronises).
cudaError_t block_degree_order(cudaStream_t st, int32_t n, const int32_t* col_idx, int64_t nnz, const int32_t* block,
                               int32_t* new2old, int32_t* old2new, AllocFn af, FreeFn ff, void* actx);
// out[k] = in[perm[k]] for 4- or 8-byte elements.
cudaError_t launch_permute(cudaStream_t st, int32_t n, const int32_t* perm, const void* in, void* out, int32_t esize);
// bit k of out = bit new2old[k] of in.
cudaError_t launch_permute_bits(cudaStream_t st, int32_t n, const int32_t* new2old, const uint32_t* in_bits,
                                uint32_t* out_bits);
// ------------------------------------------------ batched personalised PageRank
// k queries ("slots") iterate together over one A^T: ranks are stored as
// [k-tile][n][32 V] FP32 -- lane l of a warp owns the V consecutive slots
// l V .. l V + V - 1 of a k-tile (V = 1, 2 or 4, the vector width) -- so the
// gather of a source vertex's values for a k-tile is 128 V contiguous bytes.
constexpr int PPR_LANES = 32;
constexpr int PPR_BLOCK = 512;
constexpr int PPR_MAX_SLOTS = GRB_PPR_MAX_SLOTS;   // 4 k-tiles

struct PprParams {
    // A^T and its row-gather plan
    const int32_t* col_idx = nullptr;
    int32_t nrows = 0, nnz = 0, ntiles = 0;
    const uint32_t* tile_meta = nullptr;
    const uint32_t* rowend_bits = nullptr;
    const int32_t* ne_rows = nullptr;
    int32_t n_ne = 0;
    const int32_t* empty_rows = nullptr;
    int32_t n_empty = 0;
    const FixDesc* fix = nullptr;
    // ranks and gather values, [kt][n][32 vw]
    int32_t kt = 0;
    int32_t vw = 1;                     // slots per lane
    const float* r_old = nullptr;
    float* r_new = nullptr;
    const float* w_old = nullptr;
    float* w_new = nullptr;
    const float* dd = nullptr;          // n: max(outdeg, 1) / damping
    const uint32_t* sinkbits = nullptr; // n bits: no out-edges
    float* agg = nullptr;               // [kt][ntiles][32 vw] carry of the row open at a tile's end
    float* first = nullptr;             // [kt][ntiles][32 vw] a tile's part of its split first row
    // teleport (1 - damping) v_s: seeds sorted by (k-tile, row, lane)
    const uint32_t* seedbits = nullptr; // n bits: a seed of some slot
    const int32_t* seed_ptr = nullptr;  // kt + 1 offsets
    const int32_t* seed_row = nullptr;
    const int32_t* seed_lane = nullptr;  // slot within the k-tile
    const float* seed_val = nullptr;
    // slot state
    const int32_t* active = nullptr;    // kt*32
    const float* tele_base = nullptr;   // kt*32: damping * D_s / n
    double* part = nullptr;             // [grid][kt*32][2] residual, dangling mass
    int32_t* status = nullptr;          // context status words (bounds-checked builds)
};

struct PprFinish {
    int32_t slots = 0, grid_a = 0, grid_b = 0;
    const double* part_a = nullptr;
    const double* part_b = nullptr;
    int32_t* active = nullptr;
    int32_t* iters = nullptr;
    const int32_t* itermax = nullptr;
    const double* tol = nullptr;
    double* resid = nullptr;
    float* tele_base = nullptr;
    int32_t* final_buf = nullptr;   // per slot: rank buffer of its last body
    int32_t out_buf = 0;            // rank buffer this body writes
    double damping = 0.85;
    int64_t n = 0;
};

// Admission of queued queries into their slots, all in one pass: zero each
// slot's column of the current rank / gather buffers, place its start vector
// (1/|S| on its seeds), its first dangling-mass term and its loop state.
struct PprInitBatch {
    int32_t np = 0, nrows = 0;
    int32_t width = PPR_LANES;          // slots per k-tile (32 vw)
    int32_t cur = 0;                    // current rank buffer (recorded as the slot's last)
    const int32_t* slots = nullptr;     // np, ascending
    const int32_t* seed_off = nullptr;  // np + 1
    const int32_t* seeds = nullptr;     // deduplicated seeds of every queued slot
    const float* r0 = nullptr;          // np: 1 / |S|
    const int32_t* act = nullptr;       // np: loop test before the first body
    const int32_t* itermax = nullptr;   // np
    const double* tol = nullptr;        // np
    float* r = nullptr;                 // current rank buffer [kt][n][width]
    float* w = nullptr;
    const float* dd = nullptr;
    const uint32_t* sinkbits = nullptr;
    int32_t* active = nullptr;          // slot state
    int32_t* iters = nullptr;
    int32_t* itermax_out = nullptr;
    double* tol_out = nullptr;
    double* resid = nullptr;
    float* tele_base = nullptr;
    int32_t* final_buf = nullptr;
    double damping = 0.85;
};

cudaError_t launch_ppr_tiles(cudaStream_t st, const PprParams& p, int grid);
cudaError_t launch_ppr_fixups(cudaStream_t st, const PprParams& p, int grid);
cudaError_t launch_ppr_finish(cudaStream_t st, const PprFinish& f);
cudaError_t launch_ppr_init_batch(cudaStream_t st, const PprInitBatch& a);
// Bits of every seed vertex (bits cleared first; nbits words of 32).
cudaError_t launch_ppr_seedbits(cudaStream_t st, int32_t nseeds, const int32_t* rows, uint32_t* bits, int64_t nwords);
// out[i] = r[kt][i][slot within the k-tile] of one slot.
cudaError_t launch_ppr_extract(cudaStream_t st, int32_t n, const float* r, int32_t width, int32_t slot, float* out);
// FP32 divisor max(deg/damping, 1/damping) and sink bits from column counts.
cudaError_t launch_ppr_divisor(cudaStream_t st, int32_t n, const int32_t* deg, double damping, float* dd,
                               uint32_t* sinkbits);
// CTAs per SM of the batched-PPR grid, for every vector width
constexpr int PPR_CTAS_PER_SM = 2;

// One body of a batch of graphs: phase A, grid barrier, phase B over the
// block-diagonal A^T; reads rbuf[from]/wbuf[from], writes the other pair
// (cooperative launch of grid CTAs).
cudaError_t launch_pr_batch(cudaStream_t st, const PrParams& p, int from, int grid);
int pr_batch_blocks_per_sm();
cudaError_t launch_mg_init(cudaStream_t st, const MgInit& a);
// graph_of[i] = g for vptr[g] <= i < vptr[g+1]; *bad (device) += rows with
// a column outside their block.
cudaError_t launch_mg_graph_of(cudaStream_t st, int32_t ngraphs, const int64_t* vptr, int32_t n,
                               const int32_t* row_ptr, const int32_t* col_idx, int32_t* graph_of,
                               unsigned long long* bad);

// Resident CTAs per SM of the fused kernel for the given rank / gather types
// (hot_n > 0: the persistent kernel with a hot copy of hot_n entries; 0 when
// that configuration cannot run).
int pr_blocks_per_sm(int32_t rank_type, int32_t gather_type, int32_t gmode, int persistent, int32_t hot_n = 0,
                     int32_t tma_stages = 0, bool bins = false);
// Dynamic shared memory of the hot persistent kernel.
size_t pr_hot_dynamic_smem(int32_t hot_n, int32_t tma_stages);
// Static shared memory of the hot persistent kernel (bytes, upper bound).
constexpr size_t PR_HOT_STATIC_SMEM = 26 * 1024;
constexpr size_t PR_SMEM_PER_BLOCK_MAX = 227 * 1024;
// Threads per CTA of the persistent kernel with the shared-memory hot copy
// (one CTA per SM).
constexpr int PR_HOT_BLOCK = 768;
cudaError_t launch_pr(cudaStream_t st, const PrParams& p, int32_t rank_type, int32_t gather_type, int grid,
                      int persistent);
// The persistent FP32 loop of one personalised query (p.pers_bits set; the
// hot copy when p.hot_n > 0), its occupancy, and the scatter of its seeds
// into the start vector and the seed bitmap.
cudaError_t launch_pr_pers(cudaStream_t st, const PrParams& p, int grid);
int pr_pers_blocks_per_sm(int32_t hot_n);
cudaError_t launch_pr_seed_scatter(cudaStream_t st, int32_t nseeds, const int32_t* seeds, const int32_t* old2new,
                                   float val, float* r0, uint32_t* bits);
cudaError_t launch_barrier_selftest(cudaStream_t st, SyncWords* sync, int32_t* status, int64_t spin_limit, int grid);

}  // namespace grb
