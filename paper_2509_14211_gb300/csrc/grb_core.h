// Internal object model of the GB300 GraphBLAS library.
//
// A user handle (vector / scalar) points at a Version: an immutable value that
// is either materialised in device memory or still pending, i.e. the output
// of a DAG node that has not run (§II: program order defines a DAG; §III-A:
// containers hold either a materialised object or a method tree).  Methods
// never modify a version in place: they record a node whose output is a new
// version and re-point the output handle at it, so `t = r` followed by a
// write to r keeps t's old value (SSA versioning).  A version that no handle
// and no pending node outside the fused group needs is never materialised:
// that is how fusion elides intermediates (§II "elide unneeded objects").
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "grb.h"
#include "grb_kernels.h"

namespace grb {

enum class Kind : uint32_t { CONTEXT = 0x47524230u, MATRIX, VECTOR, SCALAR, PPR, PRBATCH, DEAD = 0xDEADDEADu };

struct Ctx;
struct Node;
struct Matrix;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// One immutable value (vector or scalar).
struct Version {
    Ctx* ctx = nullptr;
    uint64_t id = 0;
    int refs = 0;          // every owner (handles, nodes, planner pins)
    int handle_refs = 0;   // user handles currently pointing here
    int node_refs = 0;     // pending nodes that read this version
    bool scalar = false;
    grb_type type = GRB_FP32;
    int64_t n = 0;         // vector length (1 for scalars)
    bool ready = false;    // materialised
    grb_info err = GRB_SUCCESS;
    std::string errmsg;
    // vector storage (Fmt::ISO keeps `iso`; FULL keeps vals; BITMAP vals+present)
    Fmt fmt = Fmt::EMPTY;
    double iso = 0.0;
    DevBuf vals, present;
    // scalar storage: host value when known on the host, else a device slot
    bool host_known = false;
    double hval = 0.0;
    DevBuf slot;           // one double on the device
    Version* iso_src = nullptr;  // ISO vector whose value is this scalar version's
    int pins = 0;          // planner / loop engine references that need the data
    Node* producer = nullptr;  // non-null while pending
    // derived data cached on the version (immutable, so always valid)
    DevBuf sinkbits;       // bitmask of present entries (for sink vectors)
    // copies in the vertex order of a relabelled matrix (key = its rel_id)
    uint64_t perm_vals_key = 0, perm_bits_key = 0;
    DevBuf perm_vals, perm_sinkbits;
};

enum class OpK : int {
    APPLY = 1, APPLY_B2 = 2, APPLY_B2S = 3, ASSIGN_S = 4, EADD = 5, EMULT = 6,
    MXV = 7, REDUCE = 8, SAPPLY_B2 = 9
};

// A pending method (a node of the program-order DAG).
struct Node {
    OpK k = OpK::APPLY;
    uint64_t seq = 0;
    grb_binop op{};          // binary operator (EADD/EMULT/APPLY_B2/SAPPLY_B2)
    int unop = 0;            // APPLY
    bool has_accum = false;
    grb_binop accum{};
    grb_semiring sr = GRB_PLUS_TIMES;
    grb_monoid mon = GRB_MONOID_PLUS;
    grb_desc desc = 0;
    double cst = 0.0;        // bound constant (APPLY_B2, SAPPLY_B2)
    double k_const() const { return cst; }
    Version* u = nullptr;    // first vector input
    Version* v = nullptr;    // second vector input
    Version* s = nullptr;    // scalar input (APPLY_B2S, ASSIGN_S, SAPPLY_B2 input)
    Version* mask = nullptr;
    Version* w_old = nullptr;  // previous value of the output (accum / masked write)
    Matrix* A = nullptr;
    Version* out = nullptr;
};

// Cached launch plan of a CSR matrix for the merge-path kernels.
struct TilePlan {
    int64_t ntiles = 0;
    DevBuf meta;               // per tile: first non-empty row | continues-a-row << 31
    DevBuf rowend_bits;        // bit k: nonzero k ends its row
    DevBuf ne_rows, empty_rows;
    int64_t n_ne = 0, n_empty = 0;
    DevBuf agg, first;         // per-tile carry of the open last row / partial of the first row
    DevBuf fix;                // per-tile fixup descriptor (row of a split first row, first tile of it)
    DevBuf longfix;            // tiles whose split first row spans more than PR_LONG tiles
    int64_t nlong = 0;
    DevBuf part;               // 2 x grid_pr x 2 doubles (residual, dangling mass)
    std::vector<DevBuf> loop_bufs;
    cudaGraphExec_t graph_exec = nullptr;
    // row-length bins of the binned body (built on first use)
    DevBuf bin_rows;
    int32_t bin_off[7] = {0, 0, 0, 0, 0, 0, 0};
    bool bins_built = false;
};

struct Matrix {
    Kind kind = Kind::MATRIX;
    Ctx* ctx = nullptr;
    int refs = 1;              // the handle + pending nodes
    bool handle_alive = true;
    grb_type type = GRB_FP32;
    int64_t nrows = 0, ncols = 0, nnz = 0;
    DevBuf row_ptr, col_idx, vals;  // vals empty => iso-valued (pattern only)
    double iso_val = 1.0;
    int64_t nonempty_rows = -1;
    TilePlan* plan = nullptr;
    DevBuf coldeg;             // int32[ncols] entries per column (out-degree when this is A^T), computed once
    // degree-ordered copy of a square pattern matrix for the device loops
    Matrix* rel = nullptr;
    DevBuf new2old, old2new;
    uint64_t rel_id = 0;       // unique id of this relabelling
    bool rel_checked = false;  // the degree order was examined (rel null: not worth it)
    bool structure_checked = false;  // bounds-checked builds: row_ptr / col_idx validated on the device
    std::string err;
};

struct VectorH {
    Kind kind = Kind::VECTOR;
    Ctx* ctx = nullptr;
    grb_type type = GRB_FP32;
    int64_t n = 0;
    Version* cur = nullptr;
    std::string err;
};

struct ScalarH {
    Kind kind = Kind::SCALAR;
    Ctx* ctx = nullptr;
    grb_type type = GRB_FP64;
    Version* cur = nullptr;
    std::string err;
};

// Recorded statement of a loop body (grb_iterate_begin .. end).
struct Stmt {
    enum Kind { VCOPY, SSET, VFILL, OP, WAIT } kind = OP;
    VectorH* dstv = nullptr;   // output vector handle (OP on vectors, VCOPY, VFILL)
    ScalarH* dsts = nullptr;   // output scalar handle
    VectorH* srcv = nullptr;   // VCOPY source
    double value = 0.0;        // VFILL / SSET
    // OP payload: the node template with handle operands
    Node tmpl;
    VectorH *hu = nullptr, *hv = nullptr, *hmask = nullptr;
    ScalarH* hs = nullptr;
    Matrix* hA = nullptr;
    bool out_is_scalar = false;
};

struct Pool {
    std::multimap<size_t, void*> free_list;
    size_t held = 0;      // bytes obtained from the allocator and not returned
};

struct Ctx {
    Kind kind = Kind::CONTEXT;
    grb_mode mode = GRB_NONBLOCKING;
    cudaStream_t stream = nullptr;
    grb_alloc_fn alloc = nullptr;
    grb_free_fn freefn = nullptr;
    void* actx = nullptr;
    int device = 0, sm_count = 0;
    size_t l2_bytes = 0;
    bool fusion = true;
    int persistent = 0;
    int64_t spin_limit = int64_t(1) << 24;
    double mixed_switch = 1e-3;
    int mixed = 0;        // 0 off, 1 when the FP32 gather vector exceeds L2, 2 always
    bool relabel = true;  // device loops run on the degree-ordered copy of the matrix
    int64_t hot_bytes = 160 * 1024;  // shared-memory copy of the hottest gathered entries
    int32_t tma_stages = 0;          // bulk-copy staging depth of the hot loop (0: register prefetch)
    bool row_bins = false;           // FP32 persistent loops: row-length-binned body instead of tiles
    bool dry = false;     // replaying a loop body to inspect its DAG: never execute
    DevBuf red_scratch;   // per-block partials of the reduction kernels
    DevBuf red_counter;   // last-block counter of the reduction kernels
    uint64_t next_seq = 1, next_id = 1;
    Pool pool;
    grb_stats stats{};
    bool recording = false;
    std::vector<Stmt> body;
    DevBuf status;        // device status words (bounded waits, bounds checks), STATUS_BYTES
    DevBuf sync;          // grid-barrier words (SyncWords) of every launch on the stream; cleared with the
                          // status word after a device error
    cudaStream_t capture_stream = nullptr;   // CUDA-graph capture of device loops
    std::string err;
    std::vector<double> last_hist;    // residual history of the last device loop
    std::vector<double> last_dang;    // its dangling-mass history (uniform dangling)
    int last_mixed_phase = -1;
    // Pinned host staging of the last device loop's result slots and
    // histories, filled by asynchronous copies behind the loop kernel:
    // [0, 8) the loop slots, [8, 8 + cap) residuals, [8 + cap, 8 + 2 cap)
    // dangling masses.  stage_ev marks the copies; the histories are read
    // from the staging lazily (loop_pending) after that event.
    double* stage = nullptr;
    size_t stage_cap = 0;              // doubles
    cudaEvent_t stage_ev = nullptr;
    bool loop_pending = false;
    int64_t loop_cap = 0;              // history capacity of the pending loop
    bool loop_uniform = false, loop_mixed = false;
    // CUDA events around the last LOOP_TIMES device loops' kernels (a ring)
    static constexpr int LOOP_TIMES = 64;
    cudaEvent_t loop_ev[LOOP_TIMES][2] = {};
    int64_t loop_count = 0;
    std::vector<VectorH*> vhandles;   // live handles (grb_context_wait completes them)
    std::vector<ScalarH*> shandles;
};

// Profiler range for the duration of a scope (NVTX; free when no profiler
// is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------- memory
void* dev_alloc(Ctx* c, size_t bytes);
void dev_free(Ctx* c, void* p, size_t bytes);
DevBuf buf_alloc(Ctx* c, size_t bytes);
void buf_free(Ctx* c, DevBuf& b);
void pool_release_all(Ctx* c);

// ------------------------------------------------------------ versions
Version* new_version(Ctx* c, bool scalar, grb_type t, int64_t n);
void ver_ref(Version* v);
void ver_unref(Version* v);
void ver_free_data(Version* v);
void handle_set(VectorH* h, Version* v);
void handle_set(ScalarH* h, Version* v);
void matrix_unref(Matrix* A);
Node* new_node(Ctx* c, OpK k);
void node_attach_inputs(Node* nd);
void node_destroy(Node* nd);

// ------------------------------------------------------------- planner
grb_info materialize(Ctx* c, Version* target);
grb_info run_pending_all(Ctx* c);
grb_info record_or_run(Ctx* c, Node* nd);
grb_info iterate_end(Ctx* c, ScalarH* cond, double tol, int64_t itermax, int64_t* iters);
VIn vin_of(const Version* v);
size_t type_size(grb_type t);
grb_info cuda_check(Ctx* c, cudaError_t e, const char* what);
grb_info check_structure(Ctx* c, Matrix* A);
grb_info ensure_plan(Ctx* c, Matrix* A);
grb_info ensure_bins(Ctx* c, Matrix* A);
grb_info ensure_sinkbits(Ctx* c, Version* sinks);
grb_info ensure_relabel(Ctx* c, Matrix* A);
grb_info ensure_coldeg(Ctx* c, Matrix* A);
grb_info ensure_perm_copy(Ctx* c, Matrix* A, Version* v, bool bits);
struct Ppr;
void ppr_destroy(Ppr* P);
struct PrBatch;
void prbatch_destroy(PrBatch* B);
grb_info read_status(Ctx* c);
grb_info resolve_loop_history(Ctx* c);
int64_t last_loop_kernel_ns(Ctx* c);
void loop_resources_free(Ctx* c);
PrParams plan_params_of(Ctx* c, Matrix* A);
int pr_grid(Ctx* c, Matrix* A, int32_t T, int32_t G, int32_t gmode, int persistent, int32_t hot_n = 0,
            int32_t tma_stages = 0, bool bins = false);
double round_host(grb_type t, double x);
double host_binop(int32_t code, double k, double x, double y);
bool guaranteed_full(const Version* v);
grb_info submit_vec_op(Ctx* c, VectorH* w, Node* nd, VectorH* hu, VectorH* hv, VectorH* hmask, ScalarH* hs,
                       Matrix* A);
grb_info submit_scalar_op(Ctx* c, ScalarH* out, Node* nd, VectorH* hu, ScalarH* hs);
grb_info scalar_value(Ctx* c, Version* v, double* out);
grb_info replay_stmt(Ctx* c, const Stmt& st);
grb_info vector_fill_now(VectorH* v, double value);
grb_info scalar_set_now(ScalarH* s, double value);

}  // namespace grb
