/*
 * grb.h -- C-ABI of the GB300 nonblocking GraphBLAS library (PageRank subset).
 *
 * The calls follow the GraphBLAS C API statement that the paper builds on
 * (§II "Nonblocking execution"): destructive, output-first arguments; every
 * call validates its arguments and returns at once; in NONBLOCKING mode the
 * call only records a node of the program-order DAG (§II, §III-A), and the
 * work runs when a result is needed (grb_wait, grb_scalar_get, an extract).
 * At that point the planner fuses the pending DAG into as few GPU kernels as
 * it can (§III-B: one fused loop per materialisation), looking kernels up by
 * the DAG's signature (§III-C).  In BLOCKING mode every call completes and
 * materialises its output before returning (§II), one GPU kernel per method.
 * Both modes give the same results up to floating-point rounding order (§II).
 *
 * Conventions
 *  - Handles are opaque and library-owned; release each with grb_free.
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership.  Device pointers are accepted where a flag says so.
 *  - Device memory comes from the context's allocator callbacks (or the CUDA
 *    stream-ordered allocator when none are given); all GPU work runs on the
 *    context's stream.
 *  - Errors: API errors (null handle, dimension or domain mismatch, invalid
 *    value) are returned immediately and change nothing.  Execution errors
 *    (out of memory, index out of range, device timeout) surface when the work
 *    runs -- at grb_wait or a call that forces it -- and stick to the output
 *    object; grb_error() returns the message.
 *  - Indices are 32-bit (§IV uses 32-bit indices): n < 2^31, nnz < 2^31.
 *    The fused row-gather kernels (device loops, the fused mxv, grb_ppr_*,
 *    grb_prbatch_*) take a matrix while nrows + nnz < 2^31 - 2^24
 *    (GRB_FUSED_INDEX_LIMIT); past it, mxv and the loops run on the general
 *    kernels, and grb_ppr_new / grb_prbatch_new return GRB_INVALID_VALUE.
 */
#ifndef GRB_H
#define GRB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status */
typedef enum {
    GRB_SUCCESS = 0,
    GRB_NO_VALUE = 1,               /* scalar holds no value */
    /* API errors (returned at once) */
    GRB_NULL_POINTER = -1,
    GRB_INVALID_VALUE = -2,
    GRB_INVALID_INDEX = -3,
    GRB_DOMAIN_MISMATCH = -4,
    GRB_DIMENSION_MISMATCH = -5,
    GRB_UNINITIALIZED_OBJECT = -6,
    GRB_NOT_IMPLEMENTED = -7,
    GRB_INVALID_OBJECT = -8,        /* object carries a sticky execution error */
    /* execution errors (at wait; sticky on the object) */
    GRB_OUT_OF_MEMORY = -101,
    GRB_INDEX_OUT_OF_BOUNDS = -102,
    GRB_DEVICE_ERROR = -103,
    GRB_DEVICE_TIMEOUT = -104,      /* a bounded device-side wait ran out */
    GRB_PANIC = -105
} grb_info;

/* §II: the two execution modes. */
typedef enum { GRB_BLOCKING = 0, GRB_NONBLOCKING = 1 } grb_mode;

/* Element types.  BF16 is a storage type: arithmetic on it runs in FP32. */
typedef enum { GRB_INT32 = 1, GRB_FP32 = 2, GRB_FP64 = 3, GRB_BF16 = 4 } grb_type;

/* Predefined binary operators.  MAX_DIV_BY carries a bound parameter k and
 * computes (x, y) -> max(x / k, y), the operator the §IV PageRank listing
 * uses to build the out-degree divisor. */
typedef enum {
    GRB_FIRST = 1, GRB_SECOND = 2, GRB_PLUS = 3, GRB_MINUS = 4, GRB_TIMES = 5,
    GRB_DIV = 6, GRB_MAX = 7, GRB_MIN = 8, GRB_ABS_DIFF = 9, GRB_MAX_DIV_BY = 10
} grb_opcode;

typedef struct grb_binop {
    int32_t opcode;   /* grb_opcode */
    int32_t reserved; /* must be 0 */
    double k;         /* parameter of GRB_MAX_DIV_BY; ignored otherwise */
} grb_binop;

/* Unary operators for grb_apply. */
typedef enum { GRB_IDENTITY = 1, GRB_ABS = 2, GRB_AINV = 3, GRB_MINV = 4 } grb_unop;

/* Monoids for reductions and semiring addition. */
typedef enum { GRB_MONOID_PLUS = 1, GRB_MONOID_MAX = 2, GRB_MONOID_MIN = 3, GRB_MONOID_TIMES = 4 } grb_monoid;

/* Semirings (add monoid, multiply operator).  PLUS_SECOND is the (+, (_,x)->x)
 * semiring of the §IV listing's mxv; on an iso-1 pattern matrix PLUS_TIMES
 * gives the same values. */
typedef enum {
    GRB_PLUS_TIMES = 1, GRB_PLUS_SECOND = 2, GRB_PLUS_FIRST = 3,
    GRB_MAX_TIMES = 4, GRB_MIN_PLUS = 5, GRB_MAX_SECOND = 6
} grb_semiring;

/* Descriptor flags (bitwise OR). */
enum {
    GRB_DESC_DEFAULT = 0,
    GRB_DESC_REPLACE = 1,     /* clear output entries outside the mask */
    GRB_DESC_STRUCTURE = 2,   /* mask by presence, not by value */
    GRB_DESC_COMPLEMENT = 4   /* use the complement of the mask */
};
typedef uint32_t grb_desc;

/* grb_matrix_build_csr flags. */
enum {
    GRB_BUILD_TRANSPOSE = 1,   /* store A^T: row i lists the sources of edges j->i */
    GRB_BUILD_DROP_SELF = 2,   /* drop self loops */
    GRB_BUILD_DEDUP = 4,       /* drop duplicate (row, col) pairs */
    GRB_BUILD_DEVICE_PTRS = 8  /* src/dst/vals are device pointers */
};

typedef enum { GRB_WAIT_COMPLETE = 0, GRB_WAIT_MATERIALIZE = 1 } grb_wait_mode;

/* Context options (grb_context_set). */
typedef enum {
    GRB_OPT_FUSION = 1,        /* 1 (default): fuse at wait; 0: one kernel per method */
    GRB_OPT_PERSISTENT = 2,    /* grb_iterate_end on a fused PageRank body:
                                  0 = automatic (default), 1 = one persistent kernel
                                  for all iterations, 2 = one fused kernel per
                                  iteration captured in a CUDA graph, 3 = replay the
                                  body from the host (per-wait fusion only) */
    GRB_OPT_SPIN_LIMIT = 3,    /* iteration limit of device-side waits (>0) */
    GRB_OPT_MIXED_SWITCH = 4,  /* residual below which the BF16 gather switches to
                                  FP32, in units of 1e-9 (default 1e6, i.e. 1e-3) */
    GRB_OPT_MIXED = 5,         /* FP32 PageRank device loops gather the rank in
                                  BF16 (FP32 accumulation) until the residual
                                  falls below the switch, then in FP32:
                                  0 (default) never; 1 when the FP32 gather
                                  vector (4 n bytes) exceeds the L2 cache, the
                                  planner's choice (smaller vectors stay
                                  L2-resident, where BF16 saves nothing);
                                  2 always */
    GRB_OPT_RELABEL = 6,       /* 1 (default): device loops run on a copy of the
                                  matrix with vertices numbered by descending
                                  out-degree (built once per matrix, cached; the
                                  loop's vectors are permuted in and out), so the
                                  rank gathers touch fewer cache lines; 0: the
                                  matrix as built */
    GRB_OPT_HOT_BYTES = 7,     /* bytes of shared memory per SM that the persistent
                                  FP32 loop on a degree-ordered matrix uses for a
                                  copy of the most-gathered rank entries
                                  (0 .. GRB_HOT_BYTES_MAX; default 163840; 0 = off) */
    GRB_OPT_TMA_STAGES = 8,    /* that loop's tile arrays: 0 (default) = register
                                  prefetch one tile ahead; 2 or 3 = bulk copies
                                  (cp.async.bulk) into shared-memory stages that
                                  many tiles ahead (the hot copy shrinks to fit) */
    GRB_OPT_ROW_BINS = 9       /* FP32 persistent PageRank loops: 0 (default) =
                                  nonzero-split warp tiles; 1 = every row summed
                                  by a group sized by its length (a thread, 4, 8
                                  or 16 lanes, a warp, or a CTA for the hub rows),
                                  no split rows and no fixup phase */
} grb_option;

#define GRB_HOT_BYTES_MAX 196608
#define GRB_FUSED_INDEX_LIMIT 2130706432LL   /* 2^31 - 2^24: bound on nrows + nnz of the fused kernels */

/* Opaque handles. */
typedef struct grb_context_s* grb_context;
typedef struct grb_matrix_s* grb_matrix;
typedef struct grb_vector_s* grb_vector;
typedef struct grb_scalar_s* grb_scalar;

/* Device allocator callbacks (for example, PyTorch's caching allocator).
 * alloc returns a device pointer of at least `bytes` bytes usable on `stream`,
 * or NULL; free releases it. */
typedef void* (*grb_alloc_fn)(void* alloc_ctx, size_t bytes, void* stream);
typedef void (*grb_free_fn)(void* alloc_ctx, void* ptr, void* stream);

/* Counters for tests and benchmarks (grb_context_stats). */
typedef struct grb_stats {
    int64_t kernel_launches;    /* kernels launched by the library so far */
    int64_t fused_groups;       /* fused kernels (more than one method each) */
    int64_t unfused_nodes;      /* methods run one kernel each */
    int64_t elided_vectors;     /* intermediate vectors never materialised */
    int64_t persistent_loops;   /* grb_iterate_end calls run on the device */
    int64_t replayed_loops;     /* grb_iterate_end calls replayed from the host */
    int64_t device_bytes;       /* bytes currently held by the library */
    int64_t cache_hits;         /* signature-table hits (§III-C) */
    int64_t last_loop_kernel_ns;/* device time of the last device loop's kernels
                                   (CUDA events on the context stream; reading
                                   it waits for that loop) */
} grb_stats;

/* ------------------------------------------------------------ context */

/* New context bound to a CUDA device stream (NULL = legacy default stream) of
 * the current device, in one of the §II execution modes (GrB_init's mode in
 * the GraphBLAS C statement the paper builds on; §II "Nonblocking
 * execution").  Every object made from it shares its mode and stream.  alloc/free may be NULL (stream-ordered cudaMallocAsync
 * is then used).  Errors: GRB_NULL_POINTER, GRB_INVALID_VALUE (bad mode),
 * GRB_DEVICE_ERROR (no usable GPU). */
grb_info grb_context_new(grb_context* ctx, grb_mode mode, void* cuda_stream,
                         grb_alloc_fn alloc, grb_free_fn free_fn, void* alloc_ctx);
grb_info grb_context_set(grb_context ctx, grb_option opt, int64_t value);
grb_info grb_context_stats(grb_context ctx, grb_stats* out);
/* Device times in milliseconds of the last min(cap, 64) device loops run by
 * grb_iterate_end on this context (CUDA events around the loop kernels on
 * the context stream), oldest first; *n gets the count.  Waits for those
 * loops.  Errors: GRB_NULL_POINTER (n NULL, or ms NULL with cap > 0). */
grb_info grb_context_loop_times(grb_context ctx, double* ms, int64_t cap, int64_t* n);
/* Runs every pending method of the context and synchronises its stream. */
grb_info grb_context_wait(grb_context ctx);

/* ------------------------------------------------------------- matrix */

/* Build a CSR matrix from a COO edge list (§IV: the PageRank listing takes
 * A^T as input; 32-bit indices).  With GRB_BUILD_TRANSPOSE, row i of the
 * stored matrix lists the sources j of the edges j -> i, ascending; otherwise
 * row j lists the destinations.  vals == NULL stores a pattern-only, iso-1
 * matrix (no value array; §III-C iso-valued objects).  The build sorts on the
 * GPU, drops self loops / duplicates when asked, and is bit-exact integer
 * work.  Errors: GRB_NULL_POINTER, GRB_INVALID_VALUE (sizes beyond 2^31-1,
 * bad type), GRB_INDEX_OUT_OF_BOUNDS (an index outside [0, nrows/ncols)),
 * GRB_OUT_OF_MEMORY. */
grb_info grb_matrix_build_csr(grb_matrix* A, grb_context ctx, grb_type type, uint64_t nrows,
                              uint64_t ncols, const int32_t* src, const int32_t* dst,
                              const void* vals, uint64_t nedges, uint32_t flags);
grb_info grb_matrix_nvals(uint64_t* nvals, grb_matrix A);
grb_info grb_matrix_nrows(uint64_t* n, grb_matrix A);
/* Copy the CSR arrays out (row_ptr: nrows+1 int32, col_idx: nvals int32,
 * vals: nvals of the matrix type or NULL).  out_is_device selects device or
 * host destination pointers. */
grb_info grb_matrix_export_csr(grb_matrix A, int32_t* row_ptr, int32_t* col_idx, void* vals,
                               int out_is_device);
/* deg(j) = number of stored entries in column j of A (for A^T: the out-degree
 * of vertex j in the graph; §IV's out_degree).  deg must be an INT32 vector
 * of length ncols in A's context (else GRB_INVALID_VALUE); vertices of
 * degree 0 get no entry (GraphBLAS reduce semantics).  The counts are
 * computed once per matrix and kept with it. */
grb_info grb_matrix_col_degree(grb_vector deg, grb_matrix A);

/* ------------------------------------------------------------- vector */

/* New vector with no entries (§III-A GrBVector{T,I}(n)). */
grb_info grb_vector_new(grb_vector* v, grb_context ctx, grb_type type, uint64_t n);
/* Make v an iso-valued full vector: every entry equals *value (a double
 * rounded to v's type).  Stores no array (§III-A GrBVector(n, v)). */
grb_info grb_vector_fill(grb_vector v, double value);
/* Replace v's content by the given entries (idx ascending, distinct;
 * host or device pointers; the GraphBLAS build of a sparse vector, the
 * SparseVector of §III-A).  vals are doubles rounded to v's type.  The call
 * waits for its copy.  Errors: GRB_NULL_POINTER, GRB_INVALID_VALUE (nvals >
 * n), GRB_INVALID_INDEX (an index outside [0, n), or host indices not
 * ascending; device indices are checked by the build kernel), GRB_OUT_OF_MEMORY;
 * on an error v keeps its old value. */
grb_info grb_vector_build(grb_vector v, const int32_t* idx, const double* vals, uint64_t nvals,
                          int ptrs_on_device);
/* dst takes src's current value (O(1): the two share one immutable version;
 * this is the `t = r` of the §IV listing). */
grb_info grb_vector_copy(grb_vector dst, grb_vector src);
grb_info grb_vector_size(uint64_t* n, grb_vector v);
/* Number of entries; forces the vector's pending work. */
grb_info grb_vector_nvals(uint64_t* nvals, grb_vector v);
/* Copy the vector out as a dense array of its type (absent entries -> 0) and
 * an optional uint8 presence array (host pointers, or device pointers when
 * out_is_device; n entries each, caller-owned).  Reading a result is a
 * materialisation point (§II: a value leaves the library only through a
 * method that waits; §III-B materialize), so pending work runs first and its
 * execution errors are returned here. */
grb_info grb_vector_extract_dense(grb_vector v, void* values, uint8_t* present, int out_is_device);

/* ------------------------------------------------------------- scalar */

grb_info grb_scalar_new(grb_scalar* s, grb_context ctx, grb_type type);
grb_info grb_scalar_set(grb_scalar s, double value);
/* Read the value (forces pending work; §III footnote: a scalar is
 * materialised before it is read).  GRB_NO_VALUE if the scalar is empty. */
grb_info grb_scalar_get(grb_scalar s, double* value);
/* out = op(in, k) on a (possibly pending) scalar. */
grb_info grb_scalar_apply_bind2nd(grb_scalar out, grb_binop op, grb_scalar in, double k);

/* ------------------------------------------------------------ methods
 * All take the GraphBLAS write step: w<mask> accum= T, where `mask` may be
 * NULL (all true), `accum` may be NULL (no accumulation), and `desc` holds
 * REPLACE / STRUCTURE / COMPLEMENT.  Arithmetic runs in w's type (FP32 for
 * BF16); inputs are converted to it. */

/* w = op(u) on each entry of u (§III-B VectorApply). */
grb_info grb_apply(grb_vector w, grb_vector mask, const grb_binop* accum, grb_unop op,
                   grb_vector u, grb_desc desc);
/* w = op(u, s) with the constant s bound as the second argument. */
grb_info grb_apply_bind2nd(grb_vector w, grb_vector mask, const grb_binop* accum, grb_binop op,
                           grb_vector u, double s, grb_desc desc);
/* Same with a (possibly pending) scalar object as the bound argument. */
grb_info grb_apply_bind2nd_scalar(grb_vector w, grb_vector mask, const grb_binop* accum,
                                  grb_binop op, grb_vector u, grb_scalar s, grb_desc desc);
/* w(i) = s for every index i (GrB_assign of a scalar to all indices); s may
 * be pending. */
grb_info grb_assign_scalar(grb_vector w, grb_vector mask, const grb_binop* accum, grb_scalar s,
                           grb_desc desc);
/* w = A (+.x) u over a semiring (§III-A MxV): row i gets an entry iff some
 * A(i,j) meets an entry u(j). */
grb_info grb_mxv(grb_vector w, grb_vector mask, const grb_binop* accum, grb_semiring s,
                 grb_matrix A, grb_vector u, grb_desc desc);
/* Union of index sets; op where both present (§III-D element-wise addition). */
grb_info grb_ewise_add(grb_vector w, grb_vector mask, const grb_binop* accum, grb_binop op,
                       grb_vector u, grb_vector v, grb_desc desc);
/* Intersection of index sets (§III-D element-wise multiplication). */
grb_info grb_ewise_mult(grb_vector w, grb_vector mask, const grb_binop* accum, grb_binop op,
                        grb_vector u, grb_vector v, grb_desc desc);
/* s accum= fold of the monoid over u's entries (identity when u is empty):
 * the reduce of the §IV listing (rdiff = reduce(+, t), Fig. "The PageRank
 * implementation in AppGrB").  Accumulation runs in FP64 and rounds once to
 * s's type; the fold order is fixed, so results are reproducible. */
grb_info grb_reduce(grb_scalar s, const grb_binop* accum, grb_monoid m, grb_vector u, grb_desc desc);

/* ------------------------------------------------------ materialisation */

/* Complete the pending work that `obj` (a vector, scalar or matrix handle)
 * depends on, fusing it (§II wait; §III-B materialize), and synchronise. */
grb_info grb_wait(void* obj, grb_wait_mode mode);

/* Loop capture (an extension that keeps nonblocking semantics).  Calls made
 * between grb_iterate_begin and grb_iterate_end are recorded as one loop body
 * instead of being run.  grb_iterate_end then executes
 *     while (iters < itermax && value(cond) > tol) { body; iters++; }
 * -- the loop test of the §IV listing (Fig. "The PageRank implementation in
 * AppGrB"), tested before each body.  When the body matches the fused
 * PageRank iteration the whole loop runs on the GPU (one persistent kernel,
 * or one fused kernel per iteration in a CUDA graph); otherwise the body is
 * replayed through the normal planner each iteration.  Every handle ends with
 * the value the plain loop would give it.
 * In NONBLOCKING mode a device loop whose body count is fixed in advance
 * (tol < 0: the loop test never fails, so *iters = itermax) only enqueues
 * its work and returns, as a nonblocking method does (§II): its results are
 * pending device values, and an execution error of the loop (a bounded
 * device-side wait that ran out) is returned by the next call that waits --
 * grb_wait, an extract, grb_scalar_get -- and sticks to what that call read.
 * A loop that stops on its tolerance waits once, for its body count. */
grb_info grb_iterate_begin(grb_context ctx);
grb_info grb_iterate_end(grb_context ctx, grb_scalar cond, double tol, int64_t itermax,
                         int64_t* iters);

/* History of the last loop grb_iterate_end ran on the device (waits for
 * it): hist[k] = the loop condition's value after body k (the §IV residual
 * rdiff), dang[k] = the dangling mass of the rank after body k -- the sum of
 * the rank over vertices without out-edges that the next body spreads
 * uniformly (NaN for loops without it) -- for k < *n; at most cap entries of
 * each written; hist and dang are optional.  *mixed_phase (optional) is 1
 * when a mixed-precision loop switched to the FP32 gather, 0 when it did
 * not, -1 for other loops. */
grb_info grb_iterate_history(grb_context ctx, double* hist, double* dang, int64_t cap, int64_t* n,
                             int32_t* mixed_phase);

/* ------------------------------- batched personalised PageRank (extension)
 *
 * The paper computes one PageRank vector (§IV).  A grb_ppr runs that same
 * fused iteration for up to GRB_PPR_MAX_SLOTS personalisation vectors
 * ("slots") over one matrix at once, as one sparse x dense product per body:
 * for slot s with seed set S (duplicates collapsed),
 *     v = 1/|S| on S,  r_0 = v,
 *     r' = (1 - damping) v + damping D / n + A^T (r ./ d),
 *     d = max(out-degree, 1) / damping,  D = sum of r over vertices
 *     without out-edges (dangling mass spread uniformly),
 *     rdiff = sum |r - r'|  (FP64),
 * and the §IV loop test `while iter <= itermax && rdiff > tol` applied to
 * each slot separately after every body; a slot whose test fails keeps its
 * rank while the others go on.  Ranks are FP32.  A slot's results do not
 * depend on the other slots or on its position (fixed summation orders).
 * Slots may be set, cleared and refilled between runs, which is how a serving
 * loop admits queries while others are in flight.
 *
 * The matrix is A^T as built by grb_matrix_build_csr(TRANSPOSE): row i lists
 * the sources of the edges into i; it must be square and pattern-only; the
 * grb_ppr holds a reference to it.  Release a grb_ppr with grb_free. */
typedef struct grb_ppr_s* grb_ppr;
#define GRB_PPR_MAX_SLOTS 128

/* New batch object with `slots` slots (rounded up to a multiple of 32;
 * grb_ppr_slots returns the count), all empty, vector width 1.  Device memory: about
 * 16 * n * slots bytes.  Errors: GRB_NULL_POINTER, GRB_UNINITIALIZED_OBJECT,
 * GRB_INVALID_VALUE (non-square or valued matrix, nrows + nnz at or past
 * GRB_FUSED_INDEX_LIMIT, slots outside 1..GRB_PPR_MAX_SLOTS, damping outside
 * [0, 1)), GRB_OUT_OF_MEMORY. */
grb_info grb_ppr_new(grb_ppr* P, grb_matrix AT, double damping, int32_t slots);
grb_info grb_ppr_slots(grb_ppr P, int32_t* slots);

/* Autotuner: each lane of a warp carries V = 1, 2 or 4 consecutive slots
 * (vector width; a k-tile holds 32 V slots).  Times trial_bodies (1..100)
 * bodies of every width with all slots busy and keeps the fastest;
 * ms_per_body[3] (optional) gets the times for V = 1, 2, 4, *chosen_vw
 * (optional) the winner.  Empties every slot; the slot count may grow to
 * a multiple of 32 V (grb_ppr_slots). */
grb_info grb_ppr_tune(grb_ppr P, int64_t trial_bodies, double* ms_per_body, int32_t* chosen_vw);

/* Set the vector width (1, 2 or 4) directly; empties every slot.  Results do
 * not depend on the width.  When a re-layout (here or in grb_ppr_tune) runs
 * out of memory, the object answers GRB_INVALID_OBJECT to every other call
 * until a re-layout succeeds. */
grb_info grb_ppr_layout(grb_ppr P, int32_t vw);

/* Start a query in `slot` (replacing whatever it held): seeds are host
 * vertex ids (nseeds >= 1; copied), tol and itermax its loop test.  The
 * query is queued on the host; every queued query is placed on the device
 * in one pass at the next grb_ppr_run / status / get / clear.
 * Errors: GRB_INVALID_VALUE (slot, nseeds or itermax out of range),
 * GRB_INVALID_INDEX (a seed outside [0, n)). */
grb_info grb_ppr_set(grb_ppr P, int32_t slot, const int32_t* seeds, int64_t nseeds, double tol, int64_t itermax);

/* Stop and empty a slot. */
grb_info grb_ppr_clear(grb_ppr P, int32_t slot);

/* Enqueue `iters` bodies (0..100000) for every active slot on the context's
 * stream (captured once per iteration count as a CUDA graph) and return. */
grb_info grb_ppr_run(grb_ppr P, int64_t iters);

/* Per slot (host arrays of grb_ppr_slots entries, each optional): 1 while
 * the slot's loop goes on, the bodies it has run, its last rdiff (1 before
 * the first body).  Waits for the queued work. */
grb_info grb_ppr_status(grb_ppr P, int32_t* active, int64_t* iters, double* resid);

/* The current rank vector of a slot: n FP32 values into `ranks` (host
 * memory, or device memory when out_is_device).  Waits for the queued work. */
grb_info grb_ppr_get(grb_ppr P, int32_t slot, float* ranks, int out_is_device);

/* Serving loop (extension): answers a stream of personalised-PageRank
 * queries by continuous batching on one grb_ppr.  Query q arrives
 * arrival_s[q] seconds after the call starts (non-decreasing) with seeds
 * seed_idx[seed_ptr[q] .. seed_ptr[q+1]) (at least one).  The loop admits
 * every arrived query into a free slot, runs `chunk` bodies for all queries
 * in flight, retires the finished ones and repeats, sleeping while idle.
 * Slots: as many as mem_fraction of the free device memory holds (about
 * 16 n bytes each), at most `slots` when slots > 0 and GRB_PPR_MAX_SLOTS;
 * free memory is read again at every admission, and while other users of
 * the device hold memory the slots in use stay below what mem_fraction of
 * (free memory + the slots' own) allows; more arrivals than usable slots
 * wait in arrival order.  The vector width is picked by grb_ppr_tune before
 * the first arrival.  A slot query's result is the one it gets alone
 * (grb_ppr); a query run on the single-vector loop (single_max) follows the
 * same iteration and loop test with its rows summed in another order, so it
 * agrees with the slot result to FP32 rounding.  Returns when every query
 * is answered. */
typedef struct grb_serve_config {
    double damping;
    double tol;            /* each query's loop test: rdiff > tol */
    int64_t itermax;
    int64_t chunk;         /* bodies per scheduling step (>= 1) */
    int32_t slots;         /* 0: limited by memory only */
    double mem_fraction;   /* (0, 1] */
    int32_t single_max;    /* >= 0: while no query holds a slot and at most this
                              many arrived queries wait, the oldest runs alone
                              on the single-vector fused loop (0: never) */
} grb_serve_config;

typedef struct grb_serve_result {
    double* latency_s;     /* [nq] answer time - arrival time (caller-owned) */
    int64_t* iters;        /* [nq] bodies run */
    double* resid;         /* [nq] final rdiff */
    float* ranks;          /* [nq * n] host ranks, or NULL to skip */
    int32_t slots;         /* out: slots used */
    int32_t vector_width;  /* out: slots per lane the autotuner chose */
    int64_t steps;         /* out: scheduling steps (graph launches) */
    int64_t max_in_flight; /* out */
    double wall_s;         /* out: time from start to the last answer */
    int64_t single_queries;/* out: queries answered by the single-vector loop */
} grb_serve_result;

grb_info grb_ppr_serve(grb_matrix AT, const grb_serve_config* cfg, int64_t nq, const double* arrival_s,
                       const int64_t* seed_ptr, const int32_t* seed_idx, grb_serve_result* out);

/* -------------------------------- batch of independent graphs (extension)
 *
 * Many PageRank problems on graphs of uneven size solved together.  AT is
 * one block-diagonal A^T (grb_matrix_build_csr with TRANSPOSE over the
 * graphs' edges, vertex ids offset so that graph g owns vertices
 * vptr[g] .. vptr[g+1]-1); an edge between two graphs is an error.  Every
 * graph runs the §IV loop with uniform dangling on its own (r_0 = 1/n_g,
 * teleport (1-d)/n_g + d D_g / n_g, FP64 residual, its own loop test); FP32
 * ranks.  A body is one launch over all graphs; a solve is captured as a
 * CUDA graph.  The launch shape (resident CTAs per SM) is picked by an
 * autotuner that times each candidate on the batch (grb_prbatch_tune, or
 * automatically before the first run); results do not depend on it. */
typedef struct grb_prbatch_s* grb_prbatch;

/* vptr: host, ngraphs + 1 non-decreasing offsets with vptr[0] = 0,
 * vptr[ngraphs] = nrows(AT), every graph at least one vertex.  Holds a
 * reference to AT.  Errors: GRB_INVALID_VALUE (bad offsets, non-square or
 * valued matrix, nrows + nnz at or past GRB_FUSED_INDEX_LIMIT, an edge across
 * graphs, damping outside [0, 1)). */
grb_info grb_prbatch_new(grb_prbatch* B, grb_matrix AT, int32_t ngraphs, const int64_t* vptr, double damping);

/* Autotune: time trial_bodies (1..1000) bodies for every candidate count of
 * resident CTAs per SM; ms_per_body[q] (host, cap entries, optional) gets
 * the time for q+1 CTAs per SM, *chosen (optional) the winner. */
grb_info grb_prbatch_tune(grb_prbatch B, int64_t trial_bodies, double* ms_per_body, int32_t cap, int32_t* chosen);

/* Solve every graph from its start vector: `while iter <= itermax &&
 * rdiff > tol` per graph, bodies launched `chunk` at a time until no graph's
 * loop goes on.  Blocks until done. */
grb_info grb_prbatch_run(grb_prbatch B, double tol, int64_t itermax, int64_t chunk);

/* ranks (host, nrows floats, optional): every graph's rank at its vertex
 * offsets; iters / resid (host, ngraphs, optional): bodies run, last rdiff. */
grb_info grb_prbatch_result(grb_prbatch B, float* ranks, int64_t* iters, double* resid);

/* ------------------------------------------------ allocation-free call */

/* The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory when they need a reduction -- code inside a host
 * framework that owns the whole device memory budget, code under a hard
 * memory cap where a new allocation could fail at a bad moment,
 * latency-critical paths that cannot pay for cudaMalloc's device
 * synchronisation.
 *
 * *out = fold of the monoid over the n elements of the dense device array x
 * (type INT32, FP32 or FP64), accumulated in FP64 in a fixed order (block b
 * folds elements [4096*b, 4096*b+4096), then the block results in order).
 * x and out are caller-owned device pointers; the call is asynchronous on
 * `stream` (NULL = legacy default stream) and allocates nothing: its scratch
 * (4096 partial sums and a counter, ~32 KB) is a fixed device array that
 * every GPU loading the library keeps until the process exits.
 *  - n may be at most GRB_NOALLOC_MAX_N; larger n returns GRB_INVALID_VALUE
 *    before any GPU work.  n = 0 gives the monoid's identity (0, 1, -inf or
 *    +inf for PLUS, TIMES, MAX, MIN).
 *  - Each call clears the scratch's counter before its kernel runs, so a
 *    call never depends on what an earlier one left in the array.
 *  - The first call on a device looks up the scratch array's device address
 *    (with that device current); make that first call before any stream
 *    capture.
 *  - All calls on a device share the scratch array: calls whose executions
 *    overlap on the GPU (different streams, no ordering between them) race.
 *  - Errors: GRB_NULL_POINTER, GRB_INVALID_VALUE (type, monoid or n),
 *    GRB_DEVICE_ERROR (no device, or the launch failed). */
#define GRB_NOALLOC_MAX_N 16777216ull
grb_info grb_reduce_dense_noalloc(const void* x, grb_type type, uint64_t n, grb_monoid m, double* out,
                                  void* stream);

/* -------------------------------------------------------------- misc */

/* Release any handle (sets *obj to NULL; GrB_free of the GraphBLAS
 * statement, §II).  Pending work that other objects still need is kept
 * (their method trees hold references, §III-A). */
grb_info grb_free(void** obj);
/* Last error message of a handle ("" if none): the GraphBLAS error string
 * of §II's error model (execution errors stick to the object that carries
 * them).  The pointer stays valid until the handle is used again. */
const char* grb_error(void* obj);
/* Self-test of the bounded device-side wait: launches a grid-barrier kernel
 * in which one arrival never comes, with the given spin limit, and returns
 * GRB_DEVICE_TIMEOUT once every block gave up (the GPU context stays
 * usable).  Used by the failure-detection test. */
grb_info grb_selftest_wait_timeout(grb_context ctx, int64_t spin_limit);

#ifdef __cplusplus
}
#endif
#endif /* GRB_H */
