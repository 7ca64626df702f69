// The planner: runs the pending DAG a materialisation needs (§II wait,
// §III-B materialize), fusing it into as few kernels as the kernel table
// allows.
//
// At wait(v) the closure of v's pending nodes is collected in program order.
// A version is elided (never materialised) when no handle points at it and
// every node that reads it is in the closure (§II: implementations may elide
// unneeded objects).  Nodes are grouped backwards from the last one; each
// group is one kernel, looked up by its shape -- the signature of §III-C,
// here a fixed table of pre-built templates instead of JIT-compiled code:
//
//   PR      ewise_mult(/, t, d) -> mxv(plus.second|plus.times, A^T) ->
//           ewise_add(+, rt, .) | accum +, optionally followed by
//           reduce(+, ewise_add(|x-y|, t, .))          -> kernels_pr.cu
//   EWRED   reduce(monoid, ewise(...)) followed by scalar apply steps
//                                                       -> ew_reduce_kernel
//   SINGLE  any one method                              -> one kernel each
//
// Groups run in the order of their last node, which always respects the
// dependencies (an input of a group is the output of an earlier group's last
// node, since inner nodes of a group feed only that group).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <unordered_set>

#include "grb_core.h"

namespace grb {

// ------------------------------------------------------------- host math
double round_host(grb_type t, double x) {
    switch (t) {
        case GRB_INT32: return (double)(int32_t)x;
        case GRB_FP32: return (double)(float)x;
        case GRB_BF16: {
            float f = (float)x;
            uint32_t u;
            std::memcpy(&u, &f, 4);
            u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
            u &= 0xffff0000u;
            std::memcpy(&f, &u, 4);
            return (double)f;
        }
        default: return x;
    }
}

double host_binop(int32_t code, double k, double x, double y) {
    switch (code) {
        case GRB_FIRST: return x;
        case GRB_SECOND: return y;
        case GRB_PLUS: return x + y;
        case GRB_MINUS: return x - y;
        case GRB_TIMES: return x * y;
        case GRB_DIV: return x / y;
        case GRB_MAX: return x > y ? x : y;
        case GRB_MIN: return x < y ? x : y;
        case GRB_ABS_DIFF: return x > y ? x - y : y - x;
        case GRB_MAX_DIV_BY: { double q = x / k; return q > y ? q : y; }
    }
    return x;
}

// ------------------------------------------------------ fill estimation
// Whether every entry of v is known to be present.  Exact for materialised
// versions; for pending ones it follows the structure of the method (the
// naive metadata estimators of §III-D, restricted to the case where they are
// certain, so that a FULL output never misses an entry).
static bool node_out_full(const Node* nd);

bool guaranteed_full(const Version* v) {
    if (!v) return false;
    if (v->scalar) return true;
    if (v->ready || !v->producer) return v->fmt == Fmt::ISO || v->fmt == Fmt::FULL;
    return node_out_full(v->producer);
}

static bool node_out_full(const Node* nd) {
    bool t_full = false;
    switch (nd->k) {
        case OpK::APPLY:
        case OpK::APPLY_B2:
        case OpK::APPLY_B2S: t_full = guaranteed_full(nd->u); break;
        case OpK::ASSIGN_S: t_full = true; break;
        case OpK::EADD: t_full = guaranteed_full(nd->u) || guaranteed_full(nd->v); break;
        case OpK::EMULT: t_full = guaranteed_full(nd->u) && guaranteed_full(nd->v); break;
        case OpK::MXV:
            t_full = guaranteed_full(nd->u) && nd->A->nonempty_rows == nd->A->nrows;
            break;
        default: return true;
    }
    const bool w_full = nd->w_old && guaranteed_full(nd->w_old);
    const bool z_full = nd->has_accum ? (t_full || w_full) : t_full;
    if (nd->mask) return z_full && w_full && !(nd->desc & GRB_DESC_REPLACE);
    return z_full;
}

// ------------------------------------------------------------ helpers
static SIn sin_of(const Version* s) {
    SIn in;
    if (s->host_known) in.host = s->hval;
    else in.slot = (const double*)s->slot.p;
    return in;
}

static grb_info alloc_vec(Ctx* c, Version* v, bool full) {
    v->vals = buf_alloc(c, type_size(v->type) * (size_t)v->n);
    if (!v->vals.p) return GRB_OUT_OF_MEMORY;
    if (!full) {
        v->present = buf_alloc(c, (size_t)v->n);
        if (!v->present.p) return GRB_OUT_OF_MEMORY;
    }
    v->fmt = full ? Fmt::FULL : Fmt::BITMAP;
    return GRB_SUCCESS;
}

static grb_info alloc_slot(Ctx* c, Version* v) {
    v->slot = buf_alloc(c, sizeof(double));
    v->host_known = false;
    return v->slot.p ? GRB_SUCCESS : GRB_OUT_OF_MEMORY;
}

static void sem_ops(grb_semiring s, int32_t& add, int32_t& mul) {
    switch (s) {
        case GRB_PLUS_TIMES: add = GRB_MONOID_PLUS; mul = GRB_TIMES; break;
        case GRB_PLUS_SECOND: add = GRB_MONOID_PLUS; mul = GRB_SECOND; break;
        case GRB_PLUS_FIRST: add = GRB_MONOID_PLUS; mul = GRB_FIRST; break;
        case GRB_MAX_TIMES: add = GRB_MONOID_MAX; mul = GRB_TIMES; break;
        case GRB_MIN_PLUS: add = GRB_MONOID_MIN; mul = GRB_PLUS; break;
        case GRB_MAX_SECOND: add = GRB_MONOID_MAX; mul = GRB_SECOND; break;
    }
}

static void plan_free(Ctx* c, TilePlan* p) {
    for (DevBuf* b : {&p->meta, &p->rowend_bits, &p->ne_rows, &p->empty_rows, &p->agg, &p->first, &p->fix,
                      &p->longfix, &p->part})
        buf_free(c, *b);
    for (auto& b : p->loop_bufs) buf_free(c, b);
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    delete p;
}

// The matrix's row plan, built once; nothing is cached unless the whole plan
// was built.
// Row-length bins of the binned body: the non-empty rows by the group that
// sums them (PR_BIN_MAX), ascending within each bin; once per matrix, from
// the row offsets on the host.
grb_info ensure_bins(Ctx* c, Matrix* A) {
    grb_info st = ensure_plan(c, A);
    if (st) return st;
    TilePlan* pl = A->plan;
    if (pl->bins_built) return GRB_SUCCESS;
    const int64_t n = A->nrows;
    std::vector<int32_t> rp((size_t)n + 1);
    st = cuda_check(c, cudaMemcpyAsync(rp.data(), A->row_ptr.p, sizeof(int32_t) * (size_t)(n + 1),
                                       cudaMemcpyDeviceToHost, c->stream), "row bins");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "row bins");
    if (st) return st;
    std::vector<int32_t> bins[6];
    for (int64_t i = 0; i < n; ++i) {
        const int32_t L = rp[(size_t)i + 1] - rp[(size_t)i];
        if (L == 0) continue;
        int b = 0;
        while (b < 5 && L > PR_BIN_MAX[b]) ++b;
        bins[b].push_back((int32_t)i);
    }
    std::vector<int32_t> all;
    all.reserve((size_t)n);
    for (int b = 0; b < 6; ++b) {
        pl->bin_off[b] = (int32_t)all.size();
        all.insert(all.end(), bins[b].begin(), bins[b].end());
    }
    pl->bin_off[6] = (int32_t)all.size();
    pl->bin_rows = buf_alloc(c, sizeof(int32_t) * std::max<size_t>(all.size(), 1));
    if (!pl->bin_rows.p) return GRB_OUT_OF_MEMORY;
    if (!all.empty())
        st = cuda_check(c, cudaMemcpyAsync(pl->bin_rows.p, all.data(), sizeof(int32_t) * all.size(),
                                           cudaMemcpyHostToDevice, c->stream), "row bins");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "row bins");
    if (!st) pl->bins_built = true;
    return st;
}

// Bounds-checked builds validate a matrix's structure on the device before
// the first kernel that walks it (plan, column counts, relabelling, general
// mxv); the host reads the verdict before anything indexes with it.
grb_info check_structure(Ctx* c, Matrix* A) {
#ifdef GRB_CHECK_BOUNDS
    if (A->structure_checked) return GRB_SUCCESS;
    c->stats.kernel_launches++;
    grb_info st = cuda_check(c, launch_csr_check(c->stream, A->nrows, A->ncols, A->nnz,
                                                 (const int32_t*)A->row_ptr.p, (const int32_t*)A->col_idx.p,
                                                 (int32_t*)c->status.p), "structure check");
    if (!st) st = read_status(c);
    if (!st) A->structure_checked = true;
    return st;
#else
    (void)c;
    (void)A;
    return GRB_SUCCESS;
#endif
}

grb_info ensure_plan(Ctx* c, Matrix* A) {
    if (A->plan) return GRB_SUCCESS;
    {
        const grb_info sc = check_structure(c, A);
        if (sc) return sc;
    }
    TilePlan* p = new TilePlan();
    p->ntiles = padded_nnz(A->nnz) / PR_NZTILE;
    const int64_t n = A->nrows;
    p->meta = buf_alloc(c, sizeof(uint32_t) * p->ntiles);
    p->rowend_bits = buf_alloc(c, sizeof(uint32_t) * (size_t)p->ntiles * (PR_NZTILE / 32));
    p->ne_rows = buf_alloc(c, sizeof(int32_t) * n);
    p->empty_rows = buf_alloc(c, sizeof(int32_t) * n);
    p->agg = buf_alloc(c, sizeof(double) * p->ntiles);
    p->first = buf_alloc(c, sizeof(double) * p->ntiles);
    p->fix = buf_alloc(c, sizeof(FixDesc) * p->ntiles);
    p->longfix = buf_alloc(c, sizeof(int32_t) * (p->ntiles + 3));
    p->part = buf_alloc(c, sizeof(double) * 2 * 2 * (size_t)c->sm_count * 8);
    if (!p->meta.p || !p->rowend_bits.p || !p->ne_rows.p || !p->empty_rows.p || !p->agg.p || !p->first.p ||
        !p->fix.p || !p->longfix.p || !p->part.p) {
        plan_free(c, p);
        return GRB_OUT_OF_MEMORY;
    }
    int32_t* counts_dev = (int32_t*)p->longfix.p + p->ntiles;
    PlanArgs pa;
    pa.row_ptr = (const int32_t*)A->row_ptr.p;
    pa.nrows = (int32_t)A->nrows;
    pa.nnz = (int32_t)A->nnz;
    pa.ntiles = p->ntiles;
    pa.ne_rows = (int32_t*)p->ne_rows.p;
    pa.empty_rows = (int32_t*)p->empty_rows.p;
    pa.rowend_bits = (uint32_t*)p->rowend_bits.p;
    pa.tile_meta = (uint32_t*)p->meta.p;
    pa.fix = (FixDesc*)p->fix.p;
    pa.longfix = (int32_t*)p->longfix.p;
    pa.counts = counts_dev;
    grb_info st = cuda_check(c, build_row_plan(c->stream, pa, [](void* x, size_t b) { return dev_alloc((Ctx*)x, b); },
                                               [](void* x, void* q, size_t b) { dev_free((Ctx*)x, q, b); }, c),
                             "row plan");
    c->stats.kernel_launches += 5;
    int32_t counts[3] = {0, 0, 0};
    if (!st)
        st = cuda_check(c, cudaMemcpyAsync(counts, counts_dev, sizeof(counts), cudaMemcpyDeviceToHost, c->stream), "plan");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "plan");
    if (st) {
        cudaStreamSynchronize(c->stream);
        plan_free(c, p);
        return st;
    }
    p->n_ne = counts[0];
    p->n_empty = counts[1];
    p->nlong = counts[2];
    A->plan = p;
    return GRB_SUCCESS;
}

// Degree-ordered copy of a square pattern matrix, built once and cached on
// the matrix (matrices are immutable).  The gathers of the PageRank loop read
// w[j] for the columns j of A^T; numbering vertices by descending out-degree
// puts the most-gathered entries of w next to each other, so far fewer cache
// lines serve the same gathers.  The loop's vectors are permuted into and out
// of this order around the loop.  On graphs without hubs (the REL_TOP
// vertices of largest out-degree carry less than REL_MIN_COVER of the edges)
// the order buys nothing and no copy is made: A->rel stays null.
static constexpr int32_t REL_TOP = 32768;
static constexpr double REL_MIN_COVER = 0.10;

grb_info ensure_coldeg(Ctx* c, Matrix* A) {
    if (A->coldeg.p) return GRB_SUCCESS;
    {
        const grb_info sc = check_structure(c, A);
        if (sc) return sc;
    }
    DevBuf d = buf_alloc(c, sizeof(int32_t) * (size_t)(A->ncols > 0 ? A->ncols : 1));
    if (!d.p) return GRB_OUT_OF_MEMORY;
    c->stats.kernel_launches++;
    grb_info st = cuda_check(c, launch_col_count(c->stream, A->ncols, A->nnz, (const int32_t*)A->col_idx.p,
                                                 (int32_t*)d.p), "column count");
    if (st) {
        buf_free(c, d);
        return st;
    }
    A->coldeg = d;
    return GRB_SUCCESS;
}

grb_info ensure_relabel(Ctx* c, Matrix* A) {
    if (A->rel || A->rel_checked) return GRB_SUCCESS;
    if (A->nrows != A->ncols || A->vals.p || A->nrows <= 0) return GRB_INVALID_VALUE;
    {
        const grb_info sd = ensure_coldeg(c, A);
        if (sd) return sd;
    }
    const int64_t n = A->nrows;
    auto af = [](void* x, size_t b) { return dev_alloc((Ctx*)x, b); };
    auto ff = [](void* x, void* q, size_t b) { dev_free((Ctx*)x, q, b); };
    DevBuf n2o = buf_alloc(c, sizeof(int32_t) * (size_t)n), o2n = buf_alloc(c, sizeof(int32_t) * (size_t)n);
    grb_info st = (n2o.p && o2n.p) ? GRB_SUCCESS : GRB_OUT_OF_MEMORY;
    RelabelArgs a;
    a.n = (int32_t)n;
    a.nnz = A->nnz;
    a.row_ptr = (const int32_t*)A->row_ptr.p;
    a.col_idx = (const int32_t*)A->col_idx.p;
    a.new_row_ptr = nullptr;
    a.new_col_idx = nullptr;
    a.new2old = (int32_t*)n2o.p;
    a.old2new = (int32_t*)o2n.p;
    a.top_h = REL_TOP;
    a.coldeg = (const int32_t*)A->coldeg.p;
    unsigned long long top = 0;
    if (!st) {
        st = cuda_check(c, relabel_order(c->stream, a, &top, af, ff, c), "relabel order");
        c->stats.kernel_launches += 5;
    }
    if (!st && (double)top < REL_MIN_COVER * (double)A->nnz) {
        A->rel_checked = true;
        buf_free(c, n2o);
        buf_free(c, o2n);
        return GRB_SUCCESS;
    }
    Matrix* R = nullptr;
    if (!st) {
        R = new Matrix();
        R->ctx = c;
        R->type = A->type;
        R->nrows = A->nrows;
        R->ncols = A->ncols;
        R->nnz = A->nnz;
        R->iso_val = A->iso_val;
        R->nonempty_rows = A->nonempty_rows;
        R->row_ptr = buf_alloc(c, sizeof(int32_t) * (size_t)(n + 1));
        R->col_idx = buf_alloc(c, sizeof(int32_t) * (size_t)padded_nnz(A->nnz));
        if (!R->row_ptr.p || !R->col_idx.p) st = GRB_OUT_OF_MEMORY;
    }
    if (!st) {
        a.new_row_ptr = (int32_t*)R->row_ptr.p;
        a.new_col_idx = (int32_t*)R->col_idx.p;
        st = cuda_check(c, relabel_build(c->stream, a, af, ff, c), "relabel build");
        c->stats.kernel_launches += 4;
    }
    if (st) {
        if (R) matrix_unref(R);
        buf_free(c, n2o);
        buf_free(c, o2n);
        return st;
    }
    A->rel = R;
    A->rel_checked = true;
    A->new2old = n2o;
    A->old2new = o2n;
    A->rel_id = c->next_id++;
    return GRB_SUCCESS;
}

// A FULL vector's values (bits = false) or a sink bitmap (bits = true) in
// the vertex order of A's relabelled copy, cached on the (immutable) version.
grb_info ensure_perm_copy(Ctx* c, Matrix* A, Version* v, bool bits) {
    const int32_t n = (int32_t)v->n;
    const int32_t* n2o = (const int32_t*)A->new2old.p;
    if (bits) {
        if (v->perm_bits_key == A->rel_id && v->perm_sinkbits.p) return GRB_SUCCESS;
        buf_free(c, v->perm_sinkbits);
        v->perm_bits_key = 0;
        v->perm_sinkbits = buf_alloc(c, sizeof(uint32_t) * (size_t)((n + 31) / 32));
        if (!v->perm_sinkbits.p) return GRB_OUT_OF_MEMORY;
        c->stats.kernel_launches++;
        grb_info st = cuda_check(c, launch_permute_bits(c->stream, n, n2o, (const uint32_t*)v->sinkbits.p,
                                                        (uint32_t*)v->perm_sinkbits.p), "permute sink bits");
        if (!st) v->perm_bits_key = A->rel_id;
        return st;
    }
    if (v->fmt != Fmt::FULL) return GRB_INVALID_VALUE;
    if (v->perm_vals_key == A->rel_id && v->perm_vals.p) return GRB_SUCCESS;
    buf_free(c, v->perm_vals);
    v->perm_vals_key = 0;
    v->perm_vals = buf_alloc(c, type_size(v->type) * (size_t)n);
    if (!v->perm_vals.p) return GRB_OUT_OF_MEMORY;
    c->stats.kernel_launches++;
    grb_info st = cuda_check(c, launch_permute(c->stream, n, n2o, v->vals.p, v->perm_vals.p, (int32_t)type_size(v->type)),
                             "permute vector");
    if (!st) v->perm_vals_key = A->rel_id;
    return st;
}

grb_info ensure_sinkbits(Ctx* c, Version* s) {
    if (s->sinkbits.p) return GRB_SUCCESS;
    DevBuf b = buf_alloc(c, sizeof(uint32_t) * (size_t)((s->n + 31) / 32));
    if (!b.p) return GRB_OUT_OF_MEMORY;
    c->stats.kernel_launches++;
    grb_info st = cuda_check(c, launch_sinkbits(c->stream, s->n, vin_of(s), (uint32_t*)b.p), "sink bits");
    if (st) {
        cudaStreamSynchronize(c->stream);
        buf_free(c, b);
        return st;
    }
    s->sinkbits = b;   // cached only once built
    return GRB_SUCCESS;
}

static PrParams plan_params(Ctx* c, Matrix* A) {
    PrParams p;
    TilePlan* pl = A->plan;
    p.row_ptr = (const int32_t*)A->row_ptr.p;
    p.col_idx = (const int32_t*)A->col_idx.p;
    p.nrows = (int32_t)A->nrows;
    p.nnz = (int32_t)A->nnz;
    p.ncols = (int32_t)A->ncols;
    p.ntiles = (int32_t)pl->ntiles;
    p.tile_meta = (const uint32_t*)pl->meta.p;
    p.rowend_bits = (const uint32_t*)pl->rowend_bits.p;
    p.ne_rows = (const int32_t*)pl->ne_rows.p;
    p.n_ne = (int32_t)pl->n_ne;
    p.empty_rows = (const int32_t*)pl->empty_rows.p;
    p.n_empty = (int32_t)pl->n_empty;
    p.agg = (double*)pl->agg.p;
    p.first = (double*)pl->first.p;
    p.fix = (const FixDesc*)pl->fix.p;
    p.longfix = (const int32_t*)pl->longfix.p;
    p.nlong = (int32_t)pl->nlong;
    p.part = (double*)pl->part.p;
    p.sync = (SyncWords*)c->sync.p;
    p.status = (int32_t*)c->status.p;
    p.spin_limit = c->spin_limit;
    return p;
}

PrParams plan_params_of(Ctx* c, Matrix* A) { return plan_params(c, A); }

int pr_grid(Ctx* c, Matrix* A, int32_t T, int32_t G, int32_t gmode, int persistent, int32_t hot_n,
            int32_t tma_stages, bool bins) {
    int nb = pr_blocks_per_sm(T, G, gmode, persistent, hot_n, tma_stages, bins);
    if (nb <= 0) {
        if (persistent == 1 && hot_n > 0) return 0;   // the hot-copy kernel cannot run: caller drops it
        nb = 1;
    }
    int g = nb * c->sm_count;
    if (g > c->sm_count * 8) g = c->sm_count * 8;
    const int wpb = (persistent == 1 && hot_n > 0 ? PR_HOT_BLOCK : PR_BLOCK) / 32;
    const int64_t need = (A->plan->ntiles + wpb - 1) / wpb;   // one tile per warp at least
    if (g > need) g = (int)need;
    return g < 1 ? 1 : g;
}

grb_info read_status(Ctx* c) {
    // word 0 the code; words 1-3 what a bounds check found (checked builds)
    int32_t w[4] = {0, 0, 0, 0};
    grb_info e = cuda_check(c, cudaMemcpyAsync(w, c->status.p, STATUS_BYTES, cudaMemcpyDeviceToHost, c->stream),
                            "status read");
    if (e) return e;
    e = cuda_check(c, cudaStreamSynchronize(c->stream), "stream sync");
    if (e) return e;
    const int32_t st = w[0];
    if (st != 0) {
        cudaMemsetAsync(c->status.p, 0, STATUS_BYTES, c->stream);
        // a barrier that gave up leaves its counter mid-crossing
        cudaMemsetAsync(c->sync.p, 0, sizeof(SyncWords), c->stream);
        if (st == (int32_t)GRB_DEVICE_TIMEOUT) {
            c->err = "a bounded device-side wait ran out";
        } else if (st == (int32_t)GRB_INDEX_OUT_OF_BOUNDS) {
            long long v = 0;
            std::memcpy(&v, w + 2, sizeof(v));
            char msg[160];
            if (w[1] == BOUNDS_ROW_PTR)
                std::snprintf(msg, sizeof msg, "bounds check: row_ptr[%lld] out of order or outside [0, nnz]", v);
            else if (w[1] == BOUNDS_COLUMN)
                std::snprintf(msg, sizeof msg, "bounds check: column index %lld outside [0, ncols)", v);
            else
                std::snprintf(msg, sizeof msg, "bounds check: index %lld out of range", v);
            c->err = msg;
        } else {
            c->err = "device status error";
        }
        return (grb_info)st;
    }
    return GRB_SUCCESS;
}

// ---------------------------------------------------------- executors
static grb_info exec_ew(Ctx* c, Node* nd, Version* out) {
    // assign of a scalar to every index, unmasked: an iso vector, no kernel
    if (nd->k == OpK::ASSIGN_S && !nd->mask && !nd->has_accum) {
        if (nd->s->host_known) {
            out->iso = round_host(out->type, nd->s->hval);
        } else {
            out->iso_src = nd->s;
            ver_ref(nd->s);
        }
        out->fmt = Fmt::ISO;
        return GRB_SUCCESS;
    }
    EwSpec e;
    switch (nd->k) {
        case OpK::APPLY: e.kind = EW_APPLY; e.unop = nd->unop; break;
        case OpK::APPLY_B2: e.kind = EW_APPLY_B2; e.s.host = nd->k == OpK::APPLY_B2 ? nd->k_const() : 0.0; break;
        case OpK::APPLY_B2S: e.kind = EW_APPLY_B2; e.s = sin_of(nd->s); break;
        case OpK::ASSIGN_S: e.kind = EW_ASSIGN; e.s = sin_of(nd->s); break;
        case OpK::EADD: e.kind = EW_EADD; break;
        case OpK::EMULT: e.kind = EW_EMULT; break;
        default: return GRB_PANIC;
    }
    e.op.code = nd->op.opcode;
    e.op.k = nd->op.k;
    e.ctype = out->type;
    if (nd->u) e.u = vin_of(nd->u);
    if (nd->v) e.v = vin_of(nd->v);
    WriteSpec w;
    if (nd->mask) {
        w.use_mask = 1;
        w.mask = vin_of(nd->mask);
        w.structural = (nd->desc & GRB_DESC_STRUCTURE) ? 1 : 0;
        w.complement = (nd->desc & GRB_DESC_COMPLEMENT) ? 1 : 0;
        w.replace = (nd->desc & GRB_DESC_REPLACE) ? 1 : 0;
    }
    if (nd->has_accum) {
        w.has_accum = 1;
        w.accum.code = nd->accum.opcode;
        w.accum.k = nd->accum.k;
    }
    if (nd->w_old) w.w_old = vin_of(nd->w_old);
    const bool full = node_out_full(nd);
    grb_info st = alloc_vec(c, out, full);
    if (st) return st;
    VOut o;
    o.vals = out->vals.p;
    o.present = (uint8_t*)out->present.p;
    o.type = out->type;
    o.full = full ? 1 : 0;
    c->stats.kernel_launches++;
    return cuda_check(c, launch_ewise(c->stream, out->n, e, w, o), "ewise");
}

static bool mxv_fast_ok(const Node* nd, const Version* u, grb_type T) {
    const Matrix* A = nd->A;
    if (nd->mask) return false;
    if (A->vals.p) return false;
    if (!(nd->sr == GRB_PLUS_SECOND || (nd->sr == GRB_PLUS_TIMES && A->iso_val == 1.0))) return false;
    if (!(T == GRB_FP32 || T == GRB_FP64)) return false;
    if (A->nrows + A->nnz >= PR_INDEX_LIMIT) return false;
    if (nd->has_accum) {
        if (nd->accum.opcode != GRB_PLUS || !nd->w_old || nd->w_old->type != T) return false;
    }
    return u != nullptr && u->type == T;
}

static void set_base(PrParams& p, const Version* b) {
    p.has_base = 1;
    if (b->fmt == Fmt::ISO && b->iso_src && !b->iso_src->host_known) {
        p.tele_from_slot = 1;
        p.tele_slot = (double*)b->iso_src->slot.p;
    } else {
        p.base = vin_of(b);
    }
}

static grb_info exec_mxv(Ctx* c, Node* nd, Version* out) {
    const grb_type T = out->type;
    Matrix* A = nd->A;
    const Version* u = nd->u;
    grb_info st;
    if (mxv_fast_ok(nd, u, T) && (u->fmt == Fmt::FULL || (u->fmt == Fmt::ISO && !u->iso_src))) {
        if ((st = ensure_plan(c, A))) return st;
        PrParams p = plan_params(c, A);
        if (u->fmt == Fmt::ISO) {
            p.gmode = G_ISO;
            p.g_iso = u->iso;
        } else {
            p.gmode = G_W;
            p.w = u->vals.p;
        }
        if (nd->has_accum) set_base(p, nd->w_old);
        const bool full = node_out_full(nd);
        if ((st = alloc_vec(c, out, full))) return st;
        p.out.vals = out->vals.p;
        p.out.present = (uint8_t*)out->present.p;
        p.out.type = T;
        p.out.full = full ? 1 : 0;
        c->stats.kernel_launches++;
        return cuda_check(c, launch_pr(c->stream, p, T, T, pr_grid(c, A, T, T, p.gmode, 0), 0), "mxv");
    }
    // general semiring / masked / valued matrix: row kernel into a temporary,
    // then the write step
    Version tmp;
    tmp.ctx = c;
    tmp.type = T;
    tmp.n = out->n;
    if ((st = alloc_vec(c, &tmp, false))) { ver_free_data(&tmp); return st; }
    int32_t add = GRB_MONOID_PLUS, mul = GRB_TIMES;
    sem_ops(nd->sr, add, mul);
    VOut o;
    o.vals = tmp.vals.p;
    o.present = (uint8_t*)tmp.present.p;
    o.type = T;
    o.full = 0;
    if ((st = check_structure(c, A))) { ver_free_data(&tmp); return st; }
    c->stats.kernel_launches += 2;
    st = cuda_check(c, launch_mxv_generic(c->stream, A->nrows, (const int32_t*)A->row_ptr.p,
                                          (const int32_t*)A->col_idx.p, A->vals.p, A->type, A->iso_val, vin_of(u),
                                          add, mul, o, A->ncols, (int32_t*)c->status.p), "mxv");
    if (!st) {
        Node cp;
        cp.k = OpK::APPLY;
        cp.unop = GRB_IDENTITY;
        cp.u = &tmp;
        cp.mask = nd->mask;
        cp.desc = nd->desc;
        cp.has_accum = nd->has_accum;
        cp.accum = nd->accum;
        cp.w_old = nd->w_old;
        // node_out_full on the copy needs A for MXV only; APPLY reads u
        st = exec_ew(c, &cp, out);
        c->stats.kernel_launches--;  // counted above
        cp.u = cp.mask = cp.w_old = nullptr;
    }
    ver_free_data(&tmp);
    return st;
}

static grb_info reduce_scratch(Ctx* c) {
    if (c->red_scratch.p) return GRB_SUCCESS;
    c->red_scratch = buf_alloc(c, sizeof(double) * (size_t)c->sm_count * 8);
    c->red_counter = buf_alloc(c, sizeof(uint32_t));
    if (!c->red_scratch.p || !c->red_counter.p) return GRB_OUT_OF_MEMORY;
    return cuda_check(c, cudaMemsetAsync(c->red_counter.p, 0, sizeof(uint32_t), c->stream), "reduce counter");
}

static int reduce_grid(Ctx* c, int64_t n) {
    int64_t g = (n + 2047) / 2048;
    if (g > c->sm_count * 4) g = c->sm_count * 4;
    return g < 1 ? 1 : (int)g;
}

static void ew_spec_of(const Node* X, EwSpec& e) {
    switch (X->k) {
        case OpK::APPLY: e.kind = EW_APPLY; e.unop = X->unop; break;
        case OpK::APPLY_B2: e.kind = EW_APPLY_B2; e.s.host = X->k_const(); break;
        case OpK::APPLY_B2S: e.kind = EW_APPLY_B2; e.s = sin_of(X->s); break;
        case OpK::EADD: e.kind = EW_EADD; break;
        case OpK::EMULT: e.kind = EW_EMULT; break;
        default: e.kind = EW_COPY; break;
    }
    e.op.code = X->op.opcode;
    e.op.k = X->op.k;
    e.ctype = X->out->type;
    if (X->u) e.u = vin_of(X->u);
    if (X->v) e.v = vin_of(X->v);
}

// reduce(monoid, X or u) then the scalar chain; result into `final_out`.
static grb_info exec_reduce(Ctx* c, Node* Q, Node* X, const std::vector<Node*>& chain, Version* final_out) {
    grb_info st;
    if ((st = reduce_scratch(c))) return st;
    EwSpec e;
    int64_t n;
    if (X) {
        ew_spec_of(X, e);
        n = X->out->n;
    } else {
        e.kind = EW_COPY;
        e.u = vin_of(Q->u);
        e.ctype = Q->u->type;
        n = Q->u->n;
    }
    SChain ch;
    for (Node* S : chain) {
        ch.ops[ch.n].code = S->op.opcode;
        ch.ops[ch.n].k = S->op.k;
        ch.c[ch.n] = S->k_const();
        ch.rtype[ch.n] = S->out->type;
        ch.n++;
    }
    OpSpec acc;
    SIn s_old;
    if (Q->has_accum) {
        acc.code = Q->accum.opcode;
        acc.k = Q->accum.k;
        s_old = sin_of(Q->w_old);
    }
    if ((st = alloc_slot(c, final_out))) return st;
    c->stats.kernel_launches++;
    return cuda_check(c, launch_ew_reduce(c->stream, n, e, Q->mon, Q->has_accum ? 1 : 0, acc, s_old, ch, Q->out->type,
                                          (double*)final_out->slot.p, (double*)c->red_scratch.p,
                                          (uint32_t*)c->red_counter.p, reduce_grid(c, n)),
                      "reduce");
}

static grb_info exec_sapply(Ctx* c, Node* S, Version* out) {
    if (S->s->host_known) {
        out->host_known = true;
        out->hval = round_host(out->type, host_binop(S->op.opcode, S->op.k, S->s->hval, S->k_const()));
        return GRB_SUCCESS;
    }
    grb_info st = alloc_slot(c, out);
    if (st) return st;
    SChain ch;
    ch.n = 1;
    ch.ops[0].code = S->op.opcode;
    ch.ops[0].k = S->op.k;
    ch.c[0] = S->k_const();
    ch.rtype[0] = out->type;
    c->stats.kernel_launches++;
    return cuda_check(c, launch_scalar_chain(c->stream, sin_of(S->s), ch, out->type, (double*)out->slot.p),
                      "scalar apply");
}

static grb_info exec_single(Ctx* c, Node* nd) {
    Version* out = nd->out;
    switch (nd->k) {
        case OpK::MXV: return exec_mxv(c, nd, out);
        case OpK::REDUCE: return exec_reduce(c, nd, nullptr, {}, out);
        case OpK::SAPPLY_B2: return exec_sapply(c, nd, out);
        default: return exec_ew(c, nd, out);
    }
}

// ------------------------------------------------------------ grouping
struct Group {
    enum Kind { SINGLE, PR, EWRED } kind = SINGLE;
    Node* root = nullptr;
    std::vector<Node*> nodes;
    // PR
    Node *W = nullptr, *M = nullptr, *E = nullptr, *X = nullptr, *Q = nullptr;
    Version* rt = nullptr;
    // EWRED
    Node* red = nullptr;
    Node* ew = nullptr;
    std::vector<Node*> chain;
};

struct Closure {
    std::vector<Node*> nodes;
    std::unordered_set<Node*> in;
    std::unordered_map<const Version*, std::vector<Node*>> consumers;
    Version* target = nullptr;
    bool must_mat(const Version* v) const {
        if (v == target || v->handle_refs > 0 || v->pins > 0) return true;
        auto it = consumers.find(v);
        const int nc = it == consumers.end() ? 0 : (int)it->second.size();
        return v->node_refs > nc;
    }
    // v is produced in the closure and, of all the pending nodes, read only
    // by `only`: it can be computed inside `only`'s kernel.  A handle may
    // still point at v; v then stays pending (its node is kept, as a method
    // tree is in the paper) and is only computed if it is read later.
    bool exclusive_to(const Version* v, const Node* only) const {
        if (!v || v == target || !v->producer || !in.count(v->producer) || v->pins > 0) return false;
        auto it = consumers.find(v);
        if (it == consumers.end()) return false;
        if (v->node_refs != (int)it->second.size()) return false;
        for (Node* n : it->second)
            if (n != only) return false;
        return true;
    }
};

static void add_inputs(const Node* nd, std::vector<Version*>& xs) {
    xs.clear();
    for (Version* x : {nd->u, nd->v, nd->s, nd->mask, nd->w_old})
        if (x) xs.push_back(x);
}

// A version usable as a fused-kernel input: available before the group runs
// (ready now, or produced by an earlier group's last node) and full of type T.
static bool full_input(const Version* v, grb_type T, bool allow_iso) {
    if (!v || v->scalar || v->type != T) return false;
    if (!guaranteed_full(v)) return false;
    if (v->ready || !v->producer) return v->fmt == Fmt::FULL || (allow_iso && v->fmt == Fmt::ISO);
    // pending: produced by an earlier group; only full materialisations occur
    // for full-guaranteed methods, except unmasked scalar assigns (iso)
    if (v->producer->k == OpK::ASSIGN_S && !v->producer->mask && !v->producer->has_accum) return allow_iso;
    return true;
}

static bool match_pr_core(const Closure& C, Node* root, const std::unordered_set<Node*>& used, Group& g) {
    Node* E = nullptr;
    Node* M = nullptr;
    Version* rt = nullptr;
    if (root->k == OpK::EADD && root->op.opcode == GRB_PLUS && !root->mask && !root->has_accum) {
        for (int side = 0; side < 2 && !M; ++side) {
            Version* s = side == 0 ? root->v : root->u;
            Version* o = side == 0 ? root->u : root->v;
            if (s && s->producer && s->producer->k == OpK::MXV && C.exclusive_to(s, root) && !used.count(s->producer)) {
                M = s->producer;
                rt = o;
            }
        }
        if (!M) return false;
        E = root;
    } else if (root->k == OpK::MXV) {
        M = root;
    } else {
        return false;
    }
    const grb_type T = M->out->type;
    if (!mxv_fast_ok(M, M->u, T)) return false;
    if (E) {
        if (M->has_accum || E->out->type != T || !full_input(rt, T, true)) return false;
    } else if (M->has_accum && !full_input(M->w_old, T, true)) {
        return false;
    }
    Node* W = nullptr;
    Version* u = M->u;
    if (u->producer && C.in.count(u->producer) && !used.count(u->producer) && C.exclusive_to(u, M)) {
        Node* w = u->producer;
        if (w->k == OpK::EMULT && w->op.opcode == GRB_DIV && !w->mask && !w->has_accum && w->out->type == T &&
            full_input(w->u, T, false) && full_input(w->v, T, false))
            W = w;  // the division runs inside the gather
    }
    if (!W && (!full_input(u, T, true) || (u->fmt == Fmt::ISO && u->iso_src) ||
               (!u->ready && u->producer && u->producer->k == OpK::ASSIGN_S && !u->producer->s->host_known))) {
        return false;  // gather operands are arrays or host-known iso values
    }
    g.kind = Group::PR;
    g.W = W;
    g.M = M;
    g.E = E;
    g.rt = rt;
    g.nodes.clear();
    if (W) g.nodes.push_back(W);
    g.nodes.push_back(M);
    if (E) g.nodes.push_back(E);
    g.root = E ? E : M;
    return true;
}

static bool match_group(const Closure& C, Node* root, const std::unordered_set<Node*>& used, Group& g) {
    // PR core with the residual reduction appended
    if (root->k == OpK::REDUCE && root->mon == GRB_MONOID_PLUS && !root->has_accum) {
        Version* xv = root->u;
        if (xv->producer && C.in.count(xv->producer) && !used.count(xv->producer) && C.exclusive_to(xv, root)) {
            Node* X = xv->producer;
            if (X->k == OpK::EADD && X->op.opcode == GRB_ABS_DIFF && !X->mask && !X->has_accum) {
                for (int side = 0; side < 2; ++side) {
                    Version* R = side == 0 ? X->v : X->u;
                    Version* ref = side == 0 ? X->u : X->v;
                    if (!R->producer || !C.in.count(R->producer) || used.count(R->producer)) continue;
                    Group core;
                    if (!match_pr_core(C, R->producer, used, core)) continue;
                    const grb_type T = core.M->out->type;
                    if (X->out->type != T || !full_input(ref, T, false)) continue;
                    // R is read by X and possibly by later groups / handles
                    auto it = C.consumers.find(R);
                    bool ok = true;
                    for (Node* n : it->second) ok = ok && (n == X || !C.in.count(n) || n->seq > root->seq);
                    if (!ok) continue;
                    g = core;
                    g.X = X;
                    g.Q = root;
                    g.nodes.push_back(X);
                    g.nodes.push_back(root);
                    g.root = root;
                    return true;
                }
            }
        }
    }
    if (match_pr_core(C, root, used, g)) return true;
    // reduce(ewise) + scalar chain
    if (root->k == OpK::SAPPLY_B2 || root->k == OpK::REDUCE) {
        std::vector<Node*> chain;
        Node* cur = root;
        while (cur->k == OpK::SAPPLY_B2) {
            chain.push_back(cur);
            Version* in = cur->s;
            if (!in->producer || !C.in.count(in->producer) || used.count(in->producer) || !C.exclusive_to(in, cur))
                return false;
            cur = in->producer;
        }
        if (cur->k != OpK::REDUCE || chain.size() > 5) return false;
        std::reverse(chain.begin(), chain.end());
        Node* X = nullptr;
        Version* xv = cur->u;
        if (xv->producer && C.in.count(xv->producer) && !used.count(xv->producer) && C.exclusive_to(xv, cur)) {
            Node* p = xv->producer;
            const bool ew = p->k == OpK::EADD || p->k == OpK::EMULT || p->k == OpK::APPLY || p->k == OpK::APPLY_B2 ||
                            p->k == OpK::APPLY_B2S;
            if (ew && !p->mask && !p->has_accum) X = p;
        }
        if (!X && chain.empty()) return false;  // a plain reduce runs as a single node
        g.kind = Group::EWRED;
        g.red = cur;
        g.ew = X;
        g.chain = chain;
        g.nodes.clear();
        if (X) g.nodes.push_back(X);
        g.nodes.push_back(cur);
        for (Node* s : chain) g.nodes.push_back(s);
        g.root = root;
        return true;
    }
    return false;
}

static grb_info exec_pr_group(Ctx* c, const Closure& C, Group& g) {
    Node* M = g.M;
    Matrix* A = M->A;
    const grb_type T = M->out->type;
    grb_info st;
    if ((st = ensure_plan(c, A))) return st;
    PrParams p = plan_params(c, A);
    DevBuf wtmp;   // the quotient t ./ d, when it is computed once per vertex
    if (g.W && A->nnz >= 2 * A->nrows) {
        // Cost rule: fused into the gather, the division runs once per
        // nonzero with two random gathers (t and d); with two or more
        // nonzeros per row it is cheaper to compute w = t ./ d once per
        // vertex in a streaming pass and gather w alone.  The quotients are
        // the same values either way (rounded to the rank type).
        wtmp = buf_alloc(c, type_size(T) * (size_t)A->ncols);
        if (!wtmp.p) return GRB_OUT_OF_MEMORY;
        EwSpec e;
        e.kind = EW_EMULT;
        e.op.code = GRB_DIV;
        e.ctype = T;
        e.u = vin_of(g.W->u);
        e.v = vin_of(g.W->v);
        WriteSpec wr;
        VOut o;
        o.vals = wtmp.p;
        o.type = T;
        o.full = 1;
        c->stats.kernel_launches++;
        if ((st = cuda_check(c, launch_ewise(c->stream, A->ncols, e, wr, o), "gather values"))) {
            buf_free(c, wtmp);
            return st;
        }
        p.gmode = G_W;
        p.w = wtmp.p;
    } else if (g.W) {
        p.gmode = G_TD;
        p.t = g.W->u->vals.p;
        p.d = g.W->v->vals.p;
    } else if (M->u->fmt == Fmt::ISO) {
        p.gmode = G_ISO;
        p.g_iso = vin_of(M->u).iso;
    } else {
        p.gmode = G_W;
        p.w = M->u->vals.p;
    }
    if (g.E) set_base(p, g.rt);
    else if (M->has_accum) set_base(p, M->w_old);
    Node* core_root = g.E ? g.E : M;
    Version* R = core_root->out;
    const bool full = node_out_full(core_root);
    if ((st = alloc_vec(c, R, full))) {
        buf_free(c, wtmp);
        return st;
    }
    p.out.vals = R->vals.p;
    p.out.present = (uint8_t*)R->present.p;
    p.out.type = T;
    p.out.full = full ? 1 : 0;
    if (g.Q) {
        p.want_resid = 1;
        const Version* ref = (g.X->v == R) ? g.X->u : g.X->v;
        p.r_old = ref->vals.p;
        if ((st = alloc_slot(c, g.Q->out))) {
            buf_free(c, wtmp);
            return st;
        }
        p.resid_slot = (double*)g.Q->out->slot.p;
        p.resid_type = g.Q->out->type;
    }
    c->stats.kernel_launches++;
    if (g.nodes.size() > 1) c->stats.fused_groups++;
    else c->stats.unfused_nodes++;
    st = cuda_check(c, launch_pr(c->stream, p, T, T, pr_grid(c, A, T, T, p.gmode, 0), 0), "fused pagerank step");
    buf_free(c, wtmp);   // stream-ordered: a later allocation reuses it after this kernel
    return st;
}

// ----------------------------------------------------------- materialize
static void collect(Version* target, Closure& C) {
    std::vector<Node*> stack;
    if (target->producer) stack.push_back(target->producer);
    std::vector<Version*> xs;
    while (!stack.empty()) {
        Node* nd = stack.back();
        stack.pop_back();
        if (C.in.count(nd)) continue;
        C.in.insert(nd);
        C.nodes.push_back(nd);
        add_inputs(nd, xs);
        for (Version* x : xs)
            if (x->producer && !C.in.count(x->producer)) stack.push_back(x->producer);
    }
    std::sort(C.nodes.begin(), C.nodes.end(), [](const Node* a, const Node* b) { return a->seq < b->seq; });
    for (Node* nd : C.nodes) {
        add_inputs(nd, xs);
        for (Version* x : xs) C.consumers[x].push_back(nd);
    }
}

grb_info materialize(Ctx* c, Version* target) {
    if (target->ready || !target->producer) return target->err;
    Closure C;
    C.target = target;
    collect(target, C);

    std::vector<Group> groups;
    std::unordered_set<Node*> used;
    for (auto it = C.nodes.rbegin(); it != C.nodes.rend(); ++it) {
        Node* nd = *it;
        if (used.count(nd)) continue;
        Group g;
        if (!(c->fusion && match_group(C, nd, used, g))) {
            g = Group();
            g.kind = Group::SINGLE;
            g.root = nd;
            g.nodes = {nd};
        }
        for (Node* m : g.nodes) used.insert(m);
        groups.push_back(g);
    }
    std::sort(groups.begin(), groups.end(), [](const Group& a, const Group& b) { return a.root->seq < b.root->seq; });

    NvtxRange range("grb: wait (fused groups)");
    grb_info st = GRB_SUCCESS;
    for (Group& g : groups) {
        NvtxRange grange(g.kind == Group::PR ? "grb: PageRank group" : g.kind == Group::EWRED ? "grb: element-wise + reduce group"
                                                                                           : "grb: single method");
        if (g.kind == Group::PR) st = exec_pr_group(c, C, g);
        else if (g.kind == Group::EWRED) {
            st = exec_reduce(c, g.red, g.ew, g.chain, g.root->out);
            c->stats.fused_groups++;
        } else {
            st = exec_single(c, g.root);
            c->stats.unfused_nodes++;
        }
        if (st) break;
        for (Node* m : g.nodes) {
            const bool written = m == g.root || (g.kind == Group::PR && m == (g.E ? g.E : g.M));
            if (written) m->out->ready = true;
            else c->stats.elided_vectors++;
        }
    }
    if (st) {
        if (c->err.empty()) c->err = "execution failed";
        target->err = st;
        target->errmsg = c->err;
        target->ready = true;
    }
    // Nodes whose output was materialised are done.  Outputs computed only
    // inside a fused kernel stay pending: their nodes remain the producers
    // and are released with the version once nothing refers to it.  Detach
    // first (destroying a node may free an elided version and its producer).
    std::vector<Node*> done;
    for (Node* nd : C.nodes)
        if (nd->out->ready) {
            nd->out->producer = nullptr;
            done.push_back(nd);
        }
    for (Node* nd : done) node_destroy(nd);
    return st ? st : target->err;
}

grb_info run_pending_all(Ctx* c) {
    // materialise every pending version a live handle holds, oldest first
    std::vector<Version*> pending;
    for (VectorH* h : c->vhandles)
        if (h->cur && h->cur->producer) pending.push_back(h->cur);
    for (ScalarH* h : c->shandles)
        if (h->cur && h->cur->producer) pending.push_back(h->cur);
    std::sort(pending.begin(), pending.end(),
              [](const Version* a, const Version* b) { return a->producer->seq < b->producer->seq; });
    for (Version* v : pending) ver_ref(v);
    grb_info st = GRB_SUCCESS;
    for (Version* v : pending) {
        grb_info s2 = materialize(c, v);
        if (!st) st = s2;
    }
    for (Version* v : pending) ver_unref(v);
    return st;
}

}  // namespace grb
