// C-ABI entry points (include/grb.h): argument validation, handle management
// and recording of methods as DAG nodes (§II: a call returns once its
// arguments are validated; in blocking mode it also completes).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "grb_core.h"
#include "grb_debug.h"

using namespace grb;

namespace {

Ctx* as_ctx(grb_context c) {
    Ctx* x = reinterpret_cast<Ctx*>(c);
    return (x && x->kind == Kind::CONTEXT) ? x : nullptr;
}
VectorH* as_vec(grb_vector v) {
    VectorH* x = reinterpret_cast<VectorH*>(v);
    return (x && x->kind == Kind::VECTOR) ? x : nullptr;
}
ScalarH* as_sca(grb_scalar s) {
    ScalarH* x = reinterpret_cast<ScalarH*>(s);
    return (x && x->kind == Kind::SCALAR) ? x : nullptr;
}
Matrix* as_mat(grb_matrix m) {
    Matrix* x = reinterpret_cast<Matrix*>(m);
    return (x && x->kind == Kind::MATRIX) ? x : nullptr;
}

bool valid_type(int t) { return t == GRB_INT32 || t == GRB_FP32 || t == GRB_FP64 || t == GRB_BF16; }
bool valid_binop(const grb_binop& op) {
    return op.opcode >= GRB_FIRST && op.opcode <= GRB_MAX_DIV_BY && op.reserved == 0 &&
           (op.opcode != GRB_MAX_DIV_BY || op.k != 0.0);
}
bool valid_monoid(int m) { return m >= GRB_MONOID_PLUS && m <= GRB_MONOID_TIMES; }
bool valid_desc(grb_desc d) { return (d & ~(uint32_t)7u) == 0; }

void* pool_alloc_cb(void* ctx, size_t bytes) { return dev_alloc(static_cast<Ctx*>(ctx), bytes); }
void pool_free_cb(void* ctx, void* p, size_t bytes) { dev_free(static_cast<Ctx*>(ctx), p, bytes); }

// Common validation of the optional mask / accumulator of a vector method.
grb_info check_write(VectorH* w, grb_vector mask, const grb_binop* accum, grb_desc desc, VectorH** m_out) {
    *m_out = nullptr;
    if (!valid_desc(desc)) return GRB_INVALID_VALUE;
    if (accum && !valid_binop(*accum)) return GRB_INVALID_VALUE;
    if (mask) {
        VectorH* m = as_vec(mask);
        if (!m) return GRB_UNINITIALIZED_OBJECT;
        if (m->n != w->n) return GRB_DIMENSION_MISMATCH;
        if (m->ctx != w->ctx) return GRB_INVALID_VALUE;
        *m_out = m;
    }
    return GRB_SUCCESS;
}

void fill_write(Node* nd, const grb_binop* accum, grb_desc desc) {
    nd->desc = desc;
    if (accum) {
        nd->has_accum = true;
        nd->accum = *accum;
    }
}

grb_info finish_read(Ctx* c, Version* v) {
    grb_info st = materialize(c, v);
    grb_info s2 = read_status(c);
    if (st) return st;
    if (s2) {
        v->err = s2;
        v->errmsg = c->err;
        return s2;
    }
    return v->err;
}

}  // namespace

namespace grb {

grb_info submit_vec_op(Ctx* c, VectorH* w, Node* nd, VectorH* hu, VectorH* hv, VectorH* hmask, ScalarH* hs,
                       Matrix* A) {
    if (c->recording) {
        Stmt st;
        st.kind = Stmt::OP;
        st.tmpl = *nd;
        st.dstv = w;
        st.hu = hu;
        st.hv = hv;
        st.hmask = hmask;
        st.hs = hs;
        st.hA = A;
        c->body.push_back(st);
        delete nd;
        return GRB_SUCCESS;
    }
    nd->u = hu ? hu->cur : nullptr;
    nd->v = hv ? hv->cur : nullptr;
    nd->mask = hmask ? hmask->cur : nullptr;
    nd->s = hs ? hs->cur : nullptr;
    nd->A = A;
    const bool need_old = nd->has_accum || (nd->mask && !(nd->desc & GRB_DESC_REPLACE));
    nd->w_old = need_old ? w->cur : nullptr;
    node_attach_inputs(nd);
    Version* out = new_version(c, false, w->type, w->n);
    out->producer = nd;
    nd->out = out;
    handle_set(w, out);
    ver_unref(out);
    if (c->mode == GRB_BLOCKING && !c->dry) return materialize(c, out);
    return GRB_SUCCESS;
}

grb_info submit_scalar_op(Ctx* c, ScalarH* out_h, Node* nd, VectorH* hu, ScalarH* hs) {
    if (c->recording) {
        Stmt st;
        st.kind = Stmt::OP;
        st.tmpl = *nd;
        st.dsts = out_h;
        st.hu = hu;
        st.hs = hs;
        st.out_is_scalar = true;
        c->body.push_back(st);
        delete nd;
        return GRB_SUCCESS;
    }
    nd->u = hu ? hu->cur : nullptr;
    nd->s = hs ? hs->cur : nullptr;
    nd->w_old = nd->has_accum ? out_h->cur : nullptr;
    node_attach_inputs(nd);
    Version* out = new_version(c, true, out_h->type, 1);
    out->producer = nd;
    nd->out = out;
    handle_set(out_h, out);
    ver_unref(out);
    if (c->mode == GRB_BLOCKING && !c->dry) return materialize(c, out);
    return GRB_SUCCESS;
}

grb_info vector_fill_now(VectorH* v, double value) {
    Version* nv = new_version(v->ctx, false, v->type, v->n);
    nv->fmt = Fmt::ISO;
    nv->iso = round_host(v->type, value);
    nv->ready = true;
    handle_set(v, nv);
    ver_unref(nv);
    return GRB_SUCCESS;
}

grb_info scalar_set_now(ScalarH* s, double value) {
    Version* nv = new_version(s->ctx, true, s->type, 1);
    nv->host_known = true;
    nv->hval = round_host(s->type, value);
    nv->ready = true;
    handle_set(s, nv);
    ver_unref(nv);
    return GRB_SUCCESS;
}

grb_info scalar_value(Ctx* c, Version* v, double* out) {
    grb_info st = finish_read(c, v);
    if (st) return st;
    if (v->host_known) {
        *out = v->hval;
        return GRB_SUCCESS;
    }
    if (!v->slot.p) return GRB_NO_VALUE;
    st = cuda_check(c, cudaMemcpyAsync(out, v->slot.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "scalar read");
    if (st) return st;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "scalar read");
}

grb_info replay_stmt(Ctx* c, const Stmt& st) {
    switch (st.kind) {
        case Stmt::VCOPY:
            handle_set(st.dstv, st.srcv->cur);
            return GRB_SUCCESS;
        case Stmt::VFILL: return vector_fill_now(st.dstv, st.value);
        case Stmt::SSET: return scalar_set_now(st.dsts, st.value);
        case Stmt::WAIT:
            if (c->dry) return GRB_SUCCESS;
            if (st.dstv) return materialize(c, st.dstv->cur);
            if (st.dsts) return materialize(c, st.dsts->cur);
            return GRB_SUCCESS;
        case Stmt::OP: {
            Node* nd = new_node(c, st.tmpl.k);
            const uint64_t seq = nd->seq;
            *nd = st.tmpl;
            nd->seq = seq;
            nd->u = nd->v = nd->s = nd->mask = nd->w_old = nullptr;
            nd->A = nullptr;
            nd->out = nullptr;
            if (st.out_is_scalar) return submit_scalar_op(c, st.dsts, nd, st.hu, st.hs);
            return submit_vec_op(c, st.dstv, nd, st.hu, st.hv, st.hmask, st.hs, st.hA);
        }
    }
    return GRB_PANIC;
}

}  // namespace grb

extern "C" {

// ---------------------------------------------------------------- context
grb_info grb_context_new(grb_context* ctx, grb_mode mode, void* cuda_stream, grb_alloc_fn alloc, grb_free_fn free_fn,
                         void* alloc_ctx) {
    if (!ctx) return GRB_NULL_POINTER;
    *ctx = nullptr;
    if (mode != GRB_BLOCKING && mode != GRB_NONBLOCKING) return GRB_INVALID_VALUE;
    if ((alloc == nullptr) != (free_fn == nullptr)) return GRB_INVALID_VALUE;
    int dev = 0, sms = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return GRB_DEVICE_ERROR;
    }
    Ctx* c = new Ctx();
    c->mode = mode;
    c->stream = (cudaStream_t)cuda_stream;
    c->alloc = alloc;
    c->freefn = free_fn;
    c->actx = alloc_ctx;
    c->device = dev;
    c->sm_count = sms;
    c->l2_bytes = (size_t)l2;
    const char* f = std::getenv("GRB_FUSION");
    if (f && f[0] == '0') c->fusion = false;
    c->status = buf_alloc(c, STATUS_BYTES);
    c->sync = buf_alloc(c, sizeof(SyncWords));
    if (!c->status.p || !c->sync.p || cudaMemsetAsync(c->status.p, 0, STATUS_BYTES, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->sync.p, 0, sizeof(SyncWords), c->stream) != cudaSuccess) {
        cudaGetLastError();
        buf_free(c, c->status);
        buf_free(c, c->sync);
        delete c;
        return GRB_DEVICE_ERROR;
    }
    *ctx = reinterpret_cast<grb_context>(c);
    return GRB_SUCCESS;
}

grb_info grb_context_set(grb_context ctx, grb_option opt, int64_t value) {
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    switch (opt) {
        case GRB_OPT_FUSION: c->fusion = value != 0; return GRB_SUCCESS;
        case GRB_OPT_PERSISTENT:
            if (value < 0 || value > 3) return GRB_INVALID_VALUE;
            c->persistent = (int)value;
            return GRB_SUCCESS;
        case GRB_OPT_SPIN_LIMIT:
            if (value <= 0) return GRB_INVALID_VALUE;
            c->spin_limit = value;
            return GRB_SUCCESS;
        case GRB_OPT_MIXED_SWITCH:
            if (value <= 0) return GRB_INVALID_VALUE;
            c->mixed_switch = (double)value * 1e-9;
            return GRB_SUCCESS;
        case GRB_OPT_MIXED:
            if (value < 0 || value > 2) return GRB_INVALID_VALUE;
            c->mixed = (int)value;
            return GRB_SUCCESS;
        case GRB_OPT_RELABEL: c->relabel = value != 0; return GRB_SUCCESS;
        case GRB_OPT_TMA_STAGES:
            if (value != 0 && value != 2 && value != 3) return GRB_INVALID_VALUE;
            c->tma_stages = (int32_t)value;
            return GRB_SUCCESS;
        case GRB_OPT_ROW_BINS:
            if (value != 0 && value != 1) return GRB_INVALID_VALUE;
            c->row_bins = value != 0;
            return GRB_SUCCESS;
        case GRB_OPT_HOT_BYTES:
            if (value < 0 || value > GRB_HOT_BYTES_MAX) return GRB_INVALID_VALUE;
            c->hot_bytes = value;
            return GRB_SUCCESS;
    }
    return GRB_INVALID_VALUE;
}

grb_info grb_context_stats(grb_context ctx, grb_stats* out) {
    Ctx* c = as_ctx(ctx);
    if (!c || !out) return GRB_NULL_POINTER;
    c->stats.last_loop_kernel_ns = last_loop_kernel_ns(c);
    *out = c->stats;
    out->device_bytes = (int64_t)c->pool.held;
    return GRB_SUCCESS;
}

grb_info grb_context_loop_times(grb_context ctx, double* ms, int64_t cap, int64_t* n) {
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    if (!n || (cap > 0 && !ms) || cap < 0) return GRB_NULL_POINTER;
    const int64_t have = std::min<int64_t>(c->loop_count, Ctx::LOOP_TIMES);
    const int64_t k = std::min<int64_t>(have, cap);
    for (int64_t q = 0; q < k; ++q) {
        cudaEvent_t* ev = c->loop_ev[(c->loop_count - k + q) % Ctx::LOOP_TIMES];
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        if (e != cudaSuccess) return cuda_check(c, e, "loop times");
        ms[q] = (double)t;
    }
    *n = k;
    return GRB_SUCCESS;
}

grb_info grb_context_wait(grb_context ctx) {
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    grb_info st = run_pending_all(c);
    grb_info s2 = read_status(c);
    return st ? st : s2;
}

// ----------------------------------------------------------------- matrix
grb_info grb_matrix_build_csr(grb_matrix* Aout, grb_context ctx, grb_type type, uint64_t nrows, uint64_t ncols,
                              const int32_t* src, const int32_t* dst, const void* vals, uint64_t nedges,
                              uint32_t flags) {
    NvtxRange range("grb: CSR build");
    if (!Aout) return GRB_NULL_POINTER;
    *Aout = nullptr;
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    if (!valid_type(type)) return GRB_INVALID_VALUE;
    if (nrows == 0 || ncols == 0 || nrows >= (1ull << 31) || ncols >= (1ull << 31) || nedges >= (1ull << 31))
        return GRB_INVALID_VALUE;
    if (flags & ~15u) return GRB_INVALID_VALUE;
    if (nedges > 0 && (!src || !dst)) return GRB_NULL_POINTER;
    const bool on_dev = flags & GRB_BUILD_DEVICE_PTRS;
    const size_t esz = type_size(type);
    DevBuf ds, dd, dv;
    grb_info st = GRB_SUCCESS;
    const int32_t* dsrc = src;
    const int32_t* ddst = dst;
    const void* dvals = vals;
    if (!on_dev && nedges > 0) {
        ds = buf_alloc(c, sizeof(int32_t) * nedges);
        dd = buf_alloc(c, sizeof(int32_t) * nedges);
        if (vals) dv = buf_alloc(c, esz * nedges);
        if (!ds.p || !dd.p || (vals && !dv.p)) st = GRB_OUT_OF_MEMORY;
        if (!st) st = cuda_check(c, cudaMemcpyAsync(ds.p, src, sizeof(int32_t) * nedges, cudaMemcpyHostToDevice, c->stream), "copy src");
        if (!st) st = cuda_check(c, cudaMemcpyAsync(dd.p, dst, sizeof(int32_t) * nedges, cudaMemcpyHostToDevice, c->stream), "copy dst");
        if (!st && vals) st = cuda_check(c, cudaMemcpyAsync(dv.p, vals, esz * nedges, cudaMemcpyHostToDevice, c->stream), "copy vals");
        dsrc = (const int32_t*)ds.p;
        ddst = (const int32_t*)dd.p;
        dvals = dv.p;
    }
    Matrix* A = nullptr;
    if (!st) {
        CsrBuildArgs a;
        a.nrows = (int64_t)nrows;
        a.ncols = (int64_t)ncols;
        a.nedges = (int64_t)nedges;
        a.src = dsrc;
        a.dst = ddst;
        a.vals = vals ? dvals : nullptr;
        a.val_type = type;
        a.transpose = (flags & GRB_BUILD_TRANSPOSE) ? 1 : 0;
        a.drop_self = (flags & GRB_BUILD_DROP_SELF) ? 1 : 0;
        a.dedup = (flags & GRB_BUILD_DEDUP) ? 1 : 0;
        int32_t *rp = nullptr, *ci = nullptr;
        void* vv = nullptr;
        int64_t nnz = 0;
        int32_t bad = 0;
        st = cuda_check(c, csr_build(c->stream, a, pool_alloc_cb, pool_free_cb, c, &rp, &ci, &vv, &nnz, &bad), "csr build");
        c->stats.kernel_launches += 6;
        if (!st && bad != 0x7fffffff) st = GRB_INDEX_OUT_OF_BOUNDS;
        if (!st) {
            A = new Matrix();
            A->ctx = c;
            A->type = type;
            A->nrows = (int64_t)nrows;
            A->ncols = (int64_t)ncols;
            A->nnz = nnz;
            A->row_ptr.p = rp;
            A->row_ptr.bytes = sizeof(int32_t) * (nrows + 1);
            A->col_idx.p = ci;
            A->col_idx.bytes = sizeof(int32_t) * (size_t)padded_nnz(nnz);
            A->vals.p = vv;
            A->vals.bytes = vv ? esz * (size_t)(nnz > 0 ? nnz : 1) : 0;
            DevBuf cnt = buf_alloc(c, sizeof(unsigned long long));
            unsigned long long ne = 0;
            st = cnt.p ? GRB_SUCCESS : GRB_OUT_OF_MEMORY;
            if (!st) st = cuda_check(c, launch_nonempty_rows(c->stream, A->nrows, rp, (unsigned long long*)cnt.p), "rows");
            if (!st) st = cuda_check(c, cudaMemcpyAsync(&ne, cnt.p, sizeof(ne), cudaMemcpyDeviceToHost, c->stream), "rows");
            if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "rows");
            buf_free(c, cnt);
            A->nonempty_rows = (int64_t)ne;
        }
    }
    cudaStreamSynchronize(c->stream);
    buf_free(c, ds);
    buf_free(c, dd);
    buf_free(c, dv);
    if (st) {
        if (A) matrix_unref(A);
        return st;
    }
    *Aout = reinterpret_cast<grb_matrix>(A);
    return GRB_SUCCESS;
}

grb_info grb_matrix_nvals(uint64_t* nvals, grb_matrix Am) {
    Matrix* A = as_mat(Am);
    if (!nvals || !Am) return GRB_NULL_POINTER;
    if (!A) return GRB_UNINITIALIZED_OBJECT;
    *nvals = (uint64_t)A->nnz;
    return GRB_SUCCESS;
}

grb_info grb_matrix_nrows(uint64_t* n, grb_matrix Am) {
    Matrix* A = as_mat(Am);
    if (!n || !Am) return GRB_NULL_POINTER;
    if (!A) return GRB_UNINITIALIZED_OBJECT;
    *n = (uint64_t)A->nrows;
    return GRB_SUCCESS;
}

grb_info grb_matrix_export_csr(grb_matrix Am, int32_t* row_ptr, int32_t* col_idx, void* vals, int out_is_device) {
    Matrix* A = as_mat(Am);
    if (!Am || !row_ptr || !col_idx) return GRB_NULL_POINTER;
    if (!A) return GRB_UNINITIALIZED_OBJECT;
    Ctx* c = A->ctx;
    const cudaMemcpyKind k = out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    grb_info st = cuda_check(c, cudaMemcpyAsync(row_ptr, A->row_ptr.p, sizeof(int32_t) * (A->nrows + 1), k, c->stream), "export");
    if (!st && A->nnz > 0) st = cuda_check(c, cudaMemcpyAsync(col_idx, A->col_idx.p, sizeof(int32_t) * A->nnz, k, c->stream), "export");
    if (!st && vals && A->vals.p && A->nnz > 0)
        st = cuda_check(c, cudaMemcpyAsync(vals, A->vals.p, type_size(A->type) * A->nnz, k, c->stream), "export");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "export");
    return st;
}

grb_info grb_matrix_col_degree(grb_vector deg, grb_matrix Am) {
    VectorH* d = as_vec(deg);
    Matrix* A = as_mat(Am);
    if (!deg || !Am) return GRB_NULL_POINTER;
    if (!d || !A) return GRB_UNINITIALIZED_OBJECT;
    if (d->type != GRB_INT32) return GRB_DOMAIN_MISMATCH;
    if (d->n != A->ncols) return GRB_DIMENSION_MISMATCH;
    Ctx* c = d->ctx;
    if (A->ctx != c) return GRB_INVALID_VALUE;   // the counts are cached on the matrix, in its context
    if (c->recording) return GRB_INVALID_VALUE;
    Version* v = new_version(c, false, GRB_INT32, d->n);
    v->vals = buf_alloc(c, sizeof(int32_t) * d->n);
    v->present = buf_alloc(c, (size_t)d->n);
    grb_info st = (v->vals.p && v->present.p) ? GRB_SUCCESS : GRB_OUT_OF_MEMORY;
    // the column counts are computed once per matrix (the degree order of
    // the device loops reuses them)
    if (!st) st = ensure_coldeg(c, A);
    if (!st)
        st = cuda_check(c, cudaMemcpyAsync(v->vals.p, A->coldeg.p, sizeof(int32_t) * (size_t)A->ncols,
                                           cudaMemcpyDeviceToDevice, c->stream), "col degree");
    if (!st)
        st = cuda_check(c, launch_deg_present(c->stream, A->ncols, (const int32_t*)A->coldeg.p,
                                              (uint8_t*)v->present.p), "col degree");
    c->stats.kernel_launches++;
    v->fmt = Fmt::BITMAP;
    v->ready = true;
    if (st) {
        ver_unref(v);
        return st;
    }
    handle_set(d, v);
    ver_unref(v);
    return GRB_SUCCESS;
}

// ----------------------------------------------------------------- vector
grb_info grb_vector_new(grb_vector* v, grb_context ctx, grb_type type, uint64_t n) {
    if (!v) return GRB_NULL_POINTER;
    *v = nullptr;
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    if (!valid_type(type)) return GRB_INVALID_VALUE;
    if (n == 0 || n >= (1ull << 31)) return GRB_INVALID_VALUE;
    VectorH* h = new VectorH();
    h->ctx = c;
    h->type = type;
    h->n = (int64_t)n;
    Version* e = new_version(c, false, type, (int64_t)n);
    e->ready = true;
    handle_set(h, e);
    ver_unref(e);
    c->vhandles.push_back(h);
    *v = reinterpret_cast<grb_vector>(h);
    return GRB_SUCCESS;
}

grb_info grb_vector_fill(grb_vector vh, double value) {
    VectorH* v = as_vec(vh);
    if (!vh) return GRB_NULL_POINTER;
    if (!v) return GRB_UNINITIALIZED_OBJECT;
    if (v->ctx->recording) {
        Stmt st;
        st.kind = Stmt::VFILL;
        st.dstv = v;
        st.value = value;
        v->ctx->body.push_back(st);
        return GRB_SUCCESS;
    }
    return vector_fill_now(v, value);
}

grb_info grb_vector_build(grb_vector vh, const int32_t* idx, const double* vals, uint64_t nvals, int ptrs_on_device) {
    VectorH* v = as_vec(vh);
    if (!vh) return GRB_NULL_POINTER;
    if (!v) return GRB_UNINITIALIZED_OBJECT;
    if (nvals > 0 && (!idx || !vals)) return GRB_NULL_POINTER;
    if ((int64_t)nvals > v->n) return GRB_INVALID_VALUE;
    Ctx* c = v->ctx;
    if (c->recording) return GRB_INVALID_VALUE;
    if (!ptrs_on_device) {
        for (uint64_t k = 0; k < nvals; ++k)
            if (idx[k] < 0 || idx[k] >= v->n || (k > 0 && idx[k - 1] >= idx[k])) return GRB_INVALID_INDEX;
    }
    const bool full = !ptrs_on_device && (int64_t)nvals == v->n;
    Version* nv = new_version(c, false, v->type, v->n);
    grb_info st = GRB_SUCCESS;
    nv->vals = buf_alloc(c, type_size(v->type) * v->n);
    if (!full) nv->present = buf_alloc(c, (size_t)v->n);
    if (!nv->vals.p || (!full && !nv->present.p)) st = GRB_OUT_OF_MEMORY;
    DevBuf di, dvv, tmp_present;
    if (!st) {
        if (!full) st = cuda_check(c, cudaMemsetAsync(nv->present.p, 0, (size_t)v->n, c->stream), "build");
        if (!st) st = cuda_check(c, cudaMemsetAsync(nv->vals.p, 0, type_size(v->type) * v->n, c->stream), "build");
        const int32_t* i_d = idx;
        const double* v_d = vals;
        if (!st && !ptrs_on_device && nvals > 0) {
            di = buf_alloc(c, sizeof(int32_t) * nvals);
            dvv = buf_alloc(c, sizeof(double) * nvals);
            if (!di.p || !dvv.p) st = GRB_OUT_OF_MEMORY;
            if (!st) st = cuda_check(c, cudaMemcpyAsync(di.p, idx, sizeof(int32_t) * nvals, cudaMemcpyHostToDevice, c->stream), "build");
            if (!st) st = cuda_check(c, cudaMemcpyAsync(dvv.p, vals, sizeof(double) * nvals, cudaMemcpyHostToDevice, c->stream), "build");
            i_d = (const int32_t*)di.p;
            v_d = (const double*)dvv.p;
        }
        uint8_t* pres = (uint8_t*)nv->present.p;
        if (!st && full) {
            tmp_present = buf_alloc(c, (size_t)v->n);
            pres = (uint8_t*)tmp_present.p;
            if (!pres) st = GRB_OUT_OF_MEMORY;
        }
        if (!st && nvals > 0) {
            st = cuda_check(c, launch_build_sparse(c->stream, v->n, i_d, v_d, (int64_t)nvals, v->type, nv->vals.p, pres,
                                                   (int32_t*)c->status.p), "build");
            c->stats.kernel_launches++;
        }
        if (!st) st = read_status(c);
    }
    buf_free(c, di);
    buf_free(c, dvv);
    buf_free(c, tmp_present);
    if (st) {
        ver_unref(nv);
        return st == GRB_INVALID_INDEX ? GRB_INVALID_INDEX : st;
    }
    nv->fmt = full ? Fmt::FULL : (nvals == 0 ? Fmt::EMPTY : Fmt::BITMAP);
    if (nvals == 0) {
        buf_free(c, nv->vals);
        buf_free(c, nv->present);
    }
    nv->ready = true;
    handle_set(v, nv);
    ver_unref(nv);
    return GRB_SUCCESS;
}

grb_info grb_vector_copy(grb_vector dsth, grb_vector srch) {
    VectorH* d = as_vec(dsth);
    VectorH* s = as_vec(srch);
    if (!dsth || !srch) return GRB_NULL_POINTER;
    if (!d || !s) return GRB_UNINITIALIZED_OBJECT;
    if (d->type != s->type) return GRB_DOMAIN_MISMATCH;
    if (d->n != s->n) return GRB_DIMENSION_MISMATCH;
    if (d->ctx->recording) {
        Stmt st;
        st.kind = Stmt::VCOPY;
        st.dstv = d;
        st.srcv = s;
        d->ctx->body.push_back(st);
        return GRB_SUCCESS;
    }
    handle_set(d, s->cur);
    return GRB_SUCCESS;
}

grb_info grb_vector_size(uint64_t* n, grb_vector vh) {
    VectorH* v = as_vec(vh);
    if (!n || !vh) return GRB_NULL_POINTER;
    if (!v) return GRB_UNINITIALIZED_OBJECT;
    *n = (uint64_t)v->n;
    return GRB_SUCCESS;
}

grb_info grb_vector_nvals(uint64_t* nvals, grb_vector vh) {
    VectorH* v = as_vec(vh);
    if (!nvals || !vh) return GRB_NULL_POINTER;
    if (!v) return GRB_UNINITIALIZED_OBJECT;
    Ctx* c = v->ctx;
    if (c->recording) return GRB_INVALID_VALUE;
    Version* cur = v->cur;
    ver_ref(cur);
    grb_info st = finish_read(c, cur);
    if (!st) {
        if (cur->fmt == Fmt::EMPTY) *nvals = 0;
        else if (cur->fmt != Fmt::BITMAP) *nvals = (uint64_t)cur->n;
        else {
            DevBuf cnt = buf_alloc(c, sizeof(unsigned long long));
            unsigned long long h = 0;
            st = cnt.p ? GRB_SUCCESS : GRB_OUT_OF_MEMORY;
            if (!st) st = cuda_check(c, launch_count_present(c->stream, cur->n, (const uint8_t*)cur->present.p, (unsigned long long*)cnt.p), "nvals");
            if (!st) st = cuda_check(c, cudaMemcpyAsync(&h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "nvals");
            if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "nvals");
            buf_free(c, cnt);
            *nvals = h;
        }
    }
    ver_unref(cur);
    return st;
}

grb_info grb_vector_extract_dense(grb_vector vh, void* values, uint8_t* present, int out_is_device) {
    VectorH* v = as_vec(vh);
    if (!vh || !values) return GRB_NULL_POINTER;
    if (!v) return GRB_UNINITIALIZED_OBJECT;
    Ctx* c = v->ctx;
    if (c->recording) return GRB_INVALID_VALUE;
    Version* cur = v->cur;
    ver_ref(cur);
    grb_info st = finish_read(c, cur);
    if (!st) {
        const size_t vb = type_size(cur->type) * cur->n;
        DevBuf tv, tp;
        void* dv = values;
        uint8_t* dp = present;
        if (!out_is_device) {
            tv = buf_alloc(c, vb);
            if (present) tp = buf_alloc(c, (size_t)cur->n);
            dv = tv.p;
            dp = (uint8_t*)tp.p;
            if (!tv.p || (present && !tp.p)) st = GRB_OUT_OF_MEMORY;
        }
        if (!st) {
            if (cur->fmt == Fmt::EMPTY) {
                st = cuda_check(c, cudaMemsetAsync(dv, 0, vb, c->stream), "extract");
                if (!st && dp) st = cuda_check(c, cudaMemsetAsync(dp, 0, (size_t)cur->n, c->stream), "extract");
            } else {
                st = cuda_check(c, launch_to_dense(c->stream, cur->n, vin_of(cur), dv, dp), "extract");
                c->stats.kernel_launches++;
            }
        }
        if (!st && !out_is_device) {
            st = cuda_check(c, cudaMemcpyAsync(values, dv, vb, cudaMemcpyDeviceToHost, c->stream), "extract");
            if (!st && present) st = cuda_check(c, cudaMemcpyAsync(present, dp, (size_t)cur->n, cudaMemcpyDeviceToHost, c->stream), "extract");
        }
        if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "extract");
        buf_free(c, tv);
        buf_free(c, tp);
    }
    ver_unref(cur);
    return st;
}

// ----------------------------------------------------------------- scalar
grb_info grb_scalar_new(grb_scalar* s, grb_context ctx, grb_type type) {
    if (!s) return GRB_NULL_POINTER;
    *s = nullptr;
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    if (!valid_type(type)) return GRB_INVALID_VALUE;
    ScalarH* h = new ScalarH();
    h->ctx = c;
    h->type = type;
    Version* e = new_version(c, true, type, 1);
    e->ready = true;
    handle_set(h, e);
    ver_unref(e);
    c->shandles.push_back(h);
    *s = reinterpret_cast<grb_scalar>(h);
    return GRB_SUCCESS;
}

grb_info grb_scalar_set(grb_scalar sh, double value) {
    ScalarH* s = as_sca(sh);
    if (!sh) return GRB_NULL_POINTER;
    if (!s) return GRB_UNINITIALIZED_OBJECT;
    if (s->ctx->recording) {
        Stmt st;
        st.kind = Stmt::SSET;
        st.dsts = s;
        st.value = value;
        s->ctx->body.push_back(st);
        return GRB_SUCCESS;
    }
    return scalar_set_now(s, value);
}

grb_info grb_scalar_get(grb_scalar sh, double* value) {
    ScalarH* s = as_sca(sh);
    if (!sh || !value) return GRB_NULL_POINTER;
    if (!s) return GRB_UNINITIALIZED_OBJECT;
    Ctx* c = s->ctx;
    if (c->recording) return GRB_INVALID_VALUE;
    Version* cur = s->cur;
    ver_ref(cur);
    grb_info st = scalar_value(c, cur, value);
    ver_unref(cur);
    return st;
}

grb_info grb_scalar_apply_bind2nd(grb_scalar outh, grb_binop op, grb_scalar inh, double k) {
    ScalarH* o = as_sca(outh);
    ScalarH* i = as_sca(inh);
    if (!outh || !inh) return GRB_NULL_POINTER;
    if (!o || !i) return GRB_UNINITIALIZED_OBJECT;
    if (!valid_binop(op)) return GRB_INVALID_VALUE;
    Node* nd = new_node(o->ctx, OpK::SAPPLY_B2);
    nd->op = op;
    nd->cst = k;
    return submit_scalar_op(o->ctx, o, nd, nullptr, i);
}

// ---------------------------------------------------------------- methods
static grb_info vec_method(OpK kind, grb_vector wh, grb_vector mask, const grb_binop* accum, const grb_binop* op,
                           int unop, grb_vector uh, grb_vector vh, grb_scalar sh, double k, grb_desc desc,
                           grb_matrix Ah = nullptr, grb_semiring sr = GRB_PLUS_TIMES) {
    VectorH* w = as_vec(wh);
    if (!wh) return GRB_NULL_POINTER;
    if (!w) return GRB_UNINITIALIZED_OBJECT;
    Ctx* c = w->ctx;
    VectorH* m = nullptr;
    grb_info st = check_write(w, mask, accum, desc, &m);
    if (st) return st;
    VectorH* u = nullptr;
    VectorH* v = nullptr;
    ScalarH* s = nullptr;
    Matrix* A = nullptr;
    if (kind != OpK::ASSIGN_S) {
        if (!uh) return GRB_NULL_POINTER;
        u = as_vec(uh);
        if (!u) return GRB_UNINITIALIZED_OBJECT;
        if (u->ctx != c) return GRB_INVALID_VALUE;
    }
    if (kind == OpK::EADD || kind == OpK::EMULT) {
        if (!vh) return GRB_NULL_POINTER;
        v = as_vec(vh);
        if (!v) return GRB_UNINITIALIZED_OBJECT;
        if (v->ctx != c) return GRB_INVALID_VALUE;
        if (v->n != w->n || u->n != w->n) return GRB_DIMENSION_MISMATCH;
    }
    if (kind == OpK::APPLY || kind == OpK::APPLY_B2 || kind == OpK::APPLY_B2S) {
        if (u->n != w->n) return GRB_DIMENSION_MISMATCH;
    }
    if (kind == OpK::APPLY_B2S || kind == OpK::ASSIGN_S) {
        if (!sh) return GRB_NULL_POINTER;
        s = as_sca(sh);
        if (!s) return GRB_UNINITIALIZED_OBJECT;
    }
    if (kind == OpK::MXV) {
        if (!Ah) return GRB_NULL_POINTER;
        A = as_mat(Ah);
        if (!A) return GRB_UNINITIALIZED_OBJECT;
        if (A->nrows != w->n || A->ncols != u->n) return GRB_DIMENSION_MISMATCH;
        if (sr < GRB_PLUS_TIMES || sr > GRB_MAX_SECOND) return GRB_INVALID_VALUE;
    }
    if (op && !valid_binop(*op)) return GRB_INVALID_VALUE;
    if (kind == OpK::APPLY && (unop < GRB_IDENTITY || unop > GRB_MINV)) return GRB_INVALID_VALUE;
    Node* nd = new_node(c, kind);
    if (op) nd->op = *op;
    nd->unop = unop;
    nd->cst = k;
    nd->sr = sr;
    fill_write(nd, accum, desc);
    return submit_vec_op(c, w, nd, u, v, m, s, A);
}

grb_info grb_apply(grb_vector w, grb_vector mask, const grb_binop* accum, grb_unop op, grb_vector u, grb_desc desc) {
    return vec_method(OpK::APPLY, w, mask, accum, nullptr, op, u, nullptr, nullptr, 0.0, desc);
}

grb_info grb_apply_bind2nd(grb_vector w, grb_vector mask, const grb_binop* accum, grb_binop op, grb_vector u, double s,
                           grb_desc desc) {
    return vec_method(OpK::APPLY_B2, w, mask, accum, &op, 0, u, nullptr, nullptr, s, desc);
}

grb_info grb_apply_bind2nd_scalar(grb_vector w, grb_vector mask, const grb_binop* accum, grb_binop op, grb_vector u,
                                  grb_scalar s, grb_desc desc) {
    return vec_method(OpK::APPLY_B2S, w, mask, accum, &op, 0, u, nullptr, s, 0.0, desc);
}

grb_info grb_assign_scalar(grb_vector w, grb_vector mask, const grb_binop* accum, grb_scalar s, grb_desc desc) {
    return vec_method(OpK::ASSIGN_S, w, mask, accum, nullptr, 0, nullptr, nullptr, s, 0.0, desc);
}

grb_info grb_mxv(grb_vector w, grb_vector mask, const grb_binop* accum, grb_semiring s, grb_matrix A, grb_vector u,
                 grb_desc desc) {
    return vec_method(OpK::MXV, w, mask, accum, nullptr, 0, u, nullptr, nullptr, 0.0, desc, A, s);
}

grb_info grb_ewise_add(grb_vector w, grb_vector mask, const grb_binop* accum, grb_binop op, grb_vector u, grb_vector v,
                       grb_desc desc) {
    return vec_method(OpK::EADD, w, mask, accum, &op, 0, u, v, nullptr, 0.0, desc);
}

grb_info grb_ewise_mult(grb_vector w, grb_vector mask, const grb_binop* accum, grb_binop op, grb_vector u, grb_vector v,
                        grb_desc desc) {
    return vec_method(OpK::EMULT, w, mask, accum, &op, 0, u, v, nullptr, 0.0, desc);
}

grb_info grb_reduce(grb_scalar sh, const grb_binop* accum, grb_monoid m, grb_vector uh, grb_desc desc) {
    ScalarH* s = as_sca(sh);
    VectorH* u = as_vec(uh);
    if (!sh || !uh) return GRB_NULL_POINTER;
    if (!s || !u) return GRB_UNINITIALIZED_OBJECT;
    if (!valid_monoid(m) || !valid_desc(desc)) return GRB_INVALID_VALUE;
    if (accum && !valid_binop(*accum)) return GRB_INVALID_VALUE;
    Node* nd = new_node(s->ctx, OpK::REDUCE);
    nd->mon = m;
    if (accum) {
        nd->has_accum = true;
        nd->accum = *accum;
    }
    return submit_scalar_op(s->ctx, s, nd, u, nullptr);
}

// ------------------------------------------------------- materialisation
grb_info grb_wait(void* obj, grb_wait_mode mode) {
    if (!obj) return GRB_NULL_POINTER;
    if (mode != GRB_WAIT_COMPLETE && mode != GRB_WAIT_MATERIALIZE) return GRB_INVALID_VALUE;
    const Kind k = *reinterpret_cast<Kind*>(obj);
    if (k == Kind::CONTEXT) return grb_context_wait(reinterpret_cast<grb_context>(obj));
    if (k == Kind::MATRIX) return GRB_SUCCESS;
    if (k == Kind::VECTOR) {
        VectorH* v = reinterpret_cast<VectorH*>(obj);
        Ctx* c = v->ctx;
        if (c->recording) {
            Stmt st;
            st.kind = Stmt::WAIT;
            st.dstv = v;
            c->body.push_back(st);
            return GRB_SUCCESS;
        }
        Version* cur = v->cur;
        ver_ref(cur);
        grb_info st = finish_read(c, cur);
        ver_unref(cur);
        return st;
    }
    if (k == Kind::SCALAR) {
        ScalarH* s = reinterpret_cast<ScalarH*>(obj);
        Ctx* c = s->ctx;
        if (c->recording) {
            Stmt st;
            st.kind = Stmt::WAIT;
            st.dsts = s;
            c->body.push_back(st);
            return GRB_SUCCESS;
        }
        Version* cur = s->cur;
        ver_ref(cur);
        grb_info st = finish_read(c, cur);
        ver_unref(cur);
        return st;
    }
    return GRB_UNINITIALIZED_OBJECT;
}

grb_info grb_iterate_begin(grb_context ctx) {
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    if (c->recording) return GRB_INVALID_VALUE;
    c->recording = true;
    c->body.clear();
    return GRB_SUCCESS;
}

grb_info grb_iterate_end(grb_context ctx, grb_scalar cond, double tol, int64_t itermax, int64_t* iters) {
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    ScalarH* s = as_sca(cond);
    if (!cond || !iters) {
        c->recording = false;
        c->body.clear();
        return GRB_NULL_POINTER;
    }
    if (!c->recording) return GRB_INVALID_VALUE;
    if (!s || itermax < 0) {
        c->recording = false;
        c->body.clear();
        return s ? GRB_INVALID_VALUE : GRB_UNINITIALIZED_OBJECT;
    }
    return iterate_end(c, s, tol, itermax, iters);
}

// -------------------------------------------------------------------- misc
grb_info grb_free(void** obj) {
    if (!obj) return GRB_NULL_POINTER;
    if (!*obj) return GRB_SUCCESS;
    const Kind k = *reinterpret_cast<Kind*>(*obj);
    if (k == Kind::VECTOR) {
        VectorH* v = reinterpret_cast<VectorH*>(*obj);
        Ctx* c = v->ctx;
        c->vhandles.erase(std::remove(c->vhandles.begin(), c->vhandles.end(), v), c->vhandles.end());
        Version* cur = v->cur;
        v->cur = nullptr;
        cur->handle_refs--;
        ver_unref(cur);
        v->kind = Kind::DEAD;
        delete v;
    } else if (k == Kind::SCALAR) {
        ScalarH* s = reinterpret_cast<ScalarH*>(*obj);
        Ctx* c = s->ctx;
        c->shandles.erase(std::remove(c->shandles.begin(), c->shandles.end(), s), c->shandles.end());
        Version* cur = s->cur;
        s->cur = nullptr;
        cur->handle_refs--;
        ver_unref(cur);
        s->kind = Kind::DEAD;
        delete s;
    } else if (k == Kind::MATRIX) {
        Matrix* A = reinterpret_cast<Matrix*>(*obj);
        A->handle_alive = false;
        matrix_unref(A);
    } else if (k == Kind::PPR) {
        ppr_destroy(reinterpret_cast<Ppr*>(*obj));
    } else if (k == Kind::PRBATCH) {
        prbatch_destroy(reinterpret_cast<PrBatch*>(*obj));
    } else if (k == Kind::CONTEXT) {
        Ctx* c = reinterpret_cast<Ctx*>(*obj);
        cudaStreamSynchronize(c->stream);
        buf_free(c, c->status);
        buf_free(c, c->sync);
        buf_free(c, c->red_scratch);
        buf_free(c, c->red_counter);
        pool_release_all(c);
        cudaStreamSynchronize(c->stream);
        if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
        loop_resources_free(c);
        c->kind = Kind::DEAD;
        delete c;
    } else {
        return GRB_UNINITIALIZED_OBJECT;
    }
    *obj = nullptr;
    return GRB_SUCCESS;
}

const char* grb_error(void* obj) {
    if (!obj) return "";
    const Kind k = *reinterpret_cast<Kind*>(obj);
    if (k == Kind::CONTEXT) return reinterpret_cast<Ctx*>(obj)->err.c_str();
    if (k == Kind::VECTOR) {
        VectorH* v = reinterpret_cast<VectorH*>(obj);
        return v->cur && v->cur->err ? v->cur->errmsg.c_str() : v->err.c_str();
    }
    if (k == Kind::SCALAR) {
        ScalarH* s = reinterpret_cast<ScalarH*>(obj);
        return s->cur && s->cur->err ? s->cur->errmsg.c_str() : s->err.c_str();
    }
    if (k == Kind::MATRIX) return reinterpret_cast<Matrix*>(obj)->err.c_str();
    return "";
}

grb_info grb_iterate_history(grb_context ctx, double* hist, double* dang, int64_t cap, int64_t* n,
                             int32_t* mixed_phase) {
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    if (!n) return GRB_NULL_POINTER;
    grb_info st = resolve_loop_history(c);
    if (st) return st;
    *n = (int64_t)c->last_hist.size();
    if (hist)
        for (int64_t k = 0; k < *n && k < cap; ++k) hist[k] = c->last_hist[(size_t)k];
    if (dang)
        for (int64_t k = 0; k < *n && k < cap; ++k)
            dang[k] = k < (int64_t)c->last_dang.size() ? c->last_dang[(size_t)k] : __builtin_nan("");
    if (mixed_phase) *mixed_phase = c->last_mixed_phase;
    return GRB_SUCCESS;
}

grb_info grb_selftest_wait_timeout(grb_context ctx, int64_t spin_limit) {
    Ctx* c = as_ctx(ctx);
    if (!c) return ctx ? GRB_UNINITIALIZED_OBJECT : GRB_NULL_POINTER;
    if (spin_limit <= 0 || spin_limit > (int64_t(1) << 24)) return GRB_INVALID_VALUE;
    DevBuf sync = buf_alloc(c, sizeof(SyncWords));
    if (!sync.p) return GRB_OUT_OF_MEMORY;
    grb_info st = cuda_check(c, cudaMemsetAsync(sync.p, 0, sizeof(SyncWords), c->stream), "selftest");
    const int grid = c->sm_count < 4 ? c->sm_count : 4;
    if (!st) st = cuda_check(c, launch_barrier_selftest(c->stream, (SyncWords*)sync.p, (int32_t*)c->status.p, spin_limit, grid), "selftest");
    c->stats.kernel_launches++;
    if (!st) st = read_status(c);
    buf_free(c, sync);
    return st;
}

#ifdef GRB_CHECK_BOUNDS
grb_info grb_debug_check_csr(grb_context ctx, const int32_t* row_ptr, const int32_t* col_idx, uint64_t nrows,
                             uint64_t ncols, uint64_t nnz, int32_t* what, int64_t* value) {
    Ctx* c = as_ctx(ctx);
    if (!ctx || !row_ptr || !what || !value || (nnz > 0 && !col_idx)) return GRB_NULL_POINTER;
    if (!c) return GRB_UNINITIALIZED_OBJECT;
    if (nrows > (uint64_t)INT32_MAX || ncols > (uint64_t)INT32_MAX || nnz > (uint64_t)INT32_MAX)
        return GRB_INVALID_VALUE;
    *what = 0;
    *value = 0;
    grb_info st = read_status(c);   // nothing left over from earlier work
    if (st) return st;
    DevBuf rp = buf_alloc(c, sizeof(int32_t) * (size_t)(nrows + 1));
    DevBuf ci = buf_alloc(c, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!rp.p || !ci.p) st = GRB_OUT_OF_MEMORY;
    if (!st)
        st = cuda_check(c, cudaMemcpyAsync(rp.p, row_ptr, sizeof(int32_t) * (size_t)(nrows + 1),
                                           cudaMemcpyHostToDevice, c->stream), "check csr");
    if (!st && nnz > 0)
        st = cuda_check(c, cudaMemcpyAsync(ci.p, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice,
                                           c->stream), "check csr");
    if (!st) {
        c->stats.kernel_launches++;
        st = cuda_check(c, launch_csr_check(c->stream, (int64_t)nrows, (int64_t)ncols, (int64_t)nnz,
                                            (const int32_t*)rp.p, (const int32_t*)ci.p, (int32_t*)c->status.p),
                        "check csr");
    }
    int32_t w[4] = {0, 0, 0, 0};
    if (!st) st = cuda_check(c, cudaMemcpyAsync(w, c->status.p, STATUS_BYTES, cudaMemcpyDeviceToHost, c->stream),
                             "check csr");
    if (!st) st = cuda_check(c, cudaMemsetAsync(c->status.p, 0, STATUS_BYTES, c->stream), "check csr");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "check csr");
    buf_free(c, rp);
    buf_free(c, ci);
    if (st) return st;
    if (w[0] == 0) return GRB_SUCCESS;
    *what = w[1];
    long long v = 0;
    std::memcpy(&v, w + 2, sizeof(v));
    *value = (int64_t)v;
    return (grb_info)w[0];
}

grb_info grb_debug_set_col(grb_matrix A, uint64_t k, int32_t col) {
    Matrix* M = as_mat(A);
    if (!A) return GRB_NULL_POINTER;
    if (!M) return GRB_UNINITIALIZED_OBJECT;
    if (k >= (uint64_t)M->nnz) return GRB_INVALID_INDEX;
    Ctx* c = M->ctx;
    grb_info st = cuda_check(c, cudaStreamSynchronize(c->stream), "set col");
    if (!st)
        st = cuda_check(c, cudaMemcpyAsync((int32_t*)M->col_idx.p + k, &col, sizeof(int32_t), cudaMemcpyHostToDevice,
                                           c->stream), "set col");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "set col");
    return st;
}
#endif

}  // extern "C"
