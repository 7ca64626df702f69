// Memory pool, versions and DAG nodes.
#include <cstring>

#include "grb_core.h"

namespace grb {

// ------------------------------------------------------------------ memory
// Size classes: powers of two up to 1 MiB, then multiples of 2 MiB.  Freed
// blocks stay in a per-context free list and are reused on the context's
// stream (stream order makes the reuse safe); they go back to the allocator
// only when an allocation fails or the context is freed.
static size_t size_class(size_t b) {
    if (b < 256) b = 256;
    if (b <= (size_t(1) << 20)) {
        size_t c = 256;
        while (c < b) c <<= 1;
        return c;
    }
    const size_t two_mb = size_t(2) << 20;
    return (b + two_mb - 1) / two_mb * two_mb;
}

static void* raw_alloc(Ctx* c, size_t bytes) {
    void* p = nullptr;
    if (c->alloc) {
        p = c->alloc(c->actx, bytes, (void*)c->stream);
    } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

static void raw_free(Ctx* c, void* p) {
    if (c->freefn) c->freefn(c->actx, p, (void*)c->stream);
    else cudaFreeAsync(p, c->stream);
}

void* dev_alloc(Ctx* c, size_t bytes) {
    const size_t cls = size_class(bytes);
    auto it = c->pool.free_list.find(cls);
    if (it != c->pool.free_list.end()) {
        void* p = it->second;
        c->pool.free_list.erase(it);
        return p;
    }
    void* p = raw_alloc(c, cls);
    if (!p && !c->pool.free_list.empty()) {
        pool_release_all(c);
        p = raw_alloc(c, cls);
    }
    if (p) {
        c->pool.held += cls;
        c->stats.device_bytes = (int64_t)c->pool.held;
    }
    return p;
}

void dev_free(Ctx* c, void* p, size_t bytes) {
    if (!p) return;
    c->pool.free_list.emplace(size_class(bytes), p);
}

void pool_release_all(Ctx* c) {
    for (auto& kv : c->pool.free_list) {
        raw_free(c, kv.second);
        c->pool.held -= kv.first;
    }
    c->pool.free_list.clear();
    c->stats.device_bytes = (int64_t)c->pool.held;
}

DevBuf buf_alloc(Ctx* c, size_t bytes) {
    DevBuf b;
    b.p = dev_alloc(c, bytes);
    b.bytes = b.p ? bytes : 0;
    return b;
}

void buf_free(Ctx* c, DevBuf& b) {
    if (b.p) dev_free(c, b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
}

size_t type_size(grb_type t) {
    switch (t) {
        case GRB_INT32: return 4;
        case GRB_FP32: return 4;
        case GRB_FP64: return 8;
        case GRB_BF16: return 2;
    }
    return 8;
}

grb_info cuda_check(Ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GRB_SUCCESS;
    cudaGetLastError();
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? GRB_OUT_OF_MEMORY : GRB_DEVICE_ERROR;
}

// ---------------------------------------------------------------- versions
Version* new_version(Ctx* c, bool scalar, grb_type t, int64_t n) {
    Version* v = new Version();
    v->ctx = c;
    v->id = c->next_id++;
    v->refs = 1;
    v->scalar = scalar;
    v->type = t;
    v->n = n;
    return v;
}

void ver_ref(Version* v) {
    if (v) v->refs++;
}

void ver_free_data(Version* v) {
    Ctx* c = v->ctx;
    buf_free(c, v->vals);
    buf_free(c, v->present);
    buf_free(c, v->slot);
    buf_free(c, v->sinkbits);
    buf_free(c, v->perm_vals);
    buf_free(c, v->perm_sinkbits);
    if (v->iso_src) {
        Version* s = v->iso_src;
        v->iso_src = nullptr;
        ver_unref(s);
    }
}

void ver_unref(Version* v) {
    if (!v) return;
    if (--v->refs > 0) return;
    if (v->producer) {
        Node* nd = v->producer;
        v->producer = nullptr;
        node_destroy(nd);
    }
    ver_free_data(v);
    delete v;
}

void handle_set(VectorH* h, Version* v) {
    ver_ref(v);
    v->handle_refs++;
    Version* old = h->cur;
    h->cur = v;
    if (old) {
        old->handle_refs--;
        ver_unref(old);
    }
}

void handle_set(ScalarH* h, Version* v) {
    ver_ref(v);
    v->handle_refs++;
    Version* old = h->cur;
    h->cur = v;
    if (old) {
        old->handle_refs--;
        ver_unref(old);
    }
}

void matrix_unref(Matrix* A) {
    if (!A) return;
    if (--A->refs > 0) return;
    Ctx* c = A->ctx;
    buf_free(c, A->row_ptr);
    buf_free(c, A->col_idx);
    buf_free(c, A->vals);
    buf_free(c, A->coldeg);
    if (A->plan) {
        TilePlan* p = A->plan;
        buf_free(c, p->meta);
        buf_free(c, p->rowend_bits);
        buf_free(c, p->ne_rows);
        buf_free(c, p->empty_rows);
        buf_free(c, p->agg);
        buf_free(c, p->first);
        buf_free(c, p->fix);
        buf_free(c, p->longfix);
        buf_free(c, p->part);
        for (auto& b : p->loop_bufs) buf_free(c, b);
        buf_free(c, p->bin_rows);
        if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
        delete p;
    }
    if (A->rel) matrix_unref(A->rel);
    buf_free(c, A->new2old);
    buf_free(c, A->old2new);
    A->kind = Kind::DEAD;
    delete A;
}

// ------------------------------------------------------------------- nodes
Node* new_node(Ctx* c, OpK k) {
    Node* nd = new Node();
    nd->k = k;
    nd->seq = c->next_seq++;
    return nd;
}

static void attach(Version* v) {
    if (!v) return;
    ver_ref(v);
    v->node_refs++;
}

void node_attach_inputs(Node* nd) {
    attach(nd->u);
    attach(nd->v);
    attach(nd->s);
    attach(nd->mask);
    attach(nd->w_old);
    if (nd->A) nd->A->refs++;
}

static void detach(Version* v) {
    if (!v) return;
    v->node_refs--;
    ver_unref(v);
}

void node_destroy(Node* nd) {
    detach(nd->u);
    detach(nd->v);
    detach(nd->s);
    detach(nd->mask);
    detach(nd->w_old);
    matrix_unref(nd->A);
    delete nd;
}

// Operand descriptor of a materialised vector version.
VIn vin_of(const Version* v) {
    VIn in;
    in.type = v->type;
    in.fmt = (int32_t)v->fmt;
    in.vals = v->vals.p;
    in.present = (const uint8_t*)v->present.p;
    in.iso = v->iso;
    if (v->fmt == Fmt::ISO && v->iso_src) {
        const Version* s = v->iso_src;
        if (s->host_known) in.iso = s->hval;
        else in.iso_slot = (const double*)s->slot.p;
    }
    return in;
}

}  // namespace grb
