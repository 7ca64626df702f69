// Loop capture: grb_iterate_begin / grb_iterate_end.
//
// The recorded body is the loop of the §IV PageRank listing.  Run from the
// host, each iteration would end in a wait and a scalar read (the loop test
// `rdiff() > tolerance` needs the residual on the host).  When the body's DAG
// is the fused PageRank step, the loop instead runs on the GPU:
//
//   persistent  one cooperative kernel: prologue (w_0 = r_0 ./ d and the
//               dangling mass of r_0), then bodies separated by grid
//               barriers, the loop test evaluated on the device;
//   graph       the same prologue plus one fused kernel per body, captured
//               in a CUDA graph; each launch first re-checks the loop test.
//
// Afterwards every handle must hold what the plain loop would have left in
// it.  The rank is loop-carried; everything else the body writes is a
// function of the last two ranks r_{K-1} and r_K.  So the body is replayed
// once more without executing, from r_{K-1}: that leaves the handles pointing
// at pending versions (lazy, as in the paper's method trees), and the two
// versions the device loop computed -- r_K and the final residual -- are
// filled in directly.
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <set>

#include "grb_core.h"

namespace grb {

namespace {

struct LoopMatch {
    VectorH* r = nullptr;
    Matrix* A = nullptr;
    Version* d = nullptr;
    Version* sinks = nullptr;
    Version* rt = nullptr;
    bool uniform = false;
    SChain chain;
    grb_type T = GRB_FP32;
    grb_type resid_type = GRB_FP64;
};

void stmt_reads(const Stmt& s, std::vector<void*>& rd) {
    rd.clear();
    switch (s.kind) {
        case Stmt::VCOPY: rd.push_back(s.srcv); break;
        case Stmt::OP:
            for (void* h : {(void*)s.hu, (void*)s.hv, (void*)s.hmask, (void*)s.hs})
                if (h) rd.push_back(h);
            if (!s.out_is_scalar && (s.tmpl.has_accum || (s.hmask && !(s.tmpl.desc & GRB_DESC_REPLACE))))
                rd.push_back(s.dstv);
            if (s.out_is_scalar && s.tmpl.has_accum) rd.push_back(s.dsts);
            break;
        default: break;
    }
}

void* stmt_write(const Stmt& s) {
    switch (s.kind) {
        case Stmt::VCOPY:
        case Stmt::VFILL: return s.dstv;
        case Stmt::SSET: return s.dsts;
        case Stmt::OP: return s.out_is_scalar ? (void*)s.dsts : (void*)s.dstv;
        default: return nullptr;
    }
}

// Handles read in the body before the body writes them, and written later:
// the loop-carried variables.
std::set<void*> loop_carried(const std::vector<Stmt>& body) {
    std::set<void*> written_any, written, carried;
    for (const Stmt& s : body)
        if (void* w = stmt_write(s)) written_any.insert(w);
    std::vector<void*> rd;
    for (const Stmt& s : body) {
        stmt_reads(s, rd);
        for (void* h : rd)
            if (!written.count(h) && written_any.count(h)) carried.insert(h);
        if (void* w = stmt_write(s)) written.insert(w);
    }
    return carried;
}

bool invariant_full(const Version* v, grb_type T, bool allow_iso) {
    return v && v->ready && !v->err && !v->scalar && v->type == T &&
           (v->fmt == Fmt::FULL || (allow_iso && v->fmt == Fmt::ISO && !v->iso_src));
}

bool match_body(Version* r0, Version* Vr, Version* Vc, LoopMatch& lm) {
    const grb_type T = r0->type;
    if (!(T == GRB_FP32 || T == GRB_FP64)) return false;
    // rdiff = reduce(+, ewise_add(|x-y|, r0, r_new))
    Node* Q = Vc->producer;
    if (!Q || Q->k != OpK::REDUCE || Q->mon != GRB_MONOID_PLUS || Q->has_accum) return false;
    Node* X = Q->u->producer;
    if (!X || X->k != OpK::EADD || X->op.opcode != GRB_ABS_DIFF || X->mask || X->has_accum) return false;
    if (!((X->u == r0 && X->v == Vr) || (X->u == Vr && X->v == r0))) return false;
    if (X->out->type != T || Vr->type != T) return false;
    Node* R = Vr->producer;
    if (!R) return false;
    Node* M = nullptr;
    if (R->k == OpK::EADD && R->op.opcode == GRB_PLUS && !R->mask && !R->has_accum) {
        for (int side = 0; side < 2 && !M; ++side) {
            Version* s = side == 0 ? R->v : R->u;
            Version* o = side == 0 ? R->u : R->v;
            if (s->producer && s->producer->k == OpK::MXV && !s->producer->has_accum) {
                M = s->producer;
                lm.rt = o;
            }
        }
        // the loop kernels take the teleport as one scalar: rt must be iso
        if (!M || !invariant_full(lm.rt, T, true) || lm.rt->fmt != Fmt::ISO) return false;
    } else if (R->k == OpK::MXV && R->has_accum && R->accum.opcode == GRB_PLUS) {
        M = R;
        Version* av = R->w_old;
        Node* AS = av ? av->producer : nullptr;
        if (!AS || AS->k != OpK::ASSIGN_S || AS->mask || AS->has_accum || av->type != T) return false;
        Version* dv = AS->s;
        if (dv->ready && dv->host_known) {
            lm.rt = av;  // filled below as an iso constant
            return false;  // constant teleport through assign: use the replay path
        }
        std::vector<Node*> steps;
        Node* cur = dv->producer;
        while (cur && cur->k == OpK::SAPPLY_B2) {
            steps.push_back(cur);
            cur = cur->s->producer;
        }
        if (!cur || cur->k != OpK::REDUCE || cur->mon != GRB_MONOID_PLUS || cur->has_accum || steps.size() > 5)
            return false;
        Node* Z = cur->u->producer;
        if (!Z || Z->k != OpK::EMULT || Z->mask || Z->has_accum || Z->out->type != T) return false;
        if (Z->op.opcode == GRB_FIRST && Z->u == r0) lm.sinks = Z->v;
        else if (Z->op.opcode == GRB_SECOND && Z->v == r0) lm.sinks = Z->u;
        else return false;
        if (!lm.sinks->ready || lm.sinks->err || lm.sinks->scalar || lm.sinks->n != r0->n) return false;
        std::reverse(steps.begin(), steps.end());
        lm.chain.n = 0;
        lm.chain.ops[0].code = GRB_FIRST;  // the reduction rounds to its scalar type
        lm.chain.c[0] = 0.0;
        lm.chain.rtype[0] = cur->out->type;
        lm.chain.n = 1;
        for (Node* s : steps) {
            lm.chain.ops[lm.chain.n].code = s->op.opcode;
            lm.chain.ops[lm.chain.n].k = s->op.k;
            lm.chain.c[lm.chain.n] = s->k_const();
            lm.chain.rtype[lm.chain.n] = s->out->type;
            lm.chain.n++;
        }
        lm.uniform = true;
    } else {
        return false;
    }
    // M = mxv(plus.second | plus.times on iso-1, A, ewise_mult(/, r0, d))
    Matrix* A = M->A;
    if (M->mask || A->vals.p || M->out->type != T) return false;
    if (!(M->sr == GRB_PLUS_SECOND || (M->sr == GRB_PLUS_TIMES && A->iso_val == 1.0))) return false;
    if (A->nrows != r0->n || A->ncols != r0->n) return false;
    if (A->nrows + A->nnz >= PR_INDEX_LIMIT) return false;
    Node* W = M->u->producer;
    if (!W || W->k != OpK::EMULT || W->op.opcode != GRB_DIV || W->mask || W->has_accum || W->u != r0) return false;
    if (W->out->type != T || !invariant_full(W->v, T, false)) return false;
    lm.d = W->v;
    lm.A = A;
    lm.T = T;
    lm.resid_type = Q->out->type;
    return true;
}

void fulfil_vector(Version* v, DevBuf& vals) {
    if (v->producer) {
        Node* nd = v->producer;
        v->producer = nullptr;
        node_destroy(nd);
    }
    v->vals = vals;
    vals = DevBuf();
    v->fmt = Fmt::FULL;
    v->ready = true;
}

void fulfil_scalar(Version* v, double value) {
    if (v->producer) {
        Node* nd = v->producer;
        v->producer = nullptr;
        node_destroy(nd);
    }
    v->host_known = true;
    v->hval = value;
    v->ready = true;
}

// The same with the value in a device slot (written in stream order).
void fulfil_scalar_dev(Version* v, DevBuf& slot) {
    if (v->producer) {
        Node* nd = v->producer;
        v->producer = nullptr;
        node_destroy(nd);
    }
    v->host_known = false;
    v->slot = slot;
    slot = DevBuf();
    v->ready = true;
}

template <class H>
void save_handles(const std::vector<Stmt>& body, std::map<H*, Version*>& saved, H* Stmt::*field) {
    for (const Stmt& s : body) {
        H* h = s.*field;
        if (h && !saved.count(h)) {
            saved[h] = h->cur;
            ver_ref(h->cur);
        }
    }
}

template <class H>
void restore_handles(std::map<H*, Version*>& saved) {
    for (auto& kv : saved) {
        handle_set(kv.first, kv.second);
        ver_unref(kv.second);
    }
    saved.clear();
}

grb_info replay_dry(Ctx* c, const std::vector<Stmt>& body) {
    c->dry = true;
    grb_info st = GRB_SUCCESS;
    for (const Stmt& s : body) {
        st = replay_stmt(c, s);
        if (st) break;
    }
    c->dry = false;
    return st;
}

}  // namespace

// Pinned host staging for a loop's result slots and histories (grown on
// demand; copies of an earlier loop may still be landing in the old one).
static grb_info ensure_stage(Ctx* c, size_t ndoubles) {
    if (!c->stage_ev) {
        grb_info st = cuda_check(c, cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming), "loop event");
        if (st) return st;
    }
    if (c->stage_cap >= ndoubles) return GRB_SUCCESS;
    grb_info st = cuda_check(c, cudaStreamSynchronize(c->stream), "loop staging");
    if (st) return st;
    if (c->stage) cudaFreeHost(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    const size_t cap = std::max<size_t>(ndoubles, 1024);
    st = cuda_check(c, cudaMallocHost((void**)&c->stage, cap * sizeof(double)), "loop staging");
    if (!st) c->stage_cap = cap;
    return st;
}

// Events around the loop kernels: one pair of a ring per device loop.
static cudaEvent_t* loop_events(Ctx* c) {
    cudaEvent_t* ev = c->loop_ev[c->loop_count % Ctx::LOOP_TIMES];
    for (int k = 0; k < 2; ++k)
        if (!ev[k] && cudaEventCreate(&ev[k]) != cudaSuccess) {
            cudaGetLastError();
            ev[k] = nullptr;
        }
    return ev[0] && ev[1] ? ev : nullptr;
}

grb_info resolve_loop_history(Ctx* c) {
    if (!c->loop_pending) return GRB_SUCCESS;
    grb_info st = cuda_check(c, cudaEventSynchronize(c->stage_ev), "loop history");
    if (st) return st;
    c->loop_pending = false;
    int64_t K = 0;
    std::memcpy(&K, &c->stage[0], sizeof(int64_t));
    K = std::max<int64_t>(0, std::min<int64_t>(K, c->loop_cap));
    const double* h = c->stage + 8;
    c->last_hist.assign(h, h + K);
    if (c->loop_uniform) c->last_dang.assign(h + c->loop_cap, h + c->loop_cap + K);
    else c->last_dang.clear();
    int32_t phase = 0;
    std::memcpy(&phase, &c->stage[4], sizeof(int32_t));
    c->last_mixed_phase = c->loop_mixed ? (int)phase : -1;
    return GRB_SUCCESS;
}

int64_t last_loop_kernel_ns(Ctx* c) {
    if (c->loop_count == 0) return c->stats.last_loop_kernel_ns;
    cudaEvent_t* ev = c->loop_ev[(c->loop_count - 1) % Ctx::LOOP_TIMES];
    float ms = 0.f;
    if (ev[1] && cudaEventSynchronize(ev[1]) == cudaSuccess && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess)
        c->stats.last_loop_kernel_ns = (int64_t)(ms * 1e6);
    cudaGetLastError();
    return c->stats.last_loop_kernel_ns;
}

void loop_resources_free(Ctx* c) {
    if (c->stage) cudaFreeHost(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    if (c->stage_ev) cudaEventDestroy(c->stage_ev);
    c->stage_ev = nullptr;
    for (auto& pair : c->loop_ev)
        for (cudaEvent_t& e : pair)
            if (e) {
                cudaEventDestroy(e);
                e = nullptr;
            }
}

// The device loop.  Everything -- loop kernel, copies of the result slots
// and histories into pinned host memory, the permutes back to the caller's
// vertex order -- is enqueued on the context's stream.  A loop whose body
// count is fixed in advance (NONBLOCKING mode, tol < 0: every residual is
// >= 0 > tol) returns without waiting: its outputs are device values ordered
// behind the loop on the stream, and a device error (a bounded wait that ran
// out, or a body count other than the one assumed) surfaces at the next call
// that waits for the stream, as for any other pending method.  A loop that
// stops on its tolerance waits once, for the body count.
static grb_info device_loop(Ctx* c, const std::vector<Stmt>& body, ScalarH* cond, LoopMatch& lm, double tol,
                            int64_t itermax, double rd0, int64_t* iters_out) {
    NvtxRange range("grb: device PageRank loop");
    const grb_type T = lm.T;
    // BF16 gathers pay only once the FP32 gather vector (4n bytes) no
    // longer fits in L2: while it does, a gather costs one L2 sector
    // whatever its width, and the BF16 phase only adds bodies
    const bool mixed = T == GRB_FP32 &&
                       (c->mixed == 2 || (c->mixed == 1 && (size_t)lm.A->nrows * sizeof(float) > c->l2_bytes));
    const grb_type G = mixed ? GRB_BF16 : T;
    Matrix* A = lm.A;
    const int64_t n = A->nrows;
    // AL: the matrix the loop kernels run on (A, or its degree-ordered copy;
    // then every vector the kernels read or write is in that vertex order)
    grb_info st = GRB_SUCCESS;
    Matrix* AL = A;
    if (c->relabel) {
        st = ensure_relabel(c, A);
        if (!st && A->rel) AL = A->rel;
    }
    const bool rel = AL != A;
    if (!st) st = ensure_plan(c, AL);
    if (!st && lm.uniform) st = ensure_sinkbits(c, lm.sinks);
    if (!st && rel) st = ensure_perm_copy(c, A, lm.d, false);
    if (!st && rel && lm.uniform) st = ensure_perm_copy(c, A, lm.sinks, true);
    if (st) return st;
    const int iters = (int)std::min<int64_t>(itermax, INT_MAX - 16);
    const int mode = (c->persistent == 2 && !mixed) ? 2 : 1;
    const bool known = mode == 1 && c->mode == GRB_NONBLOCKING && tol < 0.0;
    st = ensure_stage(c, 8 + 2 * (size_t)iters);
    if (st) return st;
    Version* r0 = lm.r->cur;
    ver_ref(r0);
    const size_t tb = type_size(T) * (size_t)n, gb = type_size(G) * (size_t)n;
    DevBuf r0full, rb[2], wb[2], w32[2], hist, slots, cslot;
    rb[0] = buf_alloc(c, tb);
    rb[1] = buf_alloc(c, tb);
    wb[0] = buf_alloc(c, gb);
    wb[1] = buf_alloc(c, gb);
    if (mixed) {
        w32[0] = buf_alloc(c, sizeof(float) * n);
        w32[1] = buf_alloc(c, sizeof(float) * n);
    }
    hist = buf_alloc(c, sizeof(double) * 2 * (size_t)iters);
    slots = buf_alloc(c, sizeof(double) * 8);
    if (known) cslot = buf_alloc(c, sizeof(double));
    if (!rb[0].p || !rb[1].p || !wb[0].p || !wb[1].p || !hist.p || !slots.p || (mixed && (!w32[0].p || !w32[1].p)) ||
        (known && !cslot.p))
        st = GRB_OUT_OF_MEMORY;
    const void* r0data = r0->vals.p;
    if (!st && r0->fmt == Fmt::ISO) {
        r0full = buf_alloc(c, tb);
        if (!r0full.p) st = GRB_OUT_OF_MEMORY;
        if (!st) {
            EwSpec e;
            e.kind = EW_COPY;
            e.u = vin_of(r0);
            e.ctype = T;
            WriteSpec w;
            VOut o;
            o.vals = r0full.p;
            o.type = T;
            o.full = 1;
            c->stats.kernel_launches++;
            st = cuda_check(c, launch_ewise(c->stream, n, e, w, o), "expand start vector");
        }
        r0data = r0full.p;
    } else if (!st && rel) {
        r0full = buf_alloc(c, tb);
        if (!r0full.p) st = GRB_OUT_OF_MEMORY;
        c->stats.kernel_launches++;
        if (!st)
            st = cuda_check(c, launch_permute(c->stream, (int32_t)n, (const int32_t*)A->new2old.p, r0->vals.p, r0full.p,
                                              (int32_t)type_size(T)), "permute start vector");
        r0data = r0full.p;
    }
    double* sl = (double*)slots.p;
    int64_t* iters_done = (int64_t*)(sl + 0);
    if (!st) st = cuda_check(c, cudaMemsetAsync(slots.p, 0, sizeof(double) * 8, c->stream), "loop slots");

    PrParams p = plan_params_of(c, AL);
    p.gmode = G_W;
    p.has_base = 1;
    if (lm.uniform) {
        p.tele_from_slot = 1;
        p.tele_slot = sl + 3;
        p.want_dang = 1;
        p.sinkbits = (const uint32_t*)(rel ? lm.sinks->perm_sinkbits.p : lm.sinks->sinkbits.p);
        p.chain = lm.chain;
    } else {
        p.tele_from_slot = 0;
        p.tele_const = lm.rt->iso;   // iso teleport vector (required by the match)
    }
    p.want_resid = 1;
    p.resid_slot = sl + 1;
    p.resid_type = lm.resid_type;
    p.dang_slot = sl + 2;
    p.dd = rel ? lm.d->perm_vals.p : lm.d->vals.p;
    p.out.type = T;
    p.out.full = 1;
    p.iters = iters;
    p.tol = tol;
    p.rdiff0 = rd0;
    p.hist = (double*)hist.p;
    p.dhist = lm.uniform ? (double*)hist.p + iters : nullptr;
    p.expect_iters = known ? iters : 0;
    p.iters_done = iters_done;
    p.r0 = r0data;
    p.rbuf[0] = rb[0].p;
    p.rbuf[1] = rb[1].p;
    p.wbuf[0] = wb[0].p;
    p.wbuf[1] = wb[1].p;
    p.mixed = mixed ? 1 : 0;
    p.mixed_switch = c->mixed_switch;
    p.wbuf32[0] = w32[0].p;
    p.wbuf32[1] = w32[1].p;
    p.mixed_phase = (int32_t*)(sl + 4);

    cudaEvent_t* ev = st ? nullptr : loop_events(c);
    if (ev) cudaEventRecord(ev[0], c->stream);
    const bool bins = mode == 1 && c->row_bins && T == GRB_FP32 && !mixed;
    if (!st && bins) {
        st = ensure_bins(c, AL);
        if (!st) {
            p.bin_rows = (const int32_t*)AL->plan->bin_rows.p;
            for (int b = 0; b < 7; ++b) p.bin_off[b] = AL->plan->bin_off[b];
        }
    }
    if (!st && mode == 1) {
        // shared-memory copy of the hottest entries of w: only useful when
        // the vertices are in degree order
        if (rel && !mixed && T == GRB_FP32 && c->hot_bytes >= 16) {
            // the staging buffers share the block's shared memory with the copy
            p.tma_stages = bins ? 0 : c->tma_stages;
            const int64_t stage_b = (int64_t)pr_hot_dynamic_smem(0, p.tma_stages);
            const int64_t room = (int64_t)PR_SMEM_PER_BLOCK_MAX - (int64_t)PR_HOT_STATIC_SMEM - stage_b;
            const int64_t bytes = std::min<int64_t>(c->hot_bytes, room);
            p.hot_n = (int32_t)(std::min<int64_t>(n, bytes / (int64_t)sizeof(float)) & ~(int64_t)3);
            if (p.hot_n <= 0) p.tma_stages = 0;
        }
        int grid = p.hot_n > 0 ? pr_grid(c, AL, T, G, G_W, 1, p.hot_n, p.tma_stages, bins) : 0;
        if (grid <= 0) {
            p.hot_n = 0;
            p.tma_stages = 0;
            grid = pr_grid(c, AL, T, G, G_W, 1, 0, 0, bins);
        }
        c->stats.kernel_launches++;
        if (!st) st = cuda_check(c, launch_pr(c->stream, p, T, G, grid, 1), "persistent pagerank loop");
    } else if (!st) {
        // prologue (no bodies) + one fused kernel per body, as a CUDA graph
        const int pgrid = pr_grid(c, AL, T, G, G_W, 1);
        const int igrid = pr_grid(c, AL, T, G, G_W, 2);
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        // capture on a private stream (the context's stream may be the
        // legacy default stream, which cannot be captured); the graph is
        // then launched on the context's stream
        if (!c->capture_stream)
            st = cuda_check(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "capture stream");
        if (!st)
            st = cuda_check(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal),
                            "graph capture");
        if (!st) {
            PrParams pp = p;
            pp.iters = 0;
            cudaError_t e = launch_pr(c->capture_stream, pp, T, G, pgrid, 1);
            for (int it = 0; it < iters && e == cudaSuccess; ++it) {
                PrParams pi = p;
                pi.iter_index = it;
                e = launch_pr(c->capture_stream, pi, T, G, igrid, 2);
            }
            cudaError_t e2 = cudaStreamEndCapture(c->capture_stream, &graph);
            st = cuda_check(c, e != cudaSuccess ? e : e2, "graph capture");
        }
        if (!st) st = cuda_check(c, cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
        if (!st && ev) cudaEventRecord(ev[0], c->stream);   // time the graph's kernels only
        if (!st) st = cuda_check(c, cudaGraphLaunch(exec, c->stream), "graph launch");
        c->stats.kernel_launches += 1 + iters;
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
    if (ev) {
        cudaEventRecord(ev[1], c->stream);
        if (!st) c->loop_count++;
    }
    cudaGetLastError();
    // result slots and histories -> pinned host staging, behind the loop
    if (!st) {
        st = cuda_check(c, cudaMemcpyAsync(c->stage, slots.p, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream),
                        "loop result");
        if (!st)
            st = cuda_check(c, cudaMemcpyAsync(c->stage + 8, hist.p, sizeof(double) * 2 * (size_t)iters,
                                               cudaMemcpyDeviceToHost, c->stream), "loop history");
        if (!st) st = cuda_check(c, cudaEventRecord(c->stage_ev, c->stream), "loop history");
        if (!st) {
            c->loop_pending = true;
            c->loop_cap = iters;
            c->loop_uniform = lm.uniform;
            c->loop_mixed = mixed;
            c->stats.persistent_loops++;
        }
    }
    int64_t K = 0;
    double rd_final = 0.0;
    if (!st && known) {
        K = iters;
        st = cuda_check(c, cudaMemcpyAsync(cslot.p, sl + 1, sizeof(double), cudaMemcpyDeviceToDevice, c->stream),
                        "loop residual");
    } else if (!st) {
        // the body count is data-dependent: wait for it (and for the status)
        st = read_status(c);
        if (!st) st = resolve_loop_history(c);
        if (!st) {
            std::memcpy(&K, &c->stage[0], sizeof(int64_t));
            rd_final = c->stage[1];
        }
    }
    // back to the caller's vertex order: out[i] = buf[old2new[i]]
    auto unpermute = [&](DevBuf& b) -> grb_info {
        if (!rel) return GRB_SUCCESS;
        DevBuf o = buf_alloc(c, tb);
        if (!o.p) return GRB_OUT_OF_MEMORY;
        c->stats.kernel_launches++;
        grb_info s2 = cuda_check(c, launch_permute(c->stream, (int32_t)n, (const int32_t*)A->old2new.p, b.p, o.p,
                                                   (int32_t)type_size(T)), "unpermute rank");
        buf_free(c, b);
        b = o;
        return s2;
    };
    if (!st && K >= 2) st = unpermute(rb[(K - 2) & 1]);
    if (!st && K >= 1) st = unpermute(rb[(K - 1) & 1]);
    if (!st && K > 0) {
        // r_{K-1}: the start vector itself, or the other ping-pong buffer
        Version* rprev = r0;
        ver_ref(rprev);
        if (K >= 2) {
            ver_unref(rprev);
            rprev = new_version(c, false, T, n);
            rprev->vals = rb[(K - 2) & 1];
            rb[(K - 2) & 1] = DevBuf();
            rprev->fmt = Fmt::FULL;
            rprev->ready = true;
        }
        handle_set(lm.r, rprev);
        ver_unref(rprev);
        st = replay_dry(c, body);
        if (!st) {
            fulfil_vector(lm.r->cur, rb[(K - 1) & 1]);
            if (known) fulfil_scalar_dev(cond->cur, cslot);
            else fulfil_scalar(cond->cur, rd_final);
        }
    }
    *iters_out = K;
    ver_unref(r0);
    // back to the context's pool: later work on the same stream reuses them
    // in stream order
    for (DevBuf* b : {&r0full, &rb[0], &rb[1], &wb[0], &wb[1], &w32[0], &w32[1], &hist, &slots, &cslot})
        buf_free(c, *b);
    return st;
}

grb_info iterate_end(Ctx* c, ScalarH* cond, double tol, int64_t itermax, int64_t* iters_out) {
    std::vector<Stmt> body;
    body.swap(c->body);
    c->recording = false;
    *iters_out = 0;
    double rd = 0.0;
    grb_info st = GRB_SUCCESS;
    Version* cv = cond->cur;
    if (cv->ready && !cv->err && cv->host_known) {
        rd = cv->hval;   // set on the host: no need to wait for the stream
    } else {
        st = scalar_value(c, cv, &rd);
        if (st == GRB_NO_VALUE) rd = __builtin_inf();
        else if (st) return st;
    }
    if (itermax == 0 || !(rd > tol)) return GRB_SUCCESS;

    LoopMatch lm;
    bool device = false;
    if (c->persistent != 3) {
        std::set<void*> carried = loop_carried(body);
        VectorH* r = nullptr;
        bool ok = carried.size() == 1;
        for (const Stmt& s : body)
            if (ok && s.dstv && carried.count(s.dstv)) r = s.dstv;
        if (ok && r && r->cur->producer) {
            Version* cur = r->cur;
            ver_ref(cur);
            st = materialize(c, cur);
            ver_unref(cur);
            if (st) return st;
        }
        if (ok && r && r->cur->ready && !r->cur->err) {
            std::map<VectorH*, Version*> sv;
            std::map<ScalarH*, Version*> ss;
            save_handles(body, sv, &Stmt::dstv);
            save_handles(body, ss, &Stmt::dsts);
            Version* r0 = r->cur;
            ver_ref(r0);
            if (!replay_dry(c, body)) {
                lm.r = r;
                device = match_body(r0, r->cur, cond->cur, lm) &&
                         (r0->fmt == Fmt::FULL || (r0->fmt == Fmt::ISO && !r0->iso_src)) && r0->type == lm.T;
            }
            restore_handles(sv);
            restore_handles(ss);
            ver_unref(r0);
        }
    }
    if (device) return device_loop(c, body, cond, lm, tol, itermax, rd, iters_out);

    int64_t it = 0;
    while (it < itermax && rd > tol) {
        for (const Stmt& s : body) {
            st = replay_stmt(c, s);
            if (st) {
                *iters_out = it;
                return st;
            }
        }
        ++it;
        st = scalar_value(c, cond->cur, &rd);
        if (st) {
            *iters_out = it;
            return st;
        }
    }
    *iters_out = it;
    c->stats.replayed_loops++;
    return GRB_SUCCESS;
}

}  // namespace grb
