// Batched personalised PageRank (grb_ppr_*): k query slots over one A^T,
// iterated together by kernels_ppr.cu.  The paper runs one rank vector per
// PageRank; the slots here are that same fused iteration for many
// personalisation vectors at once, the form a serving loop needs: a slot
// can be (re)filled between runs while the others keep their state.
//
// Per slot: seeds S (deduplicated), teleport v = uniform over S, start
// vector r_0 = v, dangling mass spread uniformly, loop test of the §IV
// listing (`while iter <= itermax && rdiff > tol`) evaluated on the device
// after every body; a slot whose test fails keeps its rank.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "grb_core.h"

namespace grb {

struct Ppr {
    Kind kind = Kind::PPR;
    Ctx* c = nullptr;
    Matrix* A = nullptr;
    double damping = 0.85;
    int32_t slots = 0, kt = 0;
    int32_t vw = 1;                    // slots per lane (vector width)
    int32_t requested = 0;             // slots asked for at creation
    int64_t n = 0;
    int grid = 0;
    int cur = 0;                       // which of r[2] / w[2] holds the current iterate
    DevBuf r[2], w[2], dd, sinkbits, seedbits, agg, first, part_a, part_b;
    DevBuf active, iters, itermax, tol, resid, tele, final_buf;
    DevBuf seed_ptr, seed_row, seed_lane, seed_val;
    std::vector<std::vector<int32_t>> seeds;
    bool dirty = true;
    cudaGraphExec_t exec = nullptr;
    int64_t exec_iters = 0;
    int exec_cur = -1;
    grb_info broken = GRB_SUCCESS;    // a failed re-layout: every later call returns it
    // queries set since the last flush: admitted together before the next
    // run / status / get
    struct Pending {
        int32_t slot;
        std::vector<int32_t> seeds;
        double tol;
        int32_t itermax;
    };
    std::vector<Pending> pending;
};

namespace {

Ppr* as_ppr(grb_ppr p) {
    Ppr* x = reinterpret_cast<Ppr*>(p);
    return (x && x->kind == Kind::PPR) ? x : nullptr;
}

void drop_graph(Ppr* P) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    P->exec_cur = -1;
}

// Seed arrays sorted by (k-tile, row, lane) and the seed bitmap.
grb_info upload_seeds(Ppr* P) {
    Ctx* c = P->c;
    struct E { int32_t kt, row, lane; float val; };
    std::vector<E> es;
    for (int32_t s = 0; s < P->slots; ++s) {
        const auto& S = P->seeds[s];
        if (S.empty()) continue;
        const float val = (float)((1.0 - P->damping) * (1.0 / (double)S.size()));
        const int32_t width = PPR_LANES * P->vw;
        for (int32_t v : S) es.push_back({s / width, v, s % width, val});
    }
    std::sort(es.begin(), es.end(), [](const E& a, const E& b) {
        return a.kt != b.kt ? a.kt < b.kt : a.row != b.row ? a.row < b.row : a.lane < b.lane;
    });
    const size_t ne = es.size();
    std::vector<int32_t> ptr(P->kt + 1, 0), row(ne ? ne : 1), lane(ne ? ne : 1);
    std::vector<float> val(ne ? ne : 1);
    for (size_t q = 0; q < ne; ++q) {
        ptr[es[q].kt + 1]++;
        row[q] = es[q].row;
        lane[q] = es[q].lane;
        val[q] = es[q].val;
    }
    for (int32_t k = 0; k < P->kt; ++k) ptr[k + 1] += ptr[k];
    drop_graph(P);
    for (DevBuf* b : {&P->seed_ptr, &P->seed_row, &P->seed_lane, &P->seed_val}) buf_free(c, *b);
    P->seed_ptr = buf_alloc(c, sizeof(int32_t) * ptr.size());
    P->seed_row = buf_alloc(c, sizeof(int32_t) * row.size());
    P->seed_lane = buf_alloc(c, sizeof(int32_t) * lane.size());
    P->seed_val = buf_alloc(c, sizeof(float) * val.size());
    if (!P->seed_ptr.p || !P->seed_row.p || !P->seed_lane.p || !P->seed_val.p) return GRB_OUT_OF_MEMORY;
    grb_info st = cuda_check(c, cudaMemcpyAsync(P->seed_ptr.p, ptr.data(), sizeof(int32_t) * ptr.size(),
                                                cudaMemcpyHostToDevice, c->stream), "seed upload");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(P->seed_row.p, row.data(), sizeof(int32_t) * row.size(),
                                                cudaMemcpyHostToDevice, c->stream), "seed upload");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(P->seed_lane.p, lane.data(), sizeof(int32_t) * lane.size(),
                                                cudaMemcpyHostToDevice, c->stream), "seed upload");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(P->seed_val.p, val.data(), sizeof(float) * val.size(),
                                                cudaMemcpyHostToDevice, c->stream), "seed upload");
    if (!st) {
        c->stats.kernel_launches++;
        st = cuda_check(c, launch_ppr_seedbits(c->stream, (int32_t)ne, (const int32_t*)P->seed_row.p,
                                               (uint32_t*)P->seedbits.p, (P->n + 31) / 32), "seed bits");
    }
    // the host vectors above must outlive the copies
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "seed upload");
    if (!st) P->dirty = false;
    return st;
}

PprParams params(Ppr* P, int from) {
    TilePlan* pl = P->A->plan;
    PprParams p;
    p.col_idx = (const int32_t*)P->A->col_idx.p;
    p.nrows = (int32_t)P->n;
    p.nnz = (int32_t)P->A->nnz;
    p.ntiles = (int32_t)pl->ntiles;
    p.status = (int32_t*)P->c->status.p;
    p.tile_meta = (const uint32_t*)pl->meta.p;
    p.rowend_bits = (const uint32_t*)pl->rowend_bits.p;
    p.ne_rows = (const int32_t*)pl->ne_rows.p;
    p.n_ne = (int32_t)pl->n_ne;
    p.empty_rows = (const int32_t*)pl->empty_rows.p;
    p.n_empty = (int32_t)pl->n_empty;
    p.fix = (const FixDesc*)pl->fix.p;
    p.kt = P->kt;
    p.vw = P->vw;
    p.r_old = (const float*)P->r[from].p;
    p.r_new = (float*)P->r[from ^ 1].p;
    p.w_old = (const float*)P->w[from].p;
    p.w_new = (float*)P->w[from ^ 1].p;
    p.dd = (const float*)P->dd.p;
    p.sinkbits = (const uint32_t*)P->sinkbits.p;
    p.agg = (float*)P->agg.p;
    p.first = (float*)P->first.p;
    p.seedbits = (const uint32_t*)P->seedbits.p;
    p.seed_ptr = (const int32_t*)P->seed_ptr.p;
    p.seed_row = (const int32_t*)P->seed_row.p;
    p.seed_lane = (const int32_t*)P->seed_lane.p;
    p.seed_val = (const float*)P->seed_val.p;
    p.active = (const int32_t*)P->active.p;
    p.tele_base = (const float*)P->tele.p;
    return p;
}

grb_info record_iterations(Ppr* P, cudaStream_t st, int64_t iters) {
    const int S = P->slots;
    PprFinish f;
    f.slots = S;
    f.grid_a = P->grid;
    f.grid_b = P->grid;
    f.part_a = (const double*)P->part_a.p;
    f.part_b = (const double*)P->part_b.p;
    f.active = (int32_t*)P->active.p;
    f.iters = (int32_t*)P->iters.p;
    f.itermax = (const int32_t*)P->itermax.p;
    f.tol = (const double*)P->tol.p;
    f.resid = (double*)P->resid.p;
    f.tele_base = (float*)P->tele.p;
    f.final_buf = (int32_t*)P->final_buf.p;
    f.damping = P->damping;
    f.n = P->n;
    cudaError_t e = cudaSuccess;
    for (int64_t k = 0; k < iters && e == cudaSuccess; ++k) {
        PprParams p = params(P, (int)((P->cur + k) & 1));
        p.part = (double*)P->part_a.p;
        e = launch_ppr_tiles(st, p, P->grid);
        if (e == cudaSuccess) {
            p.part = (double*)P->part_b.p;
            e = launch_ppr_fixups(st, p, P->grid);
        }
        f.out_buf = (int32_t)((P->cur + k + 1) & 1);
        if (e == cudaSuccess) e = launch_ppr_finish(st, f);
    }
    return cuda_check(P->c, e, "ppr iteration");
}

// (Re)lay out the slot state for vector width vw: rank / gather buffers,
// carries, partials and slot arrays, all zero; every slot empty.
grb_info alloc_layout(Ppr* P, int32_t vw) {
    Ctx* c = P->c;
    drop_graph(P);
    cudaStreamSynchronize(c->stream);
    for (DevBuf* b : {&P->r[0], &P->r[1], &P->w[0], &P->w[1], &P->agg, &P->first, &P->part_a, &P->part_b,
                      &P->active, &P->iters, &P->itermax, &P->tol, &P->resid, &P->tele, &P->final_buf})
        buf_free(c, *b);
    const int32_t width = PPR_LANES * vw;
    P->vw = vw;
    P->kt = (P->requested + width - 1) / width;
    P->slots = P->kt * width;
    P->seeds.assign(P->slots, {});
    P->pending.clear();
    P->cur = 0;
    P->dirty = true;
    // the same grid at every width (two CTAs per SM; at width 4, whose CTAs
    // need a whole SM's registers, that is two waves): each warp then takes
    // the same tiles and rows, so every slot's sums are folded in the same
    // order whatever the width
    P->grid = PPR_CTAS_PER_SM * c->sm_count;
    const int64_t n = P->n, S = P->slots, nt = P->A->plan->ntiles;
    const size_t rb = sizeof(float) * (size_t)S * (size_t)n;
    for (int q = 0; q < 2; ++q) {
        P->r[q] = buf_alloc(c, rb);
        P->w[q] = buf_alloc(c, rb);
    }
    P->agg = buf_alloc(c, sizeof(float) * (size_t)S * nt);
    P->first = buf_alloc(c, sizeof(float) * (size_t)S * nt);
    P->part_a = buf_alloc(c, sizeof(double) * 2 * (size_t)P->grid * S);
    P->part_b = buf_alloc(c, sizeof(double) * 2 * (size_t)P->grid * S);
    P->active = buf_alloc(c, sizeof(int32_t) * S);
    P->iters = buf_alloc(c, sizeof(int32_t) * S);
    P->itermax = buf_alloc(c, sizeof(int32_t) * S);
    P->tol = buf_alloc(c, sizeof(double) * S);
    P->resid = buf_alloc(c, sizeof(double) * S);
    P->tele = buf_alloc(c, sizeof(float) * S);
    P->final_buf = buf_alloc(c, sizeof(int32_t) * S);
    grb_info st = GRB_SUCCESS;
    for (DevBuf* b : {&P->r[0], &P->r[1], &P->w[0], &P->w[1], &P->agg, &P->first, &P->part_a, &P->part_b,
                      &P->active, &P->iters, &P->itermax, &P->tol, &P->resid, &P->tele, &P->final_buf})
        if (!b->p) st = GRB_OUT_OF_MEMORY;
    for (DevBuf* b : {&P->r[0], &P->r[1], &P->w[0], &P->w[1], &P->active, &P->iters, &P->itermax, &P->tol,
                      &P->resid, &P->tele, &P->final_buf})
        if (!st) st = cuda_check(c, cudaMemsetAsync(b->p, 0, b->bytes, c->stream), "ppr layout");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "ppr layout");
    P->broken = st;
    return st;
}

// Admit every queued query: one upload of the queue, one kernel that clears
// the queued slots' columns (adjacent slots share cache lines) and one that
// places their start vectors and loop state.
grb_info flush_pending(Ppr* P) {
    if (P->pending.empty()) return GRB_SUCCESS;
    Ctx* c = P->c;
    std::sort(P->pending.begin(), P->pending.end(),
              [](const Ppr::Pending& a, const Ppr::Pending& b) { return a.slot < b.slot; });
    const int32_t np = (int32_t)P->pending.size();
    std::vector<int32_t> slots(np), off(np + 1, 0), act(np), im(np), seeds;
    std::vector<float> r0(np);
    std::vector<double> tol(np);
    for (int32_t k = 0; k < np; ++k) {
        const auto& q = P->pending[k];
        slots[k] = q.slot;
        off[k + 1] = off[k] + (int32_t)q.seeds.size();
        seeds.insert(seeds.end(), q.seeds.begin(), q.seeds.end());
        r0[k] = (float)(1.0 / (double)q.seeds.size());
        act[k] = (q.itermax > 0 && 1.0 > q.tol) ? 1 : 0;   // the loop test before the first body
        im[k] = q.itermax;
        tol[k] = q.tol;
    }
    // one staging buffer: doubles first, then the 4-byte arrays
    const size_t b_tol = 8 * (size_t)np, b_i = 4 * (size_t)np;
    const size_t bytes = b_tol + b_i * 4 + 4 * (size_t)(np + 1) + 4 * seeds.size();
    std::vector<char> host(bytes);
    char* h = host.data();
    size_t o = 0;
    auto put = [&](const void* src, size_t n) {
        std::memcpy(h + o, src, n);
        const size_t at = o;
        o += n;
        return at;
    };
    const size_t o_tol = put(tol.data(), b_tol), o_slots = put(slots.data(), b_i), o_r0 = put(r0.data(), b_i),
                 o_act = put(act.data(), b_i), o_im = put(im.data(), b_i),
                 o_off = put(off.data(), 4 * (size_t)(np + 1)), o_seeds = put(seeds.data(), 4 * seeds.size());
    DevBuf stage = buf_alloc(c, bytes);
    if (!stage.p) return GRB_OUT_OF_MEMORY;
    char* d = (char*)stage.p;
    grb_info st = cuda_check(c, cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c->stream), "queued queries");
    PprInitBatch a;
    a.np = np;
    a.nrows = (int32_t)P->n;
    a.width = PPR_LANES * P->vw;
    a.cur = P->cur;
    a.slots = (const int32_t*)(d + o_slots);
    a.seed_off = (const int32_t*)(d + o_off);
    a.seeds = (const int32_t*)(d + o_seeds);
    a.r0 = (const float*)(d + o_r0);
    a.act = (const int32_t*)(d + o_act);
    a.itermax = (const int32_t*)(d + o_im);
    a.tol = (const double*)(d + o_tol);
    a.r = (float*)P->r[P->cur].p;
    a.w = (float*)P->w[P->cur].p;
    a.dd = (const float*)P->dd.p;
    a.sinkbits = (const uint32_t*)P->sinkbits.p;
    a.active = (int32_t*)P->active.p;
    a.iters = (int32_t*)P->iters.p;
    a.itermax_out = (int32_t*)P->itermax.p;
    a.tol_out = (double*)P->tol.p;
    a.resid = (double*)P->resid.p;
    a.tele_base = (float*)P->tele.p;
    a.final_buf = (int32_t*)P->final_buf.p;
    a.damping = P->damping;
    if (!st) {
        c->stats.kernel_launches += 2;
        st = cuda_check(c, launch_ppr_init_batch(c->stream, a), "admit queries");
    }
    // the host staging copy must outlive the upload
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "admit queries");
    buf_free(c, stage);
    if (!st) P->pending.clear();
    return st;
}

}  // namespace

void ppr_destroy(Ppr* P) {
    Ctx* c = P->c;
    cudaStreamSynchronize(c->stream);
    drop_graph(P);
    for (DevBuf* b : {&P->r[0], &P->r[1], &P->w[0], &P->w[1], &P->dd, &P->sinkbits, &P->seedbits, &P->agg,
                      &P->first, &P->part_a, &P->part_b, &P->active, &P->iters, &P->itermax, &P->tol, &P->resid,
                      &P->tele, &P->final_buf, &P->seed_ptr, &P->seed_row, &P->seed_lane, &P->seed_val})
        buf_free(c, *b);
    matrix_unref(P->A);
    P->kind = Kind::DEAD;
    delete P;
}

}  // namespace grb

using namespace grb;

extern "C" {

grb_info grb_ppr_new(grb_ppr* out, grb_matrix Am, double damping, int32_t slots) {
    if (!out || !Am) return GRB_NULL_POINTER;
    *out = nullptr;
    Matrix* A = reinterpret_cast<Matrix*>(Am);
    if (A->kind != Kind::MATRIX) return GRB_UNINITIALIZED_OBJECT;
    if (A->nrows != A->ncols || A->vals.p) return GRB_INVALID_VALUE;      // square pattern A^T
    if (A->nrows < 1 || A->nrows + A->nnz >= PR_INDEX_LIMIT) return GRB_INVALID_VALUE;
    if (slots < 1 || slots > PPR_MAX_SLOTS || !(damping >= 0.0 && damping < 1.0)) return GRB_INVALID_VALUE;
    Ctx* c = A->ctx;
    grb_info st = ensure_plan(c, A);
    if (st) return st;
    Ppr* P = new Ppr();
    P->c = c;
    P->A = A;
    A->refs++;
    P->damping = damping;
    P->n = A->nrows;
    P->requested = slots;
    const int64_t n = P->n;
    P->dd = buf_alloc(c, sizeof(float) * n);
    P->sinkbits = buf_alloc(c, sizeof(uint32_t) * ((n + 31) / 32));
    P->seedbits = buf_alloc(c, sizeof(uint32_t) * ((n + 31) / 32));
    if (!P->dd.p || !P->sinkbits.p || !P->seedbits.p) st = GRB_OUT_OF_MEMORY;
    if (!st) st = alloc_layout(P, 1);
    DevBuf deg = buf_alloc(c, sizeof(int32_t) * n), pres = buf_alloc(c, (size_t)n);
    if (!deg.p || !pres.p) st = GRB_OUT_OF_MEMORY;
    if (!st) {
        c->stats.kernel_launches += 3;
        st = cuda_check(c, launch_col_degree(c->stream, n, A->nnz, (const int32_t*)A->col_idx.p, (int32_t*)deg.p,
                                             (uint8_t*)pres.p), "out-degree");
        if (!st) st = cuda_check(c, launch_ppr_divisor(c->stream, (int32_t)n, (const int32_t*)deg.p, damping,
                                                       (float*)P->dd.p, (uint32_t*)P->sinkbits.p), "divisor");
        if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "ppr init");
    }
    buf_free(c, deg);
    buf_free(c, pres);
    if (!st) st = upload_seeds(P);
    if (st) {
        ppr_destroy(P);
        return st;
    }
    *out = reinterpret_cast<grb_ppr>(P);
    return GRB_SUCCESS;
}

grb_info grb_ppr_layout(grb_ppr Ph, int32_t vw) {
    Ppr* P = as_ppr(Ph);
    if (!Ph) return GRB_NULL_POINTER;
    if (!P) return GRB_UNINITIALIZED_OBJECT;
    if (vw != 1 && vw != 2 && vw != 4) return GRB_INVALID_VALUE;
    return alloc_layout(P, vw);   // also the way out of a failed re-layout
}

grb_info grb_ppr_tune(grb_ppr Ph, int64_t trial_bodies, double* ms_per_body, int32_t* chosen_vw) {
    Ppr* P = as_ppr(Ph);
    if (!Ph) return GRB_NULL_POINTER;
    if (!P) return GRB_UNINITIALIZED_OBJECT;
    if (trial_bodies < 1 || trial_bodies > 100) return GRB_INVALID_VALUE;
    Ctx* c = P->c;
    const int32_t cands[3] = {1, 2, 4};
    double best = 1e300;
    int32_t best_vw = 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    grb_info st = cuda_check(c, cudaEventCreate(&e0), "ppr tune");
    if (!st) st = cuda_check(c, cudaEventCreate(&e1), "ppr tune");
    for (int q = 0; q < 3 && !st; ++q) {
        st = alloc_layout(P, cands[q]);
        // every slot busy with a one-vertex query
        for (int32_t s = 0; s < P->slots && !st; ++s) {
            const int32_t v = (int32_t)(((int64_t)s * 7919) % P->n);
            st = grb_ppr_set(Ph, s, &v, 1, -1.0, INT32_MAX);
        }
        if (!st) st = grb_ppr_run(Ph, trial_bodies);   // captures the graph, warms up
        if (!st) st = cuda_check(c, cudaEventRecord(e0, c->stream), "ppr tune");
        if (!st) st = grb_ppr_run(Ph, trial_bodies);
        if (!st) st = cuda_check(c, cudaEventRecord(e1, c->stream), "ppr tune");
        if (!st) st = cuda_check(c, cudaEventSynchronize(e1), "ppr tune");
        float ms = 0.f;
        if (!st) st = cuda_check(c, cudaEventElapsedTime(&ms, e0, e1), "ppr tune");
        if (st) break;
        // time per body for the requested slots (a wider layout may round
        // the slot count up; the extra slots do not count)
        const double per = (double)ms / (double)trial_bodies;
        if (ms_per_body) ms_per_body[q] = per;
        if (per < best) {
            best = per;
            best_vw = cands[q];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!st) st = alloc_layout(P, best_vw);
    if (!st && chosen_vw) *chosen_vw = best_vw;
    return st;
}

grb_info grb_ppr_slots(grb_ppr Ph, int32_t* slots) {
    Ppr* P = as_ppr(Ph);
    if (!Ph || !slots) return GRB_NULL_POINTER;
    if (!P) return GRB_UNINITIALIZED_OBJECT;
    if (P->broken) return GRB_INVALID_OBJECT;
    *slots = P->slots;
    return GRB_SUCCESS;
}

grb_info grb_ppr_set(grb_ppr Ph, int32_t slot, const int32_t* seeds, int64_t nseeds, double tol, int64_t itermax) {
    Ppr* P = as_ppr(Ph);
    if (!Ph || !seeds) return GRB_NULL_POINTER;
    if (!P) return GRB_UNINITIALIZED_OBJECT;
    if (P->broken) return GRB_INVALID_OBJECT;
    if (slot < 0 || slot >= P->slots || nseeds < 1 || itermax < 0 || itermax > INT32_MAX) return GRB_INVALID_VALUE;
    std::vector<int32_t> S(seeds, seeds + nseeds);
    for (int32_t v : S)
        if (v < 0 || v >= P->n) return GRB_INVALID_INDEX;
    std::sort(S.begin(), S.end());
    S.erase(std::unique(S.begin(), S.end()), S.end());
    // queued: the slot is (re)started at the next flush, with every other
    // query queued by then (one pass for all of them)
    P->pending.erase(std::remove_if(P->pending.begin(), P->pending.end(),
                                    [slot](const Ppr::Pending& q) { return q.slot == slot; }),
                     P->pending.end());
    P->pending.push_back({slot, S, tol, (int32_t)itermax});
    P->seeds[slot] = std::move(S);
    P->dirty = true;
    return GRB_SUCCESS;
}

grb_info grb_ppr_clear(grb_ppr Ph, int32_t slot) {
    Ppr* P = as_ppr(Ph);
    if (!Ph) return GRB_NULL_POINTER;
    if (!P) return GRB_UNINITIALIZED_OBJECT;
    if (P->broken) return GRB_INVALID_OBJECT;
    if (slot < 0 || slot >= P->slots) return GRB_INVALID_VALUE;
    grb_info st = flush_pending(P);
    if (st) return st;
    const int32_t zero = 0;
    st = cuda_check(P->c, cudaMemcpyAsync((int32_t*)P->active.p + slot, &zero, 4, cudaMemcpyHostToDevice,
                                          P->c->stream), "slot clear");
    if (!st) st = cuda_check(P->c, cudaStreamSynchronize(P->c->stream), "slot clear");
    if (st) return st;
    P->seeds[slot].clear();
    P->dirty = true;
    return GRB_SUCCESS;
}

grb_info grb_ppr_run(grb_ppr Ph, int64_t iters) {
    NvtxRange range("grb: personalised PageRank bodies");
    Ppr* P = as_ppr(Ph);
    if (!Ph) return GRB_NULL_POINTER;
    if (!P) return GRB_UNINITIALIZED_OBJECT;
    if (P->broken) return GRB_INVALID_OBJECT;
    if (iters < 0 || iters > 100000) return GRB_INVALID_VALUE;
    if (iters == 0) return GRB_SUCCESS;
    Ctx* c = P->c;
    grb_info st = flush_pending(P);
    if (!st && P->dirty) st = upload_seeds(P);
    if (st) return st;
    if (!P->exec || P->exec_iters != iters || P->exec_cur != P->cur) {
        drop_graph(P);
        if (!c->capture_stream)
            st = cuda_check(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t g = nullptr;
        if (!st) st = cuda_check(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal),
                                 "ppr capture");
        if (!st) {
            grb_info s1 = record_iterations(P, c->capture_stream, iters);
            grb_info s2 = cuda_check(c, cudaStreamEndCapture(c->capture_stream, &g), "ppr capture");
            st = s1 ? s1 : s2;
        }
        if (!st) st = cuda_check(c, cudaGraphInstantiate(&P->exec, g, 0), "ppr instantiate");
        if (g) cudaGraphDestroy(g);
        if (st) return st;
        P->exec_iters = iters;
        P->exec_cur = P->cur;
    }
    st = cuda_check(c, cudaGraphLaunch(P->exec, c->stream), "ppr launch");
    if (st) return st;
    c->stats.kernel_launches += 3 * iters;
    P->cur = (int)((P->cur + iters) & 1);
    return GRB_SUCCESS;
}

grb_info grb_ppr_status(grb_ppr Ph, int32_t* active, int64_t* iters, double* resid) {
    Ppr* P = as_ppr(Ph);
    if (!Ph) return GRB_NULL_POINTER;
    if (!P) return GRB_UNINITIALIZED_OBJECT;
    if (P->broken) return GRB_INVALID_OBJECT;
    Ctx* c = P->c;
    grb_info st0 = flush_pending(P);
    if (st0) return st0;
    const int S = P->slots;
    std::vector<int32_t> a(S), it(S);
    std::vector<double> rs(S);
    grb_info st = cuda_check(c, cudaMemcpyAsync(a.data(), P->active.p, 4 * S, cudaMemcpyDeviceToHost, c->stream),
                             "ppr status");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(it.data(), P->iters.p, 4 * S, cudaMemcpyDeviceToHost, c->stream),
                             "ppr status");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(rs.data(), P->resid.p, 8 * S, cudaMemcpyDeviceToHost, c->stream),
                             "ppr status");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "ppr status");
#ifdef GRB_CHECK_BOUNDS
    if (!st) st = read_status(c);   // a failed bounds check in the bodies run so far
#endif
    if (st) return st;
    for (int s = 0; s < S; ++s) {
        if (active) active[s] = a[s];
        if (iters) iters[s] = it[s];
        if (resid) resid[s] = rs[s];
    }
    return GRB_SUCCESS;
}

grb_info grb_ppr_get(grb_ppr Ph, int32_t slot, float* ranks, int out_is_device) {
    Ppr* P = as_ppr(Ph);
    if (!Ph || !ranks) return GRB_NULL_POINTER;
    if (!P) return GRB_UNINITIALIZED_OBJECT;
    if (P->broken) return GRB_INVALID_OBJECT;
    if (slot < 0 || slot >= P->slots) return GRB_INVALID_VALUE;
    Ctx* c = P->c;
    grb_info st0 = flush_pending(P);
    if (st0) return st0;
    float* dst = ranks;
    DevBuf tmp;
    if (!out_is_device) {
        tmp = buf_alloc(c, sizeof(float) * P->n);
        if (!tmp.p) return GRB_OUT_OF_MEMORY;
        dst = (float*)tmp.p;
    }
    // an active slot's rank is in the current buffer; a finished one's where
    // its last body left it
    int32_t act = 0, fb = 0;
    grb_info st = cuda_check(c, cudaMemcpyAsync(&act, (int32_t*)P->active.p + slot, 4, cudaMemcpyDeviceToHost,
                                                c->stream), "ppr extract");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(&fb, (int32_t*)P->final_buf.p + slot, 4, cudaMemcpyDeviceToHost,
                                                c->stream), "ppr extract");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "ppr extract");
    const int buf = act ? P->cur : (fb & 1);
    c->stats.kernel_launches++;
    if (!st)
        st = cuda_check(c, launch_ppr_extract(c->stream, (int32_t)P->n, (const float*)P->r[buf].p, PPR_LANES * P->vw, slot, dst),
                        "ppr extract");
    if (!st && !out_is_device)
        st = cuda_check(c, cudaMemcpyAsync(ranks, tmp.p, sizeof(float) * P->n, cudaMemcpyDeviceToHost, c->stream),
                        "ppr extract");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "ppr extract");
    buf_free(c, tmp);
    return st;
}

}  // extern "C"
