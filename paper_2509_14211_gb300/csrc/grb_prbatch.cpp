// A batch of independent PageRank problems (grb_prbatch_*): many graphs of
// uneven size solved together.  The caller builds one block-diagonal A^T
// (graph g owns rows and columns vptr[g] .. vptr[g+1]); every body is one
// cooperative launch of the fused tile kernel over all graphs' nonzeros (so
// a launch is as large as the sum of the graphs, however small each one is)
// that ends with the per-graph folds, and a whole solve is captured as one
// CUDA graph.  Each graph follows the §IV loop with uniform dangling
// on its own: teleport (1-d)/n_g, its own dangling mass, residual and loop
// test; a graph whose test fails keeps its rank while the others go on.
//
// Launch shape: an autotuner times every candidate number of resident CTAs
// per SM (1 .. the occupancy limit) on the batch itself and keeps the
// fastest.  The per-graph folds do not depend on the launch shape, so the
// results are the same for every candidate.
#include <algorithm>
#include <cstring>
#include <vector>

#include "grb_core.h"

namespace grb {

struct PrBatch {
    Kind kind = Kind::PRBATCH;
    Ctx* c = nullptr;
    Matrix* A = nullptr;       // the matrix the kernels run on (A_in, or its copy renumbered inside the blocks)
    Matrix* A_in = nullptr;    // the caller's matrix
    std::vector<int32_t> old2new_h;   // empty: no renumbering
    int32_t ng = 0;
    int64_t n = 0;
    double damping = 0.85;
    std::vector<int64_t> vptr_h;
    DevBuf vptr, graph_of, dd, sinkbits, row_res, row_dang, r[2], w[2];
    DevBuf chunk_lo, chunk_graph, g_chunk, chunk_part;   // the fold's chunks (MG_CHUNK rows of one graph)
    int32_t nchunks = 0;
    DevBuf active, iters, resid, tele, final_buf;
    int grid = 0;          // tuned cooperative grid (0: not tuned yet)
    std::vector<double> tune_ms;   // per candidate CTAs/SM, ms per body
    int cur = 0;
    double tol = 0.0;
    int64_t itermax = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t exec_iters = -1;
    int exec_cur = -1, exec_grid = -1;
};

namespace {

PrBatch* as_batch(grb_prbatch b) {
    PrBatch* x = reinterpret_cast<PrBatch*>(b);
    return (x && x->kind == Kind::PRBATCH) ? x : nullptr;
}

void drop_graph(PrBatch* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    B->exec_iters = -1;
}

PrParams batch_params(PrBatch* B) {
    PrParams p = plan_params_of(B->c, B->A);
    p.gmode = G_W;
    p.want_dang = 1;
    p.want_resid = 1;
    p.sinkbits = (const uint32_t*)B->sinkbits.p;
    p.dd = B->dd.p;
    p.rbuf[0] = B->r[0].p;
    p.rbuf[1] = B->r[1].p;
    p.wbuf[0] = B->w[0].p;
    p.wbuf[1] = B->w[1].p;
    p.graph_of = (const int32_t*)B->graph_of.p;
    p.g_active = (const int32_t*)B->active.p;
    p.g_tele = (const float*)B->tele.p;
    p.row_res = (float*)B->row_res.p;
    p.row_dang = (float*)B->row_dang.p;
    MgFinish& f = p.mg;
    f.ngraphs = B->ng;
    f.vptr = (const int64_t*)B->vptr.p;
    f.row_res = (const float*)B->row_res.p;
    f.row_dang = (const float*)B->row_dang.p;
    f.nchunks = B->nchunks;
    f.chunk_lo = (const int32_t*)B->chunk_lo.p;
    f.chunk_graph = (const int32_t*)B->chunk_graph.p;
    f.g_chunk = (const int32_t*)B->g_chunk.p;
    f.chunk_part = (double*)B->chunk_part.p;
    f.active = (int32_t*)B->active.p;
    f.iters = (int32_t*)B->iters.p;
    f.itermax = (int32_t)std::min<int64_t>(B->itermax, INT32_MAX);
    f.tol = B->tol;
    f.resid = (double*)B->resid.p;
    f.tele = (float*)B->tele.p;
    f.final_buf = (int32_t*)B->final_buf.p;
    f.damping = B->damping;
    return p;
}

grb_info init_state(PrBatch* B) {
    MgInit a;
    a.ngraphs = B->ng;
    a.vptr = (const int64_t*)B->vptr.p;
    a.dd = (const float*)B->dd.p;
    a.sinkbits = (const uint32_t*)B->sinkbits.p;
    a.r = (float*)B->r[0].p;
    a.w = (float*)B->w[0].p;
    a.active = (int32_t*)B->active.p;
    a.iters = (int32_t*)B->iters.p;
    a.resid = (double*)B->resid.p;
    a.tele = (float*)B->tele.p;
    a.final_buf = (int32_t*)B->final_buf.p;
    a.start_active = (B->itermax > 0 && 1.0 > B->tol) ? 1 : 0;
    a.damping = B->damping;
    B->cur = 0;
    B->c->stats.kernel_launches++;
    return cuda_check(B->c, launch_mg_init(B->c->stream, a), "batch init");
}

// `iters` bodies starting from buffer `from`, on stream st.
grb_info record_bodies(PrBatch* B, cudaStream_t st, int64_t iters, int from, int grid) {
    PrParams p = batch_params(B);
    cudaError_t e = cudaSuccess;
    for (int64_t k = 0; k < iters && e == cudaSuccess; ++k) e = launch_pr_batch(st, p, (int)((from + k) & 1), grid);
    return cuda_check(B->c, e, "batch body");
}

grb_info run_bodies(PrBatch* B, int64_t iters) {
    Ctx* c = B->c;
    grb_info st = GRB_SUCCESS;
    if (!B->exec || B->exec_iters != iters || B->exec_cur != B->cur || B->exec_grid != B->grid) {
        drop_graph(B);
        if (!c->capture_stream)
            st = cuda_check(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t g = nullptr;
        if (!st) st = cuda_check(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal),
                                 "batch capture");
        if (!st) {
            grb_info s1 = record_bodies(B, c->capture_stream, iters, B->cur, B->grid);
            grb_info s2 = cuda_check(c, cudaStreamEndCapture(c->capture_stream, &g), "batch capture");
            st = s1 ? s1 : s2;
        }
        if (!st) st = cuda_check(c, cudaGraphInstantiate(&B->exec, g, 0), "batch instantiate");
        if (g) cudaGraphDestroy(g);
        if (st) return st;
        B->exec_iters = iters;
        B->exec_cur = B->cur;
        B->exec_grid = B->grid;
    }
    st = cuda_check(c, cudaGraphLaunch(B->exec, c->stream), "batch launch");
    c->stats.kernel_launches += iters;
    B->cur = (int)((B->cur + iters) & 1);
    return st;
}

// Autotuner: every CTAs-per-SM count up to the occupancy limit, timed on
// `trial` bodies of this batch (from its start state); the fastest wins.
grb_info tune(PrBatch* B, int64_t trial) {
    Ctx* c = B->c;
    const int maxb = pr_batch_blocks_per_sm();
    const double save_tol = B->tol;
    const int64_t save_itermax = B->itermax;
    B->tol = -1.0;            // every graph runs every trial body
    B->itermax = INT32_MAX;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    grb_info st = cuda_check(c, cudaEventCreate(&e0), "tune");
    if (!st) st = cuda_check(c, cudaEventCreate(&e1), "tune");
    B->tune_ms.assign(maxb, 0.0);
    double best = 1e300;
    int best_b = maxb;
    for (int b = 1; b <= maxb && !st; ++b) {
        B->grid = b * c->sm_count;
        st = init_state(B);
        if (!st) st = run_bodies(B, trial);   // capture + warm-up
        if (!st) st = init_state(B);
        if (!st) st = cuda_check(c, cudaEventRecord(e0, c->stream), "tune");
        if (!st) st = run_bodies(B, trial);
        if (!st) st = cuda_check(c, cudaEventRecord(e1, c->stream), "tune");
        if (!st) st = cuda_check(c, cudaEventSynchronize(e1), "tune");
        float ms = 0.f;
        if (!st) st = cuda_check(c, cudaEventElapsedTime(&ms, e0, e1), "tune");
        if (!st) st = read_status(c);
        if (st) break;
        B->tune_ms[b - 1] = ms / (double)trial;
        if (ms < best) {
            best = ms;
            best_b = b;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    drop_graph(B);
    B->grid = best_b * c->sm_count;
    B->tol = save_tol;
    B->itermax = save_itermax;
    return st;
}

}  // namespace

void prbatch_destroy(PrBatch* B) {
    Ctx* c = B->c;
    cudaStreamSynchronize(c->stream);
    drop_graph(B);
    for (DevBuf* b : {&B->vptr, &B->graph_of, &B->dd, &B->sinkbits, &B->row_res, &B->row_dang, &B->r[0], &B->r[1],
                      &B->w[0], &B->w[1], &B->active, &B->iters, &B->resid, &B->tele, &B->final_buf, &B->chunk_lo,
                      &B->chunk_graph, &B->g_chunk, &B->chunk_part})
        buf_free(c, *b);
    if (B->A && B->A != B->A_in) matrix_unref(B->A);
    matrix_unref(B->A_in);
    B->kind = Kind::DEAD;
    delete B;
}

}  // namespace grb

using namespace grb;

extern "C" {

grb_info grb_prbatch_new(grb_prbatch* out, grb_matrix Am, int32_t ngraphs, const int64_t* vptr, double damping) {
    if (!out || !Am || !vptr) return GRB_NULL_POINTER;
    *out = nullptr;
    Matrix* A = reinterpret_cast<Matrix*>(Am);
    if (A->kind != Kind::MATRIX) return GRB_UNINITIALIZED_OBJECT;
    if (A->nrows != A->ncols || A->vals.p || A->nrows + A->nnz >= PR_INDEX_LIMIT) return GRB_INVALID_VALUE;
    if (ngraphs < 1 || !(damping >= 0.0 && damping < 1.0)) return GRB_INVALID_VALUE;
    if (vptr[0] != 0 || vptr[ngraphs] != A->nrows) return GRB_INVALID_VALUE;
    for (int32_t g = 0; g < ngraphs; ++g)
        if (vptr[g + 1] <= vptr[g]) return GRB_INVALID_VALUE;   // every graph has a vertex
    Ctx* c = A->ctx;
    grb_info st = ensure_plan(c, A);
    if (st) return st;
    PrBatch* B = new PrBatch();
    B->c = c;
    B->A = A;
    B->A_in = A;
    A->refs++;
    B->ng = ngraphs;
    B->n = A->nrows;
    B->damping = damping;
    B->vptr_h.assign(vptr, vptr + ngraphs + 1);
    const int64_t n = B->n;
    B->vptr = buf_alloc(c, sizeof(int64_t) * (ngraphs + 1));
    B->graph_of = buf_alloc(c, sizeof(int32_t) * n);
    B->dd = buf_alloc(c, sizeof(float) * n);
    B->sinkbits = buf_alloc(c, sizeof(uint32_t) * ((n + 31) / 32));
    B->row_res = buf_alloc(c, sizeof(float) * n);
    B->row_dang = buf_alloc(c, sizeof(float) * n);
    for (int q = 0; q < 2; ++q) {
        B->r[q] = buf_alloc(c, sizeof(float) * n);
        B->w[q] = buf_alloc(c, sizeof(float) * n);
    }
    B->active = buf_alloc(c, sizeof(int32_t) * ngraphs);
    B->iters = buf_alloc(c, sizeof(int32_t) * ngraphs);
    B->resid = buf_alloc(c, sizeof(double) * ngraphs);
    B->tele = buf_alloc(c, sizeof(float) * ngraphs);
    B->final_buf = buf_alloc(c, sizeof(int32_t) * ngraphs);
    // the fold's chunks: each graph's rows cut into pieces of at most
    // MG_CHUNK rows (host-side, from the offsets; fixed for the batch)
    std::vector<int32_t> clo, cgr, gch(ngraphs + 1);
    for (int32_t g = 0; g < ngraphs; ++g) {
        gch[g] = (int32_t)clo.size();
        for (int64_t i = vptr[g]; i < vptr[g + 1]; i += MG_CHUNK) {
            clo.push_back((int32_t)i);
            cgr.push_back(g);
        }
    }
    gch[ngraphs] = (int32_t)clo.size();
    B->nchunks = (int32_t)clo.size();
    clo.push_back((int32_t)n);
    B->chunk_lo = buf_alloc(c, sizeof(int32_t) * clo.size());
    B->chunk_graph = buf_alloc(c, sizeof(int32_t) * cgr.size());
    B->g_chunk = buf_alloc(c, sizeof(int32_t) * gch.size());
    B->chunk_part = buf_alloc(c, sizeof(double) * 2 * cgr.size());
    DevBuf deg = buf_alloc(c, sizeof(int32_t) * n), pres = buf_alloc(c, (size_t)n),
           bad = buf_alloc(c, sizeof(unsigned long long));
    for (DevBuf* b : {&B->vptr, &B->graph_of, &B->dd, &B->sinkbits, &B->row_res, &B->row_dang, &B->r[0], &B->r[1],
                      &B->w[0], &B->w[1], &B->active, &B->iters, &B->resid, &B->tele, &B->final_buf, &B->chunk_lo,
                      &B->chunk_graph, &B->g_chunk, &B->chunk_part, &deg, &pres, &bad})
        if (!b->p) st = GRB_OUT_OF_MEMORY;
    unsigned long long nbad = 0;
    if (!st) st = cuda_check(c, cudaMemcpyAsync(B->vptr.p, vptr, sizeof(int64_t) * (ngraphs + 1),
                                                cudaMemcpyHostToDevice, c->stream), "batch offsets");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(B->chunk_lo.p, clo.data(), sizeof(int32_t) * clo.size(),
                                                cudaMemcpyHostToDevice, c->stream), "batch chunks");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(B->chunk_graph.p, cgr.data(), sizeof(int32_t) * cgr.size(),
                                                cudaMemcpyHostToDevice, c->stream), "batch chunks");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(B->g_chunk.p, gch.data(), sizeof(int32_t) * gch.size(),
                                                cudaMemcpyHostToDevice, c->stream), "batch chunks");
    if (!st) {
        c->stats.kernel_launches += 4;
        st = cuda_check(c, launch_mg_graph_of(c->stream, ngraphs, (const int64_t*)B->vptr.p, (int32_t)n,
                                              (const int32_t*)A->row_ptr.p, (const int32_t*)A->col_idx.p,
                                              (int32_t*)B->graph_of.p, (unsigned long long*)bad.p), "graph ids");
        if (!st) st = cuda_check(c, launch_col_degree(c->stream, n, A->nnz, (const int32_t*)A->col_idx.p,
                                                      (int32_t*)deg.p, (uint8_t*)pres.p), "out-degree");
        if (!st) st = cuda_check(c, launch_ppr_divisor(c->stream, (int32_t)n, (const int32_t*)deg.p, damping,
                                                       (float*)B->dd.p, (uint32_t*)B->sinkbits.p), "divisor");
        if (!st) st = cuda_check(c, cudaMemcpyAsync(&nbad, bad.p, sizeof(nbad), cudaMemcpyDeviceToHost, c->stream),
                                 "graph ids");
        if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "batch setup");
    }
    if (!st && nbad) st = GRB_INVALID_VALUE;   // an edge between two graphs
    // Renumber each graph's vertices by descending out-degree inside its own
    // block (the block-diagonal structure stays): the most-gathered entries
    // of w become neighbours, as for the single-graph loop.
    if (!st && c->relabel) {
        auto af = [](void* x, size_t b2) { return dev_alloc((Ctx*)x, b2); };
        auto ff = [](void* x, void* q, size_t b2) { dev_free((Ctx*)x, q, b2); };
        DevBuf n2o = buf_alloc(c, sizeof(int32_t) * n), o2n = buf_alloc(c, sizeof(int32_t) * n);
        Matrix* R = new Matrix();
        R->ctx = c;
        R->type = A->type;
        R->nrows = A->nrows;
        R->ncols = A->ncols;
        R->nnz = A->nnz;
        R->iso_val = A->iso_val;
        R->nonempty_rows = A->nonempty_rows;
        R->row_ptr = buf_alloc(c, sizeof(int32_t) * (size_t)(n + 1));
        R->col_idx = buf_alloc(c, sizeof(int32_t) * (size_t)padded_nnz(A->nnz));
        if (!n2o.p || !o2n.p || !R->row_ptr.p || !R->col_idx.p) st = GRB_OUT_OF_MEMORY;
        if (!st) {
            c->stats.kernel_launches += 4;
            st = cuda_check(c, block_degree_order(c->stream, (int32_t)n, (const int32_t*)A->col_idx.p, A->nnz,
                                                  (const int32_t*)B->graph_of.p, (int32_t*)n2o.p, (int32_t*)o2n.p, af,
                                                  ff, c), "block order");
        }
        if (!st) {
            RelabelArgs ra;
            ra.n = (int32_t)n;
            ra.nnz = A->nnz;
            ra.row_ptr = (const int32_t*)A->row_ptr.p;
            ra.col_idx = (const int32_t*)A->col_idx.p;
            ra.new_row_ptr = (int32_t*)R->row_ptr.p;
            ra.new_col_idx = (int32_t*)R->col_idx.p;
            ra.new2old = (int32_t*)n2o.p;
            ra.old2new = (int32_t*)o2n.p;
            ra.top_h = 0;
            c->stats.kernel_launches += 3;
            st = cuda_check(c, relabel_build(c->stream, ra, af, ff, c), "block relabel");
        }
        if (!st) {
            B->old2new_h.resize(n);
            st = cuda_check(c, cudaMemcpy(B->old2new_h.data(), o2n.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost),
                            "block relabel");
        }
        buf_free(c, n2o);
        buf_free(c, o2n);
        if (!st) st = ensure_plan(c, R);
        if (st) {
            matrix_unref(R);
            B->old2new_h.clear();
        } else {
            B->A = R;
            // graph ids and divisors in the new numbering
            c->stats.kernel_launches += 4;
            st = cuda_check(c, launch_mg_graph_of(c->stream, ngraphs, (const int64_t*)B->vptr.p, (int32_t)n,
                                                  (const int32_t*)R->row_ptr.p, (const int32_t*)R->col_idx.p,
                                                  (int32_t*)B->graph_of.p, (unsigned long long*)bad.p), "graph ids");
            if (!st) st = cuda_check(c, launch_col_degree(c->stream, n, R->nnz, (const int32_t*)R->col_idx.p,
                                                          (int32_t*)deg.p, (uint8_t*)pres.p), "out-degree");
            if (!st) st = cuda_check(c, launch_ppr_divisor(c->stream, (int32_t)n, (const int32_t*)deg.p, damping,
                                                           (float*)B->dd.p, (uint32_t*)B->sinkbits.p), "divisor");
            if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "batch setup");
        }
    }
    buf_free(c, deg);
    buf_free(c, pres);
    buf_free(c, bad);
    if (st) {
        prbatch_destroy(B);
        return st;
    }
    *out = reinterpret_cast<grb_prbatch>(B);
    return GRB_SUCCESS;
}

grb_info grb_prbatch_tune(grb_prbatch Bh, int64_t trial_bodies, double* ms_per_body, int32_t cap, int32_t* chosen) {
    PrBatch* B = as_batch(Bh);
    if (!Bh) return GRB_NULL_POINTER;
    if (!B) return GRB_UNINITIALIZED_OBJECT;
    if (trial_bodies < 1 || trial_bodies > 1000) return GRB_INVALID_VALUE;
    grb_info st = tune(B, trial_bodies);
    if (st) return st;
    for (int32_t q = 0; ms_per_body && q < cap; ++q) ms_per_body[q] = q < (int32_t)B->tune_ms.size() ? B->tune_ms[q] : 0.0;
    if (chosen) *chosen = B->grid / B->c->sm_count;
    return GRB_SUCCESS;
}

grb_info grb_prbatch_run(grb_prbatch Bh, double tol, int64_t itermax, int64_t chunk) {
    NvtxRange range("grb: graph batch solve");
    PrBatch* B = as_batch(Bh);
    if (!Bh) return GRB_NULL_POINTER;
    if (!B) return GRB_UNINITIALIZED_OBJECT;
    if (itermax < 0 || itermax > INT32_MAX || chunk < 1) return GRB_INVALID_VALUE;
    Ctx* c = B->c;
    grb_info st = GRB_SUCCESS;
    if (!B->grid) st = tune(B, 3);
    if (st) return st;
    B->tol = tol;
    B->itermax = itermax;
    drop_graph(B);   // tol / itermax are launch parameters of the fold kernel
    st = init_state(B);
    // bodies in chunks of `chunk` (one CUDA-graph launch each) until every
    // graph's loop has ended
    std::vector<int32_t> act(B->ng);
    int64_t done = 0;
    while (!st && done < itermax) {
        const int64_t k = std::min<int64_t>(chunk, itermax - done);
        st = run_bodies(B, k);
        done += k;
        if (!st) st = cuda_check(c, cudaMemcpyAsync(act.data(), B->active.p, sizeof(int32_t) * B->ng,
                                                    cudaMemcpyDeviceToHost, c->stream), "batch state");
        if (!st) st = read_status(c);
        if (!st && std::none_of(act.begin(), act.end(), [](int32_t a) { return a != 0; })) break;
    }
    return st;
}

grb_info grb_prbatch_result(grb_prbatch Bh, float* ranks, int64_t* iters, double* resid) {
    PrBatch* B = as_batch(Bh);
    if (!Bh) return GRB_NULL_POINTER;
    if (!B) return GRB_UNINITIALIZED_OBJECT;
    Ctx* c = B->c;
    std::vector<int32_t> it(B->ng), fb(B->ng), act(B->ng);
    std::vector<double> rs(B->ng);
    grb_info st = cuda_check(c, cudaMemcpyAsync(it.data(), B->iters.p, 4 * B->ng, cudaMemcpyDeviceToHost, c->stream),
                             "batch result");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(fb.data(), B->final_buf.p, 4 * B->ng, cudaMemcpyDeviceToHost,
                                                c->stream), "batch result");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(act.data(), B->active.p, 4 * B->ng, cudaMemcpyDeviceToHost,
                                                c->stream), "batch result");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(rs.data(), B->resid.p, 8 * B->ng, cudaMemcpyDeviceToHost, c->stream),
                             "batch result");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "batch result");
    if (st) return st;
    if (ranks) {
        // each graph's rank from the buffer its last body wrote (an active
        // graph's from the current one)
        std::vector<float> h[2];
        for (int q = 0; q < 2 && !st; ++q) {
            h[q].resize(B->n);
            st = cuda_check(c, cudaMemcpy(h[q].data(), B->r[q].p, sizeof(float) * B->n, cudaMemcpyDeviceToHost),
                            "batch result");
        }
        if (st) return st;
        for (int32_t g = 0; g < B->ng; ++g) {
            const int src = act[g] ? B->cur : (fb[g] & 1);
            if (B->old2new_h.empty()) {
                std::memcpy(ranks + B->vptr_h[g], h[src].data() + B->vptr_h[g],
                            sizeof(float) * (size_t)(B->vptr_h[g + 1] - B->vptr_h[g]));
            } else {
                for (int64_t i = B->vptr_h[g]; i < B->vptr_h[g + 1]; ++i) ranks[i] = h[src][B->old2new_h[i]];
            }
        }
    }
    for (int32_t g = 0; g < B->ng; ++g) {
        if (iters) iters[g] = it[g];
        if (resid) resid[g] = rs[g];
    }
    return GRB_SUCCESS;
}

}  // extern "C"
