// Serving loop for personalised-PageRank queries (grb_ppr_serve): continuous
// batching on top of a grb_ppr.  The graph and every in-flight query's state
// stay resident on the device; a query is admitted into a free slot as soon
// as it has arrived and a slot is free, and joins the bodies already running
// for the others; a finished query leaves its slot at the next scheduling
// step.  The number of slots is chosen from the free device memory.
//
// Host loop (one thread):
//   when no query holds a slot and at most `single_max` arrived queries
//   wait, answer the oldest one alone on the single-vector loop (below);
//   otherwise admit every arrived query into a free slot (grb_ppr_set) --
//   while the slots the current free device memory allows are not all busy;
//   if nothing is in flight, sleep until the next arrival;
//   otherwise run `chunk` bodies (one CUDA-graph launch), read the slot
//   states, and retire the finished slots (latency = now - arrival).
// A slot query's result does not depend on when it was admitted or on its
// neighbours (see grb_ppr).
//
// Single-vector loop.  A k-tile of slots costs the same per body whether one
// of its slots is live or all of them are, so a lone query would wait for
// a whole k-tile's bodies.  At low load each query instead runs alone as the
// fused persistent PageRank loop (the kernel of grb_iterate_end, on the
// degree-ordered copy of A^T with the shared-memory hot copy) with its
// teleport term (1-d)/|S| added on its seed rows: the same iteration and loop
// test as a slot, with the rows summed in another order, so the result
// agrees with the slot result to FP32 rounding (not bit for bit).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <functional>
#include <queue>
#include <thread>
#include <vector>

#include "grb_core.h"

using namespace grb;

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

// The single-vector personalised loop: buffers in the loop's vertex order,
// allocated once per serving call.
struct SingleLoop {
    Ctx* c = nullptr;
    Matrix* A = nullptr;    // the caller's A^T
    Matrix* AL = nullptr;   // the matrix the loop runs on (A or its degree-ordered copy)
    int64_t n = 0;
    double damping = 0.85;
    int32_t itermax = 0;
    DevBuf dd, sinkbits, seedbits, r0, rb[2], wb[2], hist, slots, out, seeds;
    int64_t seeds_cap = 0;
    int grid = 0;
    int32_t hot_n = 0;

    grb_info setup(Ctx* cx, Matrix* Am, double d, int64_t itmax) {
        c = cx;
        A = Am;
        n = A->nrows;
        damping = d;
        itermax = (int32_t)std::min<int64_t>(std::max<int64_t>(itmax, 1), INT_MAX - 16);
        grb_info st = GRB_SUCCESS;
        AL = A;
        if (c->relabel) {
            st = ensure_relabel(c, A);
            if (!st && A->rel) AL = A->rel;
        }
        if (!st) st = ensure_plan(c, AL);
        if (!st) st = ensure_coldeg(c, AL);
        if (st) return st;
        const size_t fb = sizeof(float) * (size_t)n, bb = sizeof(uint32_t) * (size_t)((n + 31) / 32);
        dd = buf_alloc(c, fb);
        sinkbits = buf_alloc(c, bb);
        seedbits = buf_alloc(c, bb);
        r0 = buf_alloc(c, fb);
        for (int q = 0; q < 2; ++q) {
            rb[q] = buf_alloc(c, fb);
            wb[q] = buf_alloc(c, fb);
        }
        hist = buf_alloc(c, sizeof(double) * (size_t)itermax);
        slots = buf_alloc(c, sizeof(double) * 8);
        out = buf_alloc(c, fb);
        for (DevBuf* b : {&dd, &sinkbits, &seedbits, &r0, &rb[0], &rb[1], &wb[0], &wb[1], &hist, &slots, &out})
            if (!b->p) return GRB_OUT_OF_MEMORY;
        // the divisor max(outdeg, 1) / damping and the sinks, in AL's order
        c->stats.kernel_launches++;
        st = cuda_check(c, launch_ppr_divisor(c->stream, (int32_t)n, (const int32_t*)AL->coldeg.p, damping,
                                              (float*)dd.p, (uint32_t*)sinkbits.p), "single-loop divisor");
        if (st) return st;
        // the hot copy as in the device loop (degree order only)
        if (AL != A && c->hot_bytes >= 16) {
            const int64_t room = (int64_t)PR_SMEM_PER_BLOCK_MAX - (int64_t)PR_HOT_STATIC_SMEM;
            const int64_t bytes = std::min<int64_t>(c->hot_bytes, room);
            hot_n = (int32_t)(std::min<int64_t>(n, bytes / (int64_t)sizeof(float)) & ~(int64_t)3);
        }
        int nb = pr_pers_blocks_per_sm(hot_n);
        if (nb <= 0 && hot_n > 0) {
            hot_n = 0;
            nb = pr_pers_blocks_per_sm(0);
        }
        if (nb <= 0) return GRB_DEVICE_ERROR;
        const int wpb = (hot_n > 0 ? PR_HOT_BLOCK : PR_BLOCK) / 32;
        const int64_t need = (AL->plan->ntiles + wpb - 1) / wpb;
        grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nb * c->sm_count, need));
        return GRB_SUCCESS;
    }

    // One query to its loop test's end; the rank goes to host_out (n
    // floats, caller's vertex order) when given.
    grb_info run(const std::vector<int32_t>& S, double tol, int64_t itmax, float* host_out, int64_t* iters,
                 double* resid) {
        const size_t fb = sizeof(float) * (size_t)n, bb = sizeof(uint32_t) * (size_t)((n + 31) / 32);
        grb_info st = GRB_SUCCESS;
        if ((int64_t)S.size() > seeds_cap) {
            buf_free(c, seeds);
            seeds = buf_alloc(c, sizeof(int32_t) * S.size());
            if (!seeds.p) return GRB_OUT_OF_MEMORY;
            seeds_cap = (int64_t)S.size();
        }
        st = cuda_check(c, cudaMemcpyAsync(seeds.p, S.data(), sizeof(int32_t) * S.size(), cudaMemcpyHostToDevice,
                                           c->stream), "single-loop seeds");
        if (!st) st = cuda_check(c, cudaMemsetAsync(r0.p, 0, fb, c->stream), "single-loop start");
        if (!st) st = cuda_check(c, cudaMemsetAsync(seedbits.p, 0, bb, c->stream), "single-loop start");
        if (!st) st = cuda_check(c, cudaMemsetAsync(slots.p, 0, sizeof(double) * 8, c->stream), "single-loop start");
        // r_0 = v = 1/|S| on the seeds; teleport term (1-d) v
        const float v0 = (float)(1.0 / (double)S.size());
        c->stats.kernel_launches++;
        if (!st)
            st = cuda_check(c, launch_pr_seed_scatter(c->stream, (int32_t)S.size(), (const int32_t*)seeds.p,
                                                      AL != A ? (const int32_t*)A->old2new.p : nullptr, v0,
                                                      (float*)r0.p, (uint32_t*)seedbits.p), "single-loop seeds");
        double* sl = (double*)slots.p;
        PrParams p = plan_params_of(c, AL);
        p.gmode = G_W;
        p.has_base = 1;
        p.tele_from_slot = 1;
        p.tele_slot = sl + 3;
        p.want_dang = 1;
        p.sinkbits = (const uint32_t*)sinkbits.p;
        // teleport scalar d D / n: the reduction's FP64 value times d / n
        p.chain.n = 2;
        p.chain.ops[0].code = GRB_FIRST;
        p.chain.c[0] = 0.0;
        p.chain.rtype[0] = GRB_FP64;
        p.chain.ops[1].code = GRB_TIMES;
        p.chain.c[1] = damping / (double)n;
        p.chain.rtype[1] = GRB_FP64;
        p.want_resid = 1;
        p.resid_slot = sl + 1;
        p.resid_type = GRB_FP64;
        p.dang_slot = sl + 2;
        p.dd = dd.p;
        p.out.type = GRB_FP32;
        p.out.full = 1;
        p.iters = (int32_t)std::min<int64_t>(itmax, itermax);
        p.tol = tol;
        p.rdiff0 = 1.0;
        p.hist = (double*)hist.p;
        p.iters_done = (int64_t*)(sl + 0);
        p.r0 = r0.p;
        p.rbuf[0] = rb[0].p;
        p.rbuf[1] = rb[1].p;
        p.wbuf[0] = wb[0].p;
        p.wbuf[1] = wb[1].p;
        p.hot_n = hot_n;
        p.pers_bits = (const uint32_t*)seedbits.p;
        p.pers_val = (float)((1.0 - damping) * (1.0 / (double)S.size()));
        c->stats.kernel_launches++;
        if (!st) st = cuda_check(c, launch_pr_pers(c->stream, p, grid), "single-loop kernel");
        double h[8] = {0};
        if (!st) st = cuda_check(c, cudaMemcpyAsync(h, slots.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
                                 "single-loop result");
        if (!st) st = read_status(c);
        if (st) return st;
        int64_t K = 0;
        std::memcpy(&K, &h[0], sizeof(int64_t));
        *iters = K;
        *resid = K > 0 ? h[1] : 1.0;
        if (host_out) {
            const void* last = K > 0 ? rb[(K - 1) & 1].p : r0.p;
            if (AL != A) {
                c->stats.kernel_launches++;
                st = cuda_check(c, launch_permute(c->stream, (int32_t)n, (const int32_t*)A->old2new.p, last, out.p, 4),
                                "single-loop rank");
                last = out.p;
            }
            if (!st) st = cuda_check(c, cudaMemcpyAsync(host_out, last, fb, cudaMemcpyDeviceToHost, c->stream),
                                     "single-loop rank");
            if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "single-loop rank");
        }
        return st;
    }

    void release() {
        if (!c) return;
        for (DevBuf* b : {&dd, &sinkbits, &seedbits, &r0, &rb[0], &rb[1], &wb[0], &wb[1], &hist, &slots, &out, &seeds})
            buf_free(c, *b);
    }
};

}  // namespace

extern "C" {

grb_info grb_ppr_serve(grb_matrix AT, const grb_serve_config* cfg, int64_t nq, const double* arrival_s,
                       const int64_t* seed_ptr, const int32_t* seed_idx, grb_serve_result* out) {
    if (!AT || !cfg || !out || (nq > 0 && (!arrival_s || !seed_ptr || !seed_idx))) return GRB_NULL_POINTER;
    if (nq < 0 || cfg->chunk < 1 || cfg->itermax < 0 || !(cfg->mem_fraction > 0.0 && cfg->mem_fraction <= 1.0) ||
        cfg->slots < 0 || cfg->slots > GRB_PPR_MAX_SLOTS || cfg->single_max < 0)
        return GRB_INVALID_VALUE;
    if (!out->latency_s || !out->iters || !out->resid) return GRB_NULL_POINTER;
    for (int64_t q = 0; q < nq; ++q) {
        if (seed_ptr[q + 1] <= seed_ptr[q]) return GRB_INVALID_VALUE;          // every query has a seed
        if (q > 0 && arrival_s[q] < arrival_s[q - 1]) return GRB_INVALID_VALUE;  // arrivals in order
    }
    Matrix* A = reinterpret_cast<Matrix*>(AT);
    if (A->kind != Kind::MATRIX) return GRB_UNINITIALIZED_OBJECT;
    const int64_t n = A->nrows;

    // admission by memory: 4 rank/gather vectors of n floats per slot, plus
    // the slot's share of the per-tile carries
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return GRB_DEVICE_ERROR;
    const double per_slot = 16.0 * (double)n + 8.0 * (double)padded_nnz(A->nnz) / PR_NZTILE + 64.0;
    int64_t cap = (int64_t)((double)free_b * cfg->mem_fraction / per_slot);
    cap = std::min<int64_t>(cap, GRB_PPR_MAX_SLOTS);
    if (cfg->slots > 0) cap = std::min<int64_t>(cap, cfg->slots);
    if (cap >= PPR_LANES) cap = cap / PPR_LANES * PPR_LANES;
    if (cap < 1) return GRB_OUT_OF_MEMORY;

    grb_ppr P = nullptr;
    grb_info st = grb_ppr_new(&P, AT, cfg->damping, (int32_t)cap);
    if (st) return st;
    // vector width by the autotuner, before the clock starts
    st = grb_ppr_tune(P, 2, nullptr, &out->vector_width);
    if (st) {
        void* pp = P;
        grb_free(&pp);
        return st;
    }
    const int32_t S = (int32_t)std::min<int64_t>(cap, GRB_PPR_MAX_SLOTS);
    out->slots = S;
    out->single_queries = 0;
    SingleLoop one;
    if (cfg->single_max > 0) st = one.setup(A->ctx, A, cfg->damping, cfg->itermax);
    std::vector<int32_t> slot_q(S, -1), active(GRB_PPR_MAX_SLOTS);
    std::vector<int64_t> its(GRB_PPR_MAX_SLOTS);
    std::vector<double> res(GRB_PPR_MAX_SLOTS);
    // the lowest free slot first: queries pack into the low k-tiles, and a
    // k-tile with no active slot is skipped by the body, so a higher k-tile
    // runs only while more queries are in flight than the lower ones hold
    std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>> free_slots;
    for (int32_t s = 0; s < S; ++s) free_slots.push(s);
    // bytes the slot buffers hold (already allocated): free memory is read
    // again at every admission and counted together with them
    const double pool_b = per_slot * (double)S;
    int64_t next = 0, done = 0, in_flight = 0, steps = 0, max_in_flight = 0;
    const double t0 = now_s();
    while (done < nq && !st) {
        double t = now_s() - t0;
        if (cfg->single_max > 0 && in_flight == 0) {
            int64_t waiting = 0;
            while (next + waiting < nq && arrival_s[next + waiting] <= t) ++waiting;
            if (waiting >= 1 && waiting <= cfg->single_max) {
                NvtxRange one_q("grb: single-vector query");
                std::vector<int32_t> sd(seed_idx + seed_ptr[next], seed_idx + seed_ptr[next + 1]);
                for (int32_t x : sd)
                    if (x < 0 || x >= n) st = GRB_INVALID_INDEX;
                if (st) break;
                std::sort(sd.begin(), sd.end());
                sd.erase(std::unique(sd.begin(), sd.end()), sd.end());
                int64_t k = 0;
                double r = 0.0;
                st = one.run(sd, cfg->tol, cfg->itermax, out->ranks ? out->ranks + (size_t)next * (size_t)n : nullptr,
                             &k, &r);
                if (st) break;
                out->latency_s[next] = (now_s() - t0) - arrival_s[next];
                out->iters[next] = k;
                out->resid[next] = r;
                out->single_queries++;
                max_in_flight = std::max<int64_t>(max_in_flight, 1);
                ++next;
                ++done;
                continue;
            }
        }
        // slots usable now: the pool, or fewer if other users of the device
        // have taken memory since the start
        int64_t usable = S;
        {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
                usable = std::min<int64_t>(S, (int64_t)(((double)fr + pool_b) * cfg->mem_fraction / per_slot));
            else
                cudaGetLastError();
            usable = std::max<int64_t>(usable, 1);
        }
        while (next < nq && arrival_s[next] <= t && !free_slots.empty() && in_flight < usable) {
            const int32_t s = free_slots.top();
            free_slots.pop();
            st = grb_ppr_set(P, s, seed_idx + seed_ptr[next], seed_ptr[next + 1] - seed_ptr[next], cfg->tol,
                             cfg->itermax);
            if (st) break;
            slot_q[s] = (int32_t)next;
            ++next;
            ++in_flight;
        }
        if (st) break;
        max_in_flight = std::max(max_in_flight, in_flight);
        if (in_flight == 0) {
            if (next < nq) {
                const double wait = arrival_s[next] - (now_s() - t0);
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
            }
            continue;
        }
        NvtxRange step("grb: serving step");
        st = grb_ppr_run(P, cfg->chunk);
        if (!st) st = grb_ppr_status(P, active.data(), its.data(), res.data());
        if (st) break;
        ++steps;
        t = now_s() - t0;
        for (int32_t s = 0; s < S && !st; ++s) {
            const int32_t q = slot_q[s];
            if (q < 0 || active[s]) continue;
            out->latency_s[q] = t - arrival_s[q];
            out->iters[q] = its[s];
            out->resid[q] = res[s];
            if (out->ranks) st = grb_ppr_get(P, s, out->ranks + (size_t)q * (size_t)n, 0);
            slot_q[s] = -1;
            free_slots.push(s);
            --in_flight;
            ++done;
        }
    }
    out->wall_s = now_s() - t0;
    out->steps = steps;
    out->max_in_flight = max_in_flight;
    one.release();
    void* pp = P;
    grb_free(&pp);
    return st;
}

}  // extern "C"
