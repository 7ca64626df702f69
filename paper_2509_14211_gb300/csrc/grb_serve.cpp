// Serving loop for personalised-PageRank queries (grb_ppr_serve): continuous
// batching on top of a grb_ppr.  The graph and every in-flight query's state
// stay resident on the device; a query is admitted into a free slot as soon
// as it has arrived and a slot is free, and joins the bodies already running
// for the others; a finished query leaves its slot at the next scheduling
// step.  The number of slots is chosen from the free device memory.
//
// Host loop (one thread):
//   admit every arrived query into a free slot (grb_ppr_set);
//   if nothing is in flight, sleep until the next arrival;
//   otherwise run `chunk` bodies (one CUDA-graph launch), read the slot
//   states, and retire the finished slots (latency = now - arrival).
// A query's result does not depend on when it was admitted or on its
// neighbours (see grb_ppr).
#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "grb_core.h"

using namespace grb;

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

}  // namespace

extern "C" {

grb_info grb_ppr_serve(grb_matrix AT, const grb_serve_config* cfg, int64_t nq, const double* arrival_s,
                       const int64_t* seed_ptr, const int32_t* seed_idx, grb_serve_result* out) {
    if (!AT || !cfg || !out || (nq > 0 && (!arrival_s || !seed_ptr || !seed_idx))) return GRB_NULL_POINTER;
    if (nq < 0 || cfg->chunk < 1 || cfg->itermax < 0 || !(cfg->mem_fraction > 0.0 && cfg->mem_fraction <= 1.0) ||
        cfg->slots < 0 || cfg->slots > GRB_PPR_MAX_SLOTS)
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
    std::vector<int32_t> slot_q(S, -1), free_slots, active(GRB_PPR_MAX_SLOTS);
    std::vector<int64_t> its(GRB_PPR_MAX_SLOTS);
    std::vector<double> res(GRB_PPR_MAX_SLOTS);
    for (int32_t s = S - 1; s >= 0; --s) free_slots.push_back(s);
    int64_t next = 0, done = 0, in_flight = 0, steps = 0, max_in_flight = 0;
    const double t0 = now_s();
    while (done < nq && !st) {
        double t = now_s() - t0;
        while (next < nq && arrival_s[next] <= t && !free_slots.empty()) {
            const int32_t s = free_slots.back();
            free_slots.pop_back();
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
            free_slots.push_back(s);
            --in_flight;
            ++done;
        }
    }
    out->wall_s = now_s() - t0;
    out->steps = steps;
    out->max_in_flight = max_in_flight;
    void* pp = P;
    grb_free(&pp);
    return st;
}

}  // extern "C"
