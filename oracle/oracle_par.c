/*
 * CPU ORACLE, MULTI-CORE TIMING VARIANT -- test and benchmark infrastructure
 * only (the tests and the benchmark's CPU-baseline leg load it; the GPU
 * library never does, and it shares no code with it).
 *
 * The same PageRank as oracle_pagerank in oracle.c -- the pagerank_gap
 * listing of §IV (Fig. "The PageRank implementation in AppGrB"), every
 * method materialised into a new vector, FP64 -- with each vector held densely
 * as values plus presence flags, so that every element-wise method, the mxv
 * and the two reductions are plain loops over the n rows, run by OpenMP on
 * all host cores.  The GraphBLAS semantics are unchanged: ewise_add is a
 * union of the present entries, ewise_mult an intersection, mxv gives an entry
 * only to rows with a contributing term, and each row sums its terms in
 * ascending column order.  Only the order in which the reductions add their
 * terms depends on the thread count, so the results agree with oracle.c to
 * FP64 rounding, not bit for bit; a CPU test checks that.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { int64_t n; double* val; unsigned char* has; } dvec;

int oracle_par_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int dv_alloc(dvec* v, int64_t n) {
    v->n = n;
    v->val = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    v->has = (unsigned char*)malloc((size_t)(n > 0 ? n : 1));
    return (v->val && v->has) ? 0 : -1;
}

static void dv_release(dvec* v) { free(v->val); free(v->has); v->val = NULL; v->has = NULL; }

/* full(s): every entry present and equal to s */
static int dv_full(dvec* v, int64_t n, double s) {
    if (dv_alloc(v, n)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) { v->val[i] = s; v->has[i] = 1; }
    return 0;
}

static int dv_copy(dvec* out, const dvec* in) {
    if (dv_alloc(out, in->n)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < in->n; ++i) { out->val[i] = in->val[i]; out->has[i] = in->has[i]; }
    return 0;
}

/* Sum of the present entries (the monoid plus). */
static double dv_reduce_plus(const dvec* u) {
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int64_t i = 0; i < u->n; ++i) if (u->has[i]) s += u->val[i];
    return s;
}

/* See oracle_pagerank (oracle.c) for the listing; this follows it line by
 * line.  Outputs: r_out (n, dense), *iters = bodies executed, rdiff_hist[k]
 * = rdiff after body k. */
int oracle_pagerank_par(int64_t n, const int64_t* ptr, const int64_t* col, const int64_t* outdeg,
                        double damping, double tolerance, int64_t itermax, int mode,
                        double* r_out, int64_t* iters, double* rdiff_hist) {
    if (n < 1) return -2;
    const double teleport = (1.0 - damping) / (double)n;
    double rdiff = 1.0;
    dvec r, d, sinks, vt;
    /* r = full(1/n) */
    if (dv_full(&r, n, 1.0 / (double)n)) return -1;
    /* d = ewise_add(max(x/damping, y), conv(out_degree), full(1/damping)):
     * the union is every index; where the degree is present (> 0) both
     * operands are, and the operator applies */
    if (dv_alloc(&d, n)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double y = 1.0 / damping;
        if (outdeg[i] > 0) { const double q = (double)outdeg[i] / damping; d.val[i] = q > y ? q : y; }
        else d.val[i] = y;
        d.has[i] = 1;
    }
    /* sinks: the vertices without out-edges (value 1) */
    if (dv_alloc(&sinks, n)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) { sinks.val[i] = 1.0; sinks.has[i] = outdeg[i] == 0; }
    if (dv_full(&vt, n, teleport)) return -1;

    int rc = 0;
    int64_t iter = 1;
    while (iter <= itermax && rdiff > tolerance) {
        dvec t, w, s, rt, tmp, diff;
        if (dv_copy(&t, &r)) { rc = -1; break; }                                      /* t = r */
        if (dv_alloc(&w, n)) { rc = -1; break; }                                      /* w = t ./ d */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            w.has[i] = t.has[i] && d.has[i];
            w.val[i] = w.has[i] ? t.val[i] / d.val[i] : 0.0;
        }
        if (dv_alloc(&s, n)) { rc = -1; break; }                                      /* s = A^T (+.second) w */
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            int found = 0;
            for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) {
                const int64_t j = col[p];
                if (!w.has[j]) continue;
                acc = acc + w.val[j];
                found = 1;
            }
            s.val[i] = found ? acc : 0.0;
            s.has[i] = (unsigned char)found;
        }
        dv_release(&w);
        if (mode == 1) {
            /* D = reduce(+, ewise_mult(first, t, sinks)); rt = vt + full(damping D / n) */
            dvec z;
            if (dv_alloc(&z, n)) { rc = -1; break; }
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) { z.has[i] = t.has[i] && sinks.has[i]; z.val[i] = z.has[i] ? t.val[i] : 0.0; }
            const double D = dv_reduce_plus(&z);
            dv_release(&z);
            if (dv_alloc(&rt, n)) { rc = -1; break; }
            const double spread = damping * D / (double)n;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) { rt.has[i] = 1; rt.val[i] = vt.has[i] ? vt.val[i] + spread : spread; }
        } else {
            if (dv_copy(&rt, &vt)) { rc = -1; break; }
        }
        if (dv_alloc(&tmp, n)) { rc = -1; break; }                                    /* r = rt + s */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            tmp.has[i] = rt.has[i] || s.has[i];
            tmp.val[i] = rt.has[i] && s.has[i] ? rt.val[i] + s.val[i] : (rt.has[i] ? rt.val[i] : s.val[i]);
        }
        dv_release(&s); dv_release(&rt);
        dv_release(&r); r = tmp;
        if (dv_alloc(&diff, n)) { rc = -1; break; }                                   /* t = |t - r| */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            diff.has[i] = t.has[i] || r.has[i];
            diff.val[i] = t.has[i] && r.has[i] ? fabs(t.val[i] - r.val[i]) : (t.has[i] ? t.val[i] : r.val[i]);
        }
        rdiff = dv_reduce_plus(&diff);                                                /* rdiff = sum(t) */
        dv_release(&diff); dv_release(&t);
        if (rdiff_hist) rdiff_hist[iter - 1] = rdiff;
        iter += 1;
    }
    if (rc == 0) {
        for (int64_t i = 0; i < n; ++i) r_out[i] = r.has[i] ? r.val[i] : 0.0;
        *iters = iter - 1;
    }
    dv_release(&r); dv_release(&d); dv_release(&sinks); dv_release(&vt);
    return rc;
}
