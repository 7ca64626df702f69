/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A plain, slow, blocking-mode GraphBLAS subset in FP64, written so that a
 * reader can check it against the paper by eye.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the GPU library.
 *
 * Every operation materialises its result as a sparse vector (sorted index
 * list + values), the "SparseVector" of §III-A; a full vector is a sparse
 * vector with all n entries present.  Semantics follow the GraphBLAS C API
 * statement the paper builds on (§II): ewise_add is a set union, ewise_mult
 * an intersection, mxv over a semiring yields an entry only for rows with at
 * least one contributing term, and the optional mask / accumulator / replace
 * step is applied last.
 *
 * oracle_pagerank follows the pagerank_gap listing of §IV (Fig. "The PageRank
 * implementation in AppGrB") step by step, with one optional addition: in
 * "uniform" dangling mode the rank held by vertices without out-edges is
 * spread evenly over all n vertices, by adding damping*D/n to the teleport
 * term, D being the rank summed over those vertices.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int64_t n, nvals; int64_t* idx; double* val; } ovec;
typedef struct { int32_t code; double k; } obinop;

enum { O_FIRST = 1, O_SECOND, O_PLUS, O_MINUS, O_TIMES, O_DIV, O_MAX, O_MIN,
       O_ABS_DIFF, O_MAX_DIV_BY };
enum { OU_IDENTITY = 1, OU_ABS, OU_AINV, OU_MINV };

/* ---------------------------------------------------------------- helpers */

void oracle_free(void* p) { free(p); }

static int vec_alloc(ovec* v, int64_t n, int64_t cap) {
    v->n = n; v->nvals = 0;
    v->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
    v->val = (double*)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    return (v->idx && v->val) ? 0 : -1;
}

static void vec_release(ovec* v) { free(v->idx); free(v->val); v->idx = NULL; v->val = NULL; }

static void vec_push(ovec* v, int64_t i, double x) { v->idx[v->nvals] = i; v->val[v->nvals] = x; v->nvals++; }

static double binop(const obinop* op, double x, double y) {
    switch (op->code) {
        case O_FIRST: return x;
        case O_SECOND: return y;
        case O_PLUS: return x + y;
        case O_MINUS: return x - y;
        case O_TIMES: return x * y;
        case O_DIV: return x / y;
        case O_MAX: return x > y ? x : y;
        case O_MIN: return x < y ? x : y;
        case O_ABS_DIFF: return fabs(x - y);
        case O_MAX_DIV_BY: { double q = x / op->k; return q > y ? q : y; } /* (x,y) -> max(x/k, y), §IV */
    }
    return NAN;
}

static double unop(int code, double x) {
    switch (code) {
        case OU_IDENTITY: return x;
        case OU_ABS: return fabs(x);
        case OU_AINV: return -x;
        case OU_MINV: return 1.0 / x;
    }
    return NAN;
}

static double monoid_identity(int code) {
    switch (code) {
        case O_PLUS: return 0.0;
        case O_TIMES: return 1.0;
        case O_MAX: return -INFINITY;
        case O_MIN: return INFINITY;
    }
    return NAN;
}

/* -------------------------------------------------- element-wise methods */

/* Union of the index sets; op applied where both are present (§III-D:
 * element-wise addition). */
int oracle_ewise_add(ovec* out, const obinop* op, const ovec* u, const ovec* v) {
    if (u->n != v->n) return -2;
    if (vec_alloc(out, u->n, u->nvals + v->nvals)) return -1;
    int64_t a = 0, b = 0;
    while (a < u->nvals || b < v->nvals) {
        if (b >= v->nvals || (a < u->nvals && u->idx[a] < v->idx[b])) { vec_push(out, u->idx[a], u->val[a]); a++; }
        else if (a >= u->nvals || v->idx[b] < u->idx[a]) { vec_push(out, v->idx[b], v->val[b]); b++; }
        else { vec_push(out, u->idx[a], binop(op, u->val[a], v->val[b])); a++; b++; }
    }
    return 0;
}

/* Intersection of the index sets (§III-D: element-wise multiplication). */
int oracle_ewise_mult(ovec* out, const obinop* op, const ovec* u, const ovec* v) {
    if (u->n != v->n) return -2;
    if (vec_alloc(out, u->n, u->nvals < v->nvals ? u->nvals : v->nvals)) return -1;
    int64_t a = 0, b = 0;
    while (a < u->nvals && b < v->nvals) {
        if (u->idx[a] < v->idx[b]) a++;
        else if (v->idx[b] < u->idx[a]) b++;
        else { vec_push(out, u->idx[a], binop(op, u->val[a], v->val[b])); a++; b++; }
    }
    return 0;
}

/* apply with a unary operator (§III-B, VectorApply). */
int oracle_apply(ovec* out, int unop_code, const ovec* u) {
    if (vec_alloc(out, u->n, u->nvals)) return -1;
    for (int64_t a = 0; a < u->nvals; ++a) vec_push(out, u->idx[a], unop(unop_code, u->val[a]));
    return 0;
}

/* apply with a binary operator whose second argument is the scalar s. */
int oracle_apply_bind2nd(ovec* out, const obinop* op, const ovec* u, double s) {
    if (vec_alloc(out, u->n, u->nvals)) return -1;
    for (int64_t a = 0; a < u->nvals; ++a) vec_push(out, u->idx[a], binop(op, u->val[a], s));
    return 0;
}

/* Full vector with every entry equal to s (GrB_assign of a scalar to all
 * indices; the iso-valued full vectors of §III-A). */
int oracle_full(ovec* out, int64_t n, double s) {
    if (vec_alloc(out, n, n)) return -1;
    for (int64_t i = 0; i < n; ++i) vec_push(out, i, s);
    return 0;
}

/* --------------------------------------------------------------- mxv */

/* w = A (+.x) u over a semiring: row i gets an entry iff some j in row i of A
 * has u_j present; the value folds add over mul(A_ij, u_j) in ascending j
 * (the MxV node of §III-A, Fig. "The MxV Julia struct").  A is CSR; a NULL
 * value array means every stored A_ij equals a_iso. */
int oracle_mxv(ovec* out, int add_code, const obinop* mul, int64_t nrows, int64_t ncols,
               const int64_t* ptr, const int64_t* col, const double* aval, double a_iso,
               const ovec* u) {
    if (u->n != ncols) return -2;
    double* dense = (double*)calloc((size_t)(ncols > 0 ? ncols : 1), sizeof(double));
    unsigned char* has = (unsigned char*)calloc((size_t)(ncols > 0 ? ncols : 1), 1);
    if (!dense || !has || vec_alloc(out, nrows, nrows)) { free(dense); free(has); return -1; }
    for (int64_t a = 0; a < u->nvals; ++a) { dense[u->idx[a]] = u->val[a]; has[u->idx[a]] = 1; }
    const obinop add = { add_code, 0.0 };
    for (int64_t i = 0; i < nrows; ++i) {
        double acc = monoid_identity(add_code);
        int found = 0;
        for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) {
            const int64_t j = col[p];
            if (!has[j]) continue;
            const double aij = aval ? aval[p] : a_iso;
            acc = binop(&add, acc, binop(mul, aij, dense[j]));
            found = 1;
        }
        if (found) vec_push(out, i, acc);
    }
    free(dense); free(has);
    return 0;
}

/* ------------------------------------------------------------ reduce */

/* Fold a monoid over the present entries in index order. */
double oracle_reduce(int add_code, const ovec* u) {
    const obinop add = { add_code, 0.0 };
    double s = monoid_identity(add_code);
    for (int64_t a = 0; a < u->nvals; ++a) s = binop(&add, s, u->val[a]);
    return s;
}

/* ------------------------------------------- mask / accumulate / replace */

/* w<mask> accum= t.  Z = accum ? ewise_add(accum, w_old, t) : t; then every
 * index where the (possibly complemented, structural or valued) mask is true
 * takes Z's entry (or becomes absent); elsewhere w keeps its old entry, or
 * becomes absent when `replace` is set. */
int oracle_write(ovec* out, const ovec* w_old, const ovec* t, const obinop* accum,
                 const ovec* mask, int structural, int complement, int replace) {
    const int64_t n = w_old->n;
    if (t->n != n || (mask && mask->n != n)) return -2;
    ovec z;
    if (accum) { if (oracle_ewise_add(&z, accum, w_old, t)) return -1; }
    else {
        if (vec_alloc(&z, n, t->nvals)) return -1;
        for (int64_t a = 0; a < t->nvals; ++a) vec_push(&z, t->idx[a], t->val[a]);
    }
    unsigned char* m = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!m || vec_alloc(out, n, n)) { vec_release(&z); free(m); return -1; }
    if (mask) {
        for (int64_t a = 0; a < mask->nvals; ++a)
            m[mask->idx[a]] = structural ? 1 : (mask->val[a] != 0.0);
    } else {
        memset(m, 1, (size_t)n);
    }
    if (complement) for (int64_t i = 0; i < n; ++i) m[i] = !m[i];
    int64_t a = 0, b = 0;
    for (int64_t i = 0; i < n; ++i) {
        while (a < z.nvals && z.idx[a] < i) a++;
        while (b < w_old->nvals && w_old->idx[b] < i) b++;
        const int zin = a < z.nvals && z.idx[a] == i;
        const int win = b < w_old->nvals && w_old->idx[b] == i;
        if (m[i]) { if (zin) vec_push(out, i, z.val[a]); }
        else if (!replace && win) vec_push(out, i, w_old->val[b]);
    }
    vec_release(&z); free(m);
    return 0;
}

/* ------------------------------------------------------- graph building */

static int cmp_pair(const void* x, const void* y) {
    const int64_t* a = (const int64_t*)x; const int64_t* b = (const int64_t*)y;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

/* CSR of the transposed adjacency A^T (row i lists the sources j of edges
 * j -> i, ascending), from a COO edge list: sort by (dst, src), optionally
 * drop self loops and duplicate pairs.  The pagerank_gap listing of §IV takes
 * this A^T as its input; 32-bit indices as in §IV.  *ptr has n+1 entries. */
int oracle_build_at(int64_t n, int64_t nedges, const int32_t* src, const int32_t* dst,
                    int drop_self, int dedup, int64_t** ptr_out, int64_t** col_out, int64_t* nnz_out) {
    int64_t* pairs = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)(nedges > 0 ? nedges : 1));
    if (!pairs) return -1;
    int64_t m = 0;
    for (int64_t e = 0; e < nedges; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) { free(pairs); return -3; }
        if (drop_self && src[e] == dst[e]) continue;
        pairs[2 * m] = dst[e]; pairs[2 * m + 1] = src[e]; m++;
    }
    qsort(pairs, (size_t)m, 2 * sizeof(int64_t), cmp_pair);
    int64_t k = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (dedup && k > 0 && pairs[2 * (k - 1)] == pairs[2 * e] && pairs[2 * (k - 1) + 1] == pairs[2 * e + 1]) continue;
        pairs[2 * k] = pairs[2 * e]; pairs[2 * k + 1] = pairs[2 * e + 1]; k++;
    }
    int64_t* ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* col = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    if (!ptr || !col) { free(pairs); free(ptr); free(col); return -1; }
    for (int64_t e = 0; e < k; ++e) { ptr[pairs[2 * e] + 1]++; col[e] = pairs[2 * e + 1]; }
    for (int64_t i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    free(pairs);
    *ptr_out = ptr; *col_out = col; *nnz_out = k;
    return 0;
}

/* Out-degree of every vertex j = number of entries in column j of A^T. */
int oracle_out_degree(int64_t n, const int64_t* ptr, const int64_t* col, int64_t* outdeg) {
    memset(outdeg, 0, sizeof(int64_t) * (size_t)n);
    for (int64_t p = 0; p < ptr[n]; ++p) outdeg[col[p]]++;
    return 0;
}

/* ------------------------------------------------------------ PageRank */

static int vec_copy(ovec* out, const ovec* in) {
    if (vec_alloc(out, in->n, in->nvals)) return -1;
    memcpy(out->idx, in->idx, sizeof(int64_t) * (size_t)in->nvals);
    memcpy(out->val, in->val, sizeof(double) * (size_t)in->nvals);
    out->nvals = in->nvals;
    return 0;
}

static void vec_replace(ovec* dst, ovec* src) { vec_release(dst); *dst = *src; }

/* pagerank_gap of §IV, every method materialised (blocking mode):
 *
 *   teleport = (1-damping)/n;  rdiff = 1;  r = full(1/n)
 *   d = ewise_add(max(x/damping, y), conv(out_degree), full(1/damping))
 *   rt = full(teleport);  iter = 1
 *   while iter <= itermax && rdiff > tolerance:
 *       t = r
 *       r = ewise_mult(/, t, d)
 *       r = mxv(plus, second, A^T, r)
 *       r = ewise_add(+, rt, r)
 *       t = ewise_add(|x-y|, t, r);  rdiff = reduce(+, t);  iter += 1
 *
 * mode 0 ("gap") is that listing as printed.  mode 1 ("uniform") also sums
 * D = reduce(+, ewise_mult(first, t, sinks)) over the vertices without
 * out-edges and uses rt = full(teleport + damping*D/n) in that iteration.
 * `personal` (NULL for the plain method) replaces the uniform teleport by
 * (1-damping)*v and the start vector by v, v a sparse probability vector.
 *
 * Outputs: r_out (n, dense), *iters = number of loop bodies executed (the
 * listing's returned iter is *iters + 1), rdiff_hist[k] = rdiff after body k. */
int oracle_pagerank(int64_t n, const int64_t* ptr, const int64_t* col, const int64_t* outdeg,
                    double damping, double tolerance, int64_t itermax, int mode,
                    const ovec* personal, double* r_out, int64_t* iters, double* rdiff_hist) {
    if (n < 1) return -2;
    const obinop o_div = { O_DIV, 0 }, o_second = { O_SECOND, 0 }, o_plus = { O_PLUS, 0 };
    const obinop o_absdiff = { O_ABS_DIFF, 0 }, o_first = { O_FIRST, 0 }, o_times = { O_TIMES, 0 };
    const obinop o_maxdiv = { O_MAX_DIV_BY, damping };
    const double scaled_damping = (1.0 - damping) / (double)n;
    const double teleport = scaled_damping;
    double rdiff = 1.0;
    ovec r, d, deg, rt, sinks, vt;
    int rc = 0;

    /* r = full(1/n), or the personalisation vector v */
    if (personal) { if (vec_copy(&r, personal)) return -1; }
    else if (oracle_full(&r, n, 1.0 / (double)n)) return -1;

    /* d = ewise_add(max(x/damping, y), conv(out_degree), full(1/damping)) */
    if (vec_alloc(&deg, n, n)) return -1;
    for (int64_t i = 0; i < n; ++i) if (outdeg[i] > 0) vec_push(&deg, i, (double)outdeg[i]);
    { ovec dfill; if (oracle_full(&dfill, n, 1.0 / damping)) return -1;
      if (oracle_ewise_add(&d, &o_maxdiv, &deg, &dfill)) return -1; vec_release(&dfill); }

    /* sinks: vertices without out-edges (iso value 1) */
    if (vec_alloc(&sinks, n, n)) return -1;
    for (int64_t i = 0; i < n; ++i) if (outdeg[i] == 0) vec_push(&sinks, i, 1.0);

    /* teleport part: full(teleport) or (1-damping)*v */
    if (personal) { if (oracle_apply_bind2nd(&vt, &o_times, personal, 1.0 - damping)) return -1; }
    else if (oracle_full(&vt, n, teleport)) return -1;

    int64_t iter = 1;
    while (iter <= itermax && rdiff > tolerance) {
        ovec t, w, s, tmp;
        if (vec_copy(&t, &r)) { rc = -1; break; }                                   /* t = r */
        if (oracle_ewise_mult(&w, &o_div, &t, &d)) { rc = -1; break; }              /* r = t ./ d */
        if (oracle_mxv(&s, O_PLUS, &o_second, n, n, ptr, col, NULL, 1.0, &w)) { rc = -1; break; }
        vec_release(&w);
        /* rt for this iteration */
        if (mode == 1) {
            ovec z; if (oracle_ewise_mult(&z, &o_first, &t, &sinks)) { rc = -1; break; }
            const double D = oracle_reduce(O_PLUS, &z);
            vec_release(&z);
            ovec spread; if (oracle_full(&spread, n, damping * D / (double)n)) { rc = -1; break; }
            if (oracle_ewise_add(&rt, &o_plus, &vt, &spread)) { rc = -1; break; }
            vec_release(&spread);
        } else {
            if (vec_copy(&rt, &vt)) { rc = -1; break; }
        }
        if (oracle_ewise_add(&tmp, &o_plus, &rt, &s)) { rc = -1; break; }           /* r = rt + s */
        vec_release(&s); vec_release(&rt);
        vec_replace(&r, &tmp);
        ovec diff; if (oracle_ewise_add(&diff, &o_absdiff, &t, &r)) { rc = -1; break; }
        rdiff = oracle_reduce(O_PLUS, &diff);                                       /* rdiff = sum|t-r| */
        vec_release(&diff); vec_release(&t);
        if (rdiff_hist) rdiff_hist[iter - 1] = rdiff;
        iter += 1;
    }
    if (rc == 0) {
        for (int64_t i = 0; i < n; ++i) r_out[i] = 0.0;
        for (int64_t a = 0; a < r.nvals; ++a) r_out[r.idx[a]] = r.val[a];
        *iters = iter - 1;
    }
    vec_release(&r); vec_release(&d); vec_release(&deg); vec_release(&sinks); vec_release(&vt);
    return rc;
}
