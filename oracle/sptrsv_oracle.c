/*
 * CPU oracle for the sparse lower-triangular solve and its superstep schedule.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a small shared object
 * that only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg load.  The GPU library never links, includes or calls it, and it shares
 * no source with the library.
 *
 * Everything here is deliberately plain and sequential:
 *   - oracle_solve_fp64     forward substitution, Eq. 2.1, row by row in FP64
 *   - oracle_solve_upper_fp64           backward substitution (the upper-
 *                           triangular counterpart of Eq. 2.1), row by row
 *   - oracle_solve_lower_transposed_fp64  L^T x = b from L's rows, column-
 *                           oriented backward substitution
 *   - oracle_spmv_fp64      y = A x in FP64 (used for residual checks in tests)
 *   - oracle_levels         wavefronts of the DAG of Sec. 2.2 (Fig. 1.1)
 *   - oracle_growlocal      the GrowLocal scheduler of Sec. 3 / Algorithm 3.1
 *   - oracle_growlocal_weighted  the same with explicit vertex weights (used by
 *                           the block-parallel scheduling of Sec. 3.1)
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add contraction) so
 * the FP64 results are reproducible on x86 and Arm.
 *
 * Input convention (all functions): square lower-triangular CSR, 0-based,
 * int32 row pointers and columns, columns strictly increasing within a row,
 * the diagonal present and stored last.  The Python wrapper validates this.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ solve */

/* Eq. 2.1: x_i = (b_i - sum_{j<i} A_ij x_j) / A_ii, rows in natural order,
 * the sum taken in ascending column order, one right-hand side at a time.
 * b and x are column-major with leading dimension ld. */
void oracle_solve_fp64(int32_t n, int32_t nrhs, const int32_t *rowptr, const int32_t *col,
                       const double *val, const double *b, int64_t ldb, double *x, int64_t ldx)
{
    for (int32_t r = 0; r < nrhs; ++r) {
        const double *bj = b + (int64_t)r * ldb;
        double *xj = x + (int64_t)r * ldx;
        for (int32_t i = 0; i < n; ++i) {
            double s = bj[i];
            int32_t last = rowptr[i + 1] - 1;          /* diagonal position */
            for (int32_t p = rowptr[i]; p < last; ++p)
                s = s - val[p] * xj[col[p]];
            xj[i] = s / val[last];
        }
    }
}

/* Backward substitution for upper-triangular U (the method's other direction):
 * x_i = (b_i - sum_{j>i} U_ij x_j) / U_ii for i = n-1 down to 0, the sum in
 * ascending column order.  Upper CSR convention: columns strictly increasing
 * within a row, the diagonal present and stored FIRST. */
void oracle_solve_upper_fp64(int32_t n, int32_t nrhs, const int32_t *rowptr, const int32_t *col,
                             const double *val, const double *b, int64_t ldb, double *x, int64_t ldx)
{
    for (int32_t r = 0; r < nrhs; ++r) {
        const double *bj = b + (int64_t)r * ldb;
        double *xj = x + (int64_t)r * ldx;
        for (int32_t i = n - 1; i >= 0; --i) {
            double s = bj[i];
            const int32_t d = rowptr[i];                /* diagonal position */
            for (int32_t p = d + 1; p < rowptr[i + 1]; ++p)
                s = s - val[p] * xj[col[p]];
            xj[i] = s / val[d];
        }
    }
}

/* L^T x = b for lower-triangular L given by its rows (diagonal last): since
 * (L^T x)_j = sum_k L_kj x_k, take k = n-1 down to 0, finish x_k = x_k / L_kk
 * and remove L_kj x_k from every x_j of row k (column-oriented backward
 * substitution; no transpose is formed). */
void oracle_solve_lower_transposed_fp64(int32_t n, int32_t nrhs, const int32_t *rowptr, const int32_t *col,
                                        const double *val, const double *b, int64_t ldb, double *x,
                                        int64_t ldx)
{
    for (int32_t r = 0; r < nrhs; ++r) {
        const double *bj = b + (int64_t)r * ldb;
        double *xj = x + (int64_t)r * ldx;
        for (int32_t i = 0; i < n; ++i) xj[i] = bj[i];
        for (int32_t k = n - 1; k >= 0; --k) {
            const int32_t last = rowptr[k + 1] - 1;
            xj[k] = xj[k] / val[last];
            for (int32_t p = rowptr[k]; p < last; ++p)
                xj[col[p]] = xj[col[p]] - val[p] * xj[k];
        }
    }
}

/* y = A x for one column (all stored entries, diagonal included), FP64. */
void oracle_spmv_fp64(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                      const double *x, double *y)
{
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            s = s + val[p] * x[col[p]];
        y[i] = s;
    }
}

/* ----------------------------------------------------------------- levels */

/* Wavefronts (Sec. 1, Fig. 1.1): a vertex is in wavefront 0 if it has no
 * parents, otherwise one past the deepest of its parents.  Vertex i's parents
 * are the off-diagonal columns of row i (edge (j,i) iff A_ij != 0, Sec. 2.2).
 * Natural order is topological for a lower-triangular matrix, so one pass
 * suffices.  Returns the number of wavefronts. */
int32_t oracle_levels(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t *level)
{
    int32_t nlev = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t lv = 0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (j != i && level[j] + 1 > lv)
                lv = level[j] + 1;
        }
        level[i] = lv;
        if (lv + 1 > nlev)
            nlev = lv + 1;
    }
    return nlev;
}

/* -------------------------------------------------------------- GrowLocal */

/* A plain binary min-heap of vertex ids (Rule I(ii): smallest id first). */
typedef struct {
    int32_t *a;
    int64_t size, cap;
} heap_t;

static void heap_push(heap_t *h, int32_t v)
{
    if (h->size == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 64;
        h->a = (int32_t *)realloc(h->a, (size_t)h->cap * sizeof(int32_t));
    }
    int64_t i = h->size++;
    h->a[i] = v;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p] <= h->a[i])
            break;
        int32_t t = h->a[p]; h->a[p] = h->a[i]; h->a[i] = t;
        i = p;
    }
}

static int32_t heap_pop(heap_t *h)
{
    int32_t top = h->a[0];
    h->a[0] = h->a[--h->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->size && h->a[l] < h->a[m]) m = l;
        if (r < h->size && h->a[r] < h->a[m]) m = r;
        if (m == i)
            break;
        int32_t t = h->a[m]; h->a[m] = h->a[i]; h->a[i] = t;
        i = m;
    }
    return top;
}

static void heap_copy(heap_t *dst, const heap_t *src)
{
    if (dst->cap < src->size) {
        dst->cap = src->size > 64 ? src->size : 64;
        dst->a = (int32_t *)realloc(dst->a, (size_t)dst->cap * sizeof(int32_t));
    }
    if (src->size)
        memcpy(dst->a, src->a, (size_t)src->size * sizeof(int32_t));
    dst->size = src->size;
}

#define OWNER_NONE  (-1)
#define OWNER_MANY  (-2)

/* One attempt ("iteration" of the inner loop of Algorithm 3.1) with vertex
 * budget `limit` for core 0.  Works on private copies of the superstep-start
 * state, so discarding it is the "undo new assignments" step.
 * Outputs: the assigned (vertex, core) list, the per-core weights Omega. */
typedef struct {
    int32_t n, k;
    const int32_t *cptr, *cidx;        /* children (transpose of the pattern) */
    const int64_t *w;                  /* omega(v) = nnz of row v (Sec. 2.2)  */
    const int32_t *missing;            /* parents not yet in a finished superstep */
    const heap_t *ready;               /* R: all parents finished, not assigned   */
    /* scratch */
    int32_t *miss;                     /* per attempt: parents still unassigned */
    int32_t *owner;                    /* core of this superstep's parents      */
    heap_t rcopy;
    heap_t *excl;                      /* X_p: vertices only computable on p    */
    /* result */
    int32_t *av, *ap;                  /* assigned vertices and their cores     */
    int64_t count;
    int64_t core0_taken;               /* vertices core 0 received              */
    int64_t *omega;
} attempt_t;

static int take(attempt_t *A, int32_t p, int32_t *v)
{
    /* Rule I: (i) core-exclusive vertices first, then (ii) smallest id. */
    if (A->excl[p].size) { *v = heap_pop(&A->excl[p]); return 1; }
    if (A->rcopy.size)   { *v = heap_pop(&A->rcopy);   return 1; }
    return 0;
}

static void assign(attempt_t *A, int32_t v, int32_t p)
{
    A->av[A->count] = v;
    A->ap[A->count] = p;
    A->count++;
    A->omega[p] += A->w[v];
    for (int32_t q = A->cptr[v]; q < A->cptr[v + 1]; ++q) {
        int32_t u = A->cidx[q];
        if (A->owner[u] == OWNER_NONE)
            A->owner[u] = p;
        else if (A->owner[u] != p)
            A->owner[u] = OWNER_MANY;
        if (--A->miss[u] == 0 && A->owner[u] == p)
            heap_push(&A->excl[p], u);   /* all of u's new parents sit on p */
        /* parents on several cores: u waits for the next barrier */
    }
}

static void run_attempt(attempt_t *A, int64_t limit)
{
    memcpy(A->miss, A->missing, (size_t)A->n * sizeof(int32_t));
    for (int32_t v = 0; v < A->n; ++v)
        A->owner[v] = OWNER_NONE;
    heap_copy(&A->rcopy, A->ready);
    for (int32_t p = 0; p < A->k; ++p) {
        A->excl[p].size = 0;
        A->omega[p] = 0;
    }
    A->count = 0;

    /* core 1 of the paper (index 0 here): up to alpha vertices */
    int32_t v;
    for (int64_t t = 0; t < limit; ++t) {
        if (!take(A, 0, &v))
            break;
        assign(A, v, 0);
    }
    A->core0_taken = A->count;
    /* cores 2..k in order: add vertices while Omega_p < Omega_1 */
    for (int32_t p = 1; p < A->k; ++p) {
        while (A->omega[p] < A->omega[0]) {
            if (!take(A, p, &v))
                break;
            assign(A, v, p);
        }
    }
}

/* GrowLocal (Sec. 3, Algorithm 3.1; acceptance rule of App. B).
 *
 * Inputs: the factor's pattern, the number of cores k, the starting superstep
 * length alpha0 (20), the growth factor (1.5), the barrier cost L (500) and
 * the acceptance ratio (0.97).  Outputs sigma (superstep, 0-based) and pi
 * (core, 0-based) for every vertex; returns the number of supersteps, or -1
 * on allocation failure.
 *
 * Readings where the paper is silent:
 *  - core 0 takes floor(alpha) vertices; alpha is a real number multiplied by
 *    `growth` after each attempt (alpha *= growth, IEEE double);
 *  - cores p >= 1 add vertices while Omega_p < Omega_0 (the last one may
 *    overshoot), each core drawing only from its own X_p and from R;
 *  - beta = sum_p Omega_p / (max_p Omega_p + L) in double; attempt 0 is
 *    always worthy, attempt a > 0 is worthy iff beta_a >= accept * (best beta
 *    of the worthy attempts of this superstep);
 *  - the superstep ends at the first unworthy attempt (the last worthy one is
 *    kept), or right after a worthy attempt in which core 0 took fewer than
 *    floor(alpha) vertices: it ran out of candidates, so every larger alpha
 *    would repeat the same attempt. */
int32_t oracle_growlocal_weighted(int32_t n, const int32_t *rowptr, const int32_t *col,
                                  const int64_t *weight, int32_t k, double alpha0, double growth,
                                  double L, double accept, int32_t *sigma, int32_t *pi);

int32_t oracle_growlocal(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t k,
                         double alpha0, double growth, double L, double accept,
                         int32_t *sigma, int32_t *pi)
{
    return oracle_growlocal_weighted(n, rowptr, col, NULL, k, alpha0, growth, L, accept, sigma, pi);
}

/* As oracle_growlocal, with the vertex weights omega(v) given explicitly
 * (weight == NULL: the row's stored entries).  The block-parallel scheduler of
 * Sec. 3.1 runs GrowLocal on a diagonal block whose rows lost their entries in
 * earlier blocks' columns, yet weighs each vertex by its full row. */
int32_t oracle_growlocal_weighted(int32_t n, const int32_t *rowptr, const int32_t *col,
                                  const int64_t *weight, int32_t k, double alpha0, double growth,
                                  double L, double accept, int32_t *sigma, int32_t *pi)
{
    if (n <= 0)
        return 0;
    /* DAG: parents = off-diagonal columns, children = their transpose. */
    int32_t *cptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int64_t *w = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int32_t *missing = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) {
        w[i] = weight ? weight[i] : (int64_t)(rowptr[i + 1] - rowptr[i]);
        missing[i] = 0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] != i) {
                cptr[col[p] + 1]++;
                missing[i]++;
            }
    }
    for (int32_t i = 0; i < n; ++i)
        cptr[i + 1] += cptr[i];
    int32_t *cidx = (int32_t *)malloc((size_t)(cptr[n] > 0 ? cptr[n] : 1) * sizeof(int32_t));
    int32_t *fill = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    memcpy(fill, cptr, (size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] != i)
                cidx[fill[col[p]]++] = i;          /* children in increasing id */
    free(fill);

    heap_t ready = {0};
    for (int32_t i = 0; i < n; ++i)
        if (missing[i] == 0)
            heap_push(&ready, i);

    attempt_t A;
    memset(&A, 0, sizeof(A));
    A.n = n; A.k = k; A.cptr = cptr; A.cidx = cidx; A.w = w;
    A.missing = missing; A.ready = &ready;
    A.miss = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    A.owner = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    A.excl = (heap_t *)calloc((size_t)k, sizeof(heap_t));
    A.av = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    A.ap = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    A.omega = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    /* the last worthy attempt */
    int32_t *keep_v = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *keep_p = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    char *is_done = (char *)calloc((size_t)n, 1);

    int64_t remaining = n;
    int32_t step = 0;
    while (remaining > 0) {
        double alpha = alpha0, best = 0.0;
        int64_t keep_count = 0;
        for (int attempt = 0;; ++attempt) {
            run_attempt(&A, (int64_t)floor(alpha));
            int64_t sum = 0, mx = 0;
            for (int32_t p = 0; p < k; ++p) {
                sum += A.omega[p];
                if (A.omega[p] > mx)
                    mx = A.omega[p];
            }
            double beta = (double)sum / ((double)mx + L);      /* Eq. 3.1 */
            int worthy = (attempt == 0) || (beta >= accept * best);
            if (!worthy)
                break;
            if (beta > best)
                best = beta;
            memcpy(keep_v, A.av, (size_t)A.count * sizeof(int32_t));
            memcpy(keep_p, A.ap, (size_t)A.count * sizeof(int32_t));
            keep_count = A.count;
            if (A.core0_taken < (int64_t)floor(alpha))
                break;
            alpha = alpha * growth;
        }
        /* finalize the last worthy attempt as superstep `step` */
        for (int64_t t = 0; t < keep_count; ++t) {
            int32_t v = keep_v[t];
            sigma[v] = step;
            pi[v] = keep_p[t];
            is_done[v] = 1;
        }
        remaining -= keep_count;
        /* rebuild R: drop assigned vertices, add the newly released ones */
        heap_t next = {0};
        while (ready.size) {
            int32_t v = heap_pop(&ready);
            if (!is_done[v])
                heap_push(&next, v);
        }
        for (int64_t t = 0; t < keep_count; ++t) {
            int32_t v = keep_v[t];
            for (int32_t q = cptr[v]; q < cptr[v + 1]; ++q) {
                int32_t u = cidx[q];
                /* u may itself have been finalized in this superstep */
                if (--missing[u] == 0 && !is_done[u])
                    heap_push(&next, u);
            }
        }
        free(ready.a);
        ready = next;
        step++;
    }

    free(ready.a); free(A.rcopy.a);
    for (int32_t p = 0; p < k; ++p)
        free(A.excl[p].a);
    free(A.excl); free(A.miss); free(A.owner); free(A.av); free(A.ap); free(A.omega);
    free(keep_v); free(keep_p); free(is_done);
    free(cptr); free(cidx); free(w); free(missing);
    return step;
}
