/*
 * ph0_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of the 0th persistent homology
 * barcode algorithm of Rawson, "Linear Run Time of Persistent Homology
 * Computation with GPU Parallelization" (Sec. 2), used to check the CUDA path.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load
 * it; the product path never does.  It shares no code, header or table with
 * the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (-ffp-contract=off matters on aarch64, where gcc would otherwise fuse the
 * multiply and add of the squared distance into one fmadd).
 *
 * Steps, in the paper's order (Sec. 2; Sec. 4 steps 1-5):
 *   1. pairwise distances of the N points: every pair u<v, the squared
 *      distance in binary64 from the binary32 inputs, one rounded subtraction,
 *      one rounded multiplication and one rounded addition per dimension, in
 *      dimension order (the paper leaves the precision open; this fixed
 *      sequence makes every tie reproducible);
 *   2. sort the list E of edges increasing by distance (ties: lexicographic
 *      (u, v), which the paper leaves open);
 *   3. D = E without duplicates; a(edge) = 1-based index of its distance in D;
 *   4. M = vertex-by-edge matrix over F2[t], M(i,j) = t^a(j) when vertex i is
 *      an endpoint of edge j, else 0;
 *   5. column-reduce M left to right; each remaining nonzero pivot ("diagonal")
 *      entry t^b gives the bar (0, b).
 * The pivot of a column is its lowest nonzero entry, i.e. the largest row
 * index.  The oracle never compresses or reorders anything: every column is
 * reduced to completion, there is no early exit.
 *
 * Parity pins (which keep this file honest, in tests/): exact integer
 * distances, an exact-rational replay of each rounding, the library sort,
 * Kruskal/union-find, dense Prim, brute-force epsilon sweeps, closed forms and
 * the dense F2[t] reduction below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OK 0
#define ERR_ARG -1
#define ERR_MEM -2
#define ERR_STATE -3

/* --------------------------------------------------------------------------
 * Step 1: distances (Sec. 2: the distance of every pair of points; Sec. 4
 * step 1).  Edge e enumerates pairs u<v lexicographically:
 * (0,1),(0,2),...,(0,N-1),(1,2),...  The output is the squared distance;
 * the distance itself is its square root, a monotone map, so sorting and
 * de-duplicating squared distances orders and merges the distances alike.
 * ------------------------------------------------------------------------ */
int ph0o_edge_endpoints(int64_t n, int32_t *u, int32_t *v)
{
    int64_t e = 0;
    if (n < 0) return ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            u[e] = (int32_t)i;
            v[e] = (int32_t)j;
            ++e;
        }
    return OK;
}

static double squared_distance(const float *x, int64_t ld, int32_t d,
                               int64_t i, int64_t j)
{
    volatile double s = 0.0; /* volatile: each step is its own rounded op */
    for (int32_t k = 0; k < d; ++k) {
        double a = (double)x[j * ld + k];
        double b = (double)x[i * ld + k];
        volatile double t = a - b;
        volatile double p = t * t;
        s = s + p;
    }
    return s;
}

int ph0o_distances(const float *x, int64_t n, int32_t d, int64_t ld,
                   double *d2)
{
    int64_t e = 0;
    if (n < 0 || d < 1 || ld < d) return ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            d2[e++] = squared_distance(x, ld, d, i, j);
    return OK;
}

/* --------------------------------------------------------------------------
 * Step 2: sort the edges increasing by distance (Sec. 2; Sec. 4 step 2).
 * Ties are broken by (u, v) so that the order is total and reproducible.
 * ------------------------------------------------------------------------ */
typedef struct {
    double d2;
    int32_t u, v;
    int64_t id;
} edge_rec;

static int cmp_edge(const void *pa, const void *pb)
{
    const edge_rec *a = (const edge_rec *)pa, *b = (const edge_rec *)pb;
    if (a->d2 < b->d2) return -1;
    if (a->d2 > b->d2) return 1;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return 0;
}

int ph0o_sort_edges(const double *d2, const int32_t *u, const int32_t *v,
                    int64_t m, int64_t *order)
{
    edge_rec *r;
    if (m < 0) return ERR_ARG;
    if (m == 0) return OK;
    r = (edge_rec *)malloc((size_t)m * sizeof(edge_rec));
    if (!r) return ERR_MEM;
    for (int64_t e = 0; e < m; ++e) {
        r[e].d2 = d2[e];
        r[e].u = u[e];
        r[e].v = v[e];
        r[e].id = e;
    }
    qsort(r, (size_t)m, sizeof(edge_rec), cmp_edge);
    for (int64_t p = 0; p < m; ++p) order[p] = r[p].id;
    free(r);
    return OK;
}

/* --------------------------------------------------------------------------
 * Step 3: D is E without repeated distances (Sec. 2); a(j) is
 * the index, from 1, of edge j's distance in D.  Input: distances already
 * sorted.  Output: a per sorted position, and |D|.
 * ------------------------------------------------------------------------ */
int ph0o_dedupe(const double *d2_sorted, int64_t m, uint32_t *a,
                int64_t *n_distinct)
{
    int64_t count = 0;
    if (m < 0) return ERR_ARG;
    for (int64_t p = 0; p < m; ++p) {
        if (p == 0 || d2_sorted[p] != d2_sorted[p - 1]) ++count;
        a[p] = (uint32_t)count;
    }
    *n_distinct = count;
    return OK;
}

/* --------------------------------------------------------------------------
 * Steps 4-5, sparse form: column j of M has the two rows {u_j, v_j}, both
 * with the entry t^a(j).  Reduction left to right: while column j is nonzero
 * and its pivot row L already belongs to an earlier column k, add column k
 * to column j.  Over F2[t] the addition is col_j += t^(a(j)-a(k)) col_k, which
 * keeps every entry of column j equal to t^a(j) (the dense variant below
 * checks this); the supports therefore add as sets over F2.  Columns are kept
 * as sorted row lists and added by symmetric difference, in general form
 * (nothing here assumes a column has two entries).
 *
 * low[j]      = pivot row of reduced column j, or -1 if it reduced to zero
 * pivot_of[L] = column whose pivot is row L, or -1
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t *rows;
    int32_t len, cap;
} column;

static int col_reserve(column *c, int32_t cap)
{
    if (c->cap >= cap) return OK;
    int32_t nc = c->cap ? c->cap : 4;
    while (nc < cap) nc *= 2;
    int32_t *p = (int32_t *)realloc(c->rows, (size_t)nc * sizeof(int32_t));
    if (!p) return ERR_MEM;
    c->rows = p;
    c->cap = nc;
    return OK;
}

/* dst = a (+) b, symmetric difference of sorted row lists */
static int col_symdiff(const column *a, const column *b, column *dst)
{
    int32_t i = 0, j = 0, n = 0;
    if (col_reserve(dst, a->len + b->len) != OK) return ERR_MEM;
    while (i < a->len || j < b->len) {
        if (j >= b->len || (i < a->len && a->rows[i] < b->rows[j]))
            dst->rows[n++] = a->rows[i++];
        else if (i >= a->len || b->rows[j] < a->rows[i])
            dst->rows[n++] = b->rows[j++];
        else { /* equal rows: 1 + 1 = 0 over F2 */
            ++i;
            ++j;
        }
    }
    dst->len = n;
    return OK;
}

int ph0o_reduce(int64_t n, const int32_t *u_sorted, const int32_t *v_sorted,
                int64_t m, int32_t *low, int64_t *pivot_of,
                int64_t *steps_out)
{
    column *reduced; /* reduced column of each pivot column (indexed by row) */
    column work = {0, 0, 0}, tmp = {0, 0, 0};
    int64_t steps = 0;
    int rc = OK;
    if (n < 0 || m < 0) return ERR_ARG;
    reduced = (column *)calloc((size_t)(n > 0 ? n : 1), sizeof(column));
    if (!reduced) return ERR_MEM;
    for (int64_t r = 0; r < n; ++r) pivot_of[r] = -1;

    for (int64_t j = 0; j < m; ++j) {
        int32_t a0 = u_sorted[j], b0 = v_sorted[j];
        if (col_reserve(&work, 2) != OK) { rc = ERR_MEM; break; }
        work.rows[0] = a0 < b0 ? a0 : b0;
        work.rows[1] = a0 < b0 ? b0 : a0;
        work.len = (a0 == b0) ? 0 : 2;
        low[j] = -1;
        while (work.len > 0) {
            int32_t L = work.rows[work.len - 1]; /* lowest nonzero = max row */
            int64_t k = pivot_of[L];
            if (k < 0) {
                pivot_of[L] = j;
                low[j] = L;
                if (col_reserve(&reduced[L], work.len) != OK) { rc = ERR_MEM; break; }
                memcpy(reduced[L].rows, work.rows, (size_t)work.len * sizeof(int32_t));
                reduced[L].len = work.len;
                break;
            }
            if (col_symdiff(&work, &reduced[L], &tmp) != OK) { rc = ERR_MEM; break; }
            { column t = work; work = tmp; tmp = t; }
            ++steps;
        }
        if (rc != OK) break;
    }
    for (int64_t r = 0; r < n; ++r) free(reduced[r].rows);
    free(reduced);
    free(work.rows);
    free(tmp.rows);
    if (steps_out) *steps_out = steps;
    return rc;
}

/* --------------------------------------------------------------------------
 * Steps 4-5, dense form, for tiny inputs: the literal N x E matrix whose
 * entries are polynomials in t with coefficients in {0,1}, each stored as a
 * bit set of exponents.  Column j is reduced by adding t^(a(j)-a(k)) times
 * column k (k<j, so a(k) <= a(j)).  Outputs per column: its pivot row (-1 if
 * zero), the exponent b of the pivot entry t^b (-1 if zero), and whether every
 * nonzero entry of the reduced column is exactly the monomial t^a(j).
 * ------------------------------------------------------------------------ */
int ph0o_reduce_dense(int64_t n, const int32_t *u_sorted,
                      const int32_t *v_sorted, const uint32_t *a, int64_t m,
                      int32_t *low, int32_t *b_exp, int32_t *homogeneous)
{
    int64_t maxdeg = 0, words;
    uint64_t *mat;
    int64_t *pivot_of;
    if (n < 0 || m < 0 || n > 64 || m > 4096) return ERR_ARG;
    for (int64_t j = 0; j < m; ++j)
        if ((int64_t)a[j] > maxdeg) maxdeg = (int64_t)a[j];
    /* room for exponents up to 2*maxdeg: a shifted entry that overshoots
     * maxdeg is kept (and then flagged as inhomogeneous), never dropped */
    words = (2 * maxdeg + 1) / 64 + 1;
    mat = (uint64_t *)calloc((size_t)(n * m * words + 1), sizeof(uint64_t));
    pivot_of = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!mat || !pivot_of) { free(mat); free(pivot_of); return ERR_MEM; }
#define ENTRY(i, j) (mat + ((size_t)(j) * (size_t)n + (size_t)(i)) * (size_t)words)
    /* M(i,j) = t^a(j) when i is a vertex of edge j */
    for (int64_t j = 0; j < m; ++j) {
        uint32_t aj = a[j];
        ENTRY(u_sorted[j], j)[aj / 64] ^= (uint64_t)1 << (aj % 64);
        ENTRY(v_sorted[j], j)[aj / 64] ^= (uint64_t)1 << (aj % 64);
    }
    for (int64_t r = 0; r < n; ++r) pivot_of[r] = -1;

    for (int64_t j = 0; j < m; ++j) {
        for (;;) {
            int64_t L = -1;
            for (int64_t i = n - 1; i >= 0 && L < 0; --i)  /* lowest nonzero row */
                for (int64_t w = 0; w < words; ++w)
                    if (ENTRY(i, j)[w]) { L = i; break; }
            if (L < 0) { low[j] = -1; break; }
            if (pivot_of[L] < 0) { pivot_of[L] = j; low[j] = (int32_t)L; break; }
            {
                int64_t k = pivot_of[L];
                int64_t shift = (int64_t)a[j] - (int64_t)a[k];
                if (shift < 0) { free(mat); free(pivot_of); return ERR_STATE; }
                /* col_j += t^shift * col_k (XOR of shifted exponent bit sets) */
                for (int64_t i = 0; i < n; ++i) {
                    const uint64_t *src = ENTRY(i, k);
                    uint64_t *dst = ENTRY(i, j);
                    for (int64_t bit = 0; bit <= maxdeg; ++bit)
                        if (src[bit / 64] >> (bit % 64) & 1u) {
                            int64_t nb = bit + shift;
                            if (nb / 64 >= words) { free(mat); free(pivot_of); return ERR_STATE; }
                            dst[nb / 64] ^= (uint64_t)1 << (nb % 64);
                        }
                }
            }
        }
        /* pivot exponent and homogeneity of the reduced column */
        b_exp[j] = -1;
        homogeneous[j] = 1;
        for (int64_t i = 0; i < n; ++i) {
            int64_t nbits = 0, only = -1;
            for (int64_t bit = 0; bit < words * 64; ++bit)
                if (ENTRY(i, j)[bit / 64] >> (bit % 64) & 1u) { ++nbits; only = bit; }
            if (nbits == 0) continue;
            if (nbits != 1 || only != (int64_t)a[j]) homogeneous[j] = 0;
            if (i == low[j]) b_exp[j] = (int32_t)(nbits == 1 ? only : -2);
        }
    }
#undef ENTRY
    free(mat);
    free(pivot_of);
    return OK;
}

/* --------------------------------------------------------------------------
 * Whole path (Sec. 2, Sec. 4 steps 1-5) and the bars it reads off: one bar
 * (0, b) per nonzero reduced column, b = a of that column; the distance at
 * which it dies is D[b] (reported both squared and as its square root); the
 * single row that is never a pivot carries the bar that never dies.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t u, v;      /* killing edge, u < v                      */
    uint32_t a;        /* 1-based index of its distance in D       */
    int32_t low;       /* pivot row of its reduced column          */
    int64_t order;     /* 0-based position in the sorted edge list */
    double death_sq;   /* squared distance                         */
    double death;      /* sqrt(death_sq)                           */
} ph0o_bar;

int ph0o_barcodes(const float *x, int64_t n, int32_t d, int64_t ld,
                  ph0o_bar *bars, int64_t *n_bars, int32_t *inf_vertex,
                  int64_t *n_distinct_out)
{
    int64_t m, n_distinct = 0, nb = 0;
    int32_t *u = 0, *v = 0, *us = 0, *vs = 0, *low = 0;
    int64_t *order = 0, *pivot_of = 0;
    double *d2 = 0, *d2s = 0;
    uint32_t *a = 0;
    int rc = OK;
    if (n < 1 || d < 1 || ld < d) return ERR_ARG;
    m = n * (n - 1) / 2;
    u = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    v = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    us = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    vs = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    low = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    order = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    pivot_of = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    d2 = (double *)malloc((size_t)(m + 1) * sizeof(double));
    d2s = (double *)malloc((size_t)(m + 1) * sizeof(double));
    a = (uint32_t *)malloc((size_t)(m + 1) * sizeof(uint32_t));
    if (!u || !v || !us || !vs || !low || !order || !pivot_of || !d2 || !d2s || !a) {
        rc = ERR_MEM;
        goto done;
    }
    ph0o_edge_endpoints(n, u, v);
    if ((rc = ph0o_distances(x, n, d, ld, d2)) != OK) goto done;
    if ((rc = ph0o_sort_edges(d2, u, v, m, order)) != OK) goto done;
    for (int64_t p = 0; p < m; ++p) {
        us[p] = u[order[p]];
        vs[p] = v[order[p]];
        d2s[p] = d2[order[p]];
    }
    if ((rc = ph0o_dedupe(d2s, m, a, &n_distinct)) != OK) goto done;
    if ((rc = ph0o_reduce(n, us, vs, m, low, pivot_of, 0)) != OK) goto done;
    for (int64_t p = 0; p < m; ++p) {
        if (low[p] < 0) continue;
        bars[nb].u = us[p];
        bars[nb].v = vs[p];
        bars[nb].a = a[p];
        bars[nb].low = low[p];
        bars[nb].order = p;
        bars[nb].death_sq = d2s[p];
        bars[nb].death = sqrt(d2s[p]);
        ++nb;
    }
    *inf_vertex = -1;
    for (int64_t r = 0; r < n; ++r)
        if (pivot_of[r] < 0) {
            if (*inf_vertex >= 0) { rc = ERR_STATE; goto done; }
            *inf_vertex = (int32_t)r;
        }
    *n_bars = nb;
    if (n_distinct_out) *n_distinct_out = n_distinct;
done:
    free(u); free(v); free(us); free(vs); free(low); free(order);
    free(pivot_of); free(d2); free(d2s); free(a);
    return rc;
}

/* --------------------------------------------------------------------------
 * Gradient of a loss L(death_1..death_{N-1}) with respect to the points, in
 * binary64, for fixed killing edges (the pairing is piecewise constant in the
 * points).  death_i = |x_v - x_u|, so d death_i / d x_u = (x_u - x_v)/death_i
 * and d death_i / d x_v = -(x_u - x_v)/death_i; a bar of length 0 contributes
 * nothing (its derivative is taken as 0).  grad is [n, d], zeroed here.
 * ------------------------------------------------------------------------ */
int ph0o_death_gradient(const double *x, int64_t n, int32_t d, int64_t ld,
                        const int32_t *bu, const int32_t *bv,
                        const double *dl_ddeath, int64_t n_bars, double *grad)
{
    if (n < 0 || d < 1 || ld < d) return ERR_ARG;
    memset(grad, 0, (size_t)(n * d) * sizeof(double));
    for (int64_t b = 0; b < n_bars; ++b) {
        int64_t iu = bu[b], iv = bv[b];
        double s = 0.0, death;
        for (int32_t k = 0; k < d; ++k) {
            double t = x[iu * ld + k] - x[iv * ld + k];
            s += t * t;
        }
        death = sqrt(s);
        if (death == 0.0) continue;
        for (int32_t k = 0; k < d; ++k) {
            double g = dl_ddeath[b] * (x[iu * ld + k] - x[iv * ld + k]) / death;
            grad[iu * d + k] += g;
            grad[iv * d + k] -= g;
        }
    }
    return OK;
}

/* binary64 squared distances of fp64 points (for finite differences) */
int ph0o_distances_f64(const double *x, int64_t n, int32_t d, int64_t ld,
                       double *d2)
{
    int64_t e = 0;
    if (n < 0 || d < 1 || ld < d) return ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            volatile double s = 0.0;
            for (int32_t k = 0; k < d; ++k) {
                volatile double t = x[j * ld + k] - x[i * ld + k];
                volatile double p = t * t;
                s = s + p;
            }
            d2[e++] = s;
        }
    return OK;
}

int ph0o_abi_version(void) { return 1; }

/* --------------------------------------------------------------------------
 * The whole path restricted to a prefix of the filtration: only the edges
 * whose squared distance is at most t_max enter the sort, the index a and
 * the reduction (Sec. 2, on the edges of VR at epsilon^2 = t_max).  Every
 * edge of the total order (d2, u, v) that comes before a kept edge is itself
 * kept, so a kept edge's position in the prefix is its position in the whole
 * sorted list, and its a counts the same distinct distances; the bars found
 * are exactly those of ph0o_barcodes whose death_sq is at most t_max (all
 * n - 1 of them when t_max is at least the largest death).  Memory and sort
 * time scale with the kept edges, which lets the oracle check the positions
 * and indices of every bar of clouds too large for ph0o_barcodes.
 * Outputs: bars (room for n - 1), their count, the edges kept, and the
 * distinct distances among them.
 * ------------------------------------------------------------------------ */
int ph0o_barcodes_below(const float *x, int64_t n, int32_t d, int64_t ld,
                        double t_max, ph0o_bar *bars, int64_t *n_bars,
                        int64_t *n_kept, int64_t *n_distinct_out)
{
    edge_rec *r = NULL;
    int64_t cap = 0, k = 0, nb = 0, n_distinct = 0;
    int32_t *us = NULL, *vs = NULL, *low = NULL;
    int64_t *pivot_of = NULL;
    double *d2s = NULL;
    uint32_t *a = NULL;
    int rc = OK;
    if (n < 1 || d < 1 || ld < d) return ERR_ARG;
    /* step 1, keeping the edges of the prefix */
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            const double s2 = squared_distance(x, ld, d, i, j);
            if (!(s2 <= t_max)) continue;
            if (k == cap) {
                int64_t nc = cap ? cap * 2 : 1024;
                edge_rec *p = (edge_rec *)realloc(r, (size_t)nc * sizeof(edge_rec));
                if (!p) { rc = ERR_MEM; goto done; }
                r = p;
                cap = nc;
            }
            r[k].d2 = s2;
            r[k].u = (int32_t)i;
            r[k].v = (int32_t)j;
            r[k].id = k;
            ++k;
        }
    /* step 2 */
    if (k > 0) qsort(r, (size_t)k, sizeof(edge_rec), cmp_edge);
    us = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
    vs = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
    low = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
    d2s = (double *)malloc((size_t)(k + 1) * sizeof(double));
    a = (uint32_t *)malloc((size_t)(k + 1) * sizeof(uint32_t));
    pivot_of = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!us || !vs || !low || !d2s || !a || !pivot_of) { rc = ERR_MEM; goto done; }
    for (int64_t p = 0; p < k; ++p) {
        us[p] = r[p].u;
        vs[p] = r[p].v;
        d2s[p] = r[p].d2;
    }
    free(r);
    r = NULL;
    /* steps 3-5 on the prefix */
    if ((rc = ph0o_dedupe(d2s, k, a, &n_distinct)) != OK) goto done;
    if ((rc = ph0o_reduce(n, us, vs, k, low, pivot_of, 0)) != OK) goto done;
    for (int64_t p = 0; p < k; ++p) {
        if (low[p] < 0) continue;
        if (nb >= n - 1) { rc = ERR_STATE; goto done; }
        bars[nb].u = us[p];
        bars[nb].v = vs[p];
        bars[nb].a = a[p];
        bars[nb].low = low[p];
        bars[nb].order = p;
        bars[nb].death_sq = d2s[p];
        bars[nb].death = sqrt(d2s[p]);
        ++nb;
    }
    *n_bars = nb;
    *n_kept = k;
    *n_distinct_out = n_distinct;
done:
    free(r); free(us); free(vs); free(low); free(d2s); free(a); free(pivot_of);
    return rc;
}

/* --------------------------------------------------------------------------
 * First homology (the extension the paper names in Sec. 1 and Sec. 4.2): the
 * Vietoris-Rips 2-skeleton adds a triangle on three points once its three
 * edges are present (Sec. 1, the recursive rule), i.e. at the largest of its
 * edges' distances, its diameter.  The boundary matrix has a row per edge (in
 * the sorted edge order of step 2) and a column per triangle, with the
 * triangle's three edges set; entries t^a over F2[t] reduce like the F2
 * supports (as in dimension 0).  Triangles are ordered by the position of
 * their diameter edge in the edge order, then (u, v, w) lexicographically.
 * The columns are reduced left to right with low = largest row; each nonzero
 * reduced column pairs its low edge (a positive edge: it closes a cycle)
 * with the triangle, the bar (a(edge), a(diameter of the triangle)).  The
 * 2-skeleton of the full simplex has no first homology, so every positive
 * edge is paired: n(n-1)/2 - (n-1) bars, zero-length ones included.
 * Outputs in column order; n <= 2000 (triangle counts below 2^31).
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t eu, ev;             /* birth edge, eu < ev                          */
    int32_t tu, tv, tw;         /* death triangle, tu < tv < tw                 */
    uint32_t birth_a, death_a;  /* 1-based indices in D                         */
    int32_t pad;
    int64_t birth_order;        /* position of the birth edge in the edge order */
    int64_t death_order;        /* position of the triangle's diameter edge     */
    int64_t death_rank;         /* position of the triangle in triangle order   */
    double birth_sq, death_sq;  /* squared distances                            */
} ph0o_h1bar;

typedef struct {
    int64_t diam;
    int32_t u, v, w, pad;
} tri_rec;

static int cmp_tri(const void *pa, const void *pb)
{
    const tri_rec *a = (const tri_rec *)pa, *b = (const tri_rec *)pb;
    if (a->diam != b->diam) return a->diam < b->diam ? -1 : 1;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    if (a->w != b->w) return a->w < b->w ? -1 : 1;
    return 0;
}

static int cmp_i64(const void *pa, const void *pb)
{
    const int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

int ph0o_h1(const float *x, int64_t n, int32_t d, int64_t ld, ph0o_h1bar *bars,
            int64_t *n_bars, int64_t *n_triangles)
{
    int64_t m, T, nb = 0;
    int32_t *u = 0, *v = 0;
    int64_t *order = 0, *pos_of = 0, *pivot_of = 0;
    double *d2 = 0, *d2s = 0;
    uint32_t *a = 0;
    tri_rec *tri = 0;
    column *reduced = 0;   /* reduced column of the pivot owner, by low row */
    column work = {0, 0, 0}, tmp = {0, 0, 0};
    int64_t n_distinct = 0;
    int rc = OK;
    if (n < 1 || d < 1 || ld < d || n > 2000) return ERR_ARG;
    m = n * (n - 1) / 2;
    T = n * (n - 1) * (n - 2) / 6;
    u = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    v = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    order = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    pos_of = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    pivot_of = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    d2 = (double *)malloc((size_t)(m + 1) * sizeof(double));
    d2s = (double *)malloc((size_t)(m + 1) * sizeof(double));
    a = (uint32_t *)malloc((size_t)(m + 1) * sizeof(uint32_t));
    tri = (tri_rec *)malloc((size_t)(T + 1) * sizeof(tri_rec));
    reduced = (column *)calloc((size_t)(m + 1), sizeof(column));
    if (!u || !v || !order || !pos_of || !pivot_of || !d2 || !d2s || !a || !tri || !reduced) {
        rc = ERR_MEM;
        goto done;
    }
    /* steps 1-3 of dimension 0: edge order, positions, a */
    ph0o_edge_endpoints(n, u, v);
    if ((rc = ph0o_distances(x, n, d, ld, d2)) != OK) goto done;
    if ((rc = ph0o_sort_edges(d2, u, v, m, order)) != OK) goto done;
    for (int64_t p = 0; p < m; ++p) {
        pos_of[order[p]] = p;
        d2s[p] = d2[order[p]];
        pivot_of[p] = -1;
    }
    if ((rc = ph0o_dedupe(d2s, m, a, &n_distinct)) != OK) goto done;
    /* triangles and their diameters, in triangle order */
    {
        int64_t k = 0;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j)
                for (int64_t l = j + 1; l < n; ++l) {
                    const int64_t pij = pos_of[i * (2 * n - i - 1) / 2 + (j - i - 1)];
                    const int64_t pil = pos_of[i * (2 * n - i - 1) / 2 + (l - i - 1)];
                    const int64_t pjl = pos_of[j * (2 * n - j - 1) / 2 + (l - j - 1)];
                    int64_t mx = pij > pil ? pij : pil;
                    mx = mx > pjl ? mx : pjl;
                    tri[k].diam = mx;
                    tri[k].u = (int32_t)i;
                    tri[k].v = (int32_t)j;
                    tri[k].w = (int32_t)l;
                    tri[k].pad = 0;
                    ++k;
                }
        if (T > 0) qsort(tri, (size_t)T, sizeof(tri_rec), cmp_tri);
    }
    /* column reduction, left to right, no early exit */
    for (int64_t j = 0; j < T; ++j) {
        const int64_t i0 = tri[j].u, j0 = tri[j].v, l0 = tri[j].w;
        int64_t e3[3];
        e3[0] = pos_of[i0 * (2 * n - i0 - 1) / 2 + (j0 - i0 - 1)];
        e3[1] = pos_of[i0 * (2 * n - i0 - 1) / 2 + (l0 - i0 - 1)];
        e3[2] = pos_of[j0 * (2 * n - j0 - 1) / 2 + (l0 - j0 - 1)];
        qsort(e3, 3, sizeof(int64_t), cmp_i64);
        if (col_reserve(&work, 3) != OK) { rc = ERR_MEM; goto done; }
        for (int q = 0; q < 3; ++q) work.rows[q] = (int32_t)e3[q];
        work.len = 3;
        while (work.len > 0) {
            const int32_t L = work.rows[work.len - 1];
            if (pivot_of[L] < 0) {
                const int64_t pe = L;
                pivot_of[L] = j;
                if (col_reserve(&reduced[L], work.len) != OK) { rc = ERR_MEM; goto done; }
                memcpy(reduced[L].rows, work.rows, (size_t)work.len * sizeof(int32_t));
                reduced[L].len = work.len;
                if (nb >= m) { rc = ERR_STATE; goto done; }
                bars[nb].eu = u[order[pe]];
                bars[nb].ev = v[order[pe]];
                bars[nb].tu = tri[j].u;
                bars[nb].tv = tri[j].v;
                bars[nb].tw = tri[j].w;
                bars[nb].pad = 0;
                bars[nb].birth_a = a[pe];
                bars[nb].death_a = a[tri[j].diam];
                bars[nb].birth_order = pe;
                bars[nb].death_order = tri[j].diam;
                bars[nb].death_rank = j;
                bars[nb].birth_sq = d2s[pe];
                bars[nb].death_sq = d2s[tri[j].diam];
                ++nb;
                break;
            }
            if (col_symdiff(&work, &reduced[L], &tmp) != OK) { rc = ERR_MEM; goto done; }
            { column t = work; work = tmp; tmp = t; }
        }
    }
    *n_bars = nb;
    *n_triangles = T;
done:
    if (reduced) {
        for (int64_t r = 0; r < m; ++r) free(reduced[r].rows);
        free(reduced);
    }
    free(work.rows); free(tmp.rows);
    free(u); free(v); free(order); free(pos_of); free(pivot_of);
    free(d2); free(d2s); free(a); free(tri);
    return rc;
}
