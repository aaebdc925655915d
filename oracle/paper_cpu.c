/*
 * paper_cpu.c -- the paper-style multi-core CPU baseline of the barcode
 * path (Rawson, Sec. 3: OpenMP "for" pragmas on the loops that parallelise,
 * the reduction's outer loop left sequential).  BENCHMARK BASELINE ONLY: it
 * is timed by the benchmark's CPU-baseline leg beside the GPU path and is
 * checked against the oracle (ph0_oracle.c) by the CPU tests.  It shares no
 * code with the oracle or with the CUDA library.
 *
 * Steps (Sec. 2), each on all host cores where the loop allows:
 *   1. squared distances of every pair u < v, binary64 from binary32, one
 *      rounded subtraction, product and sum per dimension in dimension order
 *      (compiled with -ffp-contract=off: no fused multiply-add), in an
 *      OpenMP "for" over u;
 *   2. sort of the records (d2, u, v) by (d2, u, v): each thread sorts a
 *      contiguous slice, then slices are merged pairwise, every merge split
 *      across the threads by output position;
 *   3. the 1-based index a of each distance in D (repeats removed): counts of
 *      new values per slice in parallel, then a running sum;
 *   4-5. the column reduction of the vertex-by-edge matrix over F2[t]
 *      (entries t^a, so the supports reduce over F2), left to right and
 *      sequential: a column {u, v} whose pivot row max(u, v) is owned by an
 *      earlier column {x, L} becomes {u, v} + {x, L}; it stops at a new pivot
 *      (a bar (0, a)) or at zero.  Once n-1 pivots exist every later column
 *      reduces to zero, so the loop ends there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

enum { P_OK = 0, P_ARG = 1, P_MEM = 2 };

typedef struct {
    double d2;
    int32_t u, v;
} rec;

typedef struct {
    int32_t u, v;
    uint32_t a;
    int32_t low;
    int64_t order;
    double death_sq;
    double death;
} pbar;

static int rec_less(const rec *a, const rec *b)
{
    if (a->d2 != b->d2) return a->d2 < b->d2;
    if (a->u != b->u) return a->u < b->u;
    return a->v < b->v;
}

static int rec_cmp(const void *pa, const void *pb)
{
    const rec *a = (const rec *)pa, *b = (const rec *)pb;
    if (rec_less(a, b)) return -1;
    if (rec_less(b, a)) return 1;
    return 0;
}

/* Number of elements taken from A among the first k of merge(A, B), with
 * ties taken from A first (the records are distinct, so ties never occur;
 * the rule only makes the split well defined). */
static int64_t co_rank(int64_t k, const rec *A, int64_t na, const rec *B, int64_t nb)
{
    int64_t lo = k > nb ? k - nb : 0, hi = k < na ? k : na;
    while (lo < hi) {
        const int64_t i = (lo + hi) / 2, j = k - i;
        /* too few from A if A[i] belongs before B[j-1] */
        if (j > 0 && i < na && rec_less(&A[i], &B[j - 1]))
            lo = i + 1;
        else
            hi = i;
    }
    return lo;
}

static void merge_range(const rec *A, int64_t na, const rec *B, int64_t nb, rec *out, int64_t k0,
                        int64_t k1)
{
    int64_t i = co_rank(k0, A, na, B, nb), j = k0 - i;
    for (int64_t k = k0; k < k1; ++k) {
        if (j >= nb || (i < na && !rec_less(&B[j], &A[i])))
            out[k] = A[i++];
        else
            out[k] = B[j++];
    }
}

/* Sorts r[0..m) by (d2, u, v) on T threads; tmp has room for m records.
 * Returns the buffer holding the result (r or tmp). */
static rec *parallel_sort(rec *r, rec *tmp, int64_t m, int T)
{
    int64_t *cut = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
    if (!cut) return NULL;
    for (int t = 0; t <= T; ++t) cut[t] = m * t / T;
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int t = 0; t < T; ++t)
        qsort(r + cut[t], (size_t)(cut[t + 1] - cut[t]), sizeof(rec), rec_cmp);
    rec *src = r, *dst = tmp;
    for (int width = 1; width < T; width *= 2) {
        /* merge runs [cut[s], cut[s+w]) and [cut[s+w], cut[s+2w]) */
        for (int s = 0; s < T; s += 2 * width) {
            const int mid = s + width < T ? s + width : T;
            const int end = s + 2 * width < T ? s + 2 * width : T;
            const int64_t a0 = cut[s], a1 = cut[mid], b1 = cut[end];
            const int64_t len = b1 - a0;
#pragma omp parallel for num_threads(T) schedule(static, 1)
            for (int t = 0; t < T; ++t) {
                const int64_t k0 = len * t / T, k1 = len * (t + 1) / T;
                merge_range(src + a0, a1 - a0, src + a1, b1 - a1, dst + a0, k0, k1);
            }
        }
        rec *x = src;
        src = dst;
        dst = x;
    }
    free(cut);
    return src;
}

int ph0p_threads(void) { return omp_get_max_threads(); }

int ph0p_barcodes(const float *x, int64_t n, int32_t d, int64_t ld, pbar *bars, int64_t *n_bars,
                  int32_t *inf_vertex, int64_t *n_distinct)
{
    const int T = omp_get_max_threads();
    int64_t m, nb = 0, count = 0;
    rec *r = NULL, *tmp = NULL, *s = NULL;
    uint32_t *a = NULL;
    int64_t *slice_new = NULL;
    int32_t *partner = NULL;
    int rc = P_OK;
    if (n < 1 || d < 1 || ld < d) return P_ARG;
    m = n * (n - 1) / 2;
    r = (rec *)malloc(sizeof(rec) * (size_t)(m + 1));
    tmp = (rec *)malloc(sizeof(rec) * (size_t)(m + 1));
    a = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m + 1));
    slice_new = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
    partner = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!r || !tmp || !a || !slice_new || !partner) {
        rc = P_MEM;
        goto done;
    }

    /* 1. distances, rows in parallel */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t u = 0; u < n - 1; ++u) {
        const float *xu = x + u * ld;
        int64_t e = u * (2 * n - u - 1) / 2;
        for (int64_t v = u + 1; v < n; ++v, ++e) {
            const float *xv = x + v * ld;
            double acc = 0.0;
            for (int32_t k = 0; k < d; ++k) {
                const double t = (double)xv[k] - (double)xu[k];
                acc = acc + t * t;
            }
            r[e].d2 = acc;
            r[e].u = (int32_t)u;
            r[e].v = (int32_t)v;
        }
    }

    /* 2. sort */
    s = m > 0 ? parallel_sort(r, tmp, m, T) : r;
    if (!s) {
        rc = P_MEM;
        goto done;
    }

    /* 3. a: new values per slice, then a running sum per slice */
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int t = 0; t < T; ++t) {
        const int64_t p0 = m * t / T, p1 = m * (t + 1) / T;
        int64_t c = 0;
        for (int64_t p = p0; p < p1; ++p) c += (p == 0 || s[p].d2 != s[p - 1].d2);
        slice_new[t + 1] = c;
    }
    for (int t = 0; t < T; ++t) slice_new[t + 1] += slice_new[t];
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int t = 0; t < T; ++t) {
        const int64_t p0 = m * t / T, p1 = m * (t + 1) / T;
        int64_t c = slice_new[t];
        for (int64_t p = p0; p < p1; ++p) {
            c += (p == 0 || s[p].d2 != s[p - 1].d2);
            a[p] = (uint32_t)c;
        }
    }
    count = slice_new[T];

    /* 4-5. sequential column reduction; partner[L] = other row of the
     * reduced column whose pivot is L (-1: no such column yet) */
    for (int64_t i = 0; i < n; ++i) partner[i] = -1;
    for (int64_t p = 0; p < m && nb < n - 1; ++p) {
        int32_t lo = s[p].u < s[p].v ? s[p].u : s[p].v;
        int32_t hi = s[p].u < s[p].v ? s[p].v : s[p].u;
        for (;;) {
            const int32_t x2 = partner[hi];
            if (x2 < 0) {  /* new pivot hi: the bar (0, a(p)) */
                partner[hi] = lo;
                bars[nb].u = s[p].u;
                bars[nb].v = s[p].v;
                bars[nb].a = a[p];
                bars[nb].low = hi;
                bars[nb].order = p;
                bars[nb].death_sq = s[p].d2;
                bars[nb].death = sqrt(s[p].d2);
                ++nb;
                break;
            }
            /* {lo, hi} + {x2, hi} = {lo, x2} (zero when lo == x2) */
            if (x2 == lo) break;
            hi = lo > x2 ? lo : x2;
            lo = lo > x2 ? x2 : lo;
        }
    }
    *inf_vertex = -1;
    for (int64_t i = 0; i < n; ++i)
        if (partner[i] < 0) {
            *inf_vertex = (int32_t)i;
            break;
        }
    *n_bars = nb;
    *n_distinct = count;
done:
    free(r);
    free(tmp);
    free(a);
    free(slice_new);
    free(partner);
    return rc;
}
