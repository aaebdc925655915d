// k_h1.cu -- first homology of the Vietoris-Rips filtration, the extension
// the paper names (Rawson, Sec. 1 and Sec. 4.2: higher-order homology).  The
// 2-skeleton adds a triangle on three points once its three edges are
// present (Sec. 1, the recursive rule): at its diameter, the latest of its
// edges in the sorted edge order of step 2.  Its boundary matrix has a row
// per edge and a column per triangle (entries t^a over F2[t], which reduce
// like their F2 supports, as in dimension 0), the triangles in the order
// (diameter position, u, v, w).  Reducing it left to right pairs each
// positive edge (one that closed a cycle) with a triangle: the bar
// (a(edge), a(diameter)).  The full simplex has no first homology, so every
// positive edge is paired: n(n-1)/2 - (n-1) bars.
//
// The GPU computes the same pairs through the coboundary matrix (the
// transpose with both orders reversed), whose left-to-right reduction has
// the same pairs (persistence pairs of homology and cohomology coincide):
// a column per edge, taken from the latest edge to the earliest, whose pivot
// is its earliest triangle.  Three facts make it short:
//   * clearing: the n-1 edges that end a class in dimension 0 are pivots of
//     the dimension-0 coboundary, so their columns are dropped;
//   * apparent pairs: when edge e is the diameter of some triangle, the
//     first such triangle t (in triangle order) is e's earliest coface and e
//     is t's latest face; no column processed before e (a later edge) can
//     contain t, so (e, t) is a pair with no column addition.  The first such
//     triangle is the one whose third vertex w is smallest (the order of
//     sorted (a, b, w) follows w);
//   * an edge that is the diameter of no triangle is either a spanning-forest
//     edge (a minimum spanning forest lies within these edges, by the cycle
//     property) or a positive edge whose column must be reduced; these are
//     few (63 at 256 uniform points in the plane, 177 at 700).
// Steps:
//   1. the dimension-0 sort and de-duplication give every edge its position
//      p and its index a(p); a matrix P[a][w] of positions;
//   2. one warp per edge: the triangles of which it is the diameter (count
//      and smallest third vertex), i.e. the apparent pairs and, by a prefix
//      sum of the counts, the rank of every triangle in triangle order;
//   3. the edges that are the diameter of no triangle, in order: Kruskal
//      (one thread) marks the spanning-forest edges; the rest are listed;
//   4. one CTA reduces the listed columns from the latest edge down: while
//      a column's pivot has an owner (the apparent pair of the pivot's
//      diameter edge, or an earlier reduced column), the owner's column is
//      added; the pivot left is claimed.  A column is a short stack of sorted
//      runs of triangle keys whose symmetric difference it is: an addition
//      pushes the owner's column as a run, runs merge (sorted symmetric
//      difference) while the one below is at most twice as long, and the
//      pivot is found at the runs' heads, so an addition costs about the
//      owner's length times the logarithm, not the column's length; the
//      reduced column is merged into one run and kept;
//   5. the bars, in triangle order, from the prefix sums of the counts.
#include "ph0_common.cuh"

namespace ph0 {

constexpr uint32_t kH1NoPos = 0xffffffffu;
constexpr int kH1VB = kH1VertexBits;
constexpr uint64_t kH1VMask = (uint64_t(1) << kH1VB) - 1;

// Key of the triangle {a, b, w} (distinct vertices) with diameter position dpos.
__device__ __forceinline__ uint64_t h1_key(uint64_t dpos, uint32_t a, uint32_t b, uint32_t w) {
    uint32_t x = a, y = b, z = w;
    if (x > y) { const uint32_t t = x; x = y; y = t; }
    if (y > z) { const uint32_t t = y; y = z; z = t; }
    if (x > y) { const uint32_t t = x; x = y; y = t; }
    return (dpos << (3 * kH1VB)) | (uint64_t(x) << (2 * kH1VB)) | (uint64_t(y) << kH1VB) | uint64_t(z);
}
__device__ __forceinline__ void h1_key_uvw(uint64_t k, uint32_t &u, uint32_t &v, uint32_t &w) {
    u = uint32_t((k >> (2 * kH1VB)) & kH1VMask);
    v = uint32_t((k >> kH1VB) & kH1VMask);
    w = uint32_t(k & kH1VMask);
}
__device__ __forceinline__ uint32_t h1_key_dpos(uint64_t k) { return uint32_t(k >> (3 * kH1VB)); }

// Endpoints a < b of the sorted edge at p; false for a record that is not an
// edge of the cloud (never, with consistent records).
__device__ __forceinline__ bool h1_uv(const uint32_t *vals, int64_t p, int64_t n, uint32_t &a, uint32_t &b) {
    record_uv(vals[p], false, n, a, b);
    return a < b && int64_t(b) < n;
}

// Column additions of one call before it stops with PH0_ETOOBIG (776 at 700
// uniform points in the plane).
constexpr unsigned long long kH1MaxAdditions = 1ull << 22;

// Counters of the last run (device; read back by h1_counters).
struct H1Counters {
    unsigned long long bars;        // bars written
    unsigned long long zero;        // edges that are the diameter of no triangle
    unsigned long long reduced;     // of them positive: columns reduced
    unsigned long long forest;      // of them spanning-forest edges
    unsigned long long additions;   // column additions
    unsigned long long max_len;     // longest column met
    unsigned long long pool_used;   // keys held by the reduced columns
    unsigned long long nodes;       // pivots claimed by reduced columns
};

// -------------------------------------------------------------- step 1 ---
// a_of[p]: 1-based index in D of the sorted edge at p, from the chunk
// prefixes of the de-duplication scan; one warp per chunk of kDedupeChunk.
__global__ void k_h1_aof(const uint64_t *keys0, const uint64_t *keys1, const Header *esort, int64_t m,
                         const uint32_t *cpref, uint32_t *a_of) {
    const uint64_t *keys = (make_plan(esort).passes & 1) ? keys1 : keys0;
    constexpr int kPer = kDedupeChunk / 32;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; c * kDedupeChunk < m; c += warps) {
        const int64_t p0 = c * kDedupeChunk + lane * kPer;
        uint32_t cnt = 0;
        uint32_t f[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int64_t p = p0 + q;
            f[q] = p < m && (p == 0 || keys[p] != keys[p - 1]) ? 1u : 0u;
            cnt += f[q];
        }
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t run = cpref[c] + inc - cnt;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            run += f[q];
            if (p0 + q < m) a_of[p0 + q] = run;
        }
    }
}

// posof[e]: position in the edge order of the edge with lexicographic index e.
__global__ void k_h1_posof(const uint32_t *vals0, const uint32_t *vals1, const Header *esort, int64_t m,
                           int64_t n, uint32_t *posof) {
    const uint32_t *vals = (make_plan(esort).passes & 1) ? vals1 : vals0;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < m; p += int64_t(gridDim.x) * blockDim.x) {
        uint32_t u, v;
        record_uv(vals[p], false, n, u, v);
        if (u < v && int64_t(v) < n) posof[edge_index(n, u, v)] = uint32_t(p);
    }
}

// P[a][w]: position of edge {a, w}; kH1NoPos on the diagonal (so that w = a
// never counts as an earlier edge).
__global__ void k_h1_pmat(const uint32_t *posof, int64_t n, uint32_t *P) {
    const int64_t nn = n * n;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nn; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t a = i / n, w = i - a * n;
        P[i] = a == w ? kH1NoPos : posof[a < w ? edge_index(n, a, w) : edge_index(n, w, a)];
    }
}

// -------------------------------------------------------------- step 2 ---
// One warp per edge position p = {a, b}: the third vertices w with both
// {a, w} and {b, w} before p are the triangles of diameter p.  tcount[p]:
// their number; tfirst[p]: the smallest w (-1 if none); scan_in[p]: 1 if
// none (for the list of step 3).
__global__ void k_h1_edges(const uint32_t *vals0, const uint32_t *vals1, const Header *esort, int64_t m,
                           int64_t n, const uint32_t *P, uint32_t *tcount, int32_t *tfirst, uint64_t *scan_in) {
    const uint32_t *vals = (make_plan(esort).passes & 1) ? vals1 : vals0;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t p = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < m; p += warps) {
        uint32_t a, b;
        if (!h1_uv(vals, p, n, a, b)) {  // left out: the bar count then shows it
            if (lane == 0) {
                tcount[p] = 0;
                tfirst[p] = -2;
                scan_in[p] = 0;
            }
            continue;
        }
        const uint32_t *Pa = P + int64_t(a) * n, *Pb = P + int64_t(b) * n;
        const uint32_t pp = uint32_t(p);
        uint32_t cnt = 0;
        int32_t first = -1;
        for (int64_t w0 = 0; w0 < n; w0 += 32) {
            const int64_t w = w0 + lane;
            const bool ok = w < n && __ldg(Pa + w) < pp && __ldg(Pb + w) < pp;
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (first < 0 && bal) first = int32_t(w0) + __ffs(bal) - 1;
            cnt += __popc(bal);
        }
        if (lane == 0) {
            tcount[p] = cnt;
            tfirst[p] = first;
            scan_in[p] = cnt == 0 ? 1u : 0u;
        }
    }
}

// ------------------------------------------------- exclusive prefix sums ---
// out[i] = in[0] + ... + in[i-1] for i <= len (out[len] = the total), over
// blocks of kH1ScanItems: per-block sums, their scan, then the blocks.
__device__ __forceinline__ uint64_t h1_block_scan(uint64_t x, uint64_t *s_warp, uint64_t &total) {
    constexpr int NW = kH1Threads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint64_t w = lane < NW ? s_warp[lane] : 0;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) s_warp[lane] = wi - w;
        if (lane == NW - 1) s_warp[NW] = wi;
    }
    __syncthreads();
    total = s_warp[NW];
    const uint64_t r = inc - x + s_warp[warp];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kH1Threads) k_h1_scan_blocks(const uint64_t *in, int64_t len, uint64_t *out,
                                                               uint64_t *bsum) {
    __shared__ uint64_t s_warp[kH1Threads / 32 + 1];
    const int64_t i0 = int64_t(blockIdx.x) * kH1ScanItems + int64_t(threadIdx.x) * 4;
    uint64_t x[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        x[q] = i0 + q < len ? in[i0 + q] : 0;
        sum += x[q];
    }
    uint64_t tot;
    uint64_t run = h1_block_scan(sum, s_warp, tot);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (i0 + q < len) out[i0 + q] = run;
        run += x[q];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One CTA: exclusive scan of the block sums in place; bsum[blocks] = total.
__global__ void __launch_bounds__(kH1Threads) k_h1_scan_sums(uint64_t *bsum, int64_t blocks) {
    __shared__ uint64_t s_warp[kH1Threads / 32 + 1];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < blocks; b0 += kH1Threads) {
        const int64_t b = b0 + threadIdx.x;
        const uint64_t x = b < blocks ? bsum[b] : 0;
        uint64_t tot;
        const uint64_t r = h1_block_scan(x, s_warp, tot);
        const uint64_t carry = s_carry;
        if (b < blocks) bsum[b] = carry + r;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blocks] = s_carry;
}

__global__ void __launch_bounds__(kH1Threads) k_h1_scan_add(uint64_t *out, int64_t len, const uint64_t *bsum,
                                                            int64_t blocks) {
    const int64_t i0 = int64_t(blockIdx.x) * kH1ScanItems + int64_t(threadIdx.x) * 4;
    const uint64_t add = bsum[blockIdx.x];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (i0 + q < len) out[i0 + q] += add;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[len] = bsum[blocks];
}

static cudaError_t h1_scan(const uint64_t *in, int64_t len, uint64_t *out, uint64_t *bsum, cudaStream_t s) {
    const int64_t blocks = (len + kH1ScanItems - 1) / kH1ScanItems;
    if (blocks == 0) return cudaMemsetAsync(out, 0, sizeof(uint64_t), s);
    k_h1_scan_blocks<<<unsigned(blocks), kH1Threads, 0, s>>>(in, len, out, bsum);
    k_h1_scan_sums<<<1, kH1Threads, 0, s>>>(bsum, blocks);
    k_h1_scan_add<<<unsigned(blocks), kH1Threads, 0, s>>>(out, len, bsum, blocks);
    return cudaGetLastError();
}

// -------------------------------------------------------------- step 3 ---
// The positions of the edges that are the diameter of no triangle, in order
// (zpref: exclusive prefix of scan_in).
__global__ void k_h1_zlist(const uint64_t *scan_in, const uint64_t *zpref, int64_t m, uint32_t *zlist) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < m; p += int64_t(gridDim.x) * blockDim.x)
        if (scan_in[p]) zlist[zpref[p]] = uint32_t(p);
}

// Kruskal over the listed edges in order (one thread; union-find with path
// halving in shared memory): an edge that joins two trees is a spanning-
// forest edge (tfirst = -2: its column is cleared), the others are positive
// and go to rlist in order.  A full simplex's forest has n-1 edges.
__global__ void __launch_bounds__(256) k_h1_forest(const uint32_t *vals0, const uint32_t *vals1, const Header *esort,
                                                   const uint32_t *zlist, const uint64_t *zpref, int64_t m, int64_t n,
                                                   int32_t *tfirst, uint32_t *rlist, H1Counters *c, Header *h) {
    __shared__ uint16_t s_par[kH1MaxN];
    const uint32_t *vals = (make_plan(esort).passes & 1) ? vals1 : vals0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_par[i] = uint16_t(i);
    __syncthreads();
    if (threadIdx.x != 0) return;
    auto find = [&](uint32_t x) {
        while (s_par[x] != x) {
            s_par[x] = s_par[s_par[x]];
            x = s_par[x];
        }
        return x;
    };
    const uint64_t Z = zpref[m];
    uint64_t forest = 0, k = 0;
    for (uint64_t z = 0; z < Z; ++z) {
        const uint32_t p = zlist[z];
        uint32_t a, b;
        if (!h1_uv(vals, p, n, a, b)) continue;
        const uint32_t ra = find(a), rb = find(b);
        if (ra != rb) {
            s_par[ra] = uint16_t(rb);
            tfirst[p] = -2;
            ++forest;
        } else {
            rlist[k++] = p;
        }
    }
    c->zero = Z;
    c->forest = forest;
    c->reduced = k;
    if (int64_t(forest) != n - 1) set_status(h, PH0_EINTERNAL);
}

// -------------------------------------------------------------- step 4 ---
struct H1Reduce {
    int64_t n;
    const uint32_t *vals0, *vals1;
    const Header *esort;
    const uint32_t *P;
    const int32_t *tfirst;
    const uint32_t *rlist;
    int32_t *head;             // [m] first claim of each diameter position, -1: none
    uint32_t *claims;          // [m] claims per diameter position
    uint64_t *node_key;        // claims: the pivot triangle,
    uint32_t *node_pos;        //   the claiming column's edge position,
    int32_t *node_next;        //   the next claim of the same diameter,
    uint32_t *node_within;     //   the pivot's rank among its diameter's triangles
    uint32_t *own_node;        // [m] the claim of each reduced column
    uint64_t *own_off;         // [m] its reduced column in the pool
    uint32_t *own_len;
    uint64_t *col_x, *col_m;
    int64_t col_cap;
    uint64_t *pool;
    int64_t pool_cap;
    H1Counters *c;
    Header *h;
};

// The coboundary of edge {a, b} at position p, sorted, into s_keys: n-2 keys
// (the rest of the power of two padded with ~0).  All threads.
__device__ void h1_cobound(const uint32_t *P, int64_t n, uint32_t a, uint32_t b, uint32_t p, uint64_t *s_keys) {
    int n2 = 2;
    while (n2 < n) n2 <<= 1;
    const uint32_t *Pa = P + int64_t(a) * n, *Pb = P + int64_t(b) * n;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        uint64_t k = ~0ull;
        if (i < n && uint32_t(i) != a && uint32_t(i) != b) {
            uint32_t d = p;
            const uint32_t x = Pa[i], y = Pb[i];
            d = x > d ? x : d;
            d = y > d ? y : d;
            k = h1_key(d, a, b, uint32_t(i));
        }
        s_keys[i] = k;
    }
    __syncthreads();
    for (int kk = 2; kk <= n2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t x = s_keys[i], y = s_keys[ixj];
                    const bool up = (i & kk) == 0;
                    if ((x > y) == up) {
                        s_keys[i] = y;
                        s_keys[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Merge-path split: the number of items of A among the first d of the merge
// of A and B (ascending; A first among equal keys).
__device__ __forceinline__ int64_t h1_split(const uint64_t *A, int64_t LA, const uint64_t *B, int64_t LB, int64_t d) {
    int64_t lo = d > LB ? d - LB : 0, hi = d < LA ? d : LA;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// C = A (+) B over F2: the symmetric difference of two ascending lists of
// distinct keys (M: room for LA + LB, the merge with the pairs of equal keys
// side by side); returns its length, or -1 (nothing written to C) above cap.
// All threads.
__device__ int64_t h1_symdiff(const uint64_t *A, int64_t LA, const uint64_t *B, int64_t LB, uint64_t *M,
                              uint64_t *C, int64_t cap, uint64_t *s_warp) {
    const int64_t total = LA + LB, T = blockDim.x, t = threadIdx.x;
    const int64_t d0 = total * t / T, d1 = total * (t + 1) / T;
    int64_t i = h1_split(A, LA, B, LB, d0), j = d0 - i;
    for (int64_t k = d0; k < d1; ++k) {
        if (j >= LB || (i < LA && A[i] <= B[j])) M[k] = A[i++];
        else M[k] = B[j++];
    }
    __syncthreads();
    auto keep = [&](int64_t k) {
        const uint64_t x = M[k];
        return !((k > 0 && M[k - 1] == x) || (k + 1 < total && M[k + 1] == x));
    };
    uint64_t cnt = 0;
    for (int64_t k = d0; k < d1; ++k) cnt += keep(k) ? 1u : 0u;
    uint64_t kept;
    uint64_t off = h1_block_scan(cnt, s_warp, kept);
    if (int64_t(kept) > cap) return -1;
    for (int64_t k = d0; k < d1; ++k)
        if (keep(k)) C[off++] = M[k];
    __syncthreads();
    return int64_t(kept);
}

// The column under reduction: up to kH1Runs sorted runs of keys in X,
// stacked in allocation order; the column is the symmetric difference of
// their live parts [head, end) (heads advance over keys that cancel in
// pairs).  Kept in shared memory, changed by thread 0 between barriers.
struct H1Runs {
    int64_t off[kH1Runs], head[kH1Runs], end[kH1Runs];
    int64_t top;  // first free key of X
    int nr;
};

// Merge the top two runs into the lower one's place (all threads).  The
// result is no longer than the two, and h1_symdiff reads its inputs only
// before its first barrier, so it may overwrite them.
__device__ void h1_merge_top(H1Runs &S, uint64_t *X, uint64_t *M, uint64_t *s_warp) {
    const int i = S.nr - 2;
    const int64_t la = S.end[i] - S.head[i], lb = S.end[i + 1] - S.head[i + 1];
    const int64_t lc = h1_symdiff(X + S.head[i], la, X + S.head[i + 1], lb, M, X + S.off[i], la + lb, s_warp);
    if (threadIdx.x == 0) {
        S.head[i] = S.off[i];
        S.end[i] = S.off[i] + lc;
        S.top = S.end[i];
        S.nr = i + 1;
    }
    __syncthreads();
}

// Push src[0, len) as a new run (all threads), merging runs while the one
// below is at most twice as long (so lengths fall geometrically up the
// stack); when X or the run table is full, every run is merged first and the
// one left moved to the bottom.  False if it still does not fit.
__device__ bool h1_push(H1Runs &S, uint64_t *X, int64_t cap, uint64_t *M, const uint64_t *src, int64_t len,
                        uint64_t *s_warp) {
    if (S.nr == kH1Runs || S.top + len > cap) {
        while (S.nr >= 2) h1_merge_top(S, X, M, s_warp);
        if (S.nr == 1 && S.head[0] > S.off[0]) {
            const int64_t h = S.head[0], l = S.end[0] - S.head[0];
            for (int64_t i = threadIdx.x; i < l; i += blockDim.x) M[i] = X[h + i];
            __syncthreads();
            for (int64_t i = threadIdx.x; i < l; i += blockDim.x) X[i] = M[i];
            __syncthreads();
            if (threadIdx.x == 0) {
                S.off[0] = 0;
                S.head[0] = 0;
                S.end[0] = l;
                S.top = l;
            }
            __syncthreads();
        }
    }
    if (S.top + len > cap) return false;
    const int64_t o = S.top;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) X[o + i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        S.off[S.nr] = o;
        S.head[S.nr] = o;
        S.end[S.nr] = o + len;
        S.top = o + len;
        S.nr += 1;
    }
    __syncthreads();
    while (S.nr >= 2 && S.end[S.nr - 2] - S.head[S.nr - 2] <= 2 * (S.end[S.nr - 1] - S.head[S.nr - 1]))
        h1_merge_top(S, X, M, s_warp);
    return true;
}

// The pivot of the column (thread 0): the smallest key at the heads of the
// runs held by an odd number of them; keys held by an even number cancel and
// their heads advance.  False for an empty column.
__device__ bool h1_pivot(H1Runs &S, const uint64_t *X, uint64_t &piv) {
    for (;;) {
        uint64_t mn = ~0ull;
        int c = 0;
        for (int r = 0; r < S.nr; ++r) {
            if (S.head[r] >= S.end[r]) continue;
            const uint64_t k = X[S.head[r]];
            if (k < mn) {
                mn = k;
                c = 1;
            } else if (k == mn) {
                ++c;
            }
        }
        if (c == 0) return false;
        if (c & 1) {
            piv = mn;
            return true;
        }
        for (int r = 0; r < S.nr; ++r)
            if (S.head[r] < S.end[r] && X[S.head[r]] == mn) S.head[r] += 1;
    }
}

// One CTA: the listed columns from the latest edge down (see the top).
__global__ void __launch_bounds__(kH1Threads) k_h1_reduce(H1Reduce R) {
    __shared__ uint64_t s_keys[kH1MaxN];
    __shared__ uint64_t s_warp[kH1Threads / 32 + 1];
    __shared__ H1Runs S;
    __shared__ uint64_t s_piv;
    __shared__ int32_t s_owner, s_app, s_err;
    __shared__ uint32_t s_node;
    const uint32_t *vals = (make_plan(R.esort).passes & 1) ? R.vals1 : R.vals0;
    const int tid = threadIdx.x;
    const int64_t n = R.n;
    const int64_t K = int64_t(R.c->reduced);
    uint64_t *X = R.col_x, *M = R.col_m;
    unsigned long long adds = 0, maxlen = 0, pool_used = 0, nodes = 0;
    if (tid == 0) s_err = 0;
    __syncthreads();
    for (int64_t k = K - 1; k >= 0; --k) {
        const uint32_t p = R.rlist[k];
        uint32_t a, b;
        h1_uv(vals, p, n, a, b);  // listed from checked records
        if (tid == 0) {
            S.nr = 0;
            S.top = 0;
        }
        __syncthreads();
        h1_cobound(R.P, n, a, b, p, s_keys);
        h1_push(S, X, R.col_cap, M, s_keys, n - 2, s_warp);  // fits: col_cap > n
        for (;;) {
            if (tid == 0) {
                int32_t owner = -1, app = 0;
                uint64_t piv = 0;
                if (!h1_pivot(S, X, piv)) {
                    s_err = PH0_EINTERNAL;  // every positive column keeps a pivot: a bug if not
                } else {
                    const uint32_t dp = h1_key_dpos(piv);
                    uint32_t a2, b2;
                    if (!h1_uv(vals, dp, n, a2, b2)) s_err = PH0_EINTERNAL;
                    if (adds >= kH1MaxAdditions) s_err = PH0_ETOOBIG;
                    const int32_t f = R.tfirst[dp];
                    if (f >= 0 && h1_key(dp, a2, b2, uint32_t(f)) == piv) {
                        owner = int32_t(dp);
                        app = 1;
                    } else {
                        for (int32_t q = R.head[dp]; q >= 0; q = R.node_next[q])
                            if (R.node_key[q] == piv) {
                                owner = int32_t(R.node_pos[q]);
                                break;
                            }
                    }
                }
                s_piv = piv;
                s_owner = owner;
                s_app = app;
            }
            __syncthreads();
            const int32_t owner = s_owner;
            const bool app = s_app != 0;
            const bool stop = s_err != 0;
            __syncthreads();
            if (stop || owner < 0) break;
            bool ok;
            if (app) {
                uint32_t a2, b2;
                h1_uv(vals, owner, n, a2, b2);  // checked above as the pivot's diameter edge
                h1_cobound(R.P, n, a2, b2, uint32_t(owner), s_keys);
                ok = h1_push(S, X, R.col_cap, M, s_keys, n - 2, s_warp);
            } else {
                ok = h1_push(S, X, R.col_cap, M, R.pool + R.own_off[owner], R.own_len[owner], s_warp);
            }
            if (!ok) {
                if (tid == 0) s_err = PH0_ETOOBIG;
                __syncthreads();
                break;
            }
            ++adds;
        }
        __syncthreads();
        if (s_err) break;
        // claim the pivot: a node in the list of its diameter position
        const uint64_t piv = s_piv;
        const uint32_t dp = h1_key_dpos(piv);
        uint32_t a2, b2, u, v, w;
        h1_uv(vals, dp, n, a2, b2);  // checked above
        h1_key_uvw(piv, u, v, w);
        const uint32_t wt = (u != a2 && u != b2) ? u : ((v != a2 && v != b2) ? v : w);
        if (tid == 0) {
            const uint32_t q = uint32_t(nodes++);
            R.node_key[q] = piv;
            R.node_pos[q] = p;
            R.node_next[q] = R.head[dp];
            R.head[dp] = int32_t(q);
            R.claims[dp] += 1;
            R.own_node[p] = q;
            s_node = q;
        }
        // its rank among the triangles of diameter dp: third vertices before wt
        const uint32_t *Pa = R.P + int64_t(a2) * n, *Pb = R.P + int64_t(b2) * n;
        uint64_t cnt = 0;
        for (uint32_t x = tid; x < wt; x += blockDim.x) cnt += (Pa[x] < dp && Pb[x] < dp) ? 1u : 0u;
        uint64_t within;
        h1_block_scan(cnt, s_warp, within);
        if (tid == 0) R.node_within[s_node] = uint32_t(within);
        // the reduced column, one sorted run (its first key is the pivot),
        // kept for the columns below
        while (S.nr >= 2) h1_merge_top(S, X, M, s_warp);
        const int64_t h0 = S.head[0], LA = S.end[0] - S.head[0];
        if (int64_t(pool_used) + LA > R.pool_cap) {
            if (tid == 0) s_err = PH0_ETOOBIG;
            __syncthreads();
            break;
        }
        for (int64_t i = tid; i < LA; i += blockDim.x) R.pool[pool_used + i] = X[h0 + i];
        if (tid == 0) {
            R.own_off[p] = pool_used;
            R.own_len[p] = uint32_t(LA);
        }
        pool_used += uint64_t(LA);
        if (uint64_t(LA) > maxlen) maxlen = uint64_t(LA);
        __syncthreads();
    }
    if (tid == 0) {
        R.c->additions = adds;
        R.c->max_len = maxlen;
        R.c->pool_used = pool_used;
        R.c->nodes = nodes;
        if (s_err) set_status(R.h, s_err);
    }
}

// -------------------------------------------------------------- step 5 ---
// scan_in[p] = (triangles of diameter p) << 24 | (claims at p), whose
// exclusive prefix gives, at p, the rank of p's first triangle in triangle
// order (high part) and the claims of earlier diameters (low 24 bits).
__global__ void k_h1_pack(const uint32_t *tcount, const uint32_t *claims, int64_t m, uint64_t *scan_in) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < m; p += int64_t(gridDim.x) * blockDim.x)
        scan_in[p] = (uint64_t(tcount[p]) << 24) | claims[p];
}

// The bar of every positive edge at its place in triangle order: before the
// bar of apparent edge p come the apparent pairs of earlier edges (p less the
// edges with no triangle before p) and the claims of earlier diameters; before
// a claim at diameter dp come also dp's apparent pair and the claims at dp
// with a smaller rank.
__global__ void k_h1_emit(const uint64_t *ek0, const uint64_t *ek1, const uint32_t *ev0, const uint32_t *ev1,
                          const Header *esort, const uint32_t *a_of, const int32_t *tfirst, const uint64_t *zpref,
                          const uint64_t *tpref, const uint32_t *own_node, const uint64_t *node_key,
                          const uint32_t *node_within, const int32_t *head, const int32_t *node_next, int64_t m,
                          int64_t n, int64_t nbars, ph0_h1bar *bars, H1Counters *c) {
    const bool odd = make_plan(esort).passes & 1;
    const uint64_t *ekey = odd ? ek1 : ek0;
    const uint32_t *eval = odd ? ev1 : ev0;
    unsigned long long written = 0;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < m; p += int64_t(gridDim.x) * blockDim.x) {
        const int32_t f = tfirst[p];
        if (f == -2) continue;  // a spanning-forest edge
        uint32_t a, b;
        if (!h1_uv(eval, p, n, a, b)) continue;
        uint64_t tk, rank, out;
        if (f >= 0) {
            tk = h1_key(uint64_t(p), a, b, uint32_t(f));
            rank = tpref[p] >> 24;
            out = (uint64_t(p) - zpref[p]) + (tpref[p] & 0xffffffu);
        } else {
            const uint32_t q = own_node[p];
            if (q == kH1NoPos) continue;  // the reduction stopped early (its status says why)
            tk = node_key[q];
            const uint32_t dp = h1_key_dpos(tk), wq = node_within[q];
            rank = (tpref[dp] >> 24) + wq;
            uint64_t before = 0;
            for (int32_t r = head[dp]; r >= 0; r = node_next[r]) before += node_within[r] < wq ? 1u : 0u;
            out = (uint64_t(dp) - zpref[dp]) + 1 + (tpref[dp] & 0xffffffu) + before;
        }
        const uint32_t dp = h1_key_dpos(tk);
        uint32_t tu, tv, tw;
        h1_key_uvw(tk, tu, tv, tw);
        if (int64_t(out) >= nbars) continue;  // only with inconsistent counts: the host sees the bar count
        ph0_h1bar bar;
        bar.eu = int32_t(a);
        bar.ev = int32_t(b);
        bar.tu = int32_t(tu);
        bar.tv = int32_t(tv);
        bar.tw = int32_t(tw);
        bar.birth_a = a_of[p];
        bar.death_a = a_of[dp];
        bar._pad = 0;
        bar.birth_order = p;
        bar.death_order = int64_t(dp);
        bar.death_rank = int64_t(rank);
        bar.birth_sq = __longlong_as_double((long long)ekey[p]);
        bar.death_sq = __longlong_as_double((long long)ekey[dp]);
        bars[out] = bar;
        ++written;
    }
    if (written) atomicAdd(&c->bars, written);
}

// ------------------------------------------------------------------ host ---
int sm_count();

// Steps 1-5 of the first homology on a workspace whose dimension-0 part
// holds the sorted edges (buffer by esort's plan) and the de-duplication
// chunk prefixes; bars: n(n-1)/2 - (n-1) entries.  Asynchronous on s;
// after_scan / after_reduce (may be null) are recorded after steps 2 and 4.
cudaError_t run_h1(void *ws, const H1Layout &H, int64_t n, const uint64_t *ek0, const uint64_t *ek1,
                   const uint32_t *ev0, const uint32_t *ev1, const Header *esort, const uint32_t *cpref,
                   Header *h, ph0_h1bar *bars, cudaStream_t s, cudaEvent_t after_scan, cudaEvent_t after_reduce) {
    const int64_t m = n_edges(n);
    H1Counters *c = at<H1Counters>(ws, H.cnt);
    uint32_t *a_of = at<uint32_t>(ws, H.aof), *posof = at<uint32_t>(ws, H.posof), *P = at<uint32_t>(ws, H.pmat);
    uint32_t *tcount = at<uint32_t>(ws, H.tcount);
    int32_t *tfirst = at<int32_t>(ws, H.tfirst);
    uint64_t *scan_in = at<uint64_t>(ws, H.scan_in), *zpref = at<uint64_t>(ws, H.zpref);
    uint64_t *tpref = at<uint64_t>(ws, H.tpref), *bsum = at<uint64_t>(ws, H.bsum);
    uint32_t *zlist = at<uint32_t>(ws, H.zlist), *rlist = at<uint32_t>(ws, H.rlist);
    int32_t *head = at<int32_t>(ws, H.head);
    uint32_t *claims = at<uint32_t>(ws, H.claims);
    cudaError_t e = cudaMemsetAsync(c, 0, sizeof(H1Counters), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(head, 0xff, 4 * size_t(m + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(claims, 0, 4 * size_t(m + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(at<uint32_t>(ws, H.own_node), 0xff, 4 * size_t(m + 1), s);
    if (e != cudaSuccess || H.T == 0) return e;
    const int grid = sm_count() * 8;
    // 1. a and the position of every edge, the position matrix
    k_h1_aof<<<grid, 256, 0, s>>>(ek0, ek1, esort, m, cpref, a_of);
    k_h1_posof<<<grid, 256, 0, s>>>(ev0, ev1, esort, m, n, posof);
    k_h1_pmat<<<grid, 256, 0, s>>>(posof, n, P);
    // 2. the triangles of each diameter; the edges with none, in order
    k_h1_edges<<<grid, 256, 0, s>>>(ev0, ev1, esort, m, n, P, tcount, tfirst, scan_in);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = h1_scan(scan_in, m, zpref, bsum, s)) != cudaSuccess) return e;
    if (after_scan && (e = cudaEventRecord(after_scan, s)) != cudaSuccess) return e;
    // 3. the spanning forest; 4. the other columns
    k_h1_zlist<<<grid, 256, 0, s>>>(scan_in, zpref, m, zlist);
    k_h1_forest<<<1, 256, 0, s>>>(ev0, ev1, esort, zlist, zpref, m, n, tfirst, rlist, c, h);
    H1Reduce R;
    R.n = n;
    R.vals0 = ev0;
    R.vals1 = ev1;
    R.esort = esort;
    R.P = P;
    R.tfirst = tfirst;
    R.rlist = rlist;
    R.head = head;
    R.claims = claims;
    R.node_key = at<uint64_t>(ws, H.node_key);
    R.node_pos = at<uint32_t>(ws, H.node_pos);
    R.node_next = at<int32_t>(ws, H.node_next);
    R.node_within = at<uint32_t>(ws, H.node_within);
    R.own_node = at<uint32_t>(ws, H.own_node);
    R.own_off = at<uint64_t>(ws, H.own_off);
    R.own_len = at<uint32_t>(ws, H.own_len);
    R.col_x = at<uint64_t>(ws, H.col_x);
    R.col_m = at<uint64_t>(ws, H.col_m);
    R.col_cap = H.col_cap;
    R.pool = at<uint64_t>(ws, H.pool);
    R.pool_cap = H.pool_cap;
    R.c = c;
    R.h = h;
    k_h1_reduce<<<1, kH1Threads, 0, s>>>(R);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (after_reduce && (e = cudaEventRecord(after_reduce, s)) != cudaSuccess) return e;
    // 5. ranks in triangle order, the bars
    k_h1_pack<<<grid, 256, 0, s>>>(tcount, claims, m, scan_in);
    if ((e = h1_scan(scan_in, m, tpref, bsum, s)) != cudaSuccess) return e;
    k_h1_emit<<<grid, 256, 0, s>>>(ek0, ek1, ev0, ev1, esort, a_of, tfirst, zpref, tpref, R.own_node, R.node_key,
                                   R.node_within, head, R.node_next, m, n, m - (n - 1), bars, c);
    return cudaGetLastError();
}

// Counters of the last run_h1 on ws (host copy): bars, apparent pairs,
// reduced columns, additions, longest column, pool keys, and the triangle
// count from the prefix sums (n(n-1)(n-2)/6 when consistent).
cudaError_t h1_counters(const void *ws, const H1Layout &H, int64_t n, uint64_t out[7]) {
    H1Counters hc;
    cudaError_t e = cudaMemcpy(&hc, static_cast<const char *>(ws) + H.cnt, sizeof(hc), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    const int64_t m = n_edges(n);
    uint64_t tp = 0;
    e = cudaMemcpy(&tp, static_cast<const char *>(ws) + H.tpref + 8 * size_t(m), sizeof(tp), cudaMemcpyDeviceToHost);
    out[0] = hc.bars;
    out[1] = uint64_t(m) - hc.zero;
    out[2] = hc.reduced;
    out[3] = hc.additions;
    out[4] = hc.max_len;
    out[5] = hc.pool_used;
    out[6] = tp >> 24;
    return e;
}

}  // namespace ph0
