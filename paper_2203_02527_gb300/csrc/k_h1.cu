// k_h1.cu -- first homology of the Vietoris-Rips filtration, the extension
// the paper names (Rawson, Sec. 1 and Sec. 4.2: higher-order homology).  The
// 2-skeleton adds a triangle on three points once its three edges are
// present (Sec. 1, the recursive rule): at its diameter, the latest of its
// edges in the sorted edge order of step 2.  The boundary matrix has a row
// per edge and a column per triangle (its three edges, entries t^a over
// F2[t], which reduce like their F2 supports, as in dimension 0); reducing
// the columns left to right, each nonzero reduced column pairs its low edge
// (a positive edge, one that closed a cycle) with its triangle: the bar
// (a(edge), a(diameter)).  The full simplex has no first homology, so every
// positive edge is paired: n(n-1)/2 - (n-1) bars.
//
// On the GPU:
//   1. the dimension-0 path's sort and de-duplication give every edge its
//      position p in the edge order and its index a(p) (a_of);
//   2. every triangle is written as (diameter position, (u << 20) | (v << 10)
//      | w) in lexicographic order and sorted stably by diameter with the
//      radix sort of step 2: the triangle order (diameter, u, v, w);
//   3. apparent pairs: the first triangle of each diameter owns that edge
//      with its unreduced column (no earlier column can reach a low that
//      late: an earlier triangle's diameter, hence its low, is smaller);
//   4. the other triangles, in windows of consecutive positions, by a
//      persistent cooperative kernel in rounds: each column is added the
//      columns of final owners of its low until it is zero or its low has no
//      final owner (in parallel, one thread per column); then, in position
//      order, a column becomes the final owner of its low L when every
//      earlier column still under reduction has a low below L (lows only
//      fall, so none of them can reach L).  The lowest such column always
//      qualifies, so every round finalizes at least one column, and every
//      column is added only columns to its left: the pairs are those of the
//      left-to-right reduction;
//   5. the paired triangles are compacted in triangle order into the bars.
// Columns under reduction live in fixed slots of kH1Cap entries; the final
// columns of non-apparent owners in a pool.  A column that outgrows its slot,
// or a full pool, stops the kernel with PH0_ETOOBIG (uniform points in the
// plane: columns up to 384 entries at n = 1024, within the 512 of a slot).
#include "ph0_common.cuh"

namespace ph0 {

constexpr int kH1Threads = 512;

__host__ __device__ __forceinline__ uint32_t h1_pack(uint32_t u, uint32_t v, uint32_t w) {
    return (u << 20) | (v << 10) | w;
}
__device__ __forceinline__ void h1_unpack(uint32_t t, uint32_t &u, uint32_t &v, uint32_t &w) {
    u = t >> 20;
    v = (t >> 10) & 1023u;
    w = t & 1023u;
}

// Sorted positions of the three edges of triangle (u, v, w).
__device__ __forceinline__ void h1_tri_edges(const uint32_t *posof, int64_t n, uint32_t u, uint32_t v,
                                             uint32_t w, uint32_t (&e)[3]) {
    uint32_t a = posof[edge_index(n, u, v)], b = posof[edge_index(n, u, w)], c = posof[edge_index(n, v, w)];
    if (a > b) { const uint32_t t = a; a = b; b = t; }
    if (b > c) { const uint32_t t = b; b = c; c = t; }
    if (a > b) { const uint32_t t = a; a = b; b = t; }
    e[0] = a;
    e[1] = b;
    e[2] = c;
}

// out = x (+) y over F2: the symmetric difference of two ascending lists;
// returns its length, or -1 if it would exceed cap.
// (y_l2: y was written by another CTA, read it through L2)
__device__ __forceinline__ int h1_symdiff(const uint32_t *x, int nx, const uint32_t *y, int ny, uint32_t *out,
                                          int cap, bool y_l2) {
    int i = 0, j = 0, k = 0;
    uint32_t xi = nx > 0 ? x[0] : 0, yj = ny > 0 ? (y_l2 ? __ldcg(y) : y[0]) : 0;
    while (i < nx || j < ny) {
        uint32_t val;
        if (j >= ny || (i < nx && xi < yj)) {
            val = xi;
            if (++i < nx) xi = x[i];
        } else if (i >= nx || yj < xi) {
            val = yj;
            if (++j < ny) yj = y_l2 ? __ldcg(y + j) : y[j];
        } else {  // equal rows: 1 + 1 = 0
            if (++i < nx) xi = x[i];
            if (++j < ny) yj = y_l2 ? __ldcg(y + j) : y[j];
            continue;
        }
        if (k >= cap) return -1;
        out[k++] = val;
    }
    return k;
}

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

// -------------------------------------------------------------- step 2 ---
// Triangles in lexicographic order: one warp per edge (u, v), its lanes over
// the third vertices w > v; key = position of the triangle's diameter edge.
__global__ void k_h1_tris(const uint32_t *posof, int64_t n, int64_t m, uint64_t *tkey, uint32_t *tval) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t tot = n * (n - 1) * (n - 2) / 6;
    for (int64_t e = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; e < m; e += warps) {
        uint32_t u, v;
        record_uv(uint32_t(e), true, n, u, v);  // the lexicographic edge index
        // triangles (i, j, k) before (u, v, v+1): those with i < u, then
        // those with i = u and u < j < v
        const int64_t nu = n - u, nv = n - v;
        const int64_t t0 = (tot - nu * (nu - 1) * (nu - 2) / 6) + ((nu - 1) * (nu - 2) / 2 - nv * (nv - 1) / 2);
        const uint32_t puv = posof[e];
        for (int64_t w = int64_t(v) + 1 + lane; w < n; w += 32) {
            const uint32_t puw = posof[edge_index(n, u, w)], pvw = posof[edge_index(n, v, w)];
            uint32_t d = puv > puw ? puv : puw;
            d = d > pvw ? d : pvw;
            const int64_t t = t0 + (w - v - 1);
            tkey[t] = d;
            tval[t] = h1_pack(u, v, uint32_t(w));
        }
    }
}

// -------------------------------------------------------------- step 3 ---
// Apparent pairs: the first triangle of each diameter owns it.
__global__ void k_h1_apparent(const uint64_t *tk0, const uint64_t *tk1, const Header *tsort, int64_t T,
                              int32_t *own_tri, int32_t *pair_low) {
    const uint64_t *tkey = (make_plan(tsort).passes & 1) ? tk1 : tk0;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < T; j += int64_t(gridDim.x) * blockDim.x) {
        const uint64_t d = tkey[j];
        if (j == 0 || tkey[j - 1] != d) {
            own_tri[d] = int32_t(j);
            pair_low[j] = int32_t(d);
        } else {
            pair_low[j] = -1;
        }
    }
}

// -------------------------------------------------------------- step 4 ---
struct H1Counters {
    unsigned long long pool_used;
    unsigned long long bars;
    uint32_t active[2];
    uint32_t rounds;
    uint32_t max_len;
};

struct H1Args {
    int64_t n, m, T, w0, w1;
    const uint32_t *posof;
    const uint64_t *tk0, *tk1;
    const uint32_t *tv0, *tv1;
    const Header *tsort;
    const int32_t *own_tri;
    uint32_t *own_off, *own_len;
    int32_t *pair_low;
    uint32_t *slots, *slen;
    int cap;
    uint32_t *pool;
    unsigned long long pool_cap;
    H1Counters *c;
    Header *h;     // status (the call's header)
    Header *bh;    // grid barrier
};

__global__ void __launch_bounds__(kH1Threads, 1) k_h1_window(H1Args A) {
    __shared__ int s_ok;
    __shared__ uint32_t s_warp[kH1Threads / 32];
    __shared__ int32_t s_carry;
    const bool odd = make_plan(A.tsort).passes & 1;
    const uint32_t *tval = odd ? A.tv1 : A.tv0;
    const int tid = threadIdx.x;
    const int64_t W = A.w1 - A.w0;
    const int64_t gtid = int64_t(blockIdx.x) * kH1Threads + tid, gstride = int64_t(gridDim.x) * kH1Threads;
    const int cap = A.cap;
    auto slot = [&](int64_t i, uint32_t half) { return A.slots + (size_t(i) * 2 + half) * size_t(cap); };

    // A: the window's columns that are not apparent owners
    for (int64_t i = gtid; i < W; i += gstride) {
        const int64_t j = A.w0 + i;
        if (A.pair_low[j] >= 0) {
            A.slen[i] = 0;
            continue;
        }
        uint32_t u, v, w, e[3];
        h1_unpack(tval[j], u, v, w);
        h1_tri_edges(A.posof, A.n, u, v, w, e);
        uint32_t *col = slot(i, 0);
        col[0] = e[0];
        col[1] = e[1];
        col[2] = e[2];
        A.slen[i] = 3;
    }
    if (!grid_barrier(A.bh, &s_ok, kSpinLimit)) return;

    for (uint32_t round = 0;; ++round) {
        // B: add the columns of final owners of the low, while there is one
        if (blockIdx.x == 0 && tid == 0) A.c->active[round & 1] = 0;
        uint32_t longest = 0;
        for (int64_t i = gtid; i < W; i += gstride) {
            uint32_t s = __ldcg(A.slen + i);  // CTA 0 may have finalized it
            int len = int(s & 0x7fffffffu);
            if (len == 0) continue;
            uint32_t half = s >> 31;
            const uint32_t *col = slot(i, half);
            for (;;) {
                const uint32_t L = col[len - 1];
                uint32_t tri3[3];
                const uint32_t *oc;
                int olen;
                const int32_t ot = A.own_tri[L];
                if (ot >= 0) {
                    uint32_t u, v, w;
                    h1_unpack(tval[ot], u, v, w);
                    h1_tri_edges(A.posof, A.n, u, v, w, tri3);
                    oc = tri3;
                    olen = 3;
                } else if (__ldcg(A.own_off + L) != 0xffffffffu) {  // written by CTA 0 in an earlier round
                    oc = A.pool + __ldcg(A.own_off + L);
                    olen = int(__ldcg(A.own_len + L));
                } else {
                    break;  // no final owner: wait for the ordering below
                }
                uint32_t *out = slot(i, half ^ 1u);
                const int k = h1_symdiff(col, len, oc, olen, out, cap, ot < 0);
                if (k < 0) {  // the column outgrew its slot
                    set_status(A.h, PH0_ETOOBIG);
                    atomicExch(&A.bh->abort, 1);
                    len = 0;
                    break;
                }
                half ^= 1u;
                col = out;
                len = k;
                longest = uint32_t(len) > longest ? uint32_t(len) : longest;
                if (len == 0) break;
            }
            A.slen[i] = uint32_t(len) | (half << 31);
        }
        if (longest) atomicMax(&A.c->max_len, longest);
        if (!grid_barrier(A.bh, &s_ok, kSpinLimit)) return;

        // C (one CTA): in position order, a column whose low exceeds every
        // earlier active column's low becomes the final owner of that low
        if (blockIdx.x == 0) {
            if (tid == 0) s_carry = -1;
            __syncthreads();
            uint32_t left = 0;
            for (int64_t base = 0; base < W; base += kH1Threads) {
                const int64_t i = base + tid;
                int32_t low = -1;
                uint32_t s = 0;
                if (i < W) {
                    s = __ldcg(A.slen + i);  // written by other CTAs in part B
                    const int len = int(s & 0x7fffffffu);
                    if (len) low = int32_t(__ldcg(slot(i, s >> 31) + (len - 1)));
                }
                if (!__syncthreads_or(low >= 0)) continue;  // no column left here: the carry stays
                // inclusive max over the block, position order
                int32_t inc = low;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                    if ((tid & 31) >= o) inc = y > inc ? y : inc;
                }
                if ((tid & 31) == 31) s_warp[tid >> 5] = uint32_t(inc);
                __syncthreads();
                int32_t before = s_carry;
                for (int wp = 0; wp < (tid >> 5); ++wp) {
                    const int32_t y = int32_t(s_warp[wp]);
                    before = y > before ? y : before;
                }
                {
                    const int32_t y = __shfl_up_sync(0xffffffffu, inc, 1);
                    if ((tid & 31) >= 1) before = y > before ? y : before;
                }
                if (low >= 0) {
                    if (before < low) {
                        const int len = int(s & 0x7fffffffu);
                        const uint32_t *col = slot(i, s >> 31);
                        const unsigned long long off = atomicAdd(&A.c->pool_used, (unsigned long long)len);
                        if (off + len > A.pool_cap) {
                            set_status(A.h, PH0_ETOOBIG);
                            atomicExch(&A.bh->abort, 1);
                        } else {
                            for (int q = 0; q < len; ++q) A.pool[off + q] = __ldcg(col + q);
                            A.own_len[low] = uint32_t(len);
                            A.own_off[low] = uint32_t(off);
                            A.pair_low[A.w0 + i] = low;
                        }
                        A.slen[i] = 0;
                    } else {
                        ++left;
                    }
                }
                __syncthreads();
                if (tid == kH1Threads - 1) {
                    const int32_t tot = before > inc ? before : inc;
                    s_carry = tot > s_carry ? tot : s_carry;
                }
                __syncthreads();
            }
            if (left) atomicAdd(&A.c->active[round & 1], left);
            if (tid == 0) atomicAdd(&A.c->rounds, 1u);
        }
        if (!grid_barrier(A.bh, &s_ok, kSpinLimit)) return;
        if (ld_volatile(&A.c->active[round & 1]) == 0 || ld_volatile(&A.bh->abort)) break;
    }
}

// -------------------------------------------------------------- step 5 ---
__global__ void k_h1_count(const int32_t *pair_low, int64_t T, uint32_t *cnt) {
    __shared__ uint32_t s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kH1ChunkTris;
    uint32_t c = 0;
    for (int q = threadIdx.x; q < kH1ChunkTris; q += blockDim.x) {
        const int64_t j = base + q;
        c += (j < T && pair_low[j] >= 0) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_sum, c);
    __syncthreads();
    if (threadIdx.x == 0) cnt[blockIdx.x] = s_sum;
}

// Exclusive scan of the chunk counts in place (one CTA); total to *total.
__global__ void k_h1_scan(uint32_t *cnt, int64_t chunks, unsigned long long *total) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < chunks; base += blockDim.x) {
        const int64_t i = base + tid;
        const uint32_t x = i < chunks ? cnt[i] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        uint32_t before = s_carry;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        if (i < chunks) cnt[i] = before + inc - x;
        __syncthreads();
        if (tid == int(blockDim.x) - 1) s_carry = before + inc;
        __syncthreads();
    }
    if (tid == 0) *total = s_carry;
}

// The bars of one chunk of triangles, in triangle order.
__global__ void k_h1_emit(const int32_t *pair_low, int64_t T, const uint32_t *cnt, const uint64_t *tk0,
                          const uint64_t *tk1, const uint32_t *tv0, const uint32_t *tv1, const Header *tsort,
                          const uint64_t *ek0, const uint64_t *ek1, const uint32_t *ev0, const uint32_t *ev1,
                          const Header *esort, const uint32_t *a_of, int64_t n, int64_t nbars, ph0_h1bar *bars) {
    __shared__ uint32_t s_warp[kH1Threads / 32];
    __shared__ uint32_t s_carry;
    const bool todd = make_plan(tsort).passes & 1, eodd = make_plan(esort).passes & 1;
    const uint64_t *tkey = todd ? tk1 : tk0;
    const uint32_t *tval = todd ? tv1 : tv0;
    const uint64_t *ekey = eodd ? ek1 : ek0;
    const uint32_t *eval = eodd ? ev1 : ev0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = cnt[blockIdx.x];
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kH1ChunkTris;
    for (int q0 = 0; q0 < kH1ChunkTris; q0 += kH1Threads) {
        const int64_t j = base + q0 + tid;
        const bool has = j < T && pair_low[j] >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, has);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = s_carry;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        before += __popc(bal & ((1u << lane) - 1u));
        if (has && int64_t(before) < nbars) {
            const uint32_t p = uint32_t(pair_low[j]);
            const uint32_t dpos = uint32_t(tkey[j]);
            uint32_t eu, ev, tu, tv, tw;
            record_uv(eval[p], false, n, eu, ev);
            h1_unpack(tval[j], tu, tv, tw);
            ph0_h1bar b;
            b.eu = int32_t(eu);
            b.ev = int32_t(ev);
            b.tu = int32_t(tu);
            b.tv = int32_t(tv);
            b.tw = int32_t(tw);
            b.birth_a = a_of[p];
            b.death_a = a_of[dpos];
            b._pad = 0;
            b.birth_order = int64_t(p);
            b.death_order = int64_t(dpos);
            b.death_rank = j;
            b.birth_sq = __longlong_as_double((long long)ekey[p]);
            b.death_sq = __longlong_as_double((long long)ekey[dpos]);
            bars[before] = b;
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < kH1Threads / 32; ++w) tot += s_warp[w];
            s_carry += tot;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host ---
int sm_count();
cudaError_t launch_sort_init(Header *h, uint64_t *look0, int64_t tiles, cudaStream_t s, int top_bits,
                             int64_t sorted_edges, const int32_t *gate);
cudaError_t launch_keystats(const uint64_t *keys, int64_t m, Header *h, cudaStream_t s, const int32_t *gate);
cudaError_t launch_sort_passes(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                               int64_t m, uint64_t *look0, uint64_t *look1, Header *h,
                               cudaStream_t s, bool persist);

// Steps 1-5 of the first homology on a workspace whose dimension-0 part
// holds the sorted edges (buffer by esort's plan) and the de-duplication
// chunk prefixes; bars: n(n-1)/2 - (n-1) entries.  Asynchronous on s.
cudaError_t run_h1(void *ws, const H1Layout &H, int64_t n, const uint64_t *ek0, const uint64_t *ek1,
                   const uint32_t *ev0, const uint32_t *ev1, const Header *esort, const uint32_t *cpref,
                   Header *h, ph0_h1bar *bars, cudaStream_t s, cudaEvent_t after_sort, cudaEvent_t after_reduce) {
    const int64_t m = n_edges(n), T = H.T;
    Header *th = at<Header>(ws, H.thdr);
    H1Counters *c = at<H1Counters>(ws, H.cnt);
    uint32_t *a_of = at<uint32_t>(ws, H.aof), *posof = at<uint32_t>(ws, H.posof);
    uint64_t *tk0 = at<uint64_t>(ws, H.tkey[0]), *tk1 = at<uint64_t>(ws, H.tkey[1]);
    uint32_t *tv0 = at<uint32_t>(ws, H.tval[0]), *tv1 = at<uint32_t>(ws, H.tval[1]);
    int32_t *own_tri = at<int32_t>(ws, H.own_tri), *pair_low = at<int32_t>(ws, H.pair_low);
    uint32_t *own_off = at<uint32_t>(ws, H.own_off), *own_len = at<uint32_t>(ws, H.own_len);
    cudaError_t e = cudaMemsetAsync(th, 0, kHeaderBytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c, 0, sizeof(H1Counters), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(own_tri, 0xff, 4 * size_t(m), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(own_off, 0xff, 4 * size_t(m), s);
    if (e != cudaSuccess || T == 0) return e;
    const int grid = sm_count() * 8;
    // 1. a and the position of every edge; 2. the triangles, sorted
    k_h1_aof<<<grid, 256, 0, s>>>(ek0, ek1, esort, m, cpref, a_of);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_h1_posof<<<grid, 256, 0, s>>>(ev0, ev1, esort, m, n, posof);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_h1_tris<<<grid, 256, 0, s>>>(posof, n, m, tk0, tv0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_sort_init(th, at<uint64_t>(ws, H.tlook[0]), H.ttiles, s, kDefaultTopBits, T, nullptr);
    if (e == cudaSuccess) e = launch_keystats(tk0, T, th, s, nullptr);
    if (e == cudaSuccess)
        e = launch_sort_passes(tk0, tk1, tv0, tv1, T, at<uint64_t>(ws, H.tlook[0]), at<uint64_t>(ws, H.tlook[1]), th,
                               s, false);
    if (e == cudaSuccess && after_sort) e = cudaEventRecord(after_sort, s);
    if (e != cudaSuccess) return e;
    // 3. apparent pairs; 4. the other columns, window by window
    k_h1_apparent<<<grid, 256, 0, s>>>(tk0, tk1, th, T, own_tri, pair_low);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_h1_window, kH1Threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int wgrid = sm_count() * (per_sm > 2 ? 2 : per_sm);
    H1Args A;
    A.n = n;
    A.m = m;
    A.T = T;
    A.posof = posof;
    A.tk0 = tk0;
    A.tk1 = tk1;
    A.tv0 = tv0;
    A.tv1 = tv1;
    A.tsort = th;
    A.own_tri = own_tri;
    A.own_off = own_off;
    A.own_len = own_len;
    A.pair_low = pair_low;
    A.slots = at<uint32_t>(ws, H.slots);
    A.slen = at<uint32_t>(ws, H.slen);
    A.cap = kH1Cap;
    A.pool = at<uint32_t>(ws, H.pool);
    A.pool_cap = (unsigned long long)H.pool_cap;
    A.c = c;
    A.h = h;
    A.bh = th;
    for (int64_t w0 = 0; w0 < T; w0 += H.W) {
        A.w0 = w0;
        A.w1 = w0 + H.W < T ? w0 + H.W : T;
        H1Args args = A;
        void *params[] = {&args};
        e = cudaLaunchCooperativeKernel((const void *)k_h1_window, dim3(wgrid), dim3(kH1Threads), params, 0, s);
        if (e != cudaSuccess) return e;
    }
    if (after_reduce && (e = cudaEventRecord(after_reduce, s)) != cudaSuccess) return e;
    // 5. the bars in triangle order
    uint32_t *ccount = at<uint32_t>(ws, H.ccount);
    k_h1_count<<<unsigned(H.chunks), 256, 0, s>>>(pair_low, T, ccount);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_h1_scan<<<1, 1024, 0, s>>>(ccount, H.chunks, &c->bars);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_h1_emit<<<unsigned(H.chunks), kH1Threads, 0, s>>>(pair_low, T, ccount, tk0, tk1, tv0, tv1, th, ek0, ek1, ev0,
                                                        ev1, esort, a_of, n, m - (n - 1), bars);
    return cudaGetLastError();
}

// Counters of the last run_h1 on ws (host copy).
cudaError_t h1_counters(const void *ws, const H1Layout &H, uint64_t out[5]) {
    H1Counters hc;
    cudaError_t e = cudaMemcpy(&hc, static_cast<const char *>(ws) + H.cnt, sizeof(hc), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    out[0] = hc.bars;
    out[1] = hc.pool_used;
    out[2] = hc.rounds;
    out[3] = hc.max_len;
    int32_t tstatus = 0;  // the triangle sort's header: its status word comes first
    e = cudaMemcpy(&tstatus, static_cast<const char *>(ws) + H.thdr, sizeof(tstatus), cudaMemcpyDeviceToHost);
    out[4] = uint64_t(uint32_t(tstatus));
    return e;
}

}  // namespace ph0
