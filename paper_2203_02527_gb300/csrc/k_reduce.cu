// k_reduce.cu -- steps 4-5 of the barcode path: the boundary matrix M over
// F2[t] and its column reduction (Rawson, Sec. 2; Sec. 4 steps 3-5).
//
// Column p of M (edges in sorted order) has the two rows u_p < v_p, both
// t^a(p).  Adding column k into column j multiplies it by t^(a(j)-a(k)), so
// every entry of a reduced column j stays t^a(j) and the reduction is the F2
// reduction of the supports.  Supports are pairs; a reduced nonzero column is
// a pair {x, L} whose pivot ("low", largest row) is L.  Following the pivot
// table from a row always moves to a smaller row, so the rows reachable from a
// vertex form a tree whose root is the smallest vertex of its connected
// component, and reducing column p = {u, v} ends either in zero (u and v are
// already connected by earlier columns: no bar) or with the pivot
// L = max(root(u), root(v)) claimed by p: a bar (0, a(p)) (Sec. 2: each
// pivot entry t^b left after the reduction gives the bar (0, b)).
// This is the pairing the left-to-right reduction produces, so the kernel
// keeps, per vertex, the root of its component (a flattened pivot table) and
// never stores M.
//
// The columns are processed in windows of consecutive sorted positions by one
// persistent cooperative kernel with bounded grid barriers:
//   F (filter)  every column whose endpoints have the same root in the
//               snapshot of the window start is zero (its endpoints are joined
//               by earlier columns) and is dropped.  Of the columns left, only
//               the first with a given pair of snapshot roots can be nonzero;
//               a per-CTA hash table keeps that one.
//   R (rounds)  every surviving column looks up the current roots of its two
//               endpoints; equal roots -> zero column.  Otherwise it claims
//               both root slots with an atomic minimum of its position
//               (priority to the lower filtration position).  A column that
//               holds the slot of the larger root H is the first remaining
//               column touching H's component, so in the left-to-right order
//               nothing before it changes that component, whose minimum is H;
//               and every link made so far on the path from its other endpoint
//               to that endpoint's (smaller) root comes from an earlier column
//               (each link is made by the first remaining column touching the
//               linked component).  So the column is nonzero with pivot H; it
//               links H under the smaller root, which keeps every root the
//               minimum of its component.  Other columns retry next round.
//               Each round the lowest remaining column holds its larger root,
//               so the rounds end.  Once at most kTailCap columns are left, one
//               CTA finishes the window's rounds in shared memory.
//   flatten     every vertex's root is updated.
// Early exit: once n-1 pivots exist every later column is zero (the graph is
// connected); the window loop stops.
#include <cooperative_groups.h>
#include <type_traits>

#include "ph0_common.cuh"

namespace ph0 {

constexpr int kReduceThreads = 512;
constexpr int kFilterLoads = 4;
constexpr int kHashSize = 2048;
constexpr uint32_t kEmpty = 0xffffffffu;


__global__ void k_reduce_init(ReduceArgs A) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = tid; i < int64_t(kTraceWindows) * kTraceWords; i += stride) A.trace[i] = 0;
    for (int64_t v = tid; v < A.n; v += stride) {
        A.comp[v] = uint32_t(v);
        A.parent[v] = uint32_t(v);
        A.res[v] = ~0ull;
        A.kill_key[v] = ~0ull;
        A.kill_val[v] = 0;
    }
    if (tid == 0) {
        // XOR of 0..n-1; k_emit folds in every pivot row, leaving the vertex
        // that is no pivot row: the bar that never dies
        const uint64_t top = A.n > 0 ? uint64_t(A.n - 1) : 0;
        const uint32_t x = (top & 3) == 0 ? uint32_t(top) : (top & 3) == 1 ? 1u : (top & 3) == 2 ? uint32_t(top + 1) : 0u;
        A.h->inf_xor = x;
        A.h->npiv = 0;
        A.h->nlist[0] = 0;
        A.h->nlist[1] = 0;
        A.h->bar_count = 0;
        A.h->bar_gen = 0;
        A.h->abort = 0;
    }
}

__device__ __forceinline__ uint32_t find_root(const uint32_t *parent, uint32_t r) {
    for (;;) {
        const uint32_t p = __ldcg(parent + r);
        if (p == r) return r;
        r = p;
    }
}

// Warp-aggregated append of `p` (where `take`) to a list; every lane of the
// warp must call it.
__device__ __forceinline__ void warp_append(bool take, uint32_t p, uint32_t *list, uint32_t *count) {
    const unsigned mask = __ballot_sync(0xffffffffu, take);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, uint32_t(__popc(mask)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (take) list[base + __popc(mask & ((1u << lane) - 1u))] = p;
}


__device__ __forceinline__ void record_pivot(const ReduceArgs &A, Header *h, uint32_t target,
                                             uint32_t p, uint32_t low) {
    const uint32_t j = atomicAdd(&h->npiv, 1u);
    if (j < target) {
        A.kill_key[j] = p;
        A.kill_val[j] = low;
    } else {
        set_status(h, PH0_EINTERNAL);
    }
}

__device__ __forceinline__ uint16_t local_find(uint16_t *par, uint16_t x) {
    for (;;) {
        const uint16_t p = par[x];
        if (p == x) return x;
        const uint16_t g = par[p];
        par[x] = g;  // path halving (benign race: only moves toward the root)
        x = g;
    }
}

// The candidate rounds of one window, run by a single CTA (all threads) in
// shared memory once at most kTailCap candidates are left.  Same rules as the
// grid rounds; the current roots of the candidates' endpoints get local ids
// (the snapshot array is reused as the global->local map), so every find,
// claim and link is a shared-memory access and rounds are separated by
// __syncthreads instead of grid barriers.  Returns the number of rounds.
// Vertex ids in the tail's shared arrays: 16 bits, or 32 (wide records).
template <bool WIDE>
using TailRoot = typename std::conditional<WIDE, uint32_t, uint16_t>::type;

template <bool WIDE>
__device__ uint32_t tail_rounds(const ReduceArgs &A, Header *h, const uint32_t *val,
                                const uint32_t *list, uint32_t ncur, uint16_t *s_comp,
                                unsigned char *s_tail, uint32_t target, uint32_t &claims) {
    constexpr int C = kTailCap;
    using R = TailRoot<WIDE>;
    uint32_t *s_p = reinterpret_cast<uint32_t *>(s_tail);        // [C] position
    uint32_t *s_lres = s_p + C;                                   // [2C] claim per local root
    R *s_ra = reinterpret_cast<R *>(s_lres + 2 * C);              // [C] this round's roots
    R *s_rb = s_ra + C;
    R *s_gid = s_rb + C;                                          // [2C] global id
    uint16_t *s_lu = reinterpret_cast<uint16_t *>(s_gid + 2 * C);  // [C] local root, u side
    uint16_t *s_lv = s_lu + C;                                    // [C] local root, v side
    uint16_t *s_lpar = s_lv + C;                                  // [2C] local parent
    uint8_t *s_act = reinterpret_cast<uint8_t *>(s_lpar + 2 * C);  // [C] still active
    // the map global root -> local id: the snapshot array (its window is
    // over), or for wide records the workspace's gmap (32-bit entries)
    auto map_get = [&](R g) -> uint32_t {
        if constexpr (WIDE) return __ldcg(A.gmap + g);
        else return s_comp[g];
    };
    __shared__ uint32_t s_nroots, s_left;
    const int tid = threadIdx.x;
    const int T = blockDim.x;
    if (tid == 0) {
        s_nroots = 0;
        s_left = 0;
    }
    // global roots and window-start roots of every endpoint
    for (uint32_t i = tid; i < ncur; i += T) {
        const uint32_t p = __ldcg(list + i);
        uint32_t u, v;
        rec_uv<WIDE>(val[p], p, A.hib, A.n, u, v);
        s_p[i] = p;
        s_ra[i] = R(find_root(A.parent, __ldcg(A.comp + u)));
        s_rb[i] = R(find_root(A.parent, __ldcg(A.comp + v)));
        s_act[i] = 1;
    }
    __syncthreads();
    // local ids: the map's entries of these roots are set to "unseen", then
    // the first thread to claim a root gives it the next local id
    for (uint32_t i = tid; i < ncur; i += T) {
        if constexpr (WIDE) {
            A.gmap[s_ra[i]] = 0xffffffffu;
            A.gmap[s_rb[i]] = 0xffffffffu;
        } else {
            s_comp[s_ra[i]] = 0xffffu;
            s_comp[s_rb[i]] = 0xffffu;
        }
    }
    __threadfence_block();
    __syncthreads();
    for (uint32_t i = tid; i < ncur; i += T) {
        for (int side = 0; side < 2; ++side) {
            const R g = side ? s_rb[i] : s_ra[i];
            bool first;
            if constexpr (WIDE) first = atomicCAS(A.gmap + g, 0xffffffffu, 0xfffffffeu) == 0xffffffffu;
            else
                first = atomicCAS(reinterpret_cast<unsigned short *>(s_comp + g), (unsigned short)0xffffu,
                                  (unsigned short)0xfffeu) == 0xffffu;
            if (first) {
                const uint32_t id = atomicAdd(&s_nroots, 1u);
                s_gid[id] = g;
                s_lpar[id] = uint16_t(id);
                s_lres[id] = 0xffffffffu;
                if constexpr (WIDE) atomicExch(A.gmap + g, id);
                else s_comp[g] = uint16_t(id);
            }
        }
    }
    __threadfence_block();
    __syncthreads();
    for (uint32_t i = tid; i < ncur; i += T) {
        s_lu[i] = uint16_t(map_get(s_ra[i]));
        s_lv[i] = uint16_t(map_get(s_rb[i]));
    }
    __syncthreads();
    uint32_t rounds = 0;
    for (;;) {
        ++rounds;
        for (uint32_t i = tid; i < ncur; i += T) {
            if (!s_act[i]) continue;
            const uint16_t a = local_find(s_lpar, s_lu[i]), b = local_find(s_lpar, s_lv[i]);
            if (a == b) {
                s_act[i] = 0;
                continue;
            }
            s_ra[i] = R(a);
            s_rb[i] = R(b);
            atomicMin(s_lres + a, s_p[i]);
            atomicMin(s_lres + b, s_p[i]);
            claims += 2;
        }
        __syncthreads();
        uint32_t left = 0;
        for (uint32_t i = tid; i < ncur; i += T) {
            if (!s_act[i]) continue;
            const uint16_t a = uint16_t(s_ra[i]), b = uint16_t(s_rb[i]);
            const uint32_t p = s_p[i];
            const bool a_lo = s_gid[a] < s_gid[b];
            const uint16_t lo = a_lo ? a : b, hi = a_lo ? b : a;
            if (s_lres[hi] == p) {
                s_lpar[hi] = lo;
                s_act[i] = 0;
                record_pivot(A, h, target, p, s_gid[hi]);
            } else {
                ++left;
            }
        }
        if (left) atomicAdd(&s_left, left);
        __syncthreads();
        for (uint32_t r = tid; r < s_nroots; r += T) s_lres[r] = 0xffffffffu;
        const uint32_t remaining = s_left;
        __syncthreads();
        if (tid == 0) s_left = 0;
        if (remaining == 0) break;
        __syncthreads();
    }
    // write the links back to the global root table
    __syncthreads();
    for (uint32_t r = tid; r < s_nroots; r += T)
        if (s_lpar[r] != r) A.parent[s_gid[r]] = s_gid[s_lpar[r]];
    __syncthreads();
    return rounds;
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// WIDE (records hold edge indices, n up to kMaxNWide): the window's root
// snapshot is read from the global root table instead of a 16-bit copy in
// shared memory, and root pairs are 64-bit hash keys.
template <bool WIDE>
__global__ void __launch_bounds__(kReduceThreads, 1) k_reduce(ReduceArgs A) {
    using PairT = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    constexpr PairT kPairEmpty = ~PairT(0);
    extern __shared__ uint16_t s_comp[];  // [n] root snapshot of the window (not WIDE)
    __shared__ PairT s_hkey[kHashSize];
    __shared__ uint32_t s_hval[kHashSize];
    __shared__ uint32_t s_hcount;
    __shared__ int s_ok;
    // snapshot root of vertex x at the window start
    auto snap = [&](uint32_t x) -> uint32_t {
        if constexpr (WIDE) return __ldcg(A.comp + x);
        else return s_comp[x];
    };

    Header *h = A.h;
    const int64_t n = A.n, m = A.m;
    if (m <= 0) return;
    const uint32_t *val = A.val0;
    if (A.sort_h) val = (make_plan(A.sort_h).passes & 1) ? A.val1 : A.val0;
    // the packed sort's records, unless its fallback replaced them
    if (A.valp && ld_volatile(&h->packed) != 0 && ld_volatile(&h->fixup_fallback) == 0) val = A.valp;
    const int tid = threadIdx.x;
    const int64_t G = gridDim.x;
    const int64_t gtid = int64_t(blockIdx.x) * kReduceThreads + tid;
    const int64_t gstride = G * kReduceThreads;
    const uint32_t target = uint32_t(n - 1);

    int64_t pos0 = A.start, W = A.w0;
    uint32_t round = 0;       // grid rounds: identical in every CTA (claim tags)
    int64_t tail_total = 0;   // shared-memory rounds (CTA 0)
    int windows = 0;
    int64_t candidates = 0;
    uint32_t claims = 0;          // atomic claims issued by this thread
    uint32_t rounds_max = 0;      // most claim rounds in one window (CTA 0)
    for (;;) {
        const uint32_t npiv = __ldcg(&h->npiv);
        if (pos0 >= m || npiv >= target) break;
        const int64_t wend = (m - pos0 < W) ? m : pos0 + W;
        ++windows;
        const bool tr = blockIdx.x == 0 && tid == 0 && windows <= kTraceWindows;
        uint64_t *rec = A.trace + size_t(windows - 1) * kTraceWords;
        const uint32_t round_before = round;
        const int64_t tail_before = tail_total;
        if (tr) {
            rec[0] = pos0;
            rec[1] = W;
            rec[6] = gtimer();
        }

        // ---------------- F: filter the window against the snapshot -------
        if constexpr (!WIDE)
            for (int64_t v = tid; v < n; v += kReduceThreads) s_comp[v] = uint16_t(__ldcg(A.comp + v));
        for (int i = tid; i < kHashSize; i += kReduceThreads) {
            s_hkey[i] = kPairEmpty;
            s_hval[i] = kEmpty;
        }
        if (tid == 0) s_hcount = 0;
        __syncthreads();
        // kFilterLoads 16-byte loads (4 records each) in flight per thread and
        // iteration (one CTA per SM: the filter is bound by the bytes in
        // flight and the work per record)
        const bool vec = ((reinterpret_cast<uintptr_t>(val + pos0) & 15u) == 0);
        constexpr int kSpan = kFilterLoads * 4 * kReduceThreads;  // records per CTA and iteration
        for (int64_t b = pos0 + int64_t(blockIdx.x) * kSpan; b < wend; b += G * kSpan) {
            uint32_t vq[kFilterLoads * 4];
#pragma unroll
            for (int q = 0; q < kFilterLoads; ++q) {
                const int64_t p0 = b + (int64_t(q) * kReduceThreads + tid) * 4;
                if (vec && p0 + 4 <= wend) {
                    const uint4 w = *reinterpret_cast<const uint4 *>(val + p0);
                    vq[4 * q] = w.x;
                    vq[4 * q + 1] = w.y;
                    vq[4 * q + 2] = w.z;
                    vq[4 * q + 3] = w.w;
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) vq[4 * q + r] = p0 + r < wend ? val[p0 + r] : 0u;
                }
            }
            // the endpoints' snapshot roots of every record first (bit qr of
            // `differ`: different roots); late windows have almost none, and
            // then the warp skips the candidate handling below at once
            uint32_t differ = 0;
#pragma unroll
            for (int qr = 0; qr < kFilterLoads * 4; ++qr) {
                const int64_t p = b + (int64_t(qr >> 2) * kReduceThreads + tid) * 4 + (qr & 3);
                if (p < wend) {
                    uint32_t vv = vq[qr];
                    // corrupt input: never index past n
                    const bool bad = WIDE ? (int64_t(vv) | index_hi(A.hib, p)) >= A.m_edges
                                          : ((vv >> 16) >= n || (vv & 0xffffu) >= n);
                    if (bad) {  // reported, and never a candidate
                        set_status(h, PH0_EINTERNAL);
                    } else {
                        uint32_t u, v;
                        rec_uv<WIDE>(vv, p, A.hib, n, u, v);
                        if (snap(u) != snap(v)) differ |= 1u << qr;
                    }
                }
            }
            if (!__any_sync(0xffffffffu, differ != 0)) continue;
            uint32_t direct = 0;  // bit qr: the record goes to the candidate list as it is
#pragma unroll
            for (int qr = 0; qr < kFilterLoads * 4; ++qr) {
                const int64_t p = b + (int64_t(qr >> 2) * kReduceThreads + tid) * 4 + (qr & 3);
                if ((differ >> qr) & 1u) {
                    uint32_t u, v;
                    rec_uv<WIDE>(vq[qr], p, A.hib, n, u, v);
                    const uint32_t cu = snap(u), cv = snap(v);
                    const uint32_t lo = cu < cv ? cu : cv, hi = cu < cv ? cv : cu;
                    const PairT pair = (PairT(lo) << (WIDE ? 32 : 16)) | hi;
                    bool done = false;
                    if (*(volatile uint32_t *)&s_hcount < kHashSize / 2) {
                        const uint32_t hs = (uint32_t(pair ^ (pair >> 29)) * 2654435761u) >> 21;  // 11 bits
                        for (int pr = 0; pr < 8; ++pr) {
                            const uint32_t slot = (hs + pr) & (kHashSize - 1);
                            // a slot keeps its pair for the whole window, so a plain
                            // read that finds it needs no CAS; the minimum only
                            // falls, so a plain read at or below p needs no atomic
                            // (every record of a pair hits one slot: no contention)
                            PairT old = *(volatile PairT *)&s_hkey[slot];
                            if (old != pair) {
                                old = atomicCAS(&s_hkey[slot], kPairEmpty, pair);
                                if (old == kPairEmpty) atomicAdd(&s_hcount, 1u);
                            }
                            if (old == kPairEmpty || old == pair) {
                                if (*(volatile uint32_t *)&s_hval[slot] > uint32_t(p))
                                    atomicMin(&s_hval[slot], uint32_t(p));
                                done = true;
                                break;
                            }
                        }
                    }
                    if (!done) direct |= 1u << qr;
                }
            }
            if (!__any_sync(0xffffffffu, direct != 0)) continue;
#pragma unroll
            for (int qr = 0; qr < kFilterLoads * 4; ++qr) {
                const int64_t p = b + (int64_t(qr >> 2) * kReduceThreads + tid) * 4 + (qr & 3);
                warp_append((direct >> qr) & 1u, uint32_t(p), A.cand0, &h->nlist[0]);
            }
        }
        __syncthreads();
        for (int slot = tid; slot < kHashSize; slot += kReduceThreads) {
            const bool has = s_hkey[slot] != kPairEmpty;
            warp_append(has, s_hval[slot], A.cand0, &h->nlist[0]);
        }
        if (!grid_barrier(h, &s_ok, A.spin_limit)) return;

        // ---------------- R: claim pivots in rounds ------------------------
        int cur = 0;
        uint32_t ncur = __ldcg(&h->nlist[0]);
        const uint32_t nwin = ncur;
        candidates += nwin;
        if (tr) {
            rec[2] = nwin;
            rec[7] = gtimer();
        }
        while (ncur > uint32_t(kTailCap)) {
            ++round;
            const unsigned long long tag = (unsigned long long)(0xffffffffu - round) << 32;
            const uint32_t *list = cur ? A.cand1 : A.cand0;
            uint32_t *next = cur ? A.cand0 : A.cand1;
            uint32_t *next_count = &h->nlist[cur ^ 1];
            if (blockIdx.x == 0 && tid == 0) *next_count = 0;
            // claim both current roots
            for (int64_t i = gtid; i < ncur; i += gstride) {
                const uint32_t p = __ldcg(list + i);
                uint32_t u, v;
                rec_uv<WIDE>(val[p], p, A.hib, n, u, v);
                const uint32_t ru = find_root(A.parent, __ldcg(A.comp + u));
                const uint32_t rv = find_root(A.parent, __ldcg(A.comp + v));
                if (ru == rv) {
                    A.candr[i] = ~0ull;
                } else {
                    A.candr[i] = (static_cast<unsigned long long>(ru) << 32) | rv;
                    atomicMin(A.res + ru, tag | p);
                    atomicMin(A.res + rv, tag | p);
                    claims += 2;
                }
            }
            if (!grid_barrier(h, &s_ok, A.spin_limit)) return;
            // commit the columns that hold their larger root H: pivot H
            for (int64_t b = int64_t(blockIdx.x) * kReduceThreads; b < ncur; b += gstride) {
                const int64_t i = b + tid;
                bool keep = false;
                uint32_t p = 0;
                if (i < ncur) {
                    const unsigned long long r = __ldcg(A.candr + i);
                    if (r != ~0ull) {
                        p = __ldcg(list + i);
                        const uint32_t ru = uint32_t(r >> 32), rv = uint32_t(r);
                        const uint32_t lo = ru < rv ? ru : rv, hi = ru < rv ? rv : ru;
                        if (__ldcg(A.res + hi) == (tag | p)) {
                            A.parent[hi] = lo;
                            record_pivot(A, h, target, p, hi);
                        } else {
                            keep = true;
                        }
                    }
                }
                warp_append(keep, p, next, next_count);
            }
            if (!grid_barrier(h, &s_ok, A.spin_limit)) return;
            cur ^= 1;
            ncur = __ldcg(&h->nlist[cur]);
        }
        if (tr) rec[8] = gtimer();
        if (ncur > 0) {
            // few candidates left: one CTA finishes the window in shared memory
            if (blockIdx.x == 0)
                tail_total += tail_rounds<WIDE>(
                    A, h, val, cur ? A.cand1 : A.cand0, ncur, s_comp,
                    reinterpret_cast<unsigned char *>(s_comp + (WIDE ? 0 : ((n + 7) & ~int64_t(7)))), target,
                    claims);
            if (!grid_barrier(h, &s_ok, A.spin_limit)) return;
        }

        if (tr) rec[9] = gtimer();
        // ---------------- flatten the roots -----------------------------------
        for (int64_t v = gtid; v < n; v += gstride)
            A.comp[v] = find_root(A.parent, __ldcg(A.comp + v));
        if (blockIdx.x == 0 && tid == 0) h->nlist[0] = 0;
        if (!grid_barrier(h, &s_ok, A.spin_limit)) return;

        {
            const uint32_t wr = (round - round_before) + uint32_t(tail_total - tail_before);
            rounds_max = wr > rounds_max ? wr : rounds_max;
        }
        if (tr) {
            rec[3] = round - round_before;
            rec[4] = uint64_t(tail_total - tail_before);
            rec[5] = __ldcg(&h->npiv);
            rec[10] = gtimer();
        }
        pos0 = wend;
        if (nwin * 64 < W) W *= 8;
        else if (nwin * 8 < W) W *= 4;
        else if (nwin * 2 < W) W *= 2;
        if (W > kMaxWindow) W = kMaxWindow;
    }
    claims = __reduce_add_sync(0xffffffffu, claims);
    if ((tid & 31) == 0 && claims) atomicAdd(&h->claim_attempts, (unsigned long long)claims);
    if (blockIdx.x == 0 && tid == 0) {  // a resumed launch adds to the earlier ones
        const bool add = A.start > 0;
        h->windows = (add ? h->windows : 0) + windows;
        h->edges_scanned = pos0;
        h->candidates = (add ? h->candidates : 0) + candidates;
        h->rounds = (add ? h->rounds : 0) + int64_t(round) + tail_total;
        h->n_bars = __ldcg(&h->npiv);
        // the scan stopped short of the edges (positions of the reduction stay
        // below 2^32) without n-1 pivots: not a result
        if (A.capped && __ldcg(&h->npiv) < target) set_status(h, PH0_ETOOBIG);
        atomicMax(&h->claim_rounds_max, rounds_max);
    }
}

// One warp per bar: the killing edge, its index a in D, its pivot row, its
// position, and the death value sqrt(d2) (IEEE round to nearest).  a comes
// from the caller's per-edge array, or (a == null) from the de-duplication
// scan's chunk prefix plus the new values of p's chunk up to p.  After the
// packed sort (pk.recs set, h->packed set, no fallback taken) the record at p
// is pk.recs[p], the key that of its edge index e in pk.keyidx, and the new
// values are the bits of pk.flags.
__global__ void k_emit(int64_t nb, int64_t m, Header *h, const unsigned long long *kk0, const unsigned long long *kk1,
                       const uint32_t *kv0, const uint32_t *kv1, const Header *kill_h,
                       const uint32_t *val0, const uint32_t *val1, const uint64_t *key0,
                       const uint64_t *key1, const Header *sort_h, const uint32_t *a,
                       const uint32_t *cpref, ph0_bar *bars, bool wide, int64_t n, const uint32_t *hib,
                       PackedRecs pk) {
    const int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;  // warp-uniform
    const int lane = threadIdx.x & 31;
    if (j >= nb) return;
    const bool packed = pk.recs && ld_volatile(&h->packed) != 0 && ld_volatile(&h->fixup_fallback) == 0;
    const bool kodd = kill_h && (make_plan(kill_h).passes & 1);
    const bool sodd = sort_h && (make_plan(sort_h).passes & 1);
    const unsigned long long p = kodd ? kk1[j] : kk0[j];
    const uint32_t low = kodd ? kv1[j] : kv0[j];
    if (p >= (unsigned long long)m) {  // fewer pivots than n-1: only after a reported error
        if (lane == 0) set_status(h, PH0_EINTERNAL);
        return;
    }
    const uint64_t *keys = sodd ? key1 : key0;
    uint32_t aval;
    if (a) {
        aval = a[p];
    } else if (packed) {
        const int64_t c0 = int64_t(p) & ~int64_t(kDedupeChunk - 1);
        const int64_t wq = (int64_t(p) >> 5) - (c0 >> 5);  // flag words of the chunk before p's
        uint32_t f = lane <= wq ? pk.flags[(c0 >> 5) + lane] : 0u;  // wq < kDedupeChunk / 32
        if (lane == wq && (p & 31) != 31) f &= (2u << (p & 31)) - 1u;
        aval = cpref[c0 / kDedupeChunk] + __reduce_add_sync(0xffffffffu, uint32_t(__popc(f)));
    } else {
        constexpr int kPer = kDedupeChunk / 32;
        const int64_t c0 = int64_t(p) & ~int64_t(kDedupeChunk - 1);
        uint32_t cnt = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int64_t i = c0 + lane * kPer + q;
            if (i <= int64_t(p)) {
                const uint64_t k = keys[i] & kKeyBits;
                cnt += i == 0 || k != (keys[i - 1] & kKeyBits);
            }
        }
        aval = cpref[c0 / kDedupeChunk] + __reduce_add_sync(0xffffffffu, cnt);
    }
    if (lane != 0) return;
    atomicXor(&h->inf_xor, low);
    uint32_t u, v;
    uint64_t key;
    if (packed) {
        record_uv(pk.recs[p], false, n, u, v);
        if (u >= v || int64_t(v) >= n) {  // only after a reported error
            set_status(h, PH0_EINTERNAL);
            return;
        }
        key = pk.keyidx[edge_index(n, u, v)] & kKeyBits;
    } else {
        const uint32_t vv = sodd ? val1[p] : val0[p];
        if (wide) edge_uv(int64_t(vv) | index_hi(hib, int64_t(p)), n, u, v);
        else record_uv(vv, false, n, u, v);
        key = keys[p] & kKeyBits;
    }
    ph0_bar b;
    b.u = int32_t(u);
    b.v = int32_t(v);
    b.a = aval;
    b.low = int32_t(low);
    b.order = int64_t(p);
    b.death_sq = __longlong_as_double((long long)key);
    b.death = __dsqrt_rn(b.death_sq);
    bars[j] = b;
}

// The bar that never dies: the vertex left in inf_xor once k_emit has folded
// in the n-1 pivot rows (every vertex but one is the pivot row of exactly one
// reduced column).  n = 1: vertex 0.
__global__ void k_inf(Header *h, int64_t n, ph0_inf_bar *inf) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t v = n > 1 ? ld_volatile(&h->inf_xor) : 0u;
    if (int64_t(v) >= n) {  // only after a reported error (fewer than n-1 bars)
        set_status(h, PH0_EINTERNAL);
        v = 0;
    }
    h->inf_vertex = int32_t(v);
    if (inf) {
        ph0_inf_bar b;
        b.vertex = int32_t(v);
        b._pad = 0;
        b.birth = 0.0;
        b.death = __longlong_as_double(0x7ff0000000000000ll);  // +inf
        *inf = b;
    }
}

// ------------------------------------------------------------------ host ---
int sm_count();

cudaError_t launch_inf(Header *h, int64_t n, ph0_inf_bar *inf, cudaStream_t s) {
    k_inf<<<1, 32, 0, s>>>(h, n, inf);
    return cudaGetLastError();
}

// Snapshot labels (2 B per vertex, rounded up to 16 B; none for wide
// records) plus the tail arrays (global ids of 2 or 4 bytes).
size_t reduce_dyn_smem(int64_t n, bool wide) {
    const size_t snap = wide ? 0 : sizeof(uint16_t) * size_t((n + 7) & ~int64_t(7));
    const size_t rid = wide ? 4 : 2;
    const size_t tail = size_t(kTailCap) * (4 + 4 * 2 + rid * 4 + 2 * 4 + 1);
    return snap + tail;
}

cudaError_t launch_reduce(const ReduceArgs &A, cudaStream_t s) {
    int blocks = int((A.n + 255) / 256);
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    // a launch that resumes (start > 0) keeps the roots, claims and pivots of
    // the earlier one: it ended at a window boundary, the end of its edges
    if (A.start == 0) k_reduce_init<<<blocks, 256, 0, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || A.m <= A.start) return e;

    const size_t smem = reduce_dyn_smem(A.n, A.wide);
    const void *fn = A.wide ? (const void *)k_reduce<true> : (const void *)k_reduce<false>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kReduceThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (per_sm > 2) per_sm = 2;
    // small clouds: fewer CTAs (cheaper grid barriers; other clouds may share the GPU)
    int grid = sm_count() * per_sm;
    const int64_t want = (A.n + 63) / 64;
    if (want < grid) grid = want < 4 ? 4 : int(want);
    ReduceArgs args = A;
    void *params[] = {&args};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kReduceThreads), params, smem, s);
}

cudaError_t launch_emit(int64_t nb, int64_t m, Header *h, const unsigned long long *kk0, const unsigned long long *kk1,
                        const uint32_t *kv0, const uint32_t *kv1, const Header *kill_h,
                        const uint32_t *val0, const uint32_t *val1, const uint64_t *key0,
                        const uint64_t *key1, const Header *sort_h, const uint32_t *a,
                        const uint32_t *cpref, ph0_bar *bars, bool wide, int64_t n, cudaStream_t s,
                        const uint32_t *hib, PackedRecs pk) {
    if (nb <= 0) return cudaSuccess;
    k_emit<<<unsigned((nb + 7) / 8), 256, 0, s>>>(nb, m, h, kk0, kk1, kv0, kv1, kill_h, val0, val1, key0,
                                                 key1, sort_h, a, cpref, bars, wide, n, hib, pk);
    return cudaGetLastError();
}

}  // namespace ph0
