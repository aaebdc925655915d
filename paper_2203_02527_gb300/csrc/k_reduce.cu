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
// L = max(root(u), root(v)) claimed by p: a bar (0, a(p)) (Sec. 2, "the
// remaining nonzero diagonal entries t^b correspond to the barcode (0,b)").
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
//               holds both slots is the first remaining column touching
//               either component, so in the left-to-right order nothing
//               before it changes them: it is nonzero, its pivot is the larger
//               root, and it links that root under the smaller one.  Columns
//               that lost a slot to a lower position retry in the next round.
//               Each round the lowest remaining column wins, so rounds end.
//   flatten     every vertex's root is updated.
// Early exit: once n-1 pivots exist every later column is zero (the graph is
// connected); the window loop stops.
#include <cooperative_groups.h>

#include "ph0_common.cuh"

namespace ph0 {

constexpr int kReduceThreads = 512;
constexpr int kHashSize = 2048;
constexpr uint32_t kEmpty = 0xffffffffu;
constexpr uint32_t kDead = 0xffffffffu;


__global__ void k_reduce_init(ReduceArgs A) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = tid; v < A.n; v += stride) {
        A.comp[v] = uint32_t(v);
        A.parent[v] = uint32_t(v);
        A.res[v] = ~0ull;
        A.kill_key[v] = ~0ull;
        A.kill_val[v] = 0;
    }
    if (tid == 0) {
        A.h->npiv = 0;
        A.h->nlist[0] = 0;
        A.h->nlist[1] = 0;
        A.h->bar_count = 0;
        A.h->bar_gen = 0;
        A.h->abort = 0;
    }
}

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of
// the CTA) if the kernel must stop.
__device__ bool grid_barrier(Header *h, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t nblocks = gridDim.x;
        const uint32_t gen = ld_volatile(&h->bar_gen);
        __threadfence();
        const uint32_t arrived = atomicAdd(&h->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&h->bar_count, 0u);
            __threadfence();
            atomicAdd(&h->bar_gen, 1u);
        } else {
            uint32_t spins = 0;
            while (ld_volatile(&h->bar_gen) == gen) {
                if (ld_volatile(&h->abort)) { ok = 0; break; }
                if (++spins > kSpinLimit) {
                    set_status(h, PH0_ETIMEOUT);
                    atomicExch(&h->abort, 1);
                    ok = 0;
                    break;
                }
                if (spins > 16) __nanosleep(32);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
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

__global__ void __launch_bounds__(kReduceThreads, 1) k_reduce(ReduceArgs A) {
    extern __shared__ uint16_t s_comp[];  // [n] root snapshot of the window
    __shared__ uint32_t s_hkey[kHashSize], s_hval[kHashSize];
    __shared__ uint32_t s_hcount;
    __shared__ int s_ok;

    Header *h = A.h;
    const int64_t n = A.n, m = A.m;
    if (m <= 0) return;
    const uint32_t *val = A.val0;
    if (A.sort_h) val = (make_plan(A.sort_h->kmin, A.sort_h->kmax).passes & 1) ? A.val1 : A.val0;
    const int tid = threadIdx.x;
    const int64_t G = gridDim.x;
    const int64_t gtid = int64_t(blockIdx.x) * kReduceThreads + tid;
    const int64_t gstride = G * kReduceThreads;
    const uint32_t target = uint32_t(n - 1);

    int64_t pos0 = 0, W = A.w0;
    uint32_t round = 0;
    int windows = 0;
    int64_t candidates = 0;
    for (;;) {
        const uint32_t npiv = __ldcg(&h->npiv);
        if (pos0 >= m || npiv >= target) break;
        const int64_t wend = (m - pos0 < W) ? m : pos0 + W;
        ++windows;

        // ---------------- F: filter the window against the snapshot -------
        for (int64_t v = tid; v < n; v += kReduceThreads) s_comp[v] = uint16_t(__ldcg(A.comp + v));
        for (int i = tid; i < kHashSize; i += kReduceThreads) {
            s_hkey[i] = kEmpty;
            s_hval[i] = kEmpty;
        }
        if (tid == 0) s_hcount = 0;
        __syncthreads();
        for (int64_t b = pos0 + int64_t(blockIdx.x) * kReduceThreads; b < wend; b += gstride) {
            const int64_t p = b + tid;
            bool direct = false;
            if (p < wend) {
                uint32_t vv = val[p];
                if ((vv >> 16) >= n || (vv & 0xffffu) >= n) {  // corrupt input: never index past n
                    set_status(h, PH0_EINTERNAL);
                    vv = 0;
                }
                const uint32_t cu = s_comp[vv >> 16], cv = s_comp[vv & 0xffffu];
                if (cu != cv) {
                    const uint32_t lo = cu < cv ? cu : cv, hi = cu < cv ? cv : cu;
                    const uint32_t pair = (lo << 16) | hi;
                    bool done = false;
                    if (*(volatile uint32_t *)&s_hcount < kHashSize / 2) {
                        const uint32_t hs = (pair * 2654435761u) >> 21;  // 11 bits
                        for (int pr = 0; pr < 8; ++pr) {
                            const uint32_t slot = (hs + pr) & (kHashSize - 1);
                            const uint32_t old = atomicCAS(&s_hkey[slot], kEmpty, pair);
                            if (old == kEmpty) atomicAdd(&s_hcount, 1u);
                            if (old == kEmpty || old == pair) {
                                atomicMin(&s_hval[slot], uint32_t(p));
                                done = true;
                                break;
                            }
                        }
                    }
                    direct = !done;
                }
            }
            warp_append(direct, uint32_t(p), A.cand0, &h->nlist[0]);
        }
        __syncthreads();
        for (int slot = tid; slot < kHashSize; slot += kReduceThreads) {
            const bool has = s_hkey[slot] != kEmpty;
            warp_append(has, s_hval[slot], A.cand0, &h->nlist[0]);
        }
        if (!grid_barrier(h, &s_ok)) return;

        // ---------------- R: claim pivots in rounds ------------------------
        int cur = 0;
        uint32_t ncur = __ldcg(&h->nlist[0]);
        const uint32_t nwin = ncur;
        candidates += nwin;
        while (ncur > 0) {
            ++round;
            const unsigned long long tag = (unsigned long long)(0xffffffffu - round) << 32;
            const uint32_t *list = cur ? A.cand1 : A.cand0;
            uint32_t *next = cur ? A.cand0 : A.cand1;
            uint32_t *next_count = &h->nlist[cur ^ 1];
            if (blockIdx.x == 0 && tid == 0) *next_count = 0;
            // reserve both roots
            for (int64_t i = gtid; i < ncur; i += gstride) {
                const uint32_t p = __ldcg(list + i);
                const uint32_t vv = val[p];
                const uint32_t ru = find_root(A.parent, __ldcg(A.comp + (vv >> 16)));
                const uint32_t rv = find_root(A.parent, __ldcg(A.comp + (vv & 0xffffu)));
                if (ru == rv) {
                    A.candr[i] = kDead;
                } else {
                    A.candr[i] = (ru << 16) | rv;
                    atomicMin(A.res + ru, tag | p);
                    atomicMin(A.res + rv, tag | p);
                }
            }
            if (!grid_barrier(h, &s_ok)) return;
            // commit the columns that hold both roots
            for (int64_t b = int64_t(blockIdx.x) * kReduceThreads; b < ncur; b += gstride) {
                const int64_t i = b + tid;
                bool keep = false;
                uint32_t p = 0;
                if (i < ncur) {
                    const uint32_t r = __ldcg(A.candr + i);
                    if (r != kDead) {
                        p = __ldcg(list + i);
                        const uint32_t ru = r >> 16, rv = r & 0xffffu;
                        const unsigned long long mine = tag | p;
                        if (__ldcg(A.res + ru) == mine && __ldcg(A.res + rv) == mine) {
                            const uint32_t lo = ru < rv ? ru : rv, hi = ru < rv ? rv : ru;
                            A.parent[hi] = lo;
                            const uint32_t j = atomicAdd(&h->npiv, 1u);
                            if (j < target) {
                                A.kill_key[j] = p;
                                A.kill_val[j] = hi;
                            } else {
                                set_status(h, PH0_EINTERNAL);
                            }
                        } else {
                            keep = true;
                        }
                    }
                }
                warp_append(keep, p, next, next_count);
            }
            if (!grid_barrier(h, &s_ok)) return;
            cur ^= 1;
            ncur = __ldcg(&h->nlist[cur]);
        }

        // ---------------- flatten the roots -----------------------------------
        for (int64_t v = gtid; v < n; v += gstride)
            A.comp[v] = find_root(A.parent, __ldcg(A.comp + v));
        if (blockIdx.x == 0 && tid == 0) h->nlist[0] = 0;
        if (!grid_barrier(h, &s_ok)) return;

        pos0 = wend;
        if (nwin * 64 < W) W *= 8;
        else if (nwin * 8 < W) W *= 4;
        else if (nwin * 2 < W) W *= 2;
        if (W > kMaxWindow) W = kMaxWindow;
    }
    if (blockIdx.x == 0 && tid == 0) {
        h->windows = windows;
        h->edges_scanned = pos0;
        h->candidates = candidates;
        h->rounds = round;
        h->n_bars = __ldcg(&h->npiv);
    }
}

// One thread per bar: the killing edge, its index a in D, its pivot row, its
// position, and the death value sqrt(d2) (IEEE round to nearest).
__global__ void k_emit(int64_t nb, int64_t m, Header *h, const unsigned long long *kk0, const unsigned long long *kk1,
                       const uint32_t *kv0, const uint32_t *kv1, const Header *kill_h,
                       const uint32_t *val0, const uint32_t *val1, const uint64_t *key0,
                       const uint64_t *key1, const Header *sort_h, const uint32_t *a,
                       ph0_bar *bars) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= nb) return;
    const bool kodd = kill_h && (make_plan(kill_h->kmin, kill_h->kmax).passes & 1);
    const bool sodd = sort_h && (make_plan(sort_h->kmin, sort_h->kmax).passes & 1);
    const unsigned long long p = kodd ? kk1[j] : kk0[j];
    const uint32_t low = kodd ? kv1[j] : kv0[j];
    if (p >= (unsigned long long)m) {  // fewer pivots than n-1: only after a reported error
        set_status(h, PH0_EINTERNAL);
        return;
    }
    const uint32_t vv = sodd ? val1[p] : val0[p];
    const uint64_t key = sodd ? key1[p] : key0[p];
    ph0_bar b;
    b.u = int32_t(vv >> 16);
    b.v = int32_t(vv & 0xffffu);
    b.a = a[p];
    b.low = int32_t(low);
    b.order = int64_t(p);
    b.death_sq = __longlong_as_double((long long)key);
    b.death = __dsqrt_rn(b.death_sq);
    bars[j] = b;
}

// ------------------------------------------------------------------ host ---
int sm_count();

cudaError_t launch_reduce(const ReduceArgs &A, cudaStream_t s) {
    int blocks = int((A.n + 255) / 256);
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    k_reduce_init<<<blocks, 256, 0, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || A.m <= 0) return e;

    const size_t smem = sizeof(uint16_t) * size_t(A.n);
    e = cudaFuncSetAttribute(k_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_reduce, kReduceThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (per_sm > 2) per_sm = 2;
    const int grid = sm_count() * per_sm;
    ReduceArgs args = A;
    void *params[] = {&args};
    return cudaLaunchCooperativeKernel((const void *)k_reduce, dim3(grid), dim3(kReduceThreads), params,
                                       smem, s);
}

cudaError_t launch_emit(int64_t nb, int64_t m, Header *h, const unsigned long long *kk0, const unsigned long long *kk1,
                        const uint32_t *kv0, const uint32_t *kv1, const Header *kill_h,
                        const uint32_t *val0, const uint32_t *val1, const uint64_t *key0,
                        const uint64_t *key1, const Header *sort_h, const uint32_t *a,
                        ph0_bar *bars, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    k_emit<<<unsigned((nb + 255) / 256), 256, 0, s>>>(nb, m, h, kk0, kk1, kv0, kv1, kill_h, val0, val1, key0,
                                                     key1, sort_h, a, bars);
    return cudaGetLastError();
}

}  // namespace ph0
