// k_dedupe.cu -- step 3 of the barcode path: remove duplicate distances and
// index every edge in D (Rawson, Sec. 2: D is E without duplicates; a(j) is
// the index of edge j's distance in D, from 1 to |D|).
//
// On the sorted keys, flag[p] = (p == 0) || key[p] != key[p-1] (exact
// equality of the binary64 bit patterns), and a[p] = flag[0] + ... + flag[p]
// is an inclusive prefix sum, computed in one pass: each CTA scans a tile in
// shared memory and obtains the count of all earlier tiles by decoupled
// look-back (bounded waits).  Items are striped over the threads (warp
// ballots count the new values), so every global and shared access is
// coalesced and free of bank conflicts.
#include "ph0_common.cuh"

namespace ph0 {

constexpr int kDedupeThreads = 256;
constexpr int kDedupeItems = 16;
constexpr int kDedupeTile = kDedupeThreads * kDedupeItems;

__global__ void __launch_bounds__(kDedupeThreads)
k_dedupe(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h, int64_t m,
         uint32_t *__restrict__ a, uint64_t *look, Header *h) {
    constexpr int T = kDedupeThreads, IT = kDedupeItems, TILE = kDedupeTile, NW = T / 32;
    __shared__ uint64_t s_key[TILE + 1];
    __shared__ uint32_t s_cnt[IT * NW];  // new-value count per (item row, warp), then offsets
    __shared__ uint32_t s_tile, s_total;
    __shared__ int64_t s_excl;

    const uint64_t *keys = keys0;
    if (sort_h) keys = (make_plan(sort_h).passes & 1) ? keys1 : keys0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&h->tile_counter[kMaxPasses], 1u);
    __syncthreads();
    const int64_t tile = s_tile, base = tile * TILE;
    const int valid = int(m - base < TILE ? m - base : TILE);

    // s_key[0] = predecessor of the tile, s_key[1 + i] = key[base + i]
#pragma unroll 4
    for (int i = tid; i < valid; i += T) s_key[1 + i] = keys[base + i];
    if (tid == 0) s_key[0] = base > 0 ? keys[base - 1] : ~keys[0];
    __syncthreads();

    // item (row j, warp w, lane) = j*T + w*32 + lane: striped, conflict-free
    uint32_t masks[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int i = j * T + tid;
        const bool f = i < valid && s_key[1 + i] != s_key[i];
        masks[j] = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_cnt[j * NW + warp] = __popc(masks[j]);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the IT*NW counts, in item order
        uint32_t c[IT * NW / 32], sum = 0;
#pragma unroll
        for (int q = 0; q < IT * NW / 32; ++q) {
            c[q] = s_cnt[lane * (IT * NW / 32) + q];
            sum += c[q];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int q = 0; q < IT * NW / 32; ++q) {
            s_cnt[lane * (IT * NW / 32) + q] = run;
            run += c[q];
        }
        if (lane == 31) s_total = inc;
    }
    __syncthreads();

    // decoupled look-back on the tile totals
    if (tid == 0) {
        const uint32_t total = s_total;
        uint64_t *my = look + tile;
        int64_t excl = 0;
        if (tile == 0) {
            st_volatile(my, kFlagPrefix | total);
        } else {
            st_volatile(my, kFlagAgg | total);
            int64_t t = tile - 1;
            uint32_t spins = 0;
            while (t >= 0) {
                const uint64_t w = ld_volatile(look + t);
                if ((w & kFlagMask) == 0) {
                    if (++spins > kSpinLimit || ld_volatile(&h->status) != 0) {
                        set_status(h, PH0_ETIMEOUT);
                        break;
                    }
                    if (spins > 32) __nanosleep(64);
                    continue;
                }
                excl += int64_t(w & kCountMask);
                if ((w & kFlagMask) == kFlagPrefix) break;
                --t;
            }
            st_volatile(my, kFlagPrefix | uint64_t(excl + total));
        }
        s_excl = excl;
        if (base + valid == m) h->n_distinct = excl + total;
    }
    __syncthreads();
    const int64_t excl = s_excl;
    const unsigned le = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int i = j * T + tid;
        if (i < valid) a[base + i] = uint32_t(excl + s_cnt[j * NW + warp] + __popc(masks[j] & le));
    }
}

cudaError_t launch_dedupe(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h,
                          int64_t m, uint32_t *a, uint64_t *look, Header *h, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const int64_t tiles = (m + kDedupeTile - 1) / kDedupeTile;
    cudaError_t e = cudaMemsetAsync(look, 0, sizeof(uint64_t) * size_t(tiles), s);
    if (e != cudaSuccess) return e;
    k_dedupe<<<unsigned(tiles), kDedupeThreads, 0, s>>>(keys0, keys1, sort_h, m, a, look, h);
    return cudaGetLastError();
}

}  // namespace ph0
