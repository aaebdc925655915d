// k_dedupe.cu -- step 3 of the barcode path: remove duplicate distances and
// index every edge in D (Rawson, Sec. 2: D is E without duplicates; a(j) is
// the index of edge j's distance in D, from 1 to |D|).
//
// On the sorted keys, flag[p] = (p == 0) || key[p] != key[p-1] (exact
// equality of the binary64 bit patterns), and a[p] = flag[0] + ... + flag[p]
// is an inclusive prefix sum, computed in one pass: each CTA counts the new
// values of a tile with warp ballots and obtains the count of all earlier
// tiles by decoupled look-back (one warp reads 32 predecessors at once;
// bounded waits).  Items are striped over the threads, so every global and
// shared access is coalesced and free of bank conflicts.
//
// The whole-path calls need a only at the n - 1 killing edges, so they run
// in count mode instead: a streaming pass counts the new values of every
// chunk of kDedupeChunk keys (one warp per chunk, no look-back), a small
// scan turns the counts into exclusive chunk prefixes in place, and the bar
// emitter finishes a[p] from the chunk prefix and the keys of p's chunk.
// That saves writing a (4 bytes per edge).
#include "ph0_common.cuh"

namespace ph0 {

constexpr int kDedupeThreads = 256;
constexpr int kDedupeItems = 16;
constexpr int kDedupeTile = kDedupeThreads * kDedupeItems;

// Per-edge mode: a[p] for every edge.
__global__ void __launch_bounds__(kDedupeThreads)
k_dedupe(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h, int64_t m,
         uint32_t *__restrict__ a, uint64_t *look, Header *h) {
    constexpr int T = kDedupeThreads, IT = kDedupeItems, TILE = kDedupeTile, NW = T / 32;
    __shared__ uint64_t s_key[TILE + 1];
    __shared__ uint32_t s_cnt[IT * NW];  // new-value count per (item row, warp), then offsets
    __shared__ uint32_t s_tile, s_excl;

    const uint64_t *keys = keys0;
    if (sort_h) keys = (make_plan(sort_h).passes & 1) ? keys1 : keys0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&h->tile_counter[kMaxPasses], 1u);
    __syncthreads();
    const int64_t tile = s_tile, base = tile * TILE;
    const int valid = int(m - base < TILE ? m - base : TILE);

    // s_key[0] = predecessor of the tile, s_key[1 + i] = key[base + i]; all
    // loads of a thread are issued before the first store
    {
        uint64_t kv[IT];
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const int i = j * T + tid;
            kv[j] = i < valid ? keys[base + i] & kKeyBits : 0;  // values: bit 63 may carry an index bit
        }
#pragma unroll
        for (int j = 0; j < IT; ++j) s_key[1 + j * T + tid] = kv[j];
    }
    if (tid == 0) s_key[0] = base > 0 ? keys[base - 1] & kKeyBits : ~keys[0];
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
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);

        // decoupled look-back on the tile totals, 32 predecessors at a time
        uint64_t *my = look + tile;
        uint32_t excl = 0;
        if (tile == 0) {
            if (lane == 0) st_volatile(my, kFlagPrefix | total);
        } else {
            if (lane == 0) st_volatile(my, kFlagAgg | total);
            int64_t t = tile - 1;  // nearest predecessor not yet folded
            uint32_t spins = 0;
            for (;;) {
                // lanes past tile 0 read a virtual PREFIX of 0 (never folded:
                // tile 0 itself is a PREFIX or unpublished)
                const int64_t src = t - lane;
                const uint64_t w = src >= 0 ? ld_volatile(look + src) : kFlagPrefix;
                const uint32_t hi = uint32_t(w >> 32), lo = uint32_t(w);
                const unsigned pref = __ballot_sync(0xffffffffu, hi == kHiPrefix);
                const unsigned stop = pref | __ballot_sync(0xffffffffu, hi == 0);
                if (stop == 0) {
                    excl += __reduce_add_sync(0xffffffffu, lo);
                    t -= 32;
                    continue;
                }
                const int first = __ffs(stop) - 1;  // nearest PREFIX or unpublished word
                const bool is_pref = (pref >> first) & 1u;
                const int upto = is_pref ? first : first - 1;
                excl += __reduce_add_sync(0xffffffffu, lane <= upto ? lo : 0u);
                if (is_pref) break;
                t -= first;  // wait for this tile to publish, then read on
                int gave_up = 0;
                if (lane == 0) {
                    while ((ld_volatile(look + t) & kFlagMask) == 0) {
                        if (++spins > kSpinLimit || ld_volatile(&h->status) != 0) {
                            set_status(h, PH0_ETIMEOUT);
                            gave_up = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                if (__shfl_sync(0xffffffffu, gave_up, 0)) break;
            }
            if (lane == 0) st_volatile(my, kFlagPrefix | uint64_t(excl + total));
        }
        if (lane == 0) {
            s_excl = excl;
            if (base + valid == m) h->n_distinct = int64_t(excl) + total;
        }
    }
    __syncthreads();
    const uint32_t excl = s_excl;
    const unsigned le = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int i = j * T + tid;
        if (i < valid) a[base + i] = excl + s_cnt[j * NW + warp] + __popc(masks[j] & le);
    }
}

// Count mode, pass 1: the number of new values in every chunk (flag[p] as
// above), one warp per chunk, grid-stride.
__global__ void __launch_bounds__(256)
k_chunk_count(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h, int64_t m,
              uint32_t *__restrict__ cnt, const int32_t *gate) {
    if (gate && ld_volatile(gate) == 0) return;  // counts already made (by the sort's fix-up)
    constexpr int kPer = kDedupeChunk / 32;
    const uint64_t *keys = keys0;
    if (sort_h) keys = (make_plan(sort_h).passes & 1) ? keys1 : keys0;
    const int lane = threadIdx.x & 31;
    const int64_t chunks = (m + kDedupeChunk - 1) / kDedupeChunk;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; c < chunks; c += nw) {
        const int64_t b = c * kDedupeChunk;
        uint64_t k[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int64_t i = b + q * 32 + lane;
            k[q] = i < m ? keys[i] & kKeyBits : 0;  // values: bit 63 may carry an index bit
        }
        const uint64_t before = b > 0 ? keys[b - 1] & kKeyBits : ~k[0];  // lane 0's k[0] is key[0] here
        uint32_t total = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            uint64_t prev = __shfl_up_sync(0xffffffffu, k[q], 1);
            const uint64_t row_prev = q > 0 ? __shfl_sync(0xffffffffu, k[q > 0 ? q - 1 : 0], 31) : before;
            if (lane == 0) prev = row_prev;
            const bool f = b + q * 32 + lane < m && k[q] != prev;
            total += __popc(__ballot_sync(0xffffffffu, f));
        }
        if (lane == 0) cnt[c] = total;
    }
}

// Count mode, pass 2: exclusive scan of the chunk counts, in place, one tile
// of kScanTile counts per CTA with decoupled look-back; the last tile records
// |D|.
constexpr int kScanThreads = 256, kScanItems = 16, kScanTile = kScanThreads * kScanItems;
__global__ void __launch_bounds__(kScanThreads)
k_chunk_scan(uint32_t *__restrict__ cnt, int64_t chunks, uint64_t *look, Header *h) {
    constexpr int T = kScanThreads, IT = kScanItems, NW = T / 32;
    __shared__ uint32_t s_warp[NW + 1];
    __shared__ uint32_t s_tile, s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&h->tile_counter[kMaxPasses], 1u);
    __syncthreads();
    const int64_t tile = s_tile, base = tile * kScanTile + int64_t(tid) * IT;
    uint32_t v[IT], sum = 0;
#pragma unroll
    for (int q = 0; q < IT; ++q) {  // blocked: thread tid owns IT consecutive counts
        v[q] = base + q < chunks ? cnt[base + q] : 0u;
        sum += v[q];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < NW ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) s_warp[lane] = wi - w;
        const uint32_t total = __shfl_sync(0xffffffffu, wi, 31);
        // look-back on the tile totals (chunk counts sum to at most m < 2^32)
        uint32_t excl = 0;
        if (tile == 0) {
            if (lane == 0) st_volatile(look + tile, kFlagPrefix | total);
        } else {
            if (lane == 0) st_volatile(look + tile, kFlagAgg | total);
            int64_t t = tile - 1;
            uint32_t spins = 0;
            for (;;) {
                const int64_t src = t - lane;
                const uint64_t wd = src >= 0 ? ld_volatile(look + src) : kFlagPrefix;
                const uint32_t hi = uint32_t(wd >> 32), lo = uint32_t(wd);
                const unsigned pref = __ballot_sync(0xffffffffu, hi == kHiPrefix);
                const unsigned stop = pref | __ballot_sync(0xffffffffu, hi == 0);
                if (stop == 0) {
                    excl += __reduce_add_sync(0xffffffffu, lo);
                    t -= 32;
                    continue;
                }
                const int first = __ffs(stop) - 1;
                const bool is_pref = (pref >> first) & 1u;
                const int upto = is_pref ? first : first - 1;
                excl += __reduce_add_sync(0xffffffffu, lane <= upto ? lo : 0u);
                if (is_pref) break;
                t -= first;
                int gave_up = 0;
                if (lane == 0) {
                    while ((ld_volatile(look + t) & kFlagMask) == 0) {
                        if (++spins > kSpinLimit || ld_volatile(&h->status) != 0) {
                            set_status(h, PH0_ETIMEOUT);
                            gave_up = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                if (__shfl_sync(0xffffffffu, gave_up, 0)) break;
            }
            if (lane == 0) st_volatile(look + tile, kFlagPrefix | uint64_t(excl + total));
        }
        if (lane == 0) {
            s_excl = excl;
            if ((tile + 1) * kScanTile >= chunks) h->n_distinct = int64_t(excl) + total;
        }
    }
    __syncthreads();
    uint32_t run = s_excl + s_warp[warp] + inc - sum;
#pragma unroll
    for (int q = 0; q < IT; ++q) {
        if (base + q < chunks) cnt[base + q] = run;
        run += v[q];
    }
}

cudaError_t launch_dedupe_count(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h, int64_t m,
                                uint32_t *cnt, const int32_t *gate, cudaStream_t s);
cudaError_t launch_dedupe_scan(uint32_t *cpref, int64_t m, uint64_t *look, Header *h, cudaStream_t s);

// Per-edge mode (a != null) or count mode (cpref != null, which must hold
// one word per chunk of kDedupeChunk keys).
cudaError_t launch_dedupe(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h,
                          int64_t m, uint32_t *a, uint32_t *cpref, uint64_t *look, Header *h,
                          cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    if (a) {
        const int64_t tiles = (m + kDedupeTile - 1) / kDedupeTile;
        cudaError_t e = cudaMemsetAsync(look, 0, sizeof(uint64_t) * size_t(tiles), s);
        if (e != cudaSuccess) return e;
        k_dedupe<<<unsigned(tiles), kDedupeThreads, 0, s>>>(keys0, keys1, sort_h, m, a, look, h);
        return cudaGetLastError();
    }
    cudaError_t e = launch_dedupe_count(keys0, keys1, sort_h, m, cpref, nullptr, s);
    if (e != cudaSuccess) return e;
    return launch_dedupe_scan(cpref, m, look, h, s);
}

// Count mode, pass 1 alone (gate: only if *gate != 0).
cudaError_t launch_dedupe_count(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h, int64_t m,
                                uint32_t *cnt, const int32_t *gate, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const int64_t chunks = (m + kDedupeChunk - 1) / kDedupeChunk;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (chunks + 7) / 8;  // 8 warps per block
    const int64_t cap = int64_t(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    k_chunk_count<<<unsigned(blocks), 256, 0, s>>>(keys0, keys1, sort_h, m, cnt, gate);
    return cudaGetLastError();
}

// Count mode, pass 2 alone: the chunk counts in cpref become chunk prefixes.
cudaError_t launch_dedupe_scan(uint32_t *cpref, int64_t m, uint64_t *look, Header *h, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const int64_t chunks = (m + kDedupeChunk - 1) / kDedupeChunk;
    const int64_t stiles = (chunks + kScanTile - 1) / kScanTile;
    cudaError_t e = cudaMemsetAsync(look, 0, sizeof(uint64_t) * size_t(stiles), s);
    if (e != cudaSuccess) return e;
    k_chunk_scan<<<unsigned(stiles), kScanThreads, 0, s>>>(cpref, chunks, look, h);
    return cudaGetLastError();
}

}  // namespace ph0
