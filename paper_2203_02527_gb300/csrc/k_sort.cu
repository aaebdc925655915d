// k_sort.cu -- step 2 of the barcode path: sort the edges by distance
// (Rawson, Sec. 2 "sort it in increasing order"; Sec. 4 step 2; the paper
// used a library sort, Sec. 4.1).
//
// A stable least-significant-digit radix sort of (key = binary64 bit pattern
// of the squared distance, val = (u << 16) | v) pairs, one 8-bit digit per
// pass.  The keys are non-negative doubles, so their unsigned bit patterns
// are in numeric order; the edges enter in val order, so stability gives the
// total order (distance, u, v).  Only the bits in which the keys differ are
// sorted (see make_plan).
//
// Each pass is a single kernel ("one sweep"): a CTA takes the next tile of
// kSortTile keys (tile ids from an atomic counter, so every tile it waits on
// belongs to a CTA already running), ranks the keys of its tile stably by
// digit with warp match, publishes its per-digit counts, and obtains the
// counts of all earlier tiles by decoupled look-back over per-tile status
// words.  The tile is reordered by digit in shared memory and written out as
// contiguous runs, one run per digit.  While writing, it histograms the next
// pass's digit, so no pass needs an extra read of the keys.  Every wait is
// bounded.
#include "ph0_common.cuh"

namespace ph0 {

template <int THREADS>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *s_warp, uint32_t &total) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) s_warp[lane] = wi - w;
        if (lane == NW - 1) s_warp[NW] = wi;
    }
    __syncthreads();
    total = s_warp[NW];
    uint32_t r = inc - x + s_warp[warp];
    __syncthreads();
    return r;
}

// Header fields a sort needs zeroed: histograms, key range, tile counters.
__global__ void k_sort_init(Header *h, uint64_t *look0, int64_t look_words) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    if (tid == 0) {
        h->kmin = ~0ull;
        h->kmax = 0;
        h->sort_passes = 0;
        h->key_bits = 0;
    }
    for (int64_t i = tid; i < int64_t(kMaxPasses) * kRadix; i += stride)
        (&h->hist[0][0])[i] = 0;
    for (int64_t i = tid; i < kMaxPasses + 4; i += stride) h->tile_counter[i] = 0;
    for (int64_t i = tid; i < look_words; i += stride) look0[i] = 0;
}

// Pass-0 histogram (raw low 8 bits) and key range of keys not produced by
// the distance kernel (which computes both itself).
__global__ void __launch_bounds__(256) k_keystats(const uint64_t *__restrict__ keys, int64_t m, Header *h) {
    __shared__ uint32_t s_hist[kRadix];
    __shared__ uint64_t s_min[8], s_max[8];
    s_hist[threadIdx.x] = 0;
    __syncthreads();
    uint64_t kmin = ~0ull, kmax = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
         i += int64_t(gridDim.x) * blockDim.x) {
        uint64_t k = keys[i];
        atomicAdd(&s_hist[k & (kRadix - 1)], 1u);
        kmin = k < kmin ? k : kmin;
        kmax = k > kmax ? k : kmax;
    }
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t a = __shfl_xor_sync(0xffffffffu, kmin, o);
        uint64_t b = __shfl_xor_sync(0xffffffffu, kmax, o);
        kmin = a < kmin ? a : kmin;
        kmax = b > kmax ? b : kmax;
    }
    if ((threadIdx.x & 31) == 0) {
        s_min[threadIdx.x >> 5] = kmin;
        s_max[threadIdx.x >> 5] = kmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            kmin = s_min[w] < kmin ? s_min[w] : kmin;
            kmax = s_max[w] > kmax ? s_max[w] : kmax;
        }
        if (kmin != ~0ull) {
            atomicMin((unsigned long long *)&h->kmin, (unsigned long long)kmin);
            atomicMax((unsigned long long *)&h->kmax, (unsigned long long)kmax);
        }
    }
    if (s_hist[threadIdx.x]) atomicAdd(&h->hist[0][threadIdx.x], s_hist[threadIdx.x]);
}

// One radix pass.  Pass p reads buffer p&1 and writes buffer (p+1)&1; its
// look-back words live in look[p&1], and it clears its tile's words in
// look[(p+1)&1] for the next pass (whose previous user, pass p-1, is done).
__global__ void __launch_bounds__(kSortThreads)
k_onesweep(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1, int64_t m, int pass,
           uint64_t *look0, uint64_t *look1, Header *h) {
    constexpr int THREADS = kSortThreads, ITEMS = kSortItems, TILE = kSortTile;
    constexpr int WARPS = THREADS / 32;
    static_assert(THREADS == kRadix, "one look-back thread per digit");
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint64_t *s_keys = reinterpret_cast<uint64_t *>(s_dyn);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_dyn + sizeof(uint64_t) * TILE);
    __shared__ uint32_t s_whist[WARPS][kRadix];
    __shared__ uint32_t s_lstart[kRadix];
    __shared__ int64_t s_gbase[kRadix];
    __shared__ uint32_t s_next[kRadix];
    __shared__ uint32_t s_scan[WARPS + 1];
    __shared__ uint32_t s_tile;

    const Plan plan = make_plan(h->kmin, h->kmax);
    if (pass >= plan.passes) return;
    const uint64_t *kin = (pass & 1) ? keys1 : keys0;
    uint64_t *kout = (pass & 1) ? keys0 : keys1;
    const uint32_t *vin = (pass & 1) ? vals1 : vals0;
    uint32_t *vout = (pass & 1) ? vals0 : vals1;
    uint64_t *look = (pass & 1) ? look1 : look0;
    uint64_t *look_next = (pass & 1) ? look0 : look1;
    const bool hist_next = pass + 1 < plan.passes;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&h->tile_counter[pass], 1u);
    for (int w = 0; w < WARPS; ++w) s_whist[w][tid] = 0;
    s_next[tid] = 0;
    // bucket start of digit `tid`: exclusive scan of this pass's histogram
    uint32_t total_all;
    const uint32_t bucket = block_excl_scan<THREADS>(h->hist[pass][tid], s_scan, total_all);
    const int64_t tile = s_tile;
    const int64_t base = tile * TILE;

    // ---- load (striped within each warp: coalesced) and rank stably ----
    uint64_t k[ITEMS];
    uint32_t v[ITEMS], rank[ITEMS], dig[ITEMS];
    const int64_t wbase = base + int64_t(warp) * 32 * ITEMS;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t idx = wbase + j * 32 + lane;
        const bool ok = idx < m;
        k[j] = ok ? kin[idx] : 0;
        v[j] = ok ? vin[idx] : 0;
        dig[j] = ok ? digit_of(k[j], plan, pass) : uint32_t(kRadix);
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t dj = dig[j];
        const unsigned peers = __match_any_sync(0xffffffffu, dj);
        const uint32_t before = __popc(peers & lt);
        const uint32_t cnt = __popc(peers);
        const uint32_t prior = dj < kRadix ? s_whist[warp][dj] : 0u;
        rank[j] = prior + before;
        __syncwarp();
        if (dj < kRadix && before == 0) s_whist[warp][dj] = prior + cnt;
        __syncwarp();
    }
    __syncthreads();

    // ---- per-digit tile totals and warp offsets (thread tid = digit) ----
    uint32_t total = 0;
    for (int w = 0; w < WARPS; ++w) {
        uint32_t c = s_whist[w][tid];
        s_whist[w][tid] = total;
        total += c;
    }
    // ---- decoupled look-back for digit tid ----
    uint64_t *my = look + tile * kRadix + tid;
    int64_t excl = 0;
    if (tile == 0) {
        st_volatile(my, kFlagPrefix | total);
    } else {
        st_volatile(my, kFlagAgg | total);
        int64_t t = tile - 1;
        uint32_t spins = 0;
        while (t >= 0) {
            uint64_t w = ld_volatile(look + t * kRadix + tid);
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
    s_gbase[tid] = int64_t(bucket) + excl;
    uint32_t tile_total;
    s_lstart[tid] = block_excl_scan<THREADS>(total, s_scan, tile_total);
    __syncthreads();

    // ---- reorder the tile by digit in shared memory ----
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t dj = dig[j];
        if (dj < kRadix) {
            const uint32_t pos = s_lstart[dj] + s_whist[warp][dj] + rank[j];
            s_keys[pos] = k[j];
            s_vals[pos] = v[j];
        }
    }
    __syncthreads();

    // ---- write contiguous runs; histogram the next digit ----
    const int valid = int(m - base < TILE ? m - base : TILE);
    for (int i = tid; i < valid; i += THREADS) {
        const uint64_t key = s_keys[i];
        const uint32_t d = digit_of(key, plan, pass);
        const int64_t g = s_gbase[d] + (i - int64_t(s_lstart[d]));
        kout[g] = key;
        vout[g] = s_vals[i];
        if (hist_next) atomicAdd(&s_next[digit_of(key, plan, pass + 1)], 1u);
    }
    look_next[tile * kRadix + tid] = 0;
    __syncthreads();
    if (hist_next && s_next[tid]) atomicAdd(&h->hist[pass + 1][tid], s_next[tid]);
    if (tile == 0 && tid == 0) {
        h->sort_passes = plan.passes;
        h->key_bits = plan.nbits;
    }
}

// After the passes: if the sorted data ended in buffer 1 (odd pass count),
// copy it into buffer 0 (used when the caller's buffer must hold the result).
__global__ void k_copy_if_odd(uint64_t *keys0, const uint64_t *keys1, uint32_t *vals0,
                              const uint32_t *vals1, int64_t m, const Header *h) {
    const Plan plan = make_plan(h->kmin, h->kmax);
    if ((plan.passes & 1) == 0) return;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
         i += int64_t(gridDim.x) * blockDim.x) {
        keys0[i] = keys1[i];
        vals0[i] = vals1[i];
    }
}

// ------------------------------------------------------------------ host ---
constexpr size_t kSortDynSmem = size_t(kSortTile) * (sizeof(uint64_t) + sizeof(uint32_t));

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Zero the sort's counters and first look-back buffer.
cudaError_t launch_sort_init(Header *h, uint64_t *look0, int64_t tiles, cudaStream_t s) {
    const int64_t words = tiles * kRadix;
    int blocks = int((words + 255) / 256);
    if (blocks < 8) blocks = 8;
    if (blocks > 4 * sm_count() * 8) blocks = 4 * sm_count() * 8;
    k_sort_init<<<blocks, 256, 0, s>>>(h, look0, words);
    return cudaGetLastError();
}

cudaError_t launch_keystats(const uint64_t *keys, int64_t m, Header *h, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    int64_t blocks = (m + 255) / 256;
    const int64_t cap = int64_t(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    k_keystats<<<unsigned(blocks), 256, 0, s>>>(keys, m, h);
    return cudaGetLastError();
}

// The passes over buffers (keys0, vals0) <-> (keys1, vals1); the sorted data
// ends in buffer (passes & 1), which the device records in the header.
cudaError_t launch_sort_passes(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                               int64_t m, uint64_t *look0, uint64_t *look1, Header *h,
                               cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kSortDynSmem));
    if (e != cudaSuccess) return e;
    const int64_t tiles = (m + kSortTile - 1) / kSortTile;
    for (int p = 0; p < kMaxPasses; ++p) {
        k_onesweep<<<unsigned(tiles), kSortThreads, kSortDynSmem, s>>>(keys0, keys1, vals0, vals1, m, p,
                                                                        look0, look1, h);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

const void *k_onesweep_symbol() { return (const void *)k_onesweep; }
size_t sort_dyn_smem() { return kSortDynSmem; }

// One pass (the attribute for the dynamic shared memory must be set).
cudaError_t launch_sort_pass(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                             int64_t m, int pass, uint64_t *look0, uint64_t *look1, Header *h,
                             cudaStream_t s) {
    const int64_t tiles = (m + kSortTile - 1) / kSortTile;
    k_onesweep<<<unsigned(tiles), kSortThreads, kSortDynSmem, s>>>(keys0, keys1, vals0, vals1, m, pass,
                                                                    look0, look1, h);
    return cudaGetLastError();
}

cudaError_t launch_copy_if_odd(uint64_t *keys0, const uint64_t *keys1, uint32_t *vals0,
                               const uint32_t *vals1, int64_t m, const Header *h, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    int64_t blocks = (m + 255) / 256;
    const int64_t cap = int64_t(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    k_copy_if_odd<<<unsigned(blocks), 256, 0, s>>>(keys0, keys1, vals0, vals1, m, h);
    return cudaGetLastError();
}

}  // namespace ph0
