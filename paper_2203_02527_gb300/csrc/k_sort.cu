// k_sort.cu -- step 2 of the barcode path: sort the edges by distance
// (Rawson, Sec. 2: the distances in increasing order; Sec. 4 step 2; the
// paper used a library sort, Sec. 4.1).
//
// A stable least-significant-digit radix sort of (key = binary64 bit pattern
// of the squared distance, val = (u << 16) | v) pairs.  The keys are
// non-negative doubles, so their unsigned bit patterns are in numeric order;
// the edges enter in val order, so stability gives the total order
// (distance, u, v).  The low 48 bits are six 8-bit digits; above them only
// the bits in which the keys differ are sorted, as one 9-bit digit or two
// 8-bit digits (see make_plan).
//
// Each pass is a single kernel ("one sweep"): a CTA takes the next tile of
// kSortTile keys (tile ids from an atomic counter, so every tile it waits on
// belongs to a CTA already running), ranks the keys of its tile stably by
// digit, publishes its per-digit counts, and obtains the counts of all
// earlier tiles by decoupled look-back over per-tile status words.  Ranking
// finds the lanes of a warp that share a digit by intersecting one warp
// ballot per digit bit (8-bit digits) or by one warp match (the 9-bit top
// digit, which is concentrated on few values).  The tile is reordered by
// digit in shared memory and written out as contiguous runs, one run per
// digit.  The distance kernel supplies the six low-digit histograms and a
// histogram of the top part modulo 512, which is the single top pass's
// digit histogram rotated by the minimum key's top part; when the top part
// needs two passes, the last low pass histograms their digits as it writes.
// So no pass needs an extra read of the keys.  Every wait is bounded.
//
// The whole path sorts with the short sort (launch_sort_short): the passes
// from slot 2 on, then a fix-up of the rare groups of records whose keys
// agree above bit 16 (k_sort_fixup); from 2^22 edges up to 32768 points in
// four or more dimensions it takes the packed sort of k_sortp.cu instead,
// and the short sort's kernels then return at once unless the keys do not
// pack.  The step entry point and the early path run every pass.  The early path's partition into distance classes is
// one more pass (slot kClassSlot, digit = class).
#include "sort_util.cuh"

namespace ph0 {

// Header fields a sort needs zeroed: histograms, key range, tile counters.
__global__ void k_sort_init(Header *h, uint64_t *look0, int64_t look_words, int top_bits,
                            int64_t sorted_edges, const int32_t *gate) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    if (gate && ld_volatile(gate) == 0) look_words = 0;  // a gated sort that will not run
    if (tid == 0) {
        if (sorted_edges >= 0) h->sorted_edges = sorted_edges;
        h->kmin = ~0ull;
        h->kmax = 0;
        h->sort_passes = 0;
        h->key_bits = 0;
        h->top_bits = top_bits;
    }
    for (int64_t i = tid; i < int64_t(kMaxPasses) * kMaxRadix; i += stride)
        (&h->hist[0][0])[i] = 0;
    for (int64_t i = tid; i < kMaxRadix; i += stride) h->hist_top_mod[i] = 0;
    for (int64_t i = tid; i < kMaxPasses + 4; i += stride) h->tile_counter[i] = 0;
    for (int64_t i = tid; i < look_words; i += stride) look0[i] = 0;
}

// Histograms of the six low digits and the key range of keys not produced by
// the distance kernel (which computes both itself); gate: return at once
// unless *gate is set (a fallback sort that is not needed).  lows_only: only
// the six low histograms (a packed-sort call whose keys did not pack, whose
// distance kernel took the top part's histogram and the key range).
__global__ void __launch_bounds__(256) k_keystats(const uint64_t *__restrict__ keys, int64_t m, Header *h,
                                                   const int32_t *gate, int lows_only) {
    if (gate && ld_volatile(gate) == 0) return;
    __shared__ uint32_t s_hist[kLowPasses][kRadix];
    __shared__ uint32_t s_top[kMaxRadix];
    __shared__ uint64_t s_min[8], s_max[8];
    for (int i = threadIdx.x; i < kLowPasses * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    for (int i = threadIdx.x; i < kMaxRadix; i += blockDim.x) s_top[i] = 0;
    __syncthreads();
    uint64_t kmin = ~0ull, kmax = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
         i += int64_t(gridDim.x) * blockDim.x) {
        const uint64_t k = keys[i] & kKeyBits;  // bit 63 carries an edge index bit
#pragma unroll
        for (int p = 0; p < kLowPasses; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & (kRadix - 1)], 1u);
        atomicAdd(&s_top[(k >> kTopShift) & (kMaxRadix - 1)], 1u);
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
    if (threadIdx.x == 0 && !lows_only) {
        for (int w = 1; w < 8; ++w) {
            kmin = s_min[w] < kmin ? s_min[w] : kmin;
            kmax = s_max[w] > kmax ? s_max[w] : kmax;
        }
        if (kmin != ~0ull) {
            atomicMin((unsigned long long *)&h->kmin, (unsigned long long)kmin);
            atomicMax((unsigned long long *)&h->kmax, (unsigned long long)kmax);
        }
    }
    for (int i = threadIdx.x; i < kLowPasses * kRadix; i += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&h->hist[i / kRadix][i % kRadix], c);
    }
    if (lows_only) return;
    for (int i = threadIdx.x; i < kMaxRadix; i += blockDim.x)
        if (s_top[i]) atomicAdd(&h->hist_top_mod[i], s_top[i]);
}

// The values of the top part that occur, numbered in increasing order (a
// single top pass only): when at most kRadix occur, the top pass runs on the
// 8-bit instance of slot 6 with digit top_lut[t] (t the top part less that of
// kmin), which orders the keys as t does; the digits' histogram is written to
// hist[kLowPasses].  On the benchmark cloud 211 of the 266 values in the
// top part's span occur.
__global__ void __launch_bounds__(kMaxRadix) k_top_compact(Header *h) {
    __shared__ uint32_t s_warp[kMaxRadix / 32 + 1];
    if (ld_volatile(&h->packed)) return;  // the packed sort runs instead (k_sortp.cu)
    const int t = threadIdx.x;
    const Plan plan = make_plan(h);
    uint32_t c = 0;
    if (plan.top == 1) c = h->hist_top_mod[(uint32_t(t) + uint32_t(plan.kmin >> kTopShift)) & (kMaxRadix - 1)];
    uint32_t tot;
    const uint32_t idx = block_excl_scan<kMaxRadix>(c != 0 ? 1u : 0u, s_warp, tot);
    const bool compact = plan.top == 1 && tot <= uint32_t(kRadix);
    if (compact) {
        h->top_lut[t] = uint8_t(c != 0 ? idx : 0u);  // t that occur nowhere are never looked up
        if (c != 0) h->hist[kLowPasses][idx] = c;
        if (t < kRadix && uint32_t(t) >= tot) h->hist[kLowPasses][t] = 0;
    }
    if (t == 0) h->top_compact = compact ? 1 : 0;
}

// Shared memory of one pass: the tile's keys (input, then in sorted order),
// its values (input, and in sorted order), per-warp digit counts, per-digit
// destination offsets.
// The 8-bit passes reorder the values in place (12 bytes of shared memory
// per key instead of 16), which lets four CTAs share an SM (3.51-3.69 ms per
// pass at 537M keys against 3.63-3.98 ms with three); the 9-bit pass keeps a
// separate array for the sorted values and three CTAs per SM (its larger
// counters do not leave room for a fourth: 5.20 against 4.44 ms).
template <int RADIX>
__host__ __device__ constexpr bool sort_inplace() { return RADIX == kRadix; }
template <int RADIX, int THREADS = kSortThreads>
struct SortSmem {
    static constexpr int W = THREADS / 32;
    uint64_t keys[kSortTile];          // input keys, then the tile's keys in sorted order
    uint32_t vals_in[kSortTile];       // input values (in place: then in sorted order)
    uint32_t vals[sort_inplace<RADIX>() ? 4 : kSortTile];  // values in sorted order (not in place)
    uint16_t whist[W][RADIX];          // counts, then the local position of each warp's first item
    uint32_t gofs[RADIX];              // global position of sorted tile index 0 of each digit's run (mod 2^32)
    uint32_t scan[W + 1];
    uint32_t tile;
    unsigned long long mbar;           // completion of the tile's bulk copies
};
static_assert(kMaxRadix <= kSortTile, "top-digit histogram lives in vals_in");
static_assert(2 * kRadix * 4 <= 8 * kRadix * 2, "in place: the next passes' histogram lives in whist");

// Digit of a key in pass slot SLOT: slots 0..5 are the raw bytes of bits
// 0..47; slot 6 is the top part (all of it if it has at most 9 bits, else its
// low byte), or, in the 8-bit instance of slot 6, the number of the top
// part among the values that occur (k_top_compact); slot 7 is the high byte
// of a 16-bit top part.
// Slot kClassSlot (the early path's partition): the class of the key's bin,
// the number of class bounds bound[1..nc-1] at or below the bin.
struct ClassDigit {
    uint64_t kmin;
    int shift, nc;
    const uint32_t *bound;  // shared memory
    const uint8_t *lut;     // shared memory: top_lut (the 8-bit instance of slot 6)
};
template <int SLOT, int RADIX>
__device__ __forceinline__ uint32_t slot_digit(uint64_t key, const Plan &p, const ClassDigit &cd) {
    if constexpr (SLOT == kClassSlot) {
        const uint32_t bin = uint32_t(((key & kKeyBits) - cd.kmin) >> cd.shift);
        uint32_t c = 0;
#pragma unroll
        for (int q = 1; q < kPrefixClasses; ++q) c += (q < cd.nc && bin >= cd.bound[q]) ? 1u : 0u;
        return c;
    } else {
        if (SLOT < kLowPasses) return uint32_t(key >> (kRadixBits * SLOT)) & (kRadix - 1);
        const uint32_t t = uint32_t(((key & kKeyBits) >> kTopShift) - (p.kmin >> kTopShift));
        if (SLOT == kLowPasses && RADIX == kRadix) return cd.lut[t & (kMaxRadix - 1)];
        if (SLOT == kLowPasses) return p.top == 1 ? t : (t & (kRadix - 1));
        return t >> kRadixBits;
    }
}

// One radix pass (pass index = SLOT).  Pass p reads buffer p&1 and writes
// buffer (p+1)&1; its look-back words (kMaxRadix per tile, whatever the
// pass's radix) live in look[p&1], and it clears its tile's words in
// look[(p+1)&1] for the next pass (whose previous user, pass p-1, is done).
// THREADS: 256 (kSortItems keys each), or 512 with half as many keys each
// (the same tile): one digit per thread in a 9-bit pass.
template <int RADIX, int THREADS = kSortThreads>
__host__ __device__ constexpr int sort_min_blocks() { return THREADS == kSortThreads ? (sort_inplace<RADIX>() ? 4 : 3) : 2; }

template <int RADIX, int SLOT, bool ALIGNED, bool PERSIST = false, int THREADS = kSortThreads>
__global__ void __launch_bounds__(THREADS, (sort_min_blocks<RADIX, THREADS>()))
k_onesweep(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1, int64_t m,
           uint64_t *look0, uint64_t *look1, Header *h) {
    constexpr int T = THREADS, IT = kSortTile / THREADS, TILE = kSortTile, W = T / 32;
    static_assert(IT * T == TILE, "every instance sorts the same tiles");

    constexpr int DPT = RADIX / T;  // digits per thread
    constexpr bool INPL = sort_inplace<RADIX>();
    static_assert(RADIX % T == 0 && RADIX <= kMaxRadix, "radix");
    static_assert((TILE & (TILE - 1)) == 0, "tile positions are masked to the tile");
    extern __shared__ __align__(16) unsigned char s_raw[];
    SortSmem<RADIX, T> &S = *reinterpret_cast<SortSmem<RADIX, T> *>(s_raw);

    const Plan plan = make_plan(h);
    if (SLOT != kClassSlot && SLOT >= plan.passes) return;
    if (ld_volatile(&h->packed)) return;  // the packed sort runs instead (k_sortp.cu)
    // slot 6 has two instances, launched one after the other: the 8-bit one
    // works when k_top_compact found at most kRadix top values, the other else
    constexpr bool COMPACT = SLOT == kLowPasses && RADIX == kRadix;
    if constexpr (SLOT == kLowPasses) {
        if (COMPACT != (ld_volatile(&h->top_compact) != 0)) return;
    }
    const uint64_t *kin = (SLOT & 1) ? keys1 : keys0;
    uint64_t *kout = (SLOT & 1) ? keys0 : keys1;
    const uint32_t *vin = (SLOT & 1) ? vals1 : vals0;
    uint32_t *vout = (SLOT & 1) ? vals0 : vals1;
    uint64_t *look = (SLOT & 1) ? look1 : look0;
    uint64_t *look_next = (SLOT & 1) ? look0 : look1;
    // two top passes: the last low pass histograms their digits as it writes
    const bool hist_top = SLOT != kClassSlot && plan.top == 2 && SLOT == plan.low - 1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        S.tile = atomicAdd(&h->tile_counter[SLOT], 1u);
        mbar_init(&S.mbar, 1);
    }
    ClassDigit cd{};
    if constexpr (COMPACT) {
        __shared__ uint8_t s_lut[kMaxRadix];
        for (int i = tid; i < kMaxRadix; i += T) s_lut[i] = h->top_lut[i];
        cd.lut = s_lut;
    }
    if constexpr (SLOT == kClassSlot) {
        __shared__ uint32_t s_bound[kPrefixClasses + 1];
        if (tid <= kPrefixClasses) s_bound[tid] = h->part_bound[tid];
        cd = ClassDigit{h->part_kmin, h->part_shift, h->part_nc, s_bound, nullptr};
    }
    __syncthreads();
    // PERSIST: the instance launched on fewer CTAs than tiles (passes that
    // usually return at once), where a CTA takes tiles from the counter until
    // none is left (every tile it waits on belongs to a CTA that is running);
    // the others take one tile per CTA
    uint32_t phase = 0;  // of the tile mbarrier (a persistent CTA loads tile after tile)
    for (;;) {
        const int64_t tile = S.tile;
        if constexpr (PERSIST) {
            if (tile >= (m + TILE - 1) / TILE) break;
        }
        const int64_t base = tile * TILE;
        const int valid = int(m - base < TILE ? m - base : TILE);
        // full tiles arrive in shared memory while the histogram scan below runs:
        // by two bulk copies when their rows are 16-byte aligned (the aligned
        // instances; a persistent one waits on the mbarrier's next phase each
        // tile), else by each thread's asynchronous copies of its own items;
        // the ragged last tile uses plain loads
        const bool bulk = (ALIGNED || !PERSIST) && valid == TILE &&
                          ((reinterpret_cast<uintptr_t>(kin) | reinterpret_cast<uintptr_t>(vin)) & 15u) == 0;
        const bool full = ALIGNED ? bulk : valid == TILE;
        if (bulk && tid == 0) {
            mbar_expect_tx(&S.mbar, uint32_t(TILE * (sizeof(uint64_t) + sizeof(uint32_t))));
            bulk_g2s(S.keys, kin + base, uint32_t(TILE * sizeof(uint64_t)), &S.mbar);
            bulk_g2s(S.vals_in, vin + base, uint32_t(TILE * sizeof(uint32_t)), &S.mbar);
        }
        if constexpr (!ALIGNED) {
            if (full && !bulk) {
                const int own = warp * 32 * IT + lane;
#pragma unroll
                for (int j = 0; j < IT; ++j) {
                    cp_async8(&S.keys[own + j * 32], kin + base + own + j * 32);
                    cp_async4(&S.vals_in[own + j * 32], vin + base + own + j * 32);
                }
            }
        }
        {  // each warp clears its own counter row (ranking touches only that row)
            uint32_t *row = reinterpret_cast<uint32_t *>(&S.whist[warp][0]);
#pragma unroll
            for (int i = lane; i < RADIX / 2; i += 32) row[i] = 0;
            __syncwarp();
        }
        // digit starts (tile 0 only): exclusive scan of this pass's histogram;
        // tile 0 folds them into its PREFIX, so later tiles get them by look-back
        uint32_t bucket[DPT];
#pragma unroll
        for (int q = 0; q < DPT; ++q) bucket[q] = 0;
        if (tile == 0) {
            uint32_t hsum = 0;
#pragma unroll
            for (int q = 0; q < DPT; ++q) {
                // a single top pass: its digit t = (key >> kTopShift) - (kmin >> kTopShift)
                // is below kMaxRadix, so its count is hist_top_mod[r] with
                // r = (t + (kmin >> kTopShift)) mod kMaxRadix (no other digit maps to r)
                bucket[q] = (SLOT == kLowPasses && !COMPACT && plan.top == 1)
                                ? h->hist_top_mod[(uint32_t(tid * DPT + q) + uint32_t(plan.kmin >> kTopShift)) &
                                                  (kMaxRadix - 1)]
                                : h->hist[SLOT == kClassSlot ? 0 : SLOT][tid * DPT + q];
                hsum += bucket[q];
            }
            uint32_t tot;
            uint32_t run = block_excl_scan<T>(hsum, S.scan, tot);
#pragma unroll
            for (int q = 0; q < DPT; ++q) {
                const uint32_t c = bucket[q];
                bucket[q] = run;
                run += c;
            }
        }

        // ---- keys (striped within each warp) and stable ranking ----
        uint64_t k[IT];
        uint32_t dr[IT];  // digit << 16 | rank within the warp, then the local position
        const int wloc = warp * 32 * IT;  // the warp's first item within the tile
        if (full) {  // each thread reads (and later scatters) only its own items
            if (bulk) {
                if (!mbar_wait(&S.mbar, phase)) set_status(h, PH0_ETIMEOUT);
                phase ^= 1u;
            } else {
                cp_async_wait_all();
            }
#pragma unroll
            for (int j = 0; j < IT; ++j) k[j] = S.keys[wloc + j * 32 + lane];
        } else {
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const int loc = wloc + j * 32 + lane;
                k[j] = loc < valid ? kin[base + loc] : 0;
            }
        }
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const uint32_t dj = (full || wloc + j * 32 + lane < valid) ? slot_digit<SLOT, RADIX>(k[j], plan, cd)
                                                                       : uint32_t(RADIX);
            // lanes with the same digit.  8-bit digits (raw mantissa bytes, about
            // uniform: a warp holds ~30 distinct values): intersect one ballot per
            // digit bit, much faster than a warp match on this GPU; the ragged
            // tile's sentinel digit RADIX needs one more bit.  The 9-bit top digit
            // (exponent and leading mantissa bits of d2) is concentrated on few
            // values; there one warp match and nine ballots measured the same
            // (4.65 ms at 537M keys), the pass being held by its two look-backs
            // per thread and its writes into few digit runs, not by ranking.
            unsigned peers = 0xffffffffu;
            if constexpr (RADIX == kMaxRadix) {
                peers = __match_any_sync(0xffffffffu, dj);
            } else {
                // the class digit (at most kPrefixClasses values) has 3 bits
                constexpr int kBits = SLOT == kClassSlot ? 3 : 8;
                static_assert(kPrefixClasses <= 8, "class digits fit 3 bits");
#pragma unroll
                for (int b = 0; b < kBits; ++b) {
                    const bool bit = (dj >> b) & 1u;
                    const unsigned vote = __ballot_sync(0xffffffffu, bit);
                    peers &= bit ? vote : ~vote;
                }
                if (!full) {  // the sentinel digit RADIX of the ragged tile
                    bool bit;
                    if constexpr (SLOT == kClassSlot) bit = dj >= uint32_t(1u << kBits);
                    else bit = (dj >> kBits) & 1u;
                    const unsigned vote = __ballot_sync(0xffffffffu, bit);
                    peers &= bit ? vote : ~vote;
                }
            }
            const uint32_t before = __popc(peers & lt);
            if constexpr (RADIX == kMaxRadix) {
                // 9-bit digits: the leader alone reads and advances its digit's
                // count and hands it to its peers (measured faster here)
                const int leader = __ffs(peers) - 1;
                uint32_t prior = 0;
                if (before == 0 && dj < RADIX) {
                    prior = S.whist[warp][dj];
                    S.whist[warp][dj] = uint16_t(prior + __popc(peers));
                }
                prior = __shfl_sync(0xffffffffu, prior, leader);
                dr[j] = (dj << 16) | (prior + before);
                __syncwarp();
            } else {
                // 8-bit digits: every lane reads its digit's count, then the leader
                // advances it (measured faster here)
                const uint32_t prior = dj < RADIX ? S.whist[warp][dj] : 0u;
                dr[j] = (dj << 16) | (prior + before);
                __syncwarp();
                if (dj < RADIX && before == 0) S.whist[warp][dj] = uint16_t(prior + __popc(peers));
                __syncwarp();
            }
        }
        __syncthreads();

        // ---- per digit: tile total (published at once), then local positions ----
        uint32_t total[DPT], tsum = 0;
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = tid * DPT + q;
            uint32_t t = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) t += S.whist[w][d];
            total[q] = t;
            tsum += t;
            st_volatile(look + tile * kMaxRadix + d, tile == 0 ? kFlagPrefix | (bucket[q] + t) : kFlagAgg | t);
        }
        uint32_t lstart[DPT];
        {
            uint32_t tot;
            uint32_t run = block_excl_scan<T>(tsum, S.scan, tot);
#pragma unroll
            for (int q = 0; q < DPT; ++q) {
                const int d = tid * DPT + q;
                lstart[q] = run;
                uint32_t pos = run;  // local position of the first item of each warp, digit d
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const uint32_t c = S.whist[w][d];
                    S.whist[w][d] = uint16_t(pos);
                    pos += c;
                }
                run += total[q];
            }
        }
        __syncthreads();

        // ---- reorder keys and values by digit in shared memory ----
        if constexpr (INPL) {
            // keys from registers into their array; then every value into a
            // register before any is written back into its own array
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const uint32_t dj = dr[j] >> 16;
                if (dj < RADIX) {
                    const uint32_t pos = (S.whist[warp][dj] + (dr[j] & 0xffffu)) & (TILE - 1);
                    S.keys[pos] = k[j];
                    dr[j] = (dj << 16) | pos;
                }
            }
            uint32_t vj[IT];
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const int loc = wloc + j * 32 + lane;
                vj[j] = full ? S.vals_in[loc] : (loc < valid ? vin[base + loc] : 0u);
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < IT; ++j)
                if ((dr[j] >> 16) < RADIX) S.vals_in[dr[j] & 0xffffu] = vj[j];
        } else {
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const uint32_t dj = dr[j] >> 16;
                const int loc = wloc + j * 32 + lane;
                if (dj < RADIX) {
                    const uint32_t pos = (S.whist[warp][dj] + (dr[j] & 0xffffu)) & (TILE - 1);  // in range by construction
                    S.keys[pos] = k[j];
                    S.vals[pos] = full ? S.vals_in[loc] : vin[base + loc];
                }
            }
        }

        // ---- look-back (keys and ranks are dead now), global offsets ----
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = tid * DPT + q;
            uint32_t excl = bucket[q];
            if (tile != 0) {
                excl = lookback_window(look + d, tile, h);
                st_volatile(look + tile * kMaxRadix + d, kFlagPrefix | uint64_t(excl + total[q]));
            }
            S.gofs[d] = excl - lstart[q];  // wraps below 0; positions are < 2^32
        }
        // dead once every thread has finished the scatter (in place: whist, dead after the reorder)
        uint32_t *s_next = INPL ? reinterpret_cast<uint32_t *>(&S.whist[0][0]) : S.vals_in;
        if (hist_top) {
            __syncthreads();
            for (int i = tid; i < kMaxRadix; i += T) s_next[i] = 0;
        }
        __syncthreads();

        // ---- write contiguous runs, one per digit ----
        const uint32_t m32 = uint32_t(m);  // m < 2^32
#pragma unroll 4
        for (int i = tid; i < valid; i += T) {
            const uint64_t key = S.keys[i];
            const uint32_t g = S.gofs[slot_digit<SLOT, RADIX>(key, plan, cd)] + uint32_t(i);
            if (g >= m32) continue;  // never taken when the counts are consistent
            kout[g] = key;
            vout[g] = INPL ? S.vals_in[i] : S.vals[i];
            if (hist_top) {  // the two top passes' digits: low and high byte of t
                const uint32_t t = uint32_t(((key & kKeyBits) >> kTopShift) - (plan.kmin >> kTopShift));
                atomicAdd(&s_next[t & (kRadix - 1)], 1u);
                atomicAdd(&s_next[kRadix + (t >> kRadixBits)], 1u);
            }
        }
        for (int i = tid; i < kMaxRadix; i += T) look_next[tile * kMaxRadix + i] = 0;
        if (hist_top) {
            __syncthreads();
            for (int i = tid; i < kMaxRadix; i += T) {
                const uint32_t c = s_next[i];
                if (!c) continue;
                constexpr int kNext = SLOT + 1 < kMaxPasses - 1 ? SLOT + 1 : kMaxPasses - 2;  // class slot: never
                atomicAdd(&h->hist[kNext + i / kRadix][i % kRadix], c);
            }
        }
        if (tile == 0 && tid == 0) {
            h->sort_passes = plan.passes;
            h->key_bits = plan.bits;
        }
        if constexpr (!PERSIST) {
            break;
        } else {  // the tile's shared memory is free once every thread is here
            __syncthreads();
            if (tid == 0) S.tile = atomicAdd(&h->tile_counter[SLOT], 1u);
            __syncthreads();
        }
    }
}

// After the passes: copy (src -> dst) the records when h's plan has a pass
// count of the given parity (-1: any) and, if gate is given, *gate is set.
// With parity 1, src = buffer 1 and dst = buffer 0, it moves the sorted data
// into buffer 0 (when the caller's buffer must hold the result).
__global__ void k_copy_parity(uint64_t *keys_dst, const uint64_t *keys_src, uint32_t *vals_dst,
                              const uint32_t *vals_src, int64_t m, const Header *h, int parity,
                              const int32_t *gate) {
    if (gate && ld_volatile(gate) == 0) return;
    const Plan plan = make_plan(h);
    if (parity >= 0 && (plan.passes & 1) != parity) return;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
         i += int64_t(gridDim.x) * blockDim.x) {
        keys_dst[i] = keys_src[i];
        vals_dst[i] = vals_src[i];
    }
}

// ---- the short sort: the passes over key bits 16 and up, then a fix-up ----
//
// The passes from slot kShortFirstSlot on (bytes 2..5 and the top part) sort
// the records by key >> kShortShift; as every pass is stable, each group of
// equal key >> kShortShift is still in input order, i.e. in increasing value
// (u << 16 | v).  The fix-up then sorts every group by the whole key, stably,
// which completes the sort.  Groups of two or more records are rare (their
// keys agree in all but the low 16 bits), so the fix-up is a streaming check
// of neighbours; a group of at most kFixCap records is sorted by the thread
// at its start, and an out-of-order group above kFixCap (only clouds whose
// distances crowd into tiny ranges) sets h->fixup_fallback, on which the
// caller gates a complete sort.  The first short slot is even, so the records
// end where a complete sort leaves them: buffer (passes & 1).
constexpr int kShortFirstSlot = 2;
constexpr int kShortShift = kRadixBits * kShortFirstSlot;
constexpr int kFixCap = 32;

// The de-duplication flag of every record (a new distance value: p == 0 or
// key[p] != key[p-1]) is counted per chunk of kDedupeChunk records as the
// fix-up streams the keys, so step 3 needs no pass of its own; a warp step
// covers exactly one chunk.  Sorting a group changes the flags inside it:
// the thread that sorts a group adds the difference to its chunk's count,
// and a group that would need sorting across the end of its chunk (whose
// records another warp may be counting meanwhile) is left to a second
// kernel, which sorts it once every count is written and corrects both
// chunks' counts.
// Sorts the group of sz records at p (2 <= sz <= kFixCap) by key, stably;
// returns the change in the number of new-value flags inside it, and, per
// record i, that change in dflag[i] when dflag is given.
__device__ int sort_group(uint64_t *keys, uint32_t *vals, int64_t p, int sz, int8_t *dflag) {
    uint64_t kk[kFixCap];
    uint32_t vv[kFixCap];
    if (dflag)
        for (int i = 0; i < sz; ++i) dflag[i] = 0;
    // compared by value (bit 63 of a word carries an edge index bit), moved whole
    bool sorted = true;
    for (int i = 0; i < sz; ++i) {
        kk[i] = keys[p + i];
        vv[i] = vals[p + i];
        if (i > 0 && (kk[i] & kKeyBits) < (kk[i - 1] & kKeyBits)) sorted = false;
    }
    if (sorted) return 0;
    int8_t before[kFixCap];
    for (int i = 1; i < sz; ++i) before[i] = (kk[i] & kKeyBits) != (kk[i - 1] & kKeyBits);
    for (int i = 1; i < sz; ++i) {  // stable: an equal key stays behind
        const uint64_t k = kk[i];
        const uint32_t v = vv[i];
        int j = i - 1;
        while (j >= 0 && (kk[j] & kKeyBits) > (k & kKeyBits)) {
            kk[j + 1] = kk[j];
            vv[j + 1] = vv[j];
            --j;
        }
        kk[j + 1] = k;
        vv[j + 1] = v;
    }
    int delta = 0;
    for (int i = 0; i < sz; ++i) {
        keys[p + i] = kk[i];
        vals[p + i] = vv[i];
        if (i > 0) {
            const int d = int((kk[i] & kKeyBits) != (kk[i - 1] & kKeyBits)) - before[i];
            delta += d;
            if (dflag) dflag[i] = int8_t(d);
        }
    }
    return delta;
}

// The rare cases of the check of one record at p (see fixup_at), kept out
// of line so that the streaming loop stays small: the start of a group of
// two or more records sorts its group (when it holds at most kFixCap
// records and ends in the chunk; else it defers it), adding the change of
// its flags to *delta; an inversion inside a longer group reports it.
// Returns whether a long group is out of order.
__device__ __noinline__ bool fixup_rare(uint64_t *keys, uint32_t *vals, int64_t m, int64_t p, uint64_t kp,
                                        bool start, int64_t chunk_end, uint64_t *defer_list,
                                        uint32_t *defer_count, int *delta) {
    // group ids never change here (the fix-up permutes within groups), so
    // reads that race with a fix-up see the same ids
    const uint64_t g = kp >> kShortShift;
    if (start) {
        int sz = 2;  // a group starts here: its size, up to kFixCap + 1
        while (sz <= kFixCap && p + sz < m && ((keys[p + sz] & kKeyBits) >> kShortShift) == g) ++sz;
        if (sz > kFixCap) return false;  // long: its inversions are checked at their own positions
        if (p + sz > chunk_end) {  // reaches into the next chunk: the second kernel sorts it
            defer_list[atomicAdd(defer_count, 1u)] = uint64_t(p);
            return false;
        }
        *delta += sort_group(keys, vals, p, sz, nullptr);
        return false;
    }
    // an inversion: fine inside a group of at most kFixCap (sorted by its
    // start), else the group is out of order
    int64_t st = -1;
    for (int i = 1; i <= kFixCap; ++i)
        if (p - i < 0 || ((keys[p - i] & kKeyBits) >> kShortShift) != g) {
            st = p - i + 1;
            break;
        }
    return st < 0 || (st + kFixCap < m && ((keys[st + kFixCap] & kKeyBits) >> kShortShift) == g);
}

// The check of one record at p (its key kp, the previous kq and next kn;
// ~0 beyond the ends): nothing to do unless p starts a group of two or more
// records or is an inversion.
__device__ __forceinline__ void fixup_at(uint64_t *keys, uint32_t *vals, int64_t m, int64_t p, uint64_t kp,
                                         uint64_t kq, uint64_t kn, int64_t chunk_end, uint64_t *defer_list,
                                         uint32_t *defer_count, int *delta, bool &long_unsorted) {
    const uint64_t g = kp >> kShortShift;
    const bool start = (kq >> kShortShift) != g || p == 0;
    if (start ? (kn >> kShortShift) == g : kp < kq)
        long_unsorted |= fixup_rare(keys, vals, m, p, kp, start, chunk_end, defer_list, defer_count, delta);
}

// Each thread takes kFixPer consecutive records (vector loads; a warp covers
// 32 x kFixPer records, one de-duplication chunk, at a time); neighbours come
// from its own registers, from a shuffle at its ends, or from a single load
// at the warp's ends.  Writes the chunk's count of new values to cnt.
constexpr int kFixPer = 8;
constexpr int64_t kFixChunk = 32 * kFixPer;
static_assert(kFixChunk == kDedupeChunk, "a warp step covers one de-duplication chunk");
// MASK: the records may carry an edge-index bit in bit 63 of their keys (the
// halves of the split sort): the streamed keys are masked to their values.
template <bool MASK>
__global__ void __launch_bounds__(256) k_sort_fixup(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0,
                                                     uint32_t *vals1, int64_t m, Header *h, uint32_t *cnt,
                                                     uint64_t *defer_list) {
    if (ld_volatile(&h->packed)) return;  // the packed sort runs instead (k_sortp.cu)
    const Plan plan = make_plan(h);
    uint64_t *keys = (plan.passes & 1) ? keys1 : keys0;
    uint32_t *vals = (plan.passes & 1) ? vals1 : vals0;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
    constexpr uint64_t km = MASK ? kKeyBits : ~0ull;
    bool long_unsorted = false;
    for (int64_t b = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * kFixChunk; b < m;
         b += nw * kFixChunk) {
        const int64_t p0 = b + int64_t(lane) * kFixPer;
        uint64_t k[kFixPer];
        if (vec && p0 + kFixPer <= m) {
            const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(keys + p0);
#pragma unroll
            for (int i = 0; i < kFixPer / 2; ++i) {
                const ulonglong2 w = src[i];
                k[2 * i] = w.x & km;
                k[2 * i + 1] = w.y & km;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kFixPer; ++i) k[i] = p0 + i < m ? keys[p0 + i] & km : ~0ull;  // ~0: no key
        }
        uint64_t prev = __shfl_up_sync(0xffffffffu, k[kFixPer - 1], 1);
        uint64_t next = __shfl_down_sync(0xffffffffu, k[0], 1);
        if (lane == 0) prev = b > 0 && b <= m ? keys[b - 1] & km : ~0ull;
        if (lane == 31) next = b + kFixChunk < m ? keys[b + kFixChunk] & km : ~0ull;
        int count = 0;
#pragma unroll
        for (int i = 0; i < kFixPer; ++i) {
            const int64_t p = p0 + i;
            const uint64_t kq = i > 0 ? k[i - 1] : prev;
            if (p < m) {
                count += (p == 0 || k[i] != kq) ? 1 : 0;
                fixup_at(keys, vals, m, p, k[i], kq, i + 1 < kFixPer ? k[i + 1] : next, b + kFixChunk,
                         defer_list, &h->defer_count, &count, long_unsorted);
            }
        }
        count = int(__reduce_add_sync(0xffffffffu, uint32_t(count)));
        if (lane == 0) cnt[b / kFixChunk] = uint32_t(count);
    }
    if (long_unsorted) atomicExch(&h->fixup_fallback, 1);
}

// The second kernel: sorts the groups the fix-up deferred (each reaching
// across the end of its chunk) and corrects the counts of the chunks its
// records lie in.
__global__ void __launch_bounds__(256) k_sort_fixup_deferred(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0,
                                                              uint32_t *vals1, int64_t m, const Header *h,
                                                              uint32_t *cnt, const uint64_t *defer_list) {
    if (ld_volatile(&h->packed)) return;  // the packed sort runs instead (k_sortp.cu)
    const Plan plan = make_plan(h);
    uint64_t *keys = (plan.passes & 1) ? keys1 : keys0;
    uint32_t *vals = (plan.passes & 1) ? vals1 : vals0;
    const uint32_t nd = h->defer_count;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nd; q += gridDim.x * blockDim.x) {
        const int64_t p = int64_t(defer_list[q]);
        const uint64_t g = (keys[p] & kKeyBits) >> kShortShift;
        int sz = 1;
        while (sz < kFixCap && p + sz < m && ((keys[p + sz] & kKeyBits) >> kShortShift) == g) ++sz;
        int8_t dflag[kFixCap];
        sort_group(keys, vals, p, sz, dflag);  // a zero total may still move counts between chunks
        for (int i = 1; i < sz; ++i)
            if (dflag[i]) atomicAdd(&cnt[(p + i) / kFixChunk], uint32_t(int32_t(dflag[i])));
    }
}

// ------------------------------------------------------------------ host ---
template <int RADIX, int THREADS = kSortThreads>
constexpr size_t sort_smem() { return sizeof(SortSmem<RADIX, THREADS>); }

// Threads of the non-persistent instance of a pass slot: the 9-bit top pass
// takes one digit per thread.
#ifndef PH0_TOP_THREADS
#define PH0_TOP_THREADS 256
#endif
template <int RADIX>
constexpr int slot_threads() { return RADIX == kMaxRadix ? PH0_TOP_THREADS : kSortThreads; }

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Zero the sort's counters and first look-back buffer (sized for 512 buckets).
cudaError_t launch_sort_init(Header *h, uint64_t *look0, int64_t tiles, cudaStream_t s, int top_bits,
                             int64_t sorted_edges, const int32_t *gate) {
    const int64_t words = tiles * kMaxRadix;
    int blocks = int((words + 255) / 256);
    if (blocks < 8) blocks = 8;
    if (blocks > 4 * sm_count() * 8) blocks = 4 * sm_count() * 8;
    k_sort_init<<<blocks, 256, 0, s>>>(h, look0, words, top_bits == 8 ? 8 : 9, sorted_edges, gate);
    return cudaGetLastError();
}

cudaError_t launch_keystats(const uint64_t *keys, int64_t m, Header *h, cudaStream_t s, const int32_t *gate,
                            bool lows_only) {
    if (m <= 0) return cudaSuccess;
    int64_t blocks = (m + 255) / 256;
    const int64_t cap = int64_t(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    k_keystats<<<unsigned(blocks), 256, 0, s>>>(keys, m, h, gate, lows_only ? 1 : 0);
    return cudaGetLastError();
}

template <int RADIX, int SLOT>
static cudaError_t set_attr() {
    constexpr int TT = slot_threads<RADIX>();
    const int bytes = int(sort_smem<RADIX>());
    const int tbytes = int(sort_smem<RADIX, TT>());
    cudaError_t e = cudaFuncSetAttribute(k_onesweep<RADIX, SLOT, true, false, TT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, tbytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_onesweep<RADIX, SLOT, false, false, TT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, tbytes);
    if constexpr (SLOT != kClassSlot) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_onesweep<RADIX, SLOT, false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_onesweep<RADIX, SLOT, true, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }
    return e;
}

cudaError_t prepare_sort_kernels() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr<kRadix, 0>();
    if (e == cudaSuccess) e = set_attr<kRadix, 1>();
    if (e == cudaSuccess) e = set_attr<kRadix, 2>();
    if (e == cudaSuccess) e = set_attr<kRadix, 3>();
    if (e == cudaSuccess) e = set_attr<kRadix, 4>();
    if (e == cudaSuccess) e = set_attr<kRadix, 5>();
    if (e == cudaSuccess) e = set_attr<kRadix, 6>();
    if (e == cudaSuccess) e = set_attr<kMaxRadix, 6>();
    if (e == cudaSuccess) e = set_attr<kRadix, 7>();
    if (e == cudaSuccess) e = set_attr<kRadix, kClassSlot>();
    return e;
}

// persist: run the persistent instance on sort_min_blocks<RADIX>() CTAs per SM,
// for passes that usually return at once (a grid of one CTA per tile costs
// ~0.1 ms at 131k tiles even then).
template <int RADIX, int SLOT>
static void launch_slot(unsigned tiles, uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                        int64_t m, uint64_t *look0, uint64_t *look1, Header *h, bool persist, cudaStream_t s) {
    // tiles arrive by bulk copies only when both buffers' rows are 16-byte aligned
    const bool aligned = ((reinterpret_cast<uintptr_t>(keys0) | reinterpret_cast<uintptr_t>(keys1) |
                           reinterpret_cast<uintptr_t>(vals0) | reinterpret_cast<uintptr_t>(vals1)) & 15u) == 0;
    if constexpr (SLOT != kClassSlot) {
        // the 9-bit top pass measured faster on persistent CTAs taking tile
        // after tile (4.46 against 4.65 ms at 537M keys; the 8-bit passes
        // slower: 3.87-4.08 against 3.62-3.71 ms)
        if (persist || (RADIX == kMaxRadix && aligned)) {
            const unsigned cap = unsigned(sm_count()) * sort_min_blocks<RADIX>();
            if (aligned)
                k_onesweep<RADIX, SLOT, true, true><<<tiles < cap ? tiles : cap, kSortThreads, sort_smem<RADIX>(), s>>>(
                    keys0, keys1, vals0, vals1, m, look0, look1, h);
            else
                k_onesweep<RADIX, SLOT, false, true><<<tiles < cap ? tiles : cap, kSortThreads, sort_smem<RADIX>(), s>>>(
                    keys0, keys1, vals0, vals1, m, look0, look1, h);
            return;
        }
    }
    constexpr int TT = slot_threads<RADIX>();
    if (aligned)
        k_onesweep<RADIX, SLOT, true, false, TT><<<tiles, TT, sort_smem<RADIX, TT>(), s>>>(
            keys0, keys1, vals0, vals1, m, look0, look1, h);
    else
        k_onesweep<RADIX, SLOT, false, false, TT><<<tiles, TT, sort_smem<RADIX, TT>(), s>>>(
            keys0, keys1, vals0, vals1, m, look0, look1, h);
}

// One pass slot (prepare_sort_kernels() must have run).
cudaError_t launch_sort_pass(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                             int64_t m, int pass, uint64_t *look0, uint64_t *look1, Header *h,
                             cudaStream_t s, bool persist) {
    const unsigned tiles = unsigned((m + kSortTile - 1) / kSortTile);
#define PH0_SLOT(R, S) launch_slot<R, S>(tiles, keys0, keys1, vals0, vals1, m, look0, look1, h, persist, s)
    switch (pass) {
        case 0: PH0_SLOT(kRadix, 0); break;
        case 1: PH0_SLOT(kRadix, 1); break;
        case 2: PH0_SLOT(kRadix, 2); break;
        case 3: PH0_SLOT(kRadix, 3); break;
        case 4: PH0_SLOT(kRadix, 4); break;
        case 5: PH0_SLOT(kRadix, 5); break;
        case 6:  // two instances, one of which returns at once (k_top_compact)
            k_top_compact<<<1, kMaxRadix, 0, s>>>(h);
            PH0_SLOT(kRadix, 6);
            PH0_SLOT(kMaxRadix, 6);
            break;
        case 7: PH0_SLOT(kRadix, 7); break;
        default: PH0_SLOT(kRadix, kClassSlot); break;
    }
#undef PH0_SLOT
    return cudaGetLastError();
}

// The passes over buffers (keys0, vals0) <-> (keys1, vals1); the sorted data
// ends in buffer (passes & 1), which the device records in the header.
cudaError_t launch_sort_passes(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                               int64_t m, uint64_t *look0, uint64_t *look1, Header *h,
                               cudaStream_t s, bool persist) {
    if (m <= 0) return cudaSuccess;
    cudaError_t e = prepare_sort_kernels();
    if (e != cudaSuccess) return e;
    for (int p = 0; p < kMaxPasses; ++p) {
        e = launch_sort_pass(keys0, keys1, vals0, vals1, m, p, look0, look1, h, s, persist);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The short sort of the records in buffer 0 (see k_sort_fixup): the passes
// from slot kShortFirstSlot on, then the fix-up.  look0 must be zeroed
// (launch_sort_init), h's histograms complete.  The records end sorted in
// buffer (passes & 1), unless h->fixup_fallback.
cudaError_t launch_sort_fixup(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1, int64_t m,
                              Header *h, uint32_t *cnt, uint64_t *defer_list, cudaStream_t s, bool masked);
// persist_all: every pass on its persistent instance (a short sort that
// usually returns at once: the packed sort's stand-in).
cudaError_t launch_sort_short(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                              int64_t m, uint64_t *look0, uint64_t *look1, Header *h, uint32_t *cnt,
                              cudaStream_t s, bool masked, bool persist_all) {
    if (m <= 0) return cudaSuccess;
    cudaError_t e = prepare_sort_kernels();
    if (e != cudaSuccess) return e;
    for (int p = kShortFirstSlot; p < kMaxPasses; ++p) {
        // the last slot works only for keys whose top part needs two passes
        e = launch_sort_pass(keys0, keys1, vals0, vals1, m, p, look0, look1, h, s,
                             persist_all || p == kMaxPasses - 1);
        if (e != cudaSuccess) return e;
    }
    // the deferred groups' list lives in look1, unused after the passes
    return launch_sort_fixup(keys0, keys1, vals0, vals1, m, h, cnt, look1, s, masked);
}

// The fix-up and its second kernel; cnt: one word per de-duplication chunk;
// defer_list: room for one word per chunk.
cudaError_t launch_sort_fixup(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1, int64_t m,
                              Header *h, uint32_t *cnt, uint64_t *defer_list, cudaStream_t s, bool masked) {
    if (m <= 0) return cudaSuccess;
    int64_t blocks = (m + 255) / 256;
    const int64_t cap = int64_t(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    if (masked)
        k_sort_fixup<true><<<unsigned(blocks), 256, 0, s>>>(keys0, keys1, vals0, vals1, m, h, cnt, defer_list);
    else
        k_sort_fixup<false><<<unsigned(blocks), 256, 0, s>>>(keys0, keys1, vals0, vals1, m, h, cnt, defer_list);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sort_fixup_deferred<<<unsigned(sm_count()), 256, 0, s>>>(keys0, keys1, vals0, vals1, m, h, cnt, defer_list);
    return cudaGetLastError();
}

cudaError_t launch_copy_parity(uint64_t *keys_dst, const uint64_t *keys_src, uint32_t *vals_dst,
                               const uint32_t *vals_src, int64_t m, const Header *h, int parity,
                               const int32_t *gate, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    int64_t blocks = (m + 255) / 256;
    const int64_t cap = int64_t(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    k_copy_parity<<<unsigned(blocks), 256, 0, s>>>(keys_dst, keys_src, vals_dst, vals_src, m, h, parity, gate);
    return cudaGetLastError();
}

cudaError_t launch_copy_if_odd(uint64_t *keys0, const uint64_t *keys1, uint32_t *vals0,
                               const uint32_t *vals1, int64_t m, const Header *h, cudaStream_t s) {
    return launch_copy_parity(keys0, keys1, vals0, vals1, m, h, 1, nullptr, s);
}

// ---- the merge of two sorted halves (clouds of more than 2^32 edges) ----
//
// Above kSplitEdges edges the sort takes the two halves of the edge array
// (each below 2^32 records) one after the other and merges them: by key
// value (bit 63 masked), the first half first among equal values (its edge
// indices, hence (u, v), are the smaller), which is the order of a stable
// sort of the whole array.  A tile of kMergeTile outputs per CTA: its split
// points (how many of its first output records come from the first half)
// come from k_merge_split, its inputs are staged in shared memory, and each
// thread merges kMergeItems consecutive outputs.
constexpr int kMergeThreads = 256, kMergeItems = 8, kMergeTile = kMergeThreads * kMergeItems;
static_assert(kMergeTile % 32 == 0, "tiles cover whole words of the index-bit mask");

// Of the first d records of the merge, how many come from A (A first among
// equal values).
template <class KA, class KB>
__device__ __forceinline__ int64_t merge_split(KA ka, int64_t la, KB kb, int64_t lb, int64_t d) {
    int64_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((ka[mid] & kKeyBits) <= (kb[d - 1 - mid] & kKeyBits)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_merge_split(const uint64_t *ka, int64_t la, const uint64_t *kb, int64_t lb, int64_t *split,
                              int64_t tiles) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t <= tiles; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t d = t * kMergeTile < la + lb ? t * kMergeTile : la + lb;
        split[t] = merge_split(ka, la, kb, lb, d);
    }
}

// hib: one bit per output record, bit 32 of its edge index (its key's bit
// 63), or null.
__global__ void __launch_bounds__(kMergeThreads) k_merge(const uint64_t *ka, const uint32_t *va, int64_t la,
                                                         const uint64_t *kb, const uint32_t *vb, int64_t lb,
                                                         const int64_t *split, uint64_t *ko, uint32_t *vo,
                                                         uint32_t *hib) {
    __shared__ uint64_t s_k[kMergeTile];
    __shared__ uint32_t s_v[kMergeTile];
    const int64_t total = la + lb, d0 = int64_t(blockIdx.x) * kMergeTile;
    if (d0 >= total) return;
    const int64_t d1 = d0 + kMergeTile < total ? d0 + kMergeTile : total;
    const int64_t i0 = split[blockIdx.x], i1 = split[blockIdx.x + 1];
    const int na = int(i1 - i0), nb = int((d1 - i1) - (d0 - i0)), nt = na + nb;
    const int64_t j0 = d0 - i0;
    for (int i = threadIdx.x; i < nt; i += kMergeThreads) {
        const bool fa = i < na;
        s_k[i] = fa ? ka[i0 + i] : kb[j0 + i - na];
        s_v[i] = fa ? va[i0 + i] : vb[j0 + i - na];
    }
    __syncthreads();
    const int dd = threadIdx.x * kMergeItems;
    uint64_t ok[kMergeItems];
    uint32_t ov[kMergeItems];
    uint32_t bits = 0;
    if (dd < nt) {
        const uint64_t *A = s_k, *B = s_k + na;
        int i = int(merge_split(A, na, B, nb, dd)), j = dd - i;
#pragma unroll
        for (int r = 0; r < kMergeItems; ++r) {
            if (dd + r >= nt) break;
            const bool fa = j >= nb || (i < na && (A[i] & kKeyBits) <= (B[j] & kKeyBits));
            const int src = fa ? i++ : na + j++;
            ok[r] = s_k[src];
            ov[r] = s_v[src];
            bits |= uint32_t(ok[r] >> 63) << r;
        }
#pragma unroll
        for (int r = 0; r < kMergeItems; ++r)
            if (dd + r < nt) {
                ko[d0 + dd + r] = ok[r];
                vo[d0 + dd + r] = ov[r];
            }
    }
    if (hib) {  // four threads' 8 bits make one word (tiles start on whole words)
        static_assert(kMergeItems == 8, "4 x 8 bits per word");
        const int lane = threadIdx.x & 31;
        uint32_t w = bits << (8 * (lane & 3));
        w |= __shfl_down_sync(0xffffffffu, w, 1);
        w |= __shfl_down_sync(0xffffffffu, w, 2);
        if ((lane & 3) == 0 && dd < nt) hib[(d0 + dd) >> 5] = w;
    }
}

// Merge (ka, va)[0, la) and (kb, vb)[0, lb), each sorted, into (ko, vo);
// split: room for (la + lb) / kMergeTile + 2 words.
cudaError_t launch_merge(const uint64_t *ka, const uint32_t *va, int64_t la, const uint64_t *kb,
                         const uint32_t *vb, int64_t lb, uint64_t *ko, uint32_t *vo, uint32_t *hib, int64_t *split,
                         cudaStream_t s) {
    const int64_t tiles = (la + lb + kMergeTile - 1) / kMergeTile;
    if (tiles == 0) return cudaSuccess;
    const int64_t sblocks = (tiles + 1 + 255) / 256;
    k_merge_split<<<unsigned(sblocks < 65535 ? sblocks : 65535), 256, 0, s>>>(ka, la, kb, lb, split, tiles);
    k_merge<<<unsigned(tiles), kMergeThreads, 0, s>>>(ka, va, la, kb, vb, lb, split, ko, vo, hib);
    return cudaGetLastError();
}

}  // namespace ph0
