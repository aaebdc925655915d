// k_sortp.cu -- the packed sort of the whole path: step 2 (Rawson, Sec. 2:
// the distances in increasing order; Sec. 4 step 2), with step 3's count of
// the distinct values taken on the way (Sec. 2: the set D).
//
// For clouds of at most 32768 points every edge travels through the sort as
// one 64-bit word (layout in ph0_common.cuh): the number of its key's top
// part among the values that occur, key bits 22..47, and (u << 15) | v.
// Words order as (key >> 22, edge index), so four stable passes (9, 9, 8 and
// 8 bits) over word bits 30..63 leave the edges ordered by key >> 22 and,
// inside each group of equal key >> 22, by index.  The fix-up then sorts
// every group of two or more words by the whole key, read from the distance
// kernel's output (the key of edge e at e), which completes the order
// (distance, edge index) of the other sorts; on the benchmark cloud (32,768
// points in dimension 16) 24.6% of the edges lie in such groups, none longer
// than 8.  A longer group (more than kPFixCap words: many equal distances) is
// only checked: in order when its keys do not decrease.  The fix-up also
// writes what steps 3-5 read: the record (u << 16) | v at every position and
// one bit per position marking a new distance value.
//
// A pass moves 16 bytes per edge (an 8-byte word read and written) where the
// (key, value) records of k_sort.cu move 24, and there are four passes where
// the short sort runs five.  Pass 0 reads the keys in edge order and forms
// the words as it loads them: each thread's items are edges 32 apart, so it
// finds (u, v) of its first from the edge index and steps along the rows.
//
// Gating, on the device: k_packed_prep finds whether the keys pack (their top
// part spans fewer than 512 values, of which at most 256 occur) and sets
// h->packed, else h->classic.  Every kernel here returns at once unless
// h->packed; the short sort of k_sort.cu returns at once when it is set, and
// runs (with k_keystats gated on h->classic for its histograms) when not.  A
// group of more than kPLongCap words, or a long group out of order, sets
// h->fixup_fallback, on which the caller gates the complete sort of
// k_sort.cu, which then replaces the result.
#include "sort_util.cuh"

namespace ph0 {

// Whether the keys pack; numbers the top part's values that occur (top_lut)
// and writes the top pass's histogram.  One CTA of kMaxRadix threads.
__global__ void __launch_bounds__(kMaxRadix) k_packed_prep(Header *h) {
    __shared__ uint32_t s_warp[kMaxRadix / 32 + 1];
    const int t = threadIdx.x;
    const uint64_t kmin = h->kmin, kmax = h->kmax;
    const uint64_t t0 = kmin >> kTopShift;
    const uint64_t span = kmax >= kmin ? (kmax >> kTopShift) - t0 : 0;  // top values t0 .. t0 + span
    const bool fits = span < uint64_t(kMaxRadix);
    uint32_t c = 0;
    if (fits && uint64_t(t) <= span) c = h->hist_top_mod[(uint32_t(t) + uint32_t(t0)) & (kMaxRadix - 1)];
    uint32_t tot;
    const uint32_t idx = block_excl_scan<kMaxRadix>(c != 0 ? 1u : 0u, s_warp, tot);
    const bool ok = fits && tot <= uint32_t(kRadix);
    if (ok) {
        h->top_lut[t] = uint8_t(c != 0 ? idx : 0u);  // values that occur nowhere are never looked up
        if (c != 0) h->phist[kPackPasses - 1][idx] = c;
    }
    if (t == 0) {
        h->packed = ok ? 1 : 0;
        h->classic = ok ? 0 : 1;
    }
}

// ---- the passes -----------------------------------------------------------
constexpr int kPThreads = kSortThreads;
constexpr int kPItems = kSortItems;
constexpr int kPTile = kSortTile;  // the tiling of the look-back buffers
template <int Q>
struct PSmem {
    static constexpr int R = pack_radix(Q);
    static constexpr int W = kPThreads / 32;
    uint64_t w[kPTile];       // the tile's words, then in sorted order (in place)
    uint16_t whist[W][R];     // per-warp digit counts, then each warp's first local position
    uint32_t gofs[R];         // global position of sorted tile index 0 of each digit's run (mod 2^32)
    uint32_t scan[W + 1];
    uint32_t tile;
    unsigned long long mbar;  // completion of the tile's bulk copy
    uint8_t lut[Q == 0 ? kMaxRadix : 16];  // pass 0: number of each top-part value
};

template <int Q>
__device__ __forceinline__ uint32_t pdigit(uint64_t w) {
    return uint32_t(w >> pack_shift(Q)) & uint32_t(pack_radix(Q) - 1);
}

#ifndef PH0_PSORT_MIN_BLOCKS
#define PH0_PSORT_MIN_BLOCKS 4
#endif
#ifndef PH0_PSORT0_MIN_BLOCKS
#define PH0_PSORT0_MIN_BLOCKS PH0_PSORT_MIN_BLOCKS
#endif

// Pass Q: reads `in` (pass 0: the keys by edge index of an n-point cloud;
// else words), writes the words stably ordered by digit Q to `out`.  Its
// look-back words (kMaxRadix per tile) live in `look`; it clears its tile's
// words in `look_next` for the next pass.  One tile of kPTile words per CTA,
// tiles taken from a counter (every tile a CTA waits on belongs to a CTA
// already running).
template <int Q>
__global__ void __launch_bounds__(kPThreads, Q == 0 ? PH0_PSORT0_MIN_BLOCKS : PH0_PSORT_MIN_BLOCKS)
k_psweep(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, int64_t m, int32_t n, uint64_t *look,
         uint64_t *look_next, Header *h) {
    constexpr int R = pack_radix(Q), DPT = R / kPThreads, W = kPThreads / 32, IT = kPItems, TILE = kPTile;
    static_assert(R % kPThreads == 0 && IT * kPThreads == TILE, "tiling");
    extern __shared__ __align__(16) unsigned char s_raw[];
    PSmem<Q> &S = *reinterpret_cast<PSmem<Q> *>(s_raw);
    if (ld_volatile(&h->packed) == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        S.tile = atomicAdd(&h->ptile[Q], 1u);
        mbar_init(&S.mbar, 1);
    }
    uint32_t t0 = 0;
    if constexpr (Q == 0) {
        for (int i = tid; i < kMaxRadix; i += kPThreads) S.lut[i] = h->top_lut[i];
        t0 = uint32_t(h->kmin >> kTopShift);
    }
    __syncthreads();
    const int64_t tile = S.tile;
    const int64_t base = tile * TILE;
    const int valid = int(m - base < TILE ? m - base : TILE);
    // a full tile arrives in shared memory by one bulk copy while the counters
    // are cleared and tile 0 scans the histogram; the ragged last tile by loads
    const bool full = valid == TILE;
    if (full && tid == 0) {
        mbar_expect_tx(&S.mbar, uint32_t(TILE * sizeof(uint64_t)));
        bulk_g2s(S.w, in + base, uint32_t(TILE * sizeof(uint64_t)), &S.mbar);
    }
    {  // each warp clears its own counter row
        uint32_t *row = reinterpret_cast<uint32_t *>(&S.whist[warp][0]);
#pragma unroll
        for (int i = lane; i < R / 2; i += 32) row[i] = 0;
        __syncwarp();
    }
    // digit starts (tile 0 only), folded into tile 0's PREFIX words
    uint32_t bucket[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) bucket[q] = 0;
    if (tile == 0) {
        uint32_t hsum = 0;
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            bucket[q] = h->phist[Q][tid * DPT + q];
            hsum += bucket[q];
        }
        uint32_t tot;
        uint32_t run = block_excl_scan<kPThreads>(hsum, S.scan, tot);
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const uint32_t c = bucket[q];
            bucket[q] = run;
            run += c;
        }
    }

    // ---- words (striped within each warp) and stable ranking ----
    uint64_t k[IT];
    uint32_t rk[IT / 2];  // rank among the warp's items of the same digit, item j in half j & 1
    const int wloc = warp * 32 * IT;
    if (full) {
        if (!mbar_wait(&S.mbar, 0)) set_status(h, PH0_ETIMEOUT);
#pragma unroll
        for (int j = 0; j < IT; ++j) k[j] = S.w[wloc + j * 32 + lane];
    } else {
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const int loc = wloc + j * 32 + lane;
            k[j] = loc < valid ? in[base + loc] : 0;
        }
    }
    if constexpr (Q == 0) {  // form the words: top number, key bits 22..47, (u << 15) | v
        // (u, v) of the thread's first edge, then of each edge 32 further on:
        // past the row's end (v = n) the next row begins at v = u + 2
        uint32_t u = 0, v = 0;
        const int64_t e0 = base + wloc + lane;
        if (e0 < m) edge_uv(e0, n, u, v);
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            if (j > 0) edge_step(u, v, uint32_t(n), 32);
            const uint64_t key = k[j];
            const uint32_t top = S.lut[(uint32_t(key >> kTopShift) - t0) & (kMaxRadix - 1)];
            k[j] = (uint64_t(top) << 56) |
                   (((key >> kPackKeyShift) & ((uint64_t(1) << kPackKeyBits) - 1)) << kPackIdBits) |
                   uint64_t((u << 15) | (v & 0x7fffu));
        }
    }
    const unsigned lt = (1u << lane) - 1u;
    constexpr int kBits = R == 512 ? 9 : 8;
    // the digit of item j (the sentinel R past the end of the ragged tile)
    auto digit = [&](int j) -> uint32_t {
        return (full || wloc + j * 32 + lane < valid) ? pdigit<Q>(k[j]) : uint32_t(R);
    };
#pragma unroll
    for (int j = 0; j < IT; j += 2) rk[j / 2] = 0;
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const uint32_t dj = digit(j);
        // lanes with the same digit: one ballot per digit bit (the ragged
        // tile's sentinel digit R needs one more)
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < kBits; ++b) {
            const bool bit = (dj >> b) & 1u;
            const unsigned vote = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? vote : ~vote;
        }
        if (!full) {
            const bool bit = (dj >> kBits) & 1u;
            const unsigned vote = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? vote : ~vote;
        }
        const uint32_t before = __popc(peers & lt);
        const uint32_t prior = dj < uint32_t(R) ? S.whist[warp][dj] : 0u;
        rk[j / 2] |= (prior + before) << (16 * (j & 1));
        __syncwarp();
        if (dj < uint32_t(R) && before == 0) S.whist[warp][dj] = uint16_t(prior + __popc(peers));
        __syncwarp();
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
        uint32_t run = block_excl_scan<kPThreads>(tsum, S.scan, tot);
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = tid * DPT + q;
            lstart[q] = run;
            uint32_t pos = run;
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

    // ---- reorder the words by digit, in place (every thread holds its own) ----
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const uint32_t dj = digit(j);
        if (dj < uint32_t(R))
            S.w[(S.whist[warp][dj] + ((rk[j / 2] >> (16 * (j & 1))) & 0xffffu)) & (TILE - 1)] = k[j];
    }

    // ---- look-back, global offsets ----
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
    __syncthreads();

    // ---- write contiguous runs, one per digit ----
    const uint32_t m32 = uint32_t(m);  // m < 2^29
#pragma unroll 4
    for (int i = tid; i < valid; i += kPThreads) {
        const uint64_t x = S.w[i];
        const uint32_t g = S.gofs[pdigit<Q>(x)] + uint32_t(i);
        if (g >= m32) continue;  // never taken when the counts are consistent
        out[g] = x;
    }
    for (int i = tid; i < kMaxRadix; i += kPThreads) look_next[tile * kMaxRadix + i] = 0;
    if (Q == kPackPasses - 1 && tile == 0 && tid == 0) {
        h->sort_passes = kPackPasses;
        h->key_bits = 64 - kPackIdBits;
    }
}

// ---- the fix-up ------------------------------------------------------------
//
// A warp takes one de-duplication chunk of kPFixChunk positions at a time,
// kPFixPer consecutive words per lane.  A position whose word >> 30 differs
// from both neighbours' (a singleton: almost every position) is a new
// distance value.  Each lane fetches the whole keys of its positions that lie
// in groups (all such loads in flight at once) into shared memory, the lane
// at the start of a group of at most kPFixCap words that ends inside the
// chunk sorts it there, and every lane writes the records of its positions:
// (u << 16) | v, the form the reduction reads.  A group reaching into the
// next chunk, or longer than kPFixCap, is left to a second kernel, which
// sorts (or checks) it once every chunk's flags and count are written and
// adds its members' flags and counts.
constexpr int kPFixCap = 32;
constexpr int kPLongCap = 4096;
constexpr int kPFixPer = 8;
constexpr int64_t kPFixChunk = 32 * kPFixPer;
constexpr int kPFixWarps = 8;  // warps per CTA
static_assert(kPFixChunk == kDedupeChunk, "a warp step covers one de-duplication chunk");
static_assert(kPFixChunk % 32 == 0, "a chunk covers whole flag words");
static_assert(int64_t(kMaxRadix) * kPFixChunk / kSortTile >= kPFixChunk / (kPFixCap + 1) + 1,
              "the look-back buffer the list lives in holds every deferred group");

// Sorts sz (key, record) pairs in place by key, stably (an equal key stays
// behind); returns each member's new-value flag as bit i (member 0's
// predecessor lies in another group: always new).
template <class K, class R>
__device__ uint32_t sort_pairs_stable(K *kk, R *rr, int sz) {
    for (int i = 1; i < sz; ++i) {
        const uint64_t k = kk[i];
        const uint32_t r = rr[i];
        int j = i - 1;
        while (j >= 0 && uint64_t(kk[j]) > k) {
            kk[j + 1] = kk[j];
            rr[j + 1] = rr[j];
            --j;
        }
        kk[j + 1] = k;
        rr[j + 1] = r;
    }
    uint32_t fl = 1u;
    for (int i = 1; i < sz; ++i)
        if (uint64_t(kk[i]) != uint64_t(kk[i - 1])) fl |= 1u << i;
    return fl;
}

#ifndef PH0_PFIX_MIN_BLOCKS
#define PH0_PFIX_MIN_BLOCKS 4
#endif
// w: the sorted words; keyidx: the key of each edge by index; recs: the
// record (u << 16) | v at each position; flags: bit p = a new distance value
// at p; cnt: new values per chunk (step 3's count mode); defer_list: room for
// kPFixChunk / (kPFixCap + 1) + 1 words per chunk (the long groups that start
// in it and the group across its end).  A word whose (u, v) is no edge of the
// cloud (never, when the passes' counts are consistent) is reported.
__global__ void __launch_bounds__(32 * kPFixWarps, PH0_PFIX_MIN_BLOCKS)
k_pfixup(const uint64_t *__restrict__ w, int64_t m, int64_t n, const uint64_t *__restrict__ keyidx,
         uint32_t *__restrict__ recs, uint32_t *__restrict__ flags, uint32_t *__restrict__ cnt,
         uint64_t *defer_list, Header *h) {
    if (ld_volatile(&h->packed) == 0) return;
    __shared__ uint64_t s_key[kPFixWarps][kPFixChunk];  // whole keys of grouped positions
    __shared__ uint32_t s_rec[kPFixWarps][kPFixChunk];  // their records
    __shared__ uint32_t s_fl[kPFixWarps][kPFixChunk / 32];
    __shared__ uint32_t s_cont[kPFixWarps][kPFixChunk / 32];  // bit q: position q continues q-1's group
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    constexpr uint64_t kNone = ~0ull;  // above every group value (< 2^35)
    uint64_t *sk = s_key[wib];
    uint32_t *sr = s_rec[wib];
    for (int64_t b = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * kPFixChunk; b < m;
         b += nw * kPFixChunk) {
        const int64_t p0 = b + int64_t(lane) * kPFixPer;
        const int own = lane * kPFixPer;  // chunk-relative index of the lane's first position
        uint64_t x[kPFixPer], g[kPFixPer];
        if (p0 + kPFixPer <= m) {
            const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(w + p0);
#pragma unroll
            for (int i = 0; i < kPFixPer / 2; ++i) {
                const ulonglong2 v = src[i];
                x[2 * i] = v.x;
                x[2 * i + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kPFixPer; ++i) x[i] = p0 + i < m ? w[p0 + i] : 0;
        }
#pragma unroll
        for (int i = 0; i < kPFixPer; ++i) g[i] = p0 + i < m ? x[i] >> kPackIdBits : kNone;
        uint64_t prev = __shfl_up_sync(0xffffffffu, g[kPFixPer - 1], 1);
        uint64_t next = __shfl_down_sync(0xffffffffu, g[0], 1);
        if (lane == 0) prev = b > 0 ? w[b - 1] >> kPackIdBits : kNone;
        if (lane == 31) next = b + kPFixChunk < m ? w[b + kPFixChunk] >> kPackIdBits : kNone;
        // cont bit i: position i continues the group of position i-1 (both exist)
        uint32_t cont = 0;
#pragma unroll
        for (int i = 0; i < kPFixPer; ++i)
            if (p0 + i < m && (i > 0 ? g[i - 1] : prev) == g[i]) cont |= 1u << i;
        // whether the lane's last position continues into the next one
        const bool last_cont = p0 + kPFixPer - 1 < m && next == g[kPFixPer - 1];
        const uint32_t after = cont >> 1 | (last_cont ? 1u << (kPFixPer - 1) : 0u);  // bit i: i+1 continues i
        uint32_t valid = 0;
#pragma unroll
        for (int i = 0; i < kPFixPer; ++i)
            if (p0 + i < m) valid |= 1u << i;
        const uint32_t grouped = (cont | after) & valid;
        const uint32_t mine = valid & ~grouped;   // singletons: new values
        uint32_t starts = after & ~cont & valid;  // a group of two or more starts here
        const bool tail_cont = __shfl_sync(0xffffffffu, last_cont ? 1 : 0, 31) != 0;  // into the next chunk
        {  // the chunk's cont mask: lanes 4k..4k+3 make word k
            uint32_t cw = cont << ((lane & 3) * kPFixPer);
            cw |= __shfl_xor_sync(0xffffffffu, cw, 1);
            cw |= __shfl_xor_sync(0xffffffffu, cw, 2);
            if ((lane & 3) == 0) s_cont[wib][lane >> 2] = cw;
        }
        // the whole keys of the grouped positions: every load issued first
        uint64_t kk[kPFixPer];
        uint32_t r[kPFixPer];
#pragma unroll
        for (int i = 0; i < kPFixPer; ++i) {
            r[i] = pack_record(x[i]);
            const bool ok = (r[i] >> 16) < (r[i] & 0xffffu) && int64_t(r[i] & 0xffffu) < n;
            if (((valid >> i) & 1u) && !ok) set_status(h, PH0_EINTERNAL);  // never, when the counts are consistent
            kk[i] = ((grouped >> i) & 1u) && ok ? keyidx[pack_edge(x[i], uint32_t(n))] : ~0ull;
        }
#pragma unroll
        for (int i = 0; i < kPFixPer; ++i)
            if ((grouped >> i) & 1u) {
                sk[own + i] = kk[i];
                sr[own + i] = r[i];
            }
        if (lane < kPFixChunk / 32) s_fl[wib][lane] = 0;
        __syncwarp();
        atomicOr(&s_fl[wib][lane >> 2], mine << ((lane & 3) * kPFixPer));
        // each group start: its size from the cont mask, then sorted here or
        // left to the second kernel
        while (starts) {
            const int i = __ffs(starts) - 1;
            starts &= starts - 1;
            const int at = own + i;
            int sz = 2;
            while (sz <= kPFixCap && at + sz < int(kPFixChunk) && ((s_cont[wib][(at + sz) >> 5] >> ((at + sz) & 31)) & 1u))
                ++sz;
            // the last member inside the chunk is at + sz - 1; a start at the
            // chunk's last position has its second member in the next chunk
            if (sz > kPFixCap || (at + sz >= int(kPFixChunk) && tail_cont)) {
                defer_list[atomicAdd(&h->defer_count, 1u)] = uint64_t(p0 + i);
                continue;
            }
            const uint32_t fl = sort_pairs_stable(sk + at, sr + at, sz);
            for (int q = 0; q < sz; ++q)
                if ((fl >> q) & 1u) atomicOr(&s_fl[wib][(at + q) >> 5], 1u << ((at + q) & 31));
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < kPFixPer; ++i)
            if ((grouped >> i) & 1u) r[i] = sr[own + i];
        if (p0 + kPFixPer <= m) {
            uint4 *dst = reinterpret_cast<uint4 *>(recs + p0);
            dst[0] = make_uint4(r[0], r[1], r[2], r[3]);
            dst[1] = make_uint4(r[4], r[5], r[6], r[7]);
        } else {
            for (int i = 0; i < kPFixPer; ++i)
                if (p0 + i < m) recs[p0 + i] = r[i];
        }
        const uint32_t f = lane < kPFixChunk / 32 ? s_fl[wib][lane] : 0u;
        if (lane < kPFixChunk / 32 && b / 32 + lane < (m + 31) / 32) flags[b / 32 + lane] = f;
        const uint32_t count = __reduce_add_sync(0xffffffffu, uint32_t(__popc(f)));
        if (lane == 0) cnt[b / kPFixChunk] = count;
        __syncwarp();  // before the next chunk reuses the shared arrays
    }
}

// The second kernel: the groups that reach across the end of their chunk
// (sorted), and the groups of more than kPFixCap words (checked: in order
// when their keys do not decrease; up to kPLongCap words).  Anything else
// sets h->fixup_fallback.
__global__ void __launch_bounds__(256) k_pfixup_deferred(const uint64_t *w, int64_t m, int64_t n,
                                                          const uint64_t *keyidx, uint32_t *recs,
                                                          uint32_t *flags, uint32_t *cnt,
                                                          const uint64_t *defer_list, Header *h) {
    if (ld_volatile(&h->packed) == 0) return;
    const uint32_t nd = ld_volatile(&h->defer_count);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nd; q += gridDim.x * blockDim.x) {
        const int64_t p = int64_t(defer_list[q]);
        const uint64_t g = w[p] >> kPackIdBits;
        int sz = 1;
        while (sz <= kPLongCap && p + sz < m && (w[p + sz] >> kPackIdBits) == g) ++sz;
        if (sz > kPLongCap) {
            atomicExch(&h->fixup_fallback, 1);
            continue;
        }
        bool ok = true;
        for (int i = 0; i < sz; ++i) {
            const uint32_t r = pack_record(w[p + i]);
            if ((r >> 16) >= (r & 0xffffu) || int64_t(r & 0xffffu) >= n) ok = false;
        }
        if (!ok) {
            set_status(h, PH0_EINTERNAL);
            continue;
        }
        if (sz > kPFixCap) {  // long: in order, or not a result (its records stand as written)
            uint64_t kq = 0;
            for (int i = 0; i < sz && ok; ++i) {
                const uint64_t k = keyidx[pack_edge(w[p + i], uint32_t(n))];
                if (i > 0 && k < kq) ok = false;
                if (i == 0 || k != kq) {
                    atomicOr(&flags[(p + i) >> 5], 1u << ((p + i) & 31));
                    atomicAdd(&cnt[(p + i) / kPFixChunk], 1u);
                }
                kq = k;
            }
            if (!ok) atomicExch(&h->fixup_fallback, 1);
            continue;
        }
        uint64_t kk[kPFixCap];
        uint32_t rr[kPFixCap];
        for (int i = 0; i < sz; ++i) {
            kk[i] = keyidx[pack_edge(w[p + i], uint32_t(n))];
            rr[i] = pack_record(w[p + i]);
        }
        const uint32_t fl = sort_pairs_stable(kk, rr, sz);
        for (int i = 0; i < sz; ++i) {
            recs[p + i] = rr[i];
            if ((fl >> i) & 1u) {
                atomicOr(&flags[(p + i) >> 5], 1u << ((p + i) & 31));
                atomicAdd(&cnt[(p + i) / kPFixChunk], 1u);
            }
        }
    }
}

// ------------------------------------------------------------------ host ---
int sm_count();

cudaError_t launch_packed_prep(Header *h, cudaStream_t s) {
    k_packed_prep<<<1, kMaxRadix, 0, s>>>(h);
    return cudaGetLastError();
}

template <int Q>
static cudaError_t launch_psweep(const uint64_t *in, uint64_t *out, int64_t m, int32_t n, uint64_t *look,
                                 uint64_t *look_next, Header *h, cudaStream_t s) {
    constexpr size_t smem = sizeof(PSmem<Q>);
    static_assert(smem <= 48 * 1024, "within the default dynamic shared memory limit (no opt-in)");
    const unsigned tiles = unsigned((m + kPTile - 1) / kPTile);
    k_psweep<Q><<<tiles, kPThreads, smem, s>>>(in, out, m, n, look, look_next, h);
    return cudaGetLastError();
}

// The four passes: keys (by edge index of an n-point cloud) -> a -> b -> a
// -> b.  look0 must be zeroed (launch_sort_init); every buffer 16-byte aligned.
cudaError_t launch_packed_passes(const uint64_t *keys, int64_t n, uint64_t *a, uint64_t *b, uint64_t *look0,
                                 uint64_t *look1, Header *h, cudaStream_t s, cudaEvent_t *after_pass) {
    const int64_t m = n * (n - 1) / 2;
    if (m <= 0) return cudaSuccess;
    if (n > kPackMaxN) return cudaErrorInvalidValue;
    if (((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) &
         15u) != 0)
        return cudaErrorInvalidValue;
    const int32_t nn = int32_t(n);
    cudaError_t e = launch_psweep<0>(keys, a, m, nn, look0, look1, h, s);
    if (e == cudaSuccess && after_pass) e = cudaEventRecord(after_pass[0], s);
    if (e == cudaSuccess) e = launch_psweep<1>(a, b, m, nn, look1, look0, h, s);
    if (e == cudaSuccess && after_pass) e = cudaEventRecord(after_pass[1], s);
    if (e == cudaSuccess) e = launch_psweep<2>(b, a, m, nn, look0, look1, h, s);
    if (e == cudaSuccess && after_pass) e = cudaEventRecord(after_pass[2], s);
    if (e == cudaSuccess) e = launch_psweep<3>(a, b, m, nn, look1, look0, h, s);
    if (e == cudaSuccess && after_pass) e = cudaEventRecord(after_pass[3], s);
    return e;
}

// The fix-up and its second kernel (see k_pfixup); defer_list: room for
// kPFixChunk / (kPFixCap + 1) + 1 words per chunk (look[1] has kMaxRadix per
// 4096 edges, 32 per chunk).
cudaError_t launch_packed_fixup(const uint64_t *w, int64_t m, int64_t n, const uint64_t *keyidx, uint32_t *recs,
                                uint32_t *flags, uint32_t *cnt, uint64_t *defer_list, Header *h, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    if (n > kPackMaxN || ((reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(recs)) & 15u) != 0)
        return cudaErrorInvalidValue;
    int64_t blocks = (m + kPFixChunk * kPFixWarps - 1) / (kPFixChunk * kPFixWarps);
    const int64_t cap = int64_t(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    k_pfixup<<<unsigned(blocks), 32 * kPFixWarps, 0, s>>>(w, m, n, keyidx, recs, flags, cnt, defer_list, h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pfixup_deferred<<<unsigned(sm_count()), 256, 0, s>>>(w, m, n, keyidx, recs, flags, cnt, defer_list, h);
    return cudaGetLastError();
}

}  // namespace ph0
