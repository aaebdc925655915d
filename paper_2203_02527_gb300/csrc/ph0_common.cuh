// ph0_common.cuh -- shared device-side definitions of libph0 (sm_103a).
//
// Workspace layout, the device status word, bounded waits and small helpers
// used by the kernels of the barcode path (Rawson, Sec. 2; Sec. 4 steps 1-5).
#pragma once

#include <cstddef>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "ph0.h"

namespace ph0 {

// ---------------------------------------------------------------- limits ---
constexpr int64_t kMaxN = 65535;   // vertex ids packed in 16 bits: E < 2^31
// Larger clouds ("wide" records): the value of an edge is its lexicographic
// index e = u(2n-u-1)/2 + v-u-1 instead of (u << 16) | v, and every position,
// count and index a stays below 2^32 while E = n(n-1)/2 < 2^32.
constexpr int64_t kMaxNWide = 92681;
static_assert(kMaxNWide * (kMaxNWide - 1) / 2 < (int64_t(1) << 32), "wide edge indices fit 32 bits");
// Beyond (the whole path only): E < 2^33, so an edge index has 33 bits; its
// bit 32 rides in bit 63 of the record's key, which a squared distance never
// sets (it is >= +0), and every reader of a key's value masks it off with
// kKeyBits.  The sort takes the edges as two halves of fewer than 2^32
// records each, merged; positions read by the reduction stay below
// kMaxScanPos (beyond it the call reports PH0_ETOOBIG).
constexpr int64_t kMaxNHuge = 131071;
static_assert(kMaxNHuge * (kMaxNHuge - 1) / 2 < (int64_t(1) << 33), "edge indices fit 33 bits");
constexpr uint64_t kKeyBits = ~(uint64_t(1) << 63);
constexpr int64_t kSplitEdges = (int64_t(1) << 32) - 4096;  // more edges than this: two halves
constexpr int64_t kMaxScanPos = (int64_t(1) << 32) - 4096;  // a multiple of the de-duplication chunk
constexpr int32_t kMaxD = 1024;
constexpr int kMaxPasses = 8;      // 6 low digit passes + at most 2 top passes
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kLowPasses = 6;      // raw 8-bit digits of key bits 0..47
constexpr int kTopShift = 48;      // the rest, key >> 48, is sorted offset by kmin >> 48
constexpr int kMaxRadix = 512;     // one top pass of up to 9 bits

// The packed sort of the whole path (k_sortp.cu), for clouds of at most
// 32768 points (kPackMaxEdges edges): each edge (u, v) becomes one 64-bit word
//   [63:56] the number of its key's top part (key >> 48) among the values
//           that occur (at most 256 of them), [55:30] key bits 22..47,
//   [29:0]  (u << 15) | v,
// whose order is the order of (key >> 22, u, v), i.e. of (key >> 22, edge
// index); four radix passes of 9, 9, 8 and 8 bits (digit q at word bit
// pack_shift(q)) sort the words, and a fix-up orders each group of equal
// key >> 22 by the whole key, read from the distance kernel's output (key by
// edge index).
constexpr int kPackIdBits = 30;
constexpr int64_t kPackMaxN = 32768;
constexpr int64_t kPackMaxEdges = kPackMaxN * (kPackMaxN - 1) / 2;
constexpr int kPackKeyShift = 22;
constexpr int kPackKeyBits = 26;   // key bits 22..47
constexpr int kPackPasses = 4;
constexpr uint64_t kPackIdMask = (uint64_t(1) << kPackIdBits) - 1;
__host__ __device__ constexpr int pack_shift(int q) { return q == 0 ? 30 : q == 1 ? 39 : q == 2 ? 48 : 56; }
__host__ __device__ constexpr int pack_radix(int q) { return q < 2 ? 512 : 256; }
static_assert(kPackIdBits + kPackKeyBits + 8 == 64 && pack_shift(2) + 8 == pack_shift(3), "word layout");
// the key's digit that is word digit q < 3 (the distance kernel's histograms)
__host__ __device__ __forceinline__ uint32_t pack_key_digit(uint64_t key, int q) {
    return uint32_t(key >> (kPackKeyShift + 9 * q)) & uint32_t(pack_radix(q) - 1);
}
// (u, v) of the edge k places after edge (u, v) in lexicographic order
// (while it exists): past the end of row u (v = n) the next row starts at
// v = u + 2.  Each step of the loop moves to the next row.
__host__ __device__ __forceinline__ void edge_step(uint32_t &u, uint32_t &v, uint32_t n, uint32_t k) {
    v += k;
    while (v >= n && u + 2 < n) {
        ++u;
        v = v - n + u + 1;
    }
}
// The record (u << 16) | v and the edge index of a word.
__host__ __device__ __forceinline__ uint32_t pack_record(uint64_t w) {
    return (uint32_t(w >> 15) & 0x7fffu) << 16 | (uint32_t(w) & 0x7fffu);
}
__host__ __device__ __forceinline__ uint32_t pack_edge(uint64_t w, uint32_t n) {
    const uint32_t u = uint32_t(w >> 15) & 0x7fffu, v = uint32_t(w) & 0x7fffu;
    return u * (2 * n - u - 1) / 2 + (v - u - 1);  // u(2n-u-1) < 2^31 at n <= 32768
}

// Bounded device-side waits: about a second at most, then the kernel records
// PH0_ETIMEOUT in the status word and returns cleanly.
constexpr uint32_t kSpinLimit = 1u << 24;

// Radix sort tile: kSortThreads threads x kSortItems keys.
constexpr int kSortThreads = 256;
#ifndef PH0_SORT_ITEMS
#define PH0_SORT_ITEMS 16
#endif
constexpr int kSortItems = PH0_SORT_ITEMS;
constexpr int kSortTile = kSortThreads * kSortItems;

// Look-back status word: [63:62] flag, [61:0] count.
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kFlagMask = 3ull << 62;
constexpr uint64_t kCountMask = ~kFlagMask;
// Counts and prefixes stay below 2^32, so a status word's high half holds its
// flag alone and its low half its count; an unpublished word is all zero.
constexpr uint32_t kHiAgg = uint32_t(kFlagAgg >> 32), kHiPrefix = uint32_t(kFlagPrefix >> 32);

// The early-terminating path (k_prefix.cu): bins of its key histogram, and
// at most kPrefixClasses classes (consecutive bin ranges) in its partition
// of the edges, which runs as radix slot kClassSlot (digit = class).
constexpr int kPrefixBinBits = 12;
constexpr int kPrefixBins = 1 << kPrefixBinBits;
constexpr int kPrefixClasses = 8;
constexpr int kClassSlot = 8;
// Bin of a key: (key - kmin) >> shift, with shift such that the key range
// [kmin, kmax] spans at most kPrefixBins bins.
__host__ __device__ __forceinline__ int prefix_shift(uint64_t kmin, uint64_t kmax) {
    const uint64_t span = kmax > kmin ? kmax - kmin : 0;
    int bits = 0;
    for (uint64_t x = span; x; x >>= 1) ++bits;
    return bits > kPrefixBinBits ? bits - kPrefixBinBits : 0;
}

// --------------------------------------------------------------- header ---
// Lives at offset 0 of the workspace.  Every counter the kernels share.
struct Header {
    int32_t status;              // ph0_status, first device error wins
    int32_t inf_vertex;          // vertex of the bar that never dies (read with status)
    int32_t sort_passes;
    int32_t key_bits;
    int32_t windows;
    uint32_t inf_xor;            // XOR of 0..n-1 and of every pivot row emitted
    uint64_t kmin;               // min / max key over the keys being sorted
    uint64_t kmax;
    int64_t n_distinct;
    int64_t edges_scanned;
    int64_t candidates;
    int64_t rounds;
    int64_t n_bars;
    unsigned long long dist_tiles;        // distance tiles, and those on the integer path
    unsigned long long dist_tiles_exact_int;
    uint32_t tile_counter[kMaxPasses + 4];
    // grid barrier of the persistent reduction kernel
    uint32_t bar_count;
    uint32_t bar_gen;
    int32_t abort;
    uint32_t npiv;               // pivots claimed so far
    uint32_t nlist[2];           // candidate list lengths (ping-pong)
    int32_t top_bits;            // width of a single top radix pass (8 or 9)
    int32_t fixup_fallback;      // set when the short sort's fix-up meets a long unsorted group
    uint32_t defer_count;        // groups the fix-up left to its second kernel
    int32_t packed;              // the packed sort runs (set once after step 1; k_sortp.cu)
    int64_t sorted_edges;        // edges sorted: m, or the prefix of the early path
    unsigned long long claim_attempts;  // atomic claims of the reduction (grid and tail rounds)
    uint32_t claim_rounds_max;   // most claim rounds in one window
    int32_t classic;             // a packed-sort call whose keys do not pack: the short sort runs
    // class partition of the early path (radix slot kClassSlot): the key
    // bins of its histogram and the classes' bin ranges [bound[c], bound[c+1])
    uint64_t part_kmin;
    int32_t part_shift;
    int32_t part_nc;
    uint32_t part_bound[kPrefixClasses + 1];
    uint32_t hist[kMaxPasses][kMaxRadix];  // digit histogram per radix pass
    // histogram of (key >> kTopShift) mod kMaxRadix, taken with the low ones:
    // when the top part spans less than kMaxRadix values (a single top
    // pass), it is the top digit's histogram rotated by kmin >> kTopShift
    uint32_t hist_top_mod[kMaxRadix];
    // the single top pass on 8-bit digits (k_top_compact): set when at most
    // kRadix values of the top part occur; top_lut numbers them in order
    int32_t top_compact;
    uint32_t pad3;
    uint8_t top_lut[kMaxRadix];
    // the packed sort: digit histograms of its four passes (the first three
    // from the distance kernel, the top one from k_packed_prep) and tile counters
    uint32_t phist[kPackPasses][kMaxRadix];
    uint32_t ptile[kPackPasses];
};

constexpr size_t kHeaderBytes = 32768;
static_assert(sizeof(Header) <= kHeaderBytes, "header too large");

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) {
    return (x + a - 1) / a * a;
}

__host__ __device__ inline int64_t n_edges(int64_t n) { return n * (n - 1) / 2; }

// Candidate list capacity of one reduction window (edges per window).
constexpr int64_t kMaxWindow = int64_t(1) << 26;
// Trace of the reduction: kTraceWindows records of kTraceWords words:
// {pos0, window size, candidates, grid rounds, tail rounds, pivots after,
//  t_begin, t_filtered, t_grid_done, t_tail_done, t_end} (globaltimer, ns).
constexpr int kTraceWindows = 256;
constexpr int kTraceWords = 12;
// Candidate count at or below which one CTA finishes a window in shared memory.
constexpr int kTailCap = 2048;
// Keys per chunk of the de-duplication scan's count mode (one prefix each).
constexpr int kDedupeChunk = 256;
// Byte offsets of every region of the workspace for a cloud of n points in
// dimension d.  Everything is caller-owned device memory; nothing is
// allocated by the library.
struct Layout {
    int64_t n, m, tiles, ktiles;
    size_t hdr, aux_hdr;                 // main header, header of the small sorts
    size_t key[2], val[2], look[2];      // edge records, ping-pong, look-back words
    size_t cpref;                        // de-duplication prefix of every key chunk
    size_t phist;                        // key histogram of the early-terminating path
    size_t dlook;                        // look-back words of the de-duplication scan
    size_t comp, parent, res, cand[2], candr;
    size_t gmap;                         // [n] global root -> local id of the wide reduction's tail
    size_t kill_key[2], kill_val[2], kill_look[2];
    size_t grad;                         // binary64 gradient accumulator [n, d]
    size_t trace;                        // per-window trace records of the reduction
    size_t hib;                          // bit 32 of the edge index per sorted record (above kMaxN points)
    size_t total;

    __host__ __device__ Layout(int64_t n_, int32_t d_) : n(n_) {
        m = n_edges(n);
        tiles = (m + kSortTile - 1) / kSortTile;
        ktiles = (n + kSortTile - 1) / kSortTile;
        int64_t wcap = m < kMaxWindow ? m : kMaxWindow;
        size_t off = 0;
        auto take = [&](size_t bytes) {
            size_t o = off;
            off = align_up(off + bytes, 256);
            return o;
        };
        hdr = take(kHeaderBytes);
        aux_hdr = take(kHeaderBytes);
        key[0] = take(8 * size_t(m));
        key[1] = take(8 * size_t(m));
        // one region for both value buffers: the packed sort uses it as one
        // buffer of m 8-byte words
        val[0] = take(8 * size_t(m) + 256);
        val[1] = val[0] + align_up(4 * size_t(m), 256);
        cpref = take(4 * size_t((m + kDedupeChunk - 1) / kDedupeChunk + 1));
        phist = take(4 * size_t(kPrefixBins));
        look[0] = take(8 * size_t(tiles) * kMaxRadix);
        look[1] = take(8 * size_t(tiles) * kMaxRadix);
        dlook = take(8 * size_t(tiles + 1));
        comp = take(4 * size_t(n));
        parent = take(4 * size_t(n));
        res = take(8 * size_t(n));
        cand[0] = take(4 * size_t(wcap + 1));
        cand[1] = take(4 * size_t(wcap + 1));
        candr = take(8 * size_t(wcap + 1));
        gmap = take(4 * size_t(n));
        kill_key[0] = take(8 * size_t(n));
        kill_key[1] = take(8 * size_t(n));
        kill_val[0] = take(4 * size_t(n));
        kill_val[1] = take(4 * size_t(n));
        kill_look[0] = take(8 * size_t(ktiles) * kMaxRadix);
        kill_look[1] = take(8 * size_t(ktiles) * kMaxRadix);
        grad = take(8 * size_t(n) * size_t(d_ > 0 ? d_ : 1));
        trace = take(sizeof(uint64_t) * kTraceWords * kTraceWindows);
        hib = take(n > kMaxN ? 4 * size_t((m + 31) / 32 + 1) : 0);
        total = off;
    }
};

// First homology (k_h1.cu): at most kH1MaxN points.  A triangle is named by
// the 64-bit key (diameter position << 36) | (u << 24) | (v << 12) | w with
// u < v < w (12 bits per vertex, positions below 2^23 at 4096 points), whose
// order is the triangle order.  kH1ScanItems: elements per CTA of the
// prefix scans (1024 threads x 4); kH1Runs: sorted runs of a column under
// reduction.
constexpr int64_t kH1MaxN = 4096;
constexpr int kH1VertexBits = 12;
constexpr int kH1Threads = 1024;
constexpr int64_t kH1ScanItems = 4 * kH1Threads;
constexpr int kH1Runs = 32;

// The first-homology regions of a workspace, after the dimension-0 layout.
// col_cap bounds a column under reduction, pool_cap the reduced columns kept
// (PH0_ETOOBIG beyond either): the runs of a column live in col_x, col_m
// holds a merge.
struct H1Layout {
    int64_t T, blocks, col_cap, pool_cap;
    size_t cnt, aof, posof, pmat, tcount, tfirst, scan_in, zpref, tpref, bsum, zlist, rlist, head, claims,
        node_key, node_pos, node_next, node_within, own_node, own_off, own_len, col_x, col_m, pool, total;
    H1Layout(int64_t n, size_t base) {
        const int64_t m = n_edges(n);
        T = n * (n - 1) * (n - 2) / 6;
        blocks = (m + kH1ScanItems - 1) / kH1ScanItems;
        // a column holds at most T distinct keys, but a push may add a kept
        // column to it before they cancel; the kept columns together may
        // exceed T (measured: 1.1 T on a perturbed 29-point simplex)
        auto clamp = [](int64_t x, int64_t lo, int64_t hi) { return x < lo ? lo : (x > hi ? hi : x); };
        col_cap = clamp(2 * T, int64_t(1) << 18, int64_t(1) << 23) + 2 * n + 1;
        pool_cap = clamp(8 * T, int64_t(1) << 20, int64_t(1) << 26) + n + 1;
        size_t off = base;
        auto take = [&](size_t bytes) {
            size_t o = off;
            off = align_up(off + bytes, 256);
            return o;
        };
        const size_t M1 = size_t(m + 1);
        cnt = take(256);
        aof = take(4 * M1);
        posof = take(4 * M1);
        pmat = take(4 * size_t(n) * size_t(n));
        tcount = take(4 * M1);
        tfirst = take(4 * M1);
        scan_in = take(8 * M1);
        zpref = take(8 * M1);
        tpref = take(8 * M1);
        bsum = take(8 * size_t(blocks + 1));
        zlist = take(4 * M1);
        rlist = take(4 * M1);
        head = take(4 * M1);
        claims = take(4 * M1);
        node_key = take(8 * M1);
        node_pos = take(4 * M1);
        node_next = take(4 * M1);
        node_within = take(4 * M1);
        own_node = take(4 * M1);
        own_off = take(8 * M1);
        own_len = take(4 * M1);
        col_x = take(8 * size_t(col_cap));
        col_m = take(8 * size_t(col_cap));
        pool = take(8 * size_t(pool_cap));
        total = off;
    }
};

// Arguments of the persistent reduction kernel (steps 4-5).
struct ReduceArgs {
    int64_t n, m;
    const uint32_t *val0, *val1;   // sorted edge records (buffer chosen by the sort plan)
    const Header *sort_h;          // header of the sort (plan), or null: use val0
    uint32_t *comp;                // [n] root of each vertex at the window start
    uint32_t *parent;              // [n] link of each root claimed in this window
    unsigned long long *res;       // [n] claim of each root: (~round << 32) | position
    uint32_t *cand0, *cand1;       // candidate lists (ping-pong)
    unsigned long long *candr;     // [list] roots of each candidate in this round (ru << 32 | rv)
    uint32_t *gmap;                // [n] global root -> local id (wide tail rounds)
    int64_t m_edges;               // n(n-1)/2: bound of the wide records' edge indices
    bool wide;                     // records hold edge indices (n > kMaxN, or forced)
    unsigned long long *kill_key;  // [n] position of each pivot column
    uint32_t *kill_val;            // [n] its pivot row
    Header *h;
    int64_t w0;                    // first window size
    int64_t start;                 // first position to scan: 0, or where an earlier launch on the
                                   // same workspace stopped (its state carried, no re-initialization)
    const uint32_t *hib;           // bit 32 of each record's edge index (records of a merged sort), or null
    const uint32_t *valp;          // the packed sort's records, read instead of val0/val1 when
                                   // h->packed is set and h->fixup_fallback is not; or null
    bool capped;                   // m stops short of the edges: fewer than n-1 pivots is PH0_ETOOBIG
    uint64_t *trace;               // [kTraceWindows][kTraceWords]
    uint32_t spin_limit;           // polls before a grid-barrier wait gives up
};

// What steps 3-5 read after the packed sort (k_sortp.cu): the record
// (u << 16) | v at every sorted position, the keys by edge index (the
// distance kernel's output), and one bit per position marking a new distance
// value.  Null members: no packed sort.
struct PackedRecs {
    const uint32_t *recs;
    const uint64_t *keyidx;
    const uint32_t *flags;
};

// One cloud of a fused small-cloud batch (k_small.cu).
struct SmallTask {
    const float *pts;      // device [n, ld]
    int64_t *fixed;        // device scratch [n * d] int64 (fixed-point coordinates)
    ph0_bar *bars;         // device [n - 1]
    int32_t *status;       // device, two words per task: status, vertex of the infinite bar
    int32_t n, d, ld, pad;
};

template <typename T>
__host__ __device__ inline T *at(void *ws, size_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

// ------------------------------------------------------------ device util ---
__device__ __forceinline__ void set_status(Header *h, int code) {
    atomicCAS(&h->status, 0, code);
}

__device__ __forceinline__ uint64_t ld_volatile(const uint64_t *p) {
    return *reinterpret_cast<const volatile uint64_t *>(p);
}
__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ int32_t ld_volatile(const int32_t *p) {
    return *reinterpret_cast<const volatile int32_t *>(p);
}
__device__ __forceinline__ void st_volatile(uint64_t *p, uint64_t v) {
    *reinterpret_cast<volatile uint64_t *>(p) = v;
}

// Grid-wide barrier with a bounded wait (spin_limit polls).  Returns false
// (in every thread of the CTA) if the kernel must stop.
__device__ __forceinline__ bool grid_barrier(Header *h, int *s_ok, uint32_t spin_limit) {
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
                if (++spins > spin_limit) {
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

// Edge index of (u, v), u < v, in lexicographic order.
__host__ __device__ __forceinline__ int64_t edge_index(int64_t n, int64_t u, int64_t v) {
    return u * (2 * n - u - 1) / 2 + (v - u - 1);
}

// (u, v) of a record value: (u << 16) | v, or (wide) the edge index e < n(n-1)/2.
// The row u of e is the largest r with r(2n-r-1)/2 <= e: the smaller root of
// r^2 - (2n-1) r + 2e = 0, estimated in binary32 (off by at most one at
// n < 2^17) and corrected with exact integer arithmetic.
// (u, v) of the edge with lexicographic index e < n(n-1)/2.
__host__ __device__ __forceinline__ void edge_uv(int64_t e, int64_t n, uint32_t &u, uint32_t &v) {
    const int64_t b = 2 * n - 1;
    const int64_t disc = b * b - 8 * e;  // > 0 for e < n(n-1)/2
#ifdef __CUDA_ARCH__
    const float root = __fsqrt_rn(float(disc));
#else
    const float root = sqrtf(float(disc));  // also correctly rounded
#endif
    int64_t r = int64_t((float(b) - root) * 0.5f);
    r = r < 0 ? 0 : (r > n - 2 ? n - 2 : r);
    if (r * (2 * n - r - 1) / 2 > e) --r;
    if (r > 0 && r * (2 * n - r - 1) / 2 > e) --r;
    if (r + 1 <= n - 2 && (r + 1) * (2 * n - r - 2) / 2 <= e) ++r;
    if (r + 1 <= n - 2 && (r + 1) * (2 * n - r - 2) / 2 <= e) ++r;
    u = uint32_t(r);
    v = uint32_t(e - r * (2 * n - r - 1) / 2 + r + 1);
}
__host__ __device__ __forceinline__ void record_uv(uint32_t vv, bool wide, int64_t n, uint32_t &u, uint32_t &v) {
    if (!wide) {
        u = vv >> 16;
        v = vv & 0xffffu;
        return;
    }
    edge_uv(int64_t(vv), n, u, v);
}
// Bit 32 of the edge index of the record at position p, from the bitmask the
// merge of the two sorted halves writes (null: every index below 2^32).
__host__ __device__ __forceinline__ int64_t index_hi(const uint32_t *hib, int64_t p) {
    return hib ? int64_t((hib[p >> 5] >> (p & 31)) & 1u) << 32 : 0;
}
// (u, v) of the sorted record at position p with value vv.
template <bool WIDE>
__device__ __forceinline__ void rec_uv(uint32_t vv, int64_t p, const uint32_t *hib, int64_t n, uint32_t &u,
                                       uint32_t &v) {
    if constexpr (WIDE) edge_uv(int64_t(vv) | index_hi(hib, p), n, u, v);
    else record_uv(vv, false, n, u, v);
}

// Radix plan.  Bits above the highest bit in which the keys differ are
// constant and not sorted.  The low passes sort raw 8-bit digits of bits
// 0..47, whose histograms can be taken where the keys are produced (before
// the key range is known).  If the keys differ above bit 47, the top part
// T = (key >> 48) - (kmin >> 48) (in key order, since the offset is constant)
// is sorted last: in one pass of up to 9 bits (512 buckets) or in two passes
// of 8 bits; its histograms are taken during the last low pass.
struct Plan {
    uint64_t kmin;
    int low, top, passes, bits;
};
__host__ __device__ __forceinline__ int bitlen64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return x ? 64 - __clzll((long long)x) : 0;
#else
    return x ? 64 - __builtin_clzll(x) : 0;
#endif
}
__host__ __device__ __forceinline__ Plan make_plan(uint64_t kmin, uint64_t kmax, int top_bits = 9) {
    Plan p;
    p.kmin = kmin;
    if (kmax < kmin) kmax = kmin;  // no keys
    const int hi = bitlen64(kmin ^ kmax);
    if (hi <= kTopShift) {
        // at least two low passes when any bit varies: the short sort, which
        // starts at slot 2, then leaves the records in buffer (passes & 1) =
        // 0 where it ran no pass (slot 1 sorts equal bits: a stable no-op)
        const int low = (hi + kRadixBits - 1) / kRadixBits;
        p.low = hi == 0 ? 0 : (low < 2 ? 2 : low);
        p.top = 0;
        p.bits = hi;
    } else {
        const int tb = bitlen64((kmax >> kTopShift) - (kmin >> kTopShift));
        p.low = kLowPasses;
        p.top = tb <= (top_bits == 8 ? 8 : 9) ? 1 : 2;
        p.bits = kTopShift + tb;
    }
    p.passes = p.low + p.top;
    return p;
}
__host__ __device__ __forceinline__ Plan make_plan(const Header *h) {
    return make_plan(h->kmin, h->kmax, h->top_bits);
}

// Built-in tuning (ph0_tuning fields of -1).
constexpr int kDefaultDistSplit16 = 16;
constexpr int kDefaultTopBits = 9;

// Digit of a key in a pass (< 512 in a single top pass, else < 256).
__host__ __device__ __forceinline__ uint32_t digit_of(uint64_t key, const Plan &p, int pass) {
    if (pass < p.low) return uint32_t(key >> (kRadixBits * pass)) & (kRadix - 1);
    const uint32_t t = uint32_t(((key & kKeyBits) >> kTopShift) - (p.kmin >> kTopShift));
    if (p.top == 1) return t;
    return pass == p.low ? (t & (kRadix - 1)) : (t >> kRadixBits);
}

}  // namespace ph0
