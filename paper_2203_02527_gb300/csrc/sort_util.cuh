// sort_util.cuh -- device helpers shared by the radix sorts (k_sort.cu,
// k_sortp.cu): a block-wide exclusive scan, bulk copies global -> shared
// completed on an mbarrier, and the decoupled look-back over per-tile status
// words (Rawson, Sec. 4 step 2: the sort of the edges).
#pragma once
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

// ---- bulk (TMA) copies global -> shared with an mbarrier -------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared, 16-byte aligned addresses, size a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Per-thread asynchronous copies global -> shared (the source only needs the
// alignment of the copy size): a full tile whose rows are not 16-byte aligned.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Bounded wait for phase `parity` of the barrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity) {
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Decoupled look-back for one digit (column `col` of the per-tile status
// words, stride kMaxRadix): the sum of the counts of all tiles before `tile`
// (tile 0's PREFIX also holds the digit's global start).  The PREFIX of a
// recent predecessor is usually close, so kLookWindow predecessors are read
// at once and folded in order (4 measured fastest on GB300: 8-bit passes
// 3.6-3.8 ms and the 9-bit top pass 4.7-4.8 ms at 537M keys, against
// 3.8 and 5.0 ms with 16 and slower still with 2 or 32); waits on
// unpublished words are bounded.  Counts and prefixes stay below 2^32, so a
// word's low half is its count and its high half its flag alone, and an
// unpublished word is all zero.
#ifndef PH0_LOOK_WINDOW
#define PH0_LOOK_WINDOW 4
#endif
constexpr int kLookWindow = PH0_LOOK_WINDOW;
__device__ __forceinline__ uint32_t lookback_window(const uint64_t *col, int64_t tile, Header *h) {
    uint32_t excl = 0;
    int64_t t = tile - 1;  // next predecessor to fold
    uint32_t spins = 0;
    while (t >= 0) {
        uint32_t lo[kLookWindow], hi[kLookWindow];
#pragma unroll
        for (int q = 0; q < kLookWindow; ++q) {
            const uint64_t w = t - q >= 0 ? ld_volatile(col + (t - q) * kMaxRadix) : 0;
            lo[q] = uint32_t(w);
            hi[q] = uint32_t(w >> 32);
        }
        // fold AGG words up to the first PREFIX (folded too) or unpublished
        // word (count 0); past tile 0 nothing is reached, tile 0 being PREFIX
        bool live = true, done = false;
        int folded = 0;
#pragma unroll
        for (int q = 0; q < kLookWindow; ++q) {
            if (live) {
                excl += lo[q];
                done = hi[q] == kHiPrefix;
                live = hi[q] == kHiAgg;
                folded += live;
            }
        }
        if (done) break;
        t -= folded;
        if (!live) {  // an unpublished word: wait on it, then take a fresh window
            bool gave_up = false;
            while ((ld_volatile(col + t * kMaxRadix) & kFlagMask) == 0) {
                if (++spins > kSpinLimit || ld_volatile(&h->status) != 0) {
                    set_status(h, PH0_ETIMEOUT);
                    gave_up = true;
                    break;
                }
                __nanosleep(spins < 8 ? 32 : 128);
            }
            if (gave_up) break;
        }
    }
    return excl;
}

}  // namespace ph0
