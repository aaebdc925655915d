// k_dist.cu -- step 1 of the barcode path: all pairwise squared distances
// (Rawson, Sec. 2: the distance of every pair of points; Sec. 3 notes the
// factor-2 saving from symmetry; Sec. 4 step 1).
//
// One CTA per tile of the upper triangle: a block of BT row points (u) by a
// block of BT column points (v), v-block >= u-block.  The binary32
// coordinates of both blocks are staged in shared memory, dimension-major
// (as binary64, or as fixed-point integers, see below), so that a warp reads
// 32 consecutive v (no bank conflicts) and the u coordinate is a broadcast.
// A warp writes 32 consecutive edges of one row u, so the key (8 B) and val
// (4 B) stores are coalesced.
//
// The arithmetic: when, in every dimension, the tile's coordinates are exact
// integers times a common power of two with magnitudes below 2^52 (checked
// per tile), the rounded binary64 sequence is computed bit-identically from
// those integers (emu64.cuh): each square RN(t*t) exactly with integer
// operations and the running sum on the binary64 adder (the "mixed" form),
// or all of it with integer operations; the binary64 units of this GPU run
// at 1/64 of the integer rate, so the squares go to the integer units and
// only the d-1 additions per edge to the binary64 adder.  Otherwise the
// whole tile uses the literal binary64 sequence.
//
// Fused: the histograms of the six low 8-bit key digits (the low radix
// passes; for the packed sort instead its three key digits, bits 22..47 in
// 9, 9 and 8 bits) and of the top part of the key modulo 512, the min and max key
// (the sort's bit range), and the finiteness check of the input.
#include "emu64.cuh"
#include "ph0_common.cuh"

namespace ph0 {

constexpr int kDistThreads = 256;
// On integer-path tiles, rows i with (i % 16) < split16 form the squares with
// integers and take the running sums on the binary64 units (16 binary64
// operations per edge at d = 16 instead of 47); the other rows are computed
// all in integers.  The two pipes run concurrently; all rows on the mixed
// form measured fastest on GB300 for d = 16 (24 ms vs 42 ms all-integer and
// 50 ms binary64-only for 537M edges), and the autotuner picks the split per
// dimension.  All forms give identical bits.  The kernel is also compiled
// for the common dimensions and tile edges (D, BT) with the dimension loop
// unrolled: 15.9 ms instead of 19.4 ms at d = 16 on the same edges.

// Squared distance of one edge: s = 0; t = x_v - x_u; s = s + t*t per
// dimension, each operation rounded to nearest (no contraction).
__device__ __forceinline__ double sq_dist_f64(const double *__restrict__ su,
                                              const double *__restrict__ sv,
                                              int d, int bt, int i, int j) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = __dsub_rn(sv[k * bt + j], su[k * bt + i]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// Linear tile id -> (bi, bj), bi <= bj < T, row-major over the upper triangle.
__device__ __forceinline__ void tile_coords(int64_t lin, int64_t T, int64_t &bi, int64_t &bj) {
    // start(bi) = bi*T - bi*(bi-1)/2 ; solve start(bi) <= lin < start(bi+1)
    double tt = double(2 * T + 1);
    int64_t r = int64_t((tt - sqrt(tt * tt - 8.0 * double(lin))) / 2.0);
    if (r < 0) r = 0;
    if (r > T - 1) r = T - 1;
    auto start = [T](int64_t b) { return b * T - b * (b - 1) / 2; };
    while (r > 0 && start(r) > lin) --r;
    while (r < T - 1 && start(r + 1) <= lin) ++r;
    bi = r;
    bj = r + (lin - start(r));
}

// D, BT > 0: the instance for dimension D and tile edge BT (the d and bt
// arguments equal them); 0: any.
template <int D, int BT>
__global__ void __launch_bounds__(kDistThreads)
k_dist(const float *__restrict__ pts, int n, int d, int64_t ld, int bt, int hw16,
       uint64_t *__restrict__ key, uint32_t *__restrict__ val, Header *__restrict__ h,
       const int32_t *gate, int wide, int packed) {
    if (gate && ld_volatile(gate) == 0) return;  // a gated run (the sort's fallback) that is not needed
    if constexpr (D > 0) {
        d = D;
        bt = BT;
    }
    // [d][bt] u block, then [d][bt] v block: binary64 values, or int64 fixed
    // point in units of 2^g[k] on the integer path; then g[d], lo[d], hi[d]
    extern __shared__ double s_coord[];
    __shared__ uint32_t s_hist[kLowPasses][kRadix];  // packed: [3][512] digits of key bits 22..47
    static_assert(kLowPasses * kRadix == 3 * kMaxRadix, "both histogram sets fit one array");
    uint32_t *s_flat = &s_hist[0][0];
    __shared__ uint32_t s_top[kMaxRadix];  // (key >> kTopShift) mod kMaxRadix
    __shared__ uint64_t s_min[kDistThreads / 32], s_max[kDistThreads / 32];
    __shared__ int s_fixed;

    const int64_t T = (n + bt - 1) / bt;
    int64_t bi, bj;
    tile_coords(blockIdx.x, T, bi, bj);
    const int u0 = int(bi) * bt, v0 = int(bj) * bt;
    double *su = s_coord;
    double *sv = s_coord + size_t(d) * bt;
    int64_t *xu = reinterpret_cast<int64_t *>(su);
    int64_t *xv = reinterpret_cast<int64_t *>(sv);
    int32_t *s_g = reinterpret_cast<int32_t *>(s_coord + size_t(2) * d * bt);
    int32_t *s_lo = s_g + d;
    int32_t *s_hi = s_lo + d;
    uint32_t *s_narrow = reinterpret_cast<uint32_t *>(s_hi + d);  // [(d+31)/32] span <= 31 bits
    uint32_t *s_narrow30 = s_narrow + (d + 31) / 32;                // [(d+31)/32] span <= 30 bits

    for (int b = threadIdx.x; b < kLowPasses * kRadix; b += blockDim.x) (&s_hist[0][0])[b] = 0;
    for (int b = threadIdx.x; b < kMaxRadix; b += blockDim.x) s_top[b] = 0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        s_lo[k] = 1 << 30;
        s_hi[k] = -(1 << 30);
    }
    __syncthreads();
    // pass 1: finiteness and, per dimension, the span of set bits
    bool bad = false;
    for (int idx = threadIdx.x; idx < 2 * bt * d; idx += blockDim.x) {
        const int side = idx / (bt * d), r = idx % (bt * d);
        const int p = r / d, k = r % d;
        const int row = (side ? v0 : u0) + p;
        const float x = row < n ? pts[int64_t(row) * ld + k] : 0.0f;
        const uint32_t b = __float_as_uint(x);
        if ((b & 0x7f800000u) == 0x7f800000u) {
            bad = true;
        } else if (b & 0x7fffffffu) {
            int32_t lo, hi;
            emu::bit_range_f32(b, lo, hi);
            atomicMin(s_lo + k, lo);
            atomicMax(s_hi + k, hi);
        }
    }
    if (bad) set_status(h, PH0_ENONFINITE);
    __syncthreads();
    if (threadIdx.x == 0) {
        int fixed = 1;
        for (int w = 0; w < (d + 31) / 32; ++w) s_narrow[w] = s_narrow30[w] = 0;
        for (int k = 0; k < d; ++k) {
            const bool zero = s_lo[k] == (1 << 30);
            s_g[k] = zero ? 0 : s_lo[k];
            const int span = zero ? 0 : s_hi[k] + 1 - s_lo[k];
            if (span > 52) fixed = 0;
            if (span <= 31) s_narrow[k >> 5] |= 1u << (k & 31);    // |X| < 2^31: 32-bit squares
            if (span <= 30) s_narrow30[k >> 5] |= 1u << (k & 31);  // |X| < 2^30: 32-bit differences
        }
        s_fixed = fixed;
        atomicAdd(&h->dist_tiles, 1ull);
        if (fixed) atomicAdd(&h->dist_tiles_exact_int, 1ull);
    }
    __syncthreads();
    const bool fixed = s_fixed != 0;
    // pass 2: stage the coordinates, dimension-major
    for (int idx = threadIdx.x; idx < bt * d; idx += blockDim.x) {
        const int p = idx / d, k = idx % d;
        const float a = (u0 + p < n) ? pts[int64_t(u0 + p) * ld + k] : 0.0f;
        const float b = (v0 + p < n) ? pts[int64_t(v0 + p) * ld + k] : 0.0f;
        if (fixed) {
            xu[k * bt + p] = emu::to_fixed(__float_as_uint(a), s_g[k]);
            xv[k * bt + p] = emu::to_fixed(__float_as_uint(b), s_g[k]);
        } else {
            su[k * bt + p] = double(a);
            sv[k * bt + p] = double(b);
        }
    }
    __syncthreads();

    uint64_t kmin = ~0ull, kmax = 0;
    const int j = threadIdx.x % bt;                // column within the tile
    const int rows_per_pass = blockDim.x / bt;     // bt divides blockDim (bt <= 128)
    const int v = v0 + j;
    // the record of edge (u, v): key, value, histograms, key range
    auto emit = [&](int u, uint64_t kb) {
        const int64_t e = edge_index(n, u, v);
        // wide: the value is the edge index, whose bit 32 (above 92,682
        // points) rides in the key's bit 63, never set by a squared distance
        key[e] = wide ? kb | (uint64_t(e >> 32) << 63) : kb;
        val[e] = wide ? uint32_t(e) : (uint32_t(u) << 16) | uint32_t(v);
        if (packed) {
#pragma unroll
            for (int q = 0; q < kPackPasses - 1; ++q) atomicAdd(&s_flat[q * kMaxRadix + pack_key_digit(kb, q)], 1u);
        } else {
#pragma unroll
            for (int q = 0; q < kLowPasses; ++q) atomicAdd(&s_hist[q][(kb >> (8 * q)) & (kRadix - 1)], 1u);
        }
        atomicAdd(&s_top[(kb >> kTopShift) & (kMaxRadix - 1)], 1u);
        kmin = kb < kmin ? kb : kmin;
        kmax = kb > kmax ? kb : kmax;
    };
    bool unrolled = false;
    if constexpr (D > 0) {
        if (fixed && hw16 >= 16) {  // every row on the mixed form
            unrolled = true;
            const uint32_t nw = s_narrow30[0];
            for (int i = threadIdx.x / BT; i < BT; i += kDistThreads / BT) {
                const int u = u0 + i;
                if (u < v && v < n) emit(u, emu::sq_dist_mixed_ct<D, BT>(xu + i, xv + j, s_g, nw));
            }
        }
    }
    if (!unrolled) {
        for (int i = threadIdx.x / bt; i < bt; i += rows_per_pass) {
            const int u = u0 + i;
            if (u < v && v < n) {
                uint64_t kb;
                if (!fixed) kb = uint64_t(__double_as_longlong(sq_dist_f64(su, sv, d, bt, i, j)));
                else if ((i & 15) < hw16) kb = emu::sq_dist_mixed(xu + i, xv + j, s_g, d, bt, bt, s_narrow30);
                else kb = emu::sq_dist_fixed(xu + i, xv + j, s_g, d, bt, bt, s_narrow);
                emit(u, kb);
            }
        }
    }
    // block min / max of the keys
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
        for (int w = 1; w < int(blockDim.x >> 5); ++w) {
            kmin = s_min[w] < kmin ? s_min[w] : kmin;
            kmax = s_max[w] > kmax ? s_max[w] : kmax;
        }
        if (kmin != ~0ull) {
            atomicMin((unsigned long long *)&h->kmin, (unsigned long long)kmin);
            atomicMax((unsigned long long *)&h->kmax, (unsigned long long)kmax);
        }
    }
    for (int b = threadIdx.x; b < kLowPasses * kRadix; b += blockDim.x) {
        const uint32_t c = s_flat[b];
        if (!c) continue;
        if (packed) atomicAdd(&h->phist[b / kMaxRadix][b % kMaxRadix], c);
        else atomicAdd(&h->hist[b / kRadix][b % kRadix], c);
    }
    for (int b = threadIdx.x; b < kMaxRadix; b += blockDim.x)
        if (s_top[b]) atomicAdd(&h->hist_top_mod[b], s_top[b]);
}

// Shared memory of a tile: two staged blocks plus g, lo, hi per dimension.
size_t dist_smem(int bt, int d) {
    return size_t(2) * bt * d * sizeof(double) + size_t(3) * d * sizeof(int32_t) +
           size_t(2) * ((d + 31) / 32) * sizeof(uint32_t);
}

// Tile edge for dimension d: the staged blocks must fit in shared memory.
int dist_tile(int d, int want) {
    int bt = (want == 32 || want == 64) ? want : 128;
    while (bt > 8 && dist_smem(bt, d) > 160 * 1024) bt /= 2;
    return bt;
}

cudaError_t launch_dist(const float *pts, int64_t n, int32_t d, int64_t ld, uint64_t *key,
                        uint32_t *val, Header *h, cudaStream_t s, int split16, int tile,
                        const int32_t *gate, bool wide, bool packed) {
    if (n < 2) return cudaSuccess;
    const int bt = dist_tile(d, tile);
    const size_t smem = dist_smem(bt, d);
    if (smem > 160 * 1024) return cudaErrorInvalidValue;
    const int64_t T = (n + bt - 1) / bt;
    const int64_t tiles = T * (T + 1) / 2;
    const int hw16 = (split16 >= 0 && split16 <= 16) ? split16 : kDefaultDistSplit16;
    auto go = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        kernel<<<unsigned(tiles), kDistThreads, smem, s>>>(pts, int(n), int(d), ld, bt, hw16, key, val, h, gate,
                                                           wide ? 1 : 0, packed ? 1 : 0);
        return cudaGetLastError();
    };
#define PH0_DIST_CASE(DD)                                       \
    case DD:                                                    \
        if (bt == 128) return go(k_dist<DD, 128>);              \
        if (bt == 64) return go(k_dist<DD, 64>);                \
        break;
    switch (d) {
        PH0_DIST_CASE(2)
        PH0_DIST_CASE(3)
        PH0_DIST_CASE(8)
        PH0_DIST_CASE(16)
        PH0_DIST_CASE(32)
        default: break;
    }
#undef PH0_DIST_CASE
    return go(k_dist<0, 0>);
}

}  // namespace ph0
