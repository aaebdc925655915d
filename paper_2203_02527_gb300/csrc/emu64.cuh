// emu64.cuh -- the binary64 squared distance of step 1 computed with integer
// arithmetic, bit-identical to the rounded sequence
//     s = 0;  for k: t = RN(x_v[k] - x_u[k]);  s = RN(s + RN(t * t))
// (RN = IEEE round to nearest-even in binary64), for binary32 inputs.
//
// Why: the binary64 pipe of this GPU issues about 2 operations per SM per
// clock, 1/64 of its 32-bit integer rate, so the literal sequence is bound
// by it.  Exactness of the emulation:
//   * coordinates of dimension k in a tile are exact integers X times 2^g_k
//     (g_k = lowest set bit over the tile's coordinates); when every |X| is
//     below 2^52 the difference T = X_v - X_u has at most 53 bits, so t is
//     exact in binary64 (the caller checks this per tile and otherwise uses
//     the binary64 units);
//   * every other value is held as (m, e): value = m * 2^(e-63) with m in
//     [2^63, 2^64), i.e. a 64-bit significand whose lowest bit may carry a
//     sticky bit; rounding to 53 bits looks at bit 10 (round) and bits 9..0
//     (sticky) and is nearest-even; products and sums are formed exactly
//     (128-bit square, aligned 64-bit add with the shifted-out bits folded
//     into the sticky bit, which is safe because an operand's bits 10..0 are
//     zero after rounding).
// All intermediate values of the sequence are normal binary64 numbers for
// binary32 inputs (squares >= 2^-298, sums <= 2^262), so rounding to 53 bits
// is IEEE rounding.  Host and device share these functions.
#pragma once

#include <cstdint>

namespace ph0 {
namespace emu {

struct F53 {
    uint64_t m;  // 0 for zero, else in [2^63, 2^64) with bits 10..0 zero
    int32_t e;   // value = m * 2^(e - 63); zero carries kZeroExp
};

// Exponent of zero: far below any nonzero value, so that aligning zero to a
// nonzero operand shifts it out entirely (no branch for zero operands).
constexpr int32_t kZeroExp = -(1 << 20);

__host__ __device__ __forceinline__ int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Round a significand with bit 63 set (bit 0 may hold a sticky bit) to 53
// bits, nearest-even, in place (the round and sticky bits are in the low
// word).  Branch-free.
__host__ __device__ __forceinline__ F53 round53(uint64_t m, int32_t e) {
    const uint32_t lo = uint32_t(m);
    const uint32_t up = (lo >> 10) & (((lo & 0x3ffu) != 0) | (lo >> 11)) & 1u;
    const uint64_t t = m + (uint64_t(up) << 11);
    const bool over = t < m;  // carried out of bit 63: the value is 2^64
    return F53{over ? (uint64_t(1) << 63) : (t & ~uint64_t(0x7ff)), e + int32_t(over)};
}

// RN(t*t) for t = a * 2^g, 0 <= a < 2^53.  Branch-free; a = 0 gives zero.
__host__ __device__ __forceinline__ F53 square53(uint64_t a, int32_t g) {
    const int lz = clz64(a | 1u);
    const uint64_t an = a << lz;
    const uint64_t hi = mulhi64(an, an), lo = an * an;
    const int32_t ea = 63 - lz + g;  // floor(log2 t)
    const uint32_t top = uint32_t(hi >> 63);
    // significand with bit 63 set: hi, or hi:lo shifted left by one
    const uint64_t m = top ? (hi | uint64_t(lo != 0))
                           : ((hi << 1) | (lo >> 63) | uint64_t((lo << 1) != 0));
    F53 r = round53(m, 2 * ea + int32_t(top));
    if (a == 0) r = F53{0, kZeroExp};
    return r;
}

// RN(t*t) for t = a * 2^g with a < 2^32 (a 32x32 -> 64-bit product, exact).
__host__ __device__ __forceinline__ F53 square53_narrow(uint32_t a, int32_t g) {
    const uint64_t p = uint64_t(a) * a;
    const int lz = clz64(p | 1u);
    F53 r = round53(p << lz, 63 - lz + 2 * g);
    if (a == 0) r = F53{0, kZeroExp};
    return r;
}

// RN(x + y) for non-negative x, y.  Branch-free (selects only).
__host__ __device__ __forceinline__ F53 add53(F53 x, F53 y) {
    const bool sw = x.e < y.e;
    const uint64_t bm = sw ? y.m : x.m, sm = sw ? x.m : y.m;
    const int32_t be = sw ? y.e : x.e, se = sw ? x.e : y.e;
    const int32_t d = be - se;
    const int dd = d < 63 ? d : 63;
    // sm >> d with the shifted-out bits folded into bit 0
    const uint64_t lost = (sm << 1) << (63 - dd);  // bits below the shift (none when dd = 0)
    uint64_t al = (sm >> dd) | uint64_t(lost != 0);
    if (d >= 64) al = uint64_t(sm != 0);
    uint64_t s = bm + al;
    const uint32_t carry = s < bm;
    s = carry ? ((s >> 1) | (s & 1u) | (uint64_t(1) << 63)) : s;
    F53 r = round53(s, be + int32_t(carry));
    if (bm == 0) r = F53{0, kZeroExp};  // both zero
    return r;
}

// binary64 bit pattern of a value (normal range).
__host__ __device__ __forceinline__ uint64_t to_bits(F53 s) {
    if (s.m == 0) return 0;
    return (uint64_t(s.e + 1023) << 52) | ((s.m >> 11) & ((uint64_t(1) << 52) - 1));
}

// Exact split of a binary32 value: x = sign * mant * 2^exp, mant < 2^24.
// Returns false for NaN / Inf.  Zero gives mant = 0.
__host__ __device__ __forceinline__ bool split_f32(uint32_t bits, int32_t &mant, int32_t &exp) {
    const uint32_t be = (bits >> 23) & 0xffu;
    const uint32_t fr = bits & 0x7fffffu;
    if (be == 0xffu) return false;
    const int32_t m = be ? int32_t(fr | 0x800000u) : int32_t(fr);
    exp = be ? int32_t(be) - 150 : -149;
    mant = (bits >> 31) ? -m : m;
    return true;
}

// Lowest set bit exponent and floor(log2|x|) of a nonzero binary32 value.
__host__ __device__ __forceinline__ void bit_range_f32(uint32_t bits, int32_t &lo, int32_t &hi) {
    int32_t m, e;
    split_f32(bits, m, e);
    const uint32_t a = uint32_t(m < 0 ? -m : m);
#ifdef __CUDA_ARCH__
    lo = e + (__ffs(int(a)) - 1);
    hi = e + 31 - __clz(int(a));
#else
    lo = e + __builtin_ctz(a);
    hi = e + 31 - __builtin_clz(a);
#endif
}

// The integer X with x = X * 2^g (requires g <= lowest set bit of x and
// |x| < 2^(g+63)).
__host__ __device__ __forceinline__ int64_t to_fixed(uint32_t bits, int32_t g) {
    int32_t m, e;
    split_f32(bits, m, e);
    if (m == 0) return 0;
    const int32_t sh = e - g;
    return sh >= 0 ? int64_t(m) * (int64_t(1) << sh) : int64_t(m) / (int64_t(1) << -sh);
}

// Squared distance from fixed-point coordinates of one edge (X[k] in units of
// 2^g[k]); every |X| < 2^52.  Dimensions whose bit `k` is set in `narrow`
// (coordinates below 2^31 in magnitude) use the 32-bit square.
__host__ __device__ __forceinline__ uint64_t sq_dist_fixed(const int64_t *xu, const int64_t *xv,
                                                           const int32_t *g, int d, int su, int sv,
                                                           const uint32_t *narrow = nullptr) {
    F53 s{0, kZeroExp};
    for (int k = 0; k < d; ++k) {
        const int64_t t = xv[k * sv] - xu[k * su];
        const uint64_t a = uint64_t(t < 0 ? -t : t);
        F53 p;
        if (narrow && ((narrow[k >> 5] >> (k & 31)) & 1u)) p = square53_narrow(uint32_t(a), g[k]);
        else p = square53(a, g[k]);
        s = add53(s, p);
    }
    return to_bits(s);
}

// binary64 value of an F53 (normal range).
__host__ __device__ __forceinline__ double to_double(F53 s) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)to_bits(s));
#else
    const uint64_t b = to_bits(s);
    double x;
    __builtin_memcpy(&x, &b, 8);
    return x;
#endif
}

// binary64 bit pattern of RN(t*t) for t = a * 2^g with 0 <= a < 2^31: the
// exact square has at most 62 bits; after normalizing it to bit 63, adding
// the rounding increment to the 53-bit significand lets a carry flow into the
// exponent field (bits = (exponent - 1) << 52 plus the significand with its
// leading bit), so no overflow case is needed.
__host__ __device__ __forceinline__ uint64_t square_bits_narrow(uint32_t a, int32_t g) {
    const uint64_t p = uint64_t(a) * a;
    const int lz = clz64(p | 1u);
    const uint64_t pn = p << lz;
    const uint32_t lo = uint32_t(pn);
    const uint32_t up = (lo >> 10) & (((lo & 0x3ffu) != 0) | (lo >> 11)) & 1u;
    const uint64_t bits = (uint64_t(int64_t(63 - lz + 2 * g + 1023 - 1)) << 52) + ((pn >> 11) + up);
    return a ? bits : 0;
}

__host__ __device__ __forceinline__ double bits_to_double(uint64_t b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    __builtin_memcpy(&x, &b, 8);
    return x;
#endif
}

// RN(t*t) as a binary64 value for t = xv - xu (fixed point in units of
// 2^g); narrow: every |X| of the dimension is below 2^30, so t fits a 32-bit
// signed difference of the low words.
__host__ __device__ __forceinline__ double square_value(int64_t xu, int64_t xv, int32_t g, bool narrow) {
    if (narrow) {
        const int32_t t = int32_t(uint32_t(xv)) - int32_t(uint32_t(xu));
        return bits_to_double(square_bits_narrow(uint32_t(t < 0 ? -t : t), g));
    }
    const int64_t t = xv - xu;
    return to_double(square53(uint64_t(t < 0 ? -t : t), g));
}

// RN(s + p) by the binary64 adder.
__host__ __device__ __forceinline__ double add_rn(double s, double p) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(s, p);
#else
    volatile double sum = s + p;
    return sum;
#endif
}

__host__ __device__ __forceinline__ uint64_t double_bits(double s) {
#ifdef __CUDA_ARCH__
    return uint64_t(__double_as_longlong(s));
#else
    uint64_t b;
    __builtin_memcpy(&b, &s, 8);
    return b;
#endif
}

// The same squared distance with the squares RN(t*t) formed exactly with
// integers and the running sum s = RN(s + p) taken by the binary64 adder
// (16 binary64 operations per edge at d = 16 instead of 47).  `narrow` bit k:
// dimension k takes the 32-bit square (see square_value).
__host__ __device__ __forceinline__ uint64_t sq_dist_mixed(const int64_t *xu, const int64_t *xv,
                                                           const int32_t *g, int d, int su, int sv,
                                                           const uint32_t *narrow = nullptr) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const bool nk = narrow && ((narrow[k >> 5] >> (k & 31)) & 1u);
        const double p = square_value(xu[k * su], xv[k * sv], g[k], nk);
        s = k == 0 ? p : add_rn(s, p);  // 0 + p is exact
    }
    return double_bits(s);
}

// sq_dist_mixed for a dimension D <= 32 and strides S known at compile time
// (the dimension loop unrolled, the narrow bits in one word).
template <int D, int S>
__host__ __device__ __forceinline__ uint64_t sq_dist_mixed_ct(const int64_t *xu, const int64_t *xv,
                                                              const int32_t *g, uint32_t narrow) {
    static_assert(D >= 1 && D <= 32, "one word of narrow bits");
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const double p = square_value(xu[k * S], xv[k * S], g[k], (narrow >> k) & 1u);
        s = k == 0 ? p : add_rn(s, p);
    }
    return double_bits(s);
}

}  // namespace emu
}  // namespace ph0
