// Host check of the radix sort's digit plan (paper_2203_02527_gb300/csrc/
// ph0_common.cuh: make_plan, digit_of), compiled by nvcc for the host only.
// For key ranges of many widths it checks that the low slots cover key bits
// 0 .. min(hi, kTopShift) - 1 exactly once, that every digit is below
// its pass's radix, and that a stable LSD counting sort of random keys in the
// range by the plan's digits, in pass order, equals a comparison sort of
// (key, original index).  Usage: sort_plan_check <seed> ; prints
// "cases failures".
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <utility>
#include <vector>

#include "ph0_common.cuh"

using namespace ph0;

// The radix of a pass: 8-bit low digits; a single top pass of up to 9 bits
// unless top_bits is 8; two top passes of at most 8 bits each.
static int radix_of(const Plan &p, int pass, int top_bits) {
    if (pass < p.low) return kRadix;
    return (p.top == 1 && top_bits != 8) ? kMaxRadix : kRadix;
}

static bool check(uint64_t kmin, uint64_t kmax, int top_bits, std::mt19937_64 &rng) {
    const Plan p = make_plan(kmin, kmax, top_bits);
    const int hi = bitlen64(kmin ^ kmax);
    // coverage of the low bits
    uint64_t covered = 0;
    for (int q = 0; q < p.low; ++q) {
        for (int i = kRadixBits * q; i < kRadixBits * (q + 1); ++i) {
            if (covered >> i & 1) return false;  // covered twice
            covered |= 1ull << i;
        }
    }
    const int want = hi < kTopShift ? hi : kTopShift;
    const uint64_t mask = want >= 64 ? ~0ull : ((1ull << want) - 1);
    if ((covered & mask) != mask) return false;
    if (p.top == 0 && hi > kTopShift) return false;
    if (p.top > 0 && p.low != kLowPasses) return false;
    if (p.passes != p.low + p.top || p.passes > kMaxPasses) return false;
    // never a single pass: the short sort (from slot 2) relies on it
    if (p.passes == 1) return false;
    // random keys in [kmin, kmax], both ends included
    const int n = 3000;
    std::vector<std::pair<uint64_t, uint32_t>> rec(n);
    std::uniform_int_distribution<uint64_t> U(kmin, kmax);
    for (int i = 0; i < n; ++i) rec[i] = {i < 2 ? (i ? kmax : kmin) : U(rng), uint32_t(i)};
    std::vector<std::pair<uint64_t, uint32_t>> a = rec, b(n);
    for (int pass = 0; pass < p.passes; ++pass) {
        const int R = radix_of(p, pass, top_bits);
        std::vector<uint32_t> cnt(R + 1, 0);
        for (const auto &r : a) {
            const uint32_t dgt = digit_of(r.first, p, pass);
            if (dgt >= uint32_t(R)) return false;
            ++cnt[dgt + 1];
        }
        for (int i = 0; i < R; ++i) cnt[i + 1] += cnt[i];
        for (const auto &r : a) b[cnt[digit_of(r.first, p, pass)]++] = r;
        a.swap(b);
    }
    std::vector<std::pair<uint64_t, uint32_t>> ref = rec;
    std::sort(ref.begin(), ref.end());
    return a == ref;
}

int main(int argc, char **argv) {
    std::mt19937_64 rng(argc > 1 ? std::strtoull(argv[1], nullptr, 10) : 1);
    int cases = 0, bad = 0;
    // squared distances as doubles: ranges of every width, from one binade
    // fraction up to all of [0, 2^1023]
    const double lows[] = {0.0, 1e-300, 1e-30, 1e-9, 1e-4, 0.5, 1.0, 3.0, 1e10};
    const double spans[] = {0.0, 1e-12, 1e-6, 0.01, 1.0, 2.0, 10.0, 1e3, 1e9, 1e30, 1e300};
    for (double lo : lows)
        for (double sp : spans)
            for (int tb : {8, 9}) {
                const double hi_d = lo + sp * (lo > 0 ? lo : 1.0);
                uint64_t kmin, kmax;
                std::memcpy(&kmin, &lo, 8);
                std::memcpy(&kmax, &hi_d, 8);
                if (kmax < kmin) std::swap(kmin, kmax);
                ++cases;
                if (!check(kmin, kmax, tb, rng)) {
                    ++bad;
                    std::fprintf(stderr, "fail kmin=%016llx kmax=%016llx top_bits=%d\n",
                                 (unsigned long long)kmin, (unsigned long long)kmax, tb);
                }
            }
    // raw ranges of every bit width, up to the largest key value (63 bits:
    // bit 63 of a record's key word carries an edge-index bit and is masked)
    for (int w = 0; w <= 63; ++w)
        for (int tb : {8, 9}) {
            const uint64_t kmin = rng() >> 2;
            const uint64_t span = w == 0 ? 0 : (rng() >> (64 - w)) | (1ull << (w - 1));
            const uint64_t kmax = kmin + span > kKeyBits ? kKeyBits : kmin + span;
            ++cases;
            if (!check(kmin, kmax, tb, rng)) {
                ++bad;
                std::fprintf(stderr, "fail w=%d top_bits=%d\n", w, tb);
            }
        }
    std::printf("%d %d\n", cases, bad);
    return bad ? 1 : 0;
}
