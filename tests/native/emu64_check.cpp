// Host check of the integer emulation of the binary64 squared distance
// (paper_2203_02527_gb300/csrc/emu64.cuh) against the host's own IEEE binary64
// arithmetic (one rounded subtraction, product and sum per dimension).
// Usage: emu64_check <seed> <tiles> ; prints "edges mismatches skipped_tiles".
#define __host__
#define __device__
#define __forceinline__ inline
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "../../paper_2203_02527_gb300/csrc/emu64.cuh"

using namespace ph0::emu;

static double ref_d2(const float *u, const float *v, int d) {
    volatile double s = 0.0;
    for (int k = 0; k < d; ++k) {
        volatile double t = (double)v[k] - (double)u[k];
        volatile double p = t * t;
        s = s + p;
    }
    return s;
}

static uint32_t fbits(float x) { uint32_t b; std::memcpy(&b, &x, 4); return b; }

int main(int argc, char **argv) {
    const uint64_t seed = argc > 1 ? strtoull(argv[1], 0, 10) : 1;
    const long tiles = argc > 2 ? atol(argv[2]) : 1000;
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    long edges = 0, bad = 0, skipped = 0;
    const int P = 24;  // points per tile
    for (long t = 0; t < tiles; ++t) {
        const int d = 1 + int(rng() % 33);
        const int kind = int(rng() % 8);
        std::vector<float> x(size_t(P) * d);
        for (auto &v : x) {
            double r;
            switch (kind) {
                case 0: r = U(rng); break;                                   // unit cube
                case 1: r = 10.0 * U(rng) - 5.0; break;                      // signed
                case 2: r = std::floor(8.0 * U(rng)); break;                 // integers: exact ties
                case 3: r = std::ldexp(U(rng), int(rng() % 40) - 20); break; // spread binades
                case 4: r = 1.0 + std::ldexp(U(rng), -20); break;            // close values
                case 5: r = (rng() % 4 == 0) ? 0.0 : U(rng) * 1e3; break;    // zeros
                case 6: r = std::ldexp(std::floor(U(rng) * 16777216.0), int(rng() % 8) - 30); break;
                default: r = (U(rng) < 0.5 ? -1.0 : 1.0) * std::ldexp(U(rng), int(rng() % 100) - 60); break;
            }
            v = (float)r;
            if (rng() % 97 == 0) v = -0.0f;
        }
        // per-dimension scale g_k and the 52-bit bound, as the kernel does
        std::vector<int32_t> g(d);
        std::vector<uint32_t> narrow((d + 31) / 32, 0u), narrow30((d + 31) / 32, 0u);
        bool ok = true;
        for (int k = 0; k < d; ++k) {
            int32_t lo = 1 << 30, hi = -(1 << 30);
            for (int p = 0; p < P; ++p) {
                uint32_t b = fbits(x[size_t(p) * d + k]);
                if ((b & 0x7fffffffu) == 0) continue;
                int32_t l, h;
                bit_range_f32(b, l, h);
                lo = l < lo ? l : lo;
                hi = h > hi ? h : hi;
            }
            if (lo == (1 << 30)) { g[k] = 0; continue; }
            g[k] = lo;
            if (hi + 1 - lo > 52) ok = false;
            if (hi + 1 - lo <= 31) narrow[k >> 5] |= 1u << (k & 31);    // |X| < 2^31: 32-bit squares
            if (hi + 1 - lo <= 30) narrow30[k >> 5] |= 1u << (k & 31);  // |X| < 2^30: 32-bit differences
        }
        if (!ok) { ++skipped; continue; }
        std::vector<int64_t> X(size_t(P) * d);
        for (int p = 0; p < P; ++p)
            for (int k = 0; k < d; ++k) X[size_t(p) * d + k] = to_fixed(fbits(x[size_t(p) * d + k]), g[k]);
        for (int i = 0; i < P; ++i)
            for (int j = i + 1; j < P; ++j) {
                const uint64_t got = sq_dist_fixed(&X[size_t(i) * d], &X[size_t(j) * d], g.data(), d, 1, 1);
                const uint64_t got_n =
                    sq_dist_fixed(&X[size_t(i) * d], &X[size_t(j) * d], g.data(), d, 1, 1, narrow.data());
                const uint64_t got_m =
                    sq_dist_mixed(&X[size_t(i) * d], &X[size_t(j) * d], g.data(), d, 1, 1, narrow30.data());
                // the unrolled form of the dimensions compiled in
                const int64_t *xi = &X[size_t(i) * d], *xj = &X[size_t(j) * d];
                uint64_t got_c = got_m;
                switch (d) {
                    case 2: got_c = sq_dist_mixed_ct<2, 1>(xi, xj, g.data(), narrow30[0]); break;
                    case 3: got_c = sq_dist_mixed_ct<3, 1>(xi, xj, g.data(), narrow30[0]); break;
                    case 8: got_c = sq_dist_mixed_ct<8, 1>(xi, xj, g.data(), narrow30[0]); break;
                    case 16: got_c = sq_dist_mixed_ct<16, 1>(xi, xj, g.data(), narrow30[0]); break;
                    case 32: got_c = sq_dist_mixed_ct<32, 1>(xi, xj, g.data(), narrow30[0]); break;
                    default: break;
                }
                const double want = ref_d2(&x[size_t(i) * d], &x[size_t(j) * d], d);
                uint64_t wb;
                std::memcpy(&wb, &want, 8);
                ++edges;
                if (got != wb || got_n != wb || got_m != wb || got_c != wb) {
                    if (bad < 5) fprintf(stderr, "mismatch tile %ld kind %d d %d (%d,%d): %016llx vs %016llx\n",
                                         t, kind, d, i, j, (unsigned long long)got, (unsigned long long)wb);
                    ++bad;
                }
            }
    }
    printf("%ld %ld %ld\n", edges, bad, skipped);
    return bad != 0;
}
