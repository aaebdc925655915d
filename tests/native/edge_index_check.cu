// Host check of the large-cloud edge records (paper_2203_02527_gb300/csrc/
// ph0_common.cuh: record_uv), compiled by nvcc for the host only: the
// decoded (u, v) of every edge index e of an n-point cloud is the edge whose
// lexicographic index (edge_index) is e.  Exhaustive for n <= 3000, every row
// start and end (and a stride of the interior) for n up to 92681; for n up
// to 32768 also the packed sort's edge of a word holding (u << 15) | v
// (pack_edge, pack_record) and the step of its first pass from an edge to
// the edge 32 places on (edge_step).  Usage: edge_index_check ; prints
// "checked failures".
#include <cstdint>
#include <cstdio>

#include "ph0_common.cuh"

using namespace ph0;

static int64_t checked = 0, bad = 0;

static void one(int64_t n, int64_t e) {
    uint32_t u = 0, v = 0;
    record_uv(uint32_t(e), true, n, u, v);
    ++checked;
    if (!(u < v && int64_t(v) < n && edge_index(n, u, v) == e)) {
        if (bad < 10) std::printf("n=%lld e=%lld -> (%u, %u)\n", (long long)n, (long long)e, u, v);
        ++bad;
    }
    if (n <= kPackMaxN && u < v && int64_t(v) < n) {
        const uint64_t w = (uint64_t(0xabcdef) << kPackIdBits) | (uint64_t(u) << 15) | v;
        ++checked;
        if (pack_edge(w, uint32_t(n)) != uint32_t(e) || pack_record(w) != ((u << 16) | v)) {
            if (bad < 10) std::printf("packed n=%lld e=%lld\n", (long long)n, (long long)e);
            ++bad;
        }
        if (e + 32 < n * (n - 1) / 2) {
            uint32_t su = u, sv = v;
            edge_step(su, sv, uint32_t(n), 32);
            ++checked;
            if (edge_index(n, su, sv) != e + 32 || su >= sv || int64_t(sv) >= n) {
                if (bad < 10) std::printf("step n=%lld e=%lld -> (%u, %u)\n", (long long)n, (long long)e, su, sv);
                ++bad;
            }
        }
    }
}

int main() {
    for (int64_t n = 2; n <= 3000; n = n < 64 ? n + 1 : n * 5 / 4 + 1)
        for (int64_t e = 0; e < n * (n - 1) / 2; ++e) one(n, e);
    const int64_t big[] = {16384, 32767, 32768, 65536, 70001, 92680, 92681};
    for (int64_t n : big) {
        for (int64_t u = 0; u + 1 < n; ++u) {
            const int64_t s = edge_index(n, u, u + 1), t = edge_index(n, u, n - 1);
            one(n, s);
            one(n, t);
            if (s + 1 < t) one(n, s + 1);
            if (t - 1 > s) one(n, t - 1);
            for (int64_t e = s + 2; e < t - 1; e += 997) one(n, e);
        }
    }
    std::printf("%lld %lld\n", (long long)checked, (long long)bad);
    return bad != 0;
}
