// ph0_capi.cu -- the C ABI of libph0 (declared in include/ph0.h): argument
// checks, workspace carving and kernel launches for the five steps of the
// barcode path (Rawson, Sec. 2; Sec. 4 steps 1-5).  The workspace entry
// points allocate nothing: every buffer is caller-owned and every call is
// asynchronous on the caller's stream, except ph0_barcodes_early (which waits
// to decide how much of the edge order to sort).  The one piece of global
// state, and the one buffer the caller does not own, is the fixed device
// array of ph0_barcodes_noalloc (end of this file) with its per-device
// address cache; that entry point is synchronous.
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "ph0_common.cuh"

namespace ph0 {

cudaError_t launch_dist(const float *pts, int64_t n, int32_t d, int64_t ld, uint64_t *key,
                        uint32_t *val, Header *h, cudaStream_t s, int split16 = -1, int tile = -1,
                        const int32_t *gate = nullptr, bool wide = false, bool packed = false);
cudaError_t launch_sort_init(Header *h, uint64_t *look0, int64_t tiles, cudaStream_t s,
                             int top_bits = kDefaultTopBits, int64_t sorted_edges = -1,
                             const int32_t *gate = nullptr);
// masked: the records may carry an edge-index bit in bit 63 of their keys (the split sort's halves)
cudaError_t launch_sort_short(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                              int64_t m, uint64_t *look0, uint64_t *look1, Header *h, uint32_t *cnt,
                              cudaStream_t s, bool masked = false, bool persist_all = false);
cudaError_t launch_sort_fixup(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1, int64_t m,
                              Header *h, uint32_t *cnt, uint64_t *defer_list, cudaStream_t s, bool masked = false);
cudaError_t launch_dedupe_count(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h, int64_t m,
                                uint32_t *cnt, const int32_t *gate, cudaStream_t s);
cudaError_t launch_dedupe_scan(uint32_t *cpref, int64_t m, uint64_t *look, Header *h, cudaStream_t s);
cudaError_t launch_merge(const uint64_t *ka, const uint32_t *va, int64_t la, const uint64_t *kb,
                         const uint32_t *vb, int64_t lb, uint64_t *ko, uint32_t *vo, uint32_t *hib, int64_t *split,
                         cudaStream_t s);
constexpr int kShortSortFirstSlot = 2;  // = kShortFirstSlot of k_sort.cu
// The whole path's built-in choice of the packed sort: from this many edges
// (below, the short sort's fewer launches count for more than its bytes) up
// to kPackMaxN points, in dimension kPackMinD and up: in fewer dimensions the
// squared distances of uniform clouds spread over so many binades that more
// than 256 values of the top part occur (8192 uniform points in 3 dimensions),
// and the short sort then runs after the packed sort's launches, 14% slower.
constexpr int64_t kPackMinEdges = int64_t(1) << 22;
constexpr int32_t kPackMinD = 4;
// ph0_barcodes_early's built-in choice: rounds from this many edges on
constexpr int64_t kEarlyMinEdges = int64_t(1) << 27;
cudaError_t launch_prefix_hist(const uint64_t *keys, int64_t m, const Header *h, uint32_t *bins,
                               cudaStream_t s);
cudaError_t launch_keystats(const uint64_t *keys, int64_t m, Header *h, cudaStream_t s,
                            const int32_t *gate = nullptr, bool lows_only = false);
cudaError_t launch_packed_prep(Header *h, cudaStream_t s);
cudaError_t launch_packed_passes(const uint64_t *keys, int64_t n, uint64_t *a, uint64_t *b, uint64_t *look0,
                                 uint64_t *look1, Header *h, cudaStream_t s, cudaEvent_t *after_pass);
cudaError_t launch_packed_fixup(const uint64_t *w, int64_t m, int64_t n, const uint64_t *keyidx, uint32_t *recs,
                                uint32_t *flags, uint32_t *cnt, uint64_t *defer_list, Header *h, cudaStream_t s);
cudaError_t launch_sort_passes(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                               int64_t m, uint64_t *look0, uint64_t *look1, Header *h,
                               cudaStream_t s, bool persist = false);
cudaError_t launch_sort_pass(uint64_t *keys0, uint64_t *keys1, uint32_t *vals0, uint32_t *vals1,
                             int64_t m, int pass, uint64_t *look0, uint64_t *look1, Header *h,
                             cudaStream_t s, bool persist = false);
cudaError_t prepare_sort_kernels();
cudaError_t launch_copy_parity(uint64_t *keys_dst, const uint64_t *keys_src, uint32_t *vals_dst,
                               const uint32_t *vals_src, int64_t m, const Header *h, int parity,
                               const int32_t *gate, cudaStream_t s);
cudaError_t launch_copy_if_odd(uint64_t *keys0, const uint64_t *keys1, uint32_t *vals0,
                               const uint32_t *vals1, int64_t m, const Header *h, cudaStream_t s);
cudaError_t launch_dedupe(const uint64_t *keys0, const uint64_t *keys1, const Header *sort_h,
                          int64_t m, uint32_t *a, uint32_t *cpref, uint64_t *look, Header *h,
                          cudaStream_t s);
cudaError_t launch_backward(const float *pts, int64_t n, int32_t d, int64_t ld, const ph0_bar *bars,
                            int64_t nb, const double *dl, float *grad, double *acc, cudaStream_t s);

cudaError_t launch_reduce(const ReduceArgs &A, cudaStream_t s);
cudaError_t launch_inf(Header *h, int64_t n, ph0_inf_bar *inf, cudaStream_t s);
cudaError_t run_h1(void *ws, const H1Layout &H, int64_t n, const uint64_t *ek0, const uint64_t *ek1,
                   const uint32_t *ev0, const uint32_t *ev1, const Header *esort, const uint32_t *cpref,
                   Header *h, ph0_h1bar *bars, cudaStream_t s, cudaEvent_t after_sort, cudaEvent_t after_reduce);
cudaError_t h1_counters(const void *ws, const H1Layout &H, int64_t n, uint64_t out[7]);
cudaError_t launch_emit(int64_t nb, int64_t m, Header *h, const unsigned long long *kk0, const unsigned long long *kk1,
                        const uint32_t *kv0, const uint32_t *kv1, const Header *kill_h,
                        const uint32_t *val0, const uint32_t *val1, const uint64_t *key0,
                        const uint64_t *key1, const Header *sort_h, const uint32_t *a,
                        const uint32_t *cpref, ph0_bar *bars, bool wide, int64_t n, cudaStream_t s,
                        const uint32_t *hib, PackedRecs pk);

namespace {

// max_n: kMaxN for the step entry points (records (u << 16) | v), kMaxNWide
// for the whole path (edge-index records above kMaxN).
int check_sizes(int64_t n, int32_t d, int64_t ld, int64_t max_n = kMaxN) {
    if (n < 1 || d < 1 || ld < d) return PH0_EINVAL;
    if (n > max_n || d > kMaxD) return PH0_ETOOBIG;
    return PH0_OK;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Smallest n whose edge count covers m.
int64_t n_for_edges(int64_t m) {
    int64_t n = 2;
    while (n_edges(n) < m) ++n;
    return n;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? PH0_OK : PH0_ECUDA; }

// Tuning with the built-in choices filled in.
struct Tune {
    int split16 = kDefaultDistSplit16, tile = -1, top_bits = kDefaultTopBits;
    uint32_t spin_limit = kSpinLimit;
    bool wide = false;  // edge-index records (always above kMaxN points)
    bool split = false;  // the whole path's sort as two merged halves (always above kSplitEdges edges)
    bool packed = false;  // the whole path's packed sort (k_sortp.cu)
    explicit Tune(const ph0_tuning *t, int64_t n = 0, int32_t d = 0) {
        const int64_t m = n_edges(n);
        wide = n > kMaxN;
        split = m > kSplitEdges;
        packed = m >= kPackMinEdges && n <= kPackMaxN && d >= kPackMinD;
        if (!t) return;
        if (t->wide_ids == 1) wide = true;
        if (t->split_sort == 1) split = true;
        if (t->packed_sort == 0) packed = false;
        if (t->packed_sort == 1) packed = m >= 1 && n <= kPackMaxN;
        if (split || wide) packed = false;  // its words take (u, v), not an edge index
        if (t->dist_split16 >= 0 && t->dist_split16 <= 16) split16 = t->dist_split16;
        if (t->dist_tile == 32 || t->dist_tile == 64 || t->dist_tile == 128) tile = t->dist_tile;
        if (t->sort_top_bits == 8 || t->sort_top_bits == 9) top_bits = t->sort_top_bits;
        if (t->reduce_spin_limit >= 0 && uint32_t(t->reduce_spin_limit) < kSpinLimit)
            spin_limit = uint32_t(t->reduce_spin_limit);
    }
};

// Zero the header and prepare the main sort (first look-back buffer).
cudaError_t begin_call(void *ws, const Layout &L, cudaStream_t s, int top_bits = kDefaultTopBits) {
    Header *h = at<Header>(ws, L.hdr);
    cudaError_t e = cudaMemsetAsync(h, 0, kHeaderBytes, s);
    if (e != cudaSuccess) return e;
    return launch_sort_init(h, at<uint64_t>(ws, L.look[0]), L.tiles, s, top_bits, L.m);
}

// The gated fallback of the whole path's sort: when the short sort's fix-up
// met a long group out of order (h->fixup_fallback), step 1 again and the
// complete sort, in the auxiliary header; otherwise every kernel returns at
// once (the distance kernel reads the gate, the radix passes a key range that
// was never set).  Both sorts leave the records in buffer (passes & 1) of the
// same plan (the keys, hence the key range, are the same).
cudaError_t sort_fallback(void *ws, const Layout &L, const float *pts, int64_t n, int32_t d, int64_t ld,
                          const Tune &t, cudaStream_t s) {
    Header *h = at<Header>(ws, L.hdr), *fh = at<Header>(ws, L.aux_hdr);
    uint64_t *k0 = at<uint64_t>(ws, L.key[0]), *k1 = at<uint64_t>(ws, L.key[1]);
    uint32_t *v0 = at<uint32_t>(ws, L.val[0]), *v1 = at<uint32_t>(ws, L.val[1]);
    uint64_t *look0 = at<uint64_t>(ws, L.look[0]), *look1 = at<uint64_t>(ws, L.look[1]);
    const int32_t *gate = &h->fixup_fallback;
    cudaError_t e = cudaMemsetAsync(fh, 0, kHeaderBytes, s);
    if (e == cudaSuccess) e = launch_sort_init(fh, look0, L.tiles, s, t.top_bits, -1, gate);
    if (e == cudaSuccess) e = launch_dist(pts, n, d, ld, k0, v0, fh, s, t.split16, t.tile, gate, t.wide);
    // persistent grids: the passes return at once unless the flag is set
    if (e == cudaSuccess) e = launch_sort_passes(k0, k1, v0, v1, L.m, look0, look1, fh, s, true);
    // the fix-up's de-duplication counts no longer hold: count again
    if (e == cudaSuccess) e = launch_dedupe_count(k0, k1, h, L.m, at<uint32_t>(ws, L.cpref), gate, s);
    return e;
}

// Step 2 of the whole path (the records of step 1 in buffer 0, h's
// histograms complete): the short sort (the passes over key bits 16 and up,
// then a fix-up of the groups they leave, which also counts the new
// distance values of every de-duplication chunk into cpref; k_sort.cu) and
// its gated fallback.  The sorted records end in buffer (passes & 1) of h's
// plan; step 3 then needs only launch_dedupe_scan.  fallback = false leaves
// the fallback out: the result is then exact only when h->fixup_fallback
// stays 0 (a caller that waits for the call checks it and runs again).
cudaError_t sort_whole(void *ws, const Layout &L, const float *pts, int64_t n, int32_t d, int64_t ld,
                       const Tune &t, cudaStream_t s, bool fallback = true) {
    if (L.m <= 0) return cudaSuccess;
    cudaError_t e = launch_sort_short(at<uint64_t>(ws, L.key[0]), at<uint64_t>(ws, L.key[1]),
                                      at<uint32_t>(ws, L.val[0]), at<uint32_t>(ws, L.val[1]), L.m,
                                      at<uint64_t>(ws, L.look[0]), at<uint64_t>(ws, L.look[1]),
                                      at<Header>(ws, L.hdr), at<uint32_t>(ws, L.cpref), s);
    if (e != cudaSuccess || !fallback) return e;
    return sort_fallback(ws, L, pts, n, d, ld, t, s);
}

// The packed form of step 2 (and of step 3's counts) on the whole path, the
// keys of step 1 in buffer 0 and its packed histograms in h (k_sortp.cu):
// the passes and fix-up of the packed sort, then the short sort with its
// histograms, which runs only when the keys do not pack (h->classic), then
// the gated complete sort (h->fixup_fallback: a group of the packed sort too
// long to sort, or a long unsorted group of the short sort).  The packed sort
// leaves the record (u << 16) | v of each position in the key[1] region and
// the flags of new values in look[0] (packed_recs); the others leave their
// records in buffer (passes & 1) of h's plan.  after_pass: kMaxPasses
// events (those past the fourth pass recorded at once), or null.
cudaError_t sort_packed(void *ws, const Layout &L, const float *pts, int64_t n, int32_t d, int64_t ld,
                        const Tune &t, cudaStream_t s, bool fallback, cudaEvent_t *after_pass = nullptr) {
    if (L.m <= 0) return cudaSuccess;
    Header *h = at<Header>(ws, L.hdr);
    uint64_t *k0 = at<uint64_t>(ws, L.key[0]), *k1 = at<uint64_t>(ws, L.key[1]);
    uint64_t *wb = at<uint64_t>(ws, L.val[0]);  // both value buffers: m words
    uint64_t *look0 = at<uint64_t>(ws, L.look[0]), *look1 = at<uint64_t>(ws, L.look[1]);
    uint32_t *cpref = at<uint32_t>(ws, L.cpref);
    cudaError_t e = launch_packed_prep(h, s);
    if (e == cudaSuccess) e = launch_packed_passes(k0, n, k1, wb, look0, look1, h, s, after_pass);
    for (int q = kPackPasses; q < kMaxPasses && after_pass && e == cudaSuccess; ++q)
        e = cudaEventRecord(after_pass[q], s);  // no such pass
    // the deferred groups' list lives in look1, unused after the passes
    if (e == cudaSuccess)
        e = launch_packed_fixup(wb, L.m, n, k0, at<uint32_t>(ws, L.key[1]), at<uint32_t>(ws, L.look[0]), cpref,
                                look1, h, s);
    if (e == cudaSuccess) e = launch_keystats(k0, L.m, h, s, &h->classic, true);
    if (e == cudaSuccess)
        e = launch_sort_short(k0, k1, at<uint32_t>(ws, L.val[0]), at<uint32_t>(ws, L.val[1]), L.m, look0, look1, h,
                              cpref, s, false, true);
    if (e != cudaSuccess || !fallback) return e;
    return sort_fallback(ws, L, pts, n, d, ld, t, s);
}

// What the reduction and the read-out take from the packed sort.
PackedRecs packed_recs(void *ws, const Layout &L) {
    return PackedRecs{at<uint32_t>(ws, L.key[1]), at<uint64_t>(ws, L.key[0]), at<uint32_t>(ws, L.look[0])};
}

// Step 2 of the whole path above kSplitEdges edges (or when a test asks for
// it): the two halves of step 1's records, each below 2^32, sorted one after
// the other in the main header with the short sort (its fix-up's chunk counts
// are scratch: step 3 counts again on the merged records) and each with its
// gated complete sort of the half as it stands (the fix-up permutes only
// within groups of equal key >> 16, stably, so equal values keep their edge
// order); both halves end in buffer 1, their merge in buffer 0, with the
// bitmask of the edge indices' bit 32 above kMaxN points.
cudaError_t sort_split(void *ws, const Layout &L, const Tune &t, cudaStream_t s) {
    Header *h = at<Header>(ws, L.hdr);
    uint64_t *k0 = at<uint64_t>(ws, L.key[0]), *k1 = at<uint64_t>(ws, L.key[1]);
    uint32_t *v0 = at<uint32_t>(ws, L.val[0]), *v1 = at<uint32_t>(ws, L.val[1]);
    uint64_t *look0 = at<uint64_t>(ws, L.look[0]), *look1 = at<uint64_t>(ws, L.look[1]);
    uint32_t *cpref = at<uint32_t>(ws, L.cpref);
    const int64_t m = L.m, half = (m / 2) & ~int64_t(3);  // 16-byte aligned rows for both halves
    const int64_t off[2] = {0, half}, len[2] = {half, m - half};
    const int32_t *fb = &h->fixup_fallback;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (len[k] <= 0) continue;
        uint64_t *sk0 = k0 + off[k], *sk1 = k1 + off[k];
        uint32_t *sv0 = v0 + off[k], *sv1 = v1 + off[k];
        const int64_t tiles = (len[k] + kSortTile - 1) / kSortTile;
        e = cudaMemsetAsync(&h->fixup_fallback, 0, sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(&h->defer_count, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = launch_sort_init(h, look0, tiles, s, t.top_bits, -1, nullptr);
        if (e == cudaSuccess) e = launch_keystats(sk0, len[k], h, s, nullptr);
        if (e == cudaSuccess) e = launch_sort_short(sk0, sk1, sv0, sv1, len[k], look0, look1, h, cpref, s, true);
        if (e == cudaSuccess) e = launch_copy_parity(sk1, sk0, sv1, sv0, len[k], h, 0, nullptr, s);
        if (e == cudaSuccess) e = launch_copy_parity(sk0, sk1, sv0, sv1, len[k], h, -1, fb, s);
        if (e == cudaSuccess) e = launch_sort_init(h, look0, tiles, s, t.top_bits, -1, fb);
        if (e == cudaSuccess) e = launch_keystats(sk0, len[k], h, s, fb);
        if (e == cudaSuccess) e = launch_sort_passes(sk0, sk1, sv0, sv1, len[k], look0, look1, h, s, true);
        if (e == cudaSuccess) e = launch_copy_parity(sk1, sk0, sv1, sv0, len[k], h, 0, fb, s);
    }
    uint32_t *hib = L.n > kMaxN ? at<uint32_t>(ws, L.hib) : nullptr;
    if (e == cudaSuccess)
        e = launch_merge(k1, v1, len[0], k1 + half, v1 + half, len[1], k0, v0, hib,
                         reinterpret_cast<int64_t *>(look0), s);  // the sorts' look-back words are free
    return e;
}

// Steps 4-5 on the first m sorted edges (m = n(n-1)/2 on the whole path):
// the pivot claiming.  val is the workspace's ping-pong buffer (sort_h != null
// selects the one holding the sorted data) or the caller's.
cudaError_t run_reduce(void *ws, const Layout &L, int64_t n, int64_t m, const uint32_t *val0,
                       const uint32_t *val1, const Header *sort_h, cudaStream_t s,
                       uint32_t spin_limit = kSpinLimit, bool wide = false, int64_t start = 0,
                       const uint32_t *hib = nullptr, bool capped = false, const uint32_t *valp = nullptr) {
    ReduceArgs A;
    A.n = n;
    A.m = m;
    A.val0 = val0;
    A.val1 = val1;
    A.sort_h = sort_h;
    A.comp = at<uint32_t>(ws, L.comp);
    A.parent = at<uint32_t>(ws, L.parent);
    A.res = at<unsigned long long>(ws, L.res);
    A.cand0 = at<uint32_t>(ws, L.cand[0]);
    A.cand1 = at<uint32_t>(ws, L.cand[1]);
    A.candr = at<unsigned long long>(ws, L.candr);
    A.gmap = at<uint32_t>(ws, L.gmap);
    A.m_edges = n_edges(n);
    A.wide = wide;
    A.kill_key = at<unsigned long long>(ws, L.kill_key[0]);
    A.kill_val = at<uint32_t>(ws, L.kill_val[0]);
    A.h = at<Header>(ws, L.hdr);
    A.trace = at<uint64_t>(ws, L.trace);
    int64_t w0 = 2 * n > 4096 ? 2 * n : 4096;
    A.w0 = w0 < kMaxWindow ? w0 : kMaxWindow;
    A.spin_limit = spin_limit;
    A.start = start;
    A.hib = hib;
    A.capped = capped;
    A.valp = valp;
    return launch_reduce(A, s);
}

// The read-out after run_reduce: order the n-1 pivot columns by position
// (their discovery order within a window is not the filtration order) and
// emit the bars, then the bar that never dies (inf may be null).  key as val;
// a is the caller's per-edge index, or null with cpref the workspace's chunk
// prefixes of the count-mode scan.
cudaError_t order_and_emit(void *ws, const Layout &L, int64_t n, int64_t m, const uint32_t *val0,
                           const uint32_t *val1, const uint64_t *key0, const uint64_t *key1,
                           const Header *sort_h, const uint32_t *a, const uint32_t *cpref,
                           ph0_bar *bars, ph0_inf_bar *inf, cudaStream_t s, bool wide = false,
                           const uint32_t *hib = nullptr, PackedRecs pk = PackedRecs{}) {
    Header *h = at<Header>(ws, L.hdr);
    const int64_t nb = n - 1;
    if (nb <= 0) return launch_inf(h, n, inf, s);
    Header *kh = at<Header>(ws, L.aux_hdr);
    cudaError_t e = cudaMemsetAsync(kh, 0, kHeaderBytes, s);
    if (e != cudaSuccess) return e;
    const int64_t ktiles = (nb + kSortTile - 1) / kSortTile;
    e = launch_sort_init(kh, at<uint64_t>(ws, L.kill_look[0]), ktiles, s);
    if (e != cudaSuccess) return e;
    uint64_t *kk0 = at<uint64_t>(ws, L.kill_key[0]), *kk1 = at<uint64_t>(ws, L.kill_key[1]);
    uint32_t *kv0 = at<uint32_t>(ws, L.kill_val[0]), *kv1 = at<uint32_t>(ws, L.kill_val[1]);
    e = launch_keystats(kk0, nb, kh, s);
    if (e != cudaSuccess) return e;
    e = launch_sort_passes(kk0, kk1, kv0, kv1, nb, at<uint64_t>(ws, L.kill_look[0]),
                           at<uint64_t>(ws, L.kill_look[1]), kh, s);
    if (e != cudaSuccess) return e;
    e = launch_emit(nb, m, h, reinterpret_cast<const unsigned long long *>(kk0),
                    reinterpret_cast<const unsigned long long *>(kk1), kv0, kv1, kh, val0, val1,
                    key0, key1, sort_h, a, cpref, bars, wide, n, s, hib, pk);
    if (e != cudaSuccess) return e;
    return launch_inf(h, n, inf, s);
}

// Steps 4-5 plus the read-out on the m = n(n-1)/2 sorted edges, or on their
// first m_scan (the merged sort of more than 2^32 edges, hib its bitmask).
cudaError_t reduce_and_emit(void *ws, const Layout &L, int64_t n, const uint32_t *val0,
                            const uint32_t *val1, const uint64_t *key0, const uint64_t *key1,
                            const Header *sort_h, const uint32_t *a, const uint32_t *cpref,
                            ph0_bar *bars, ph0_inf_bar *inf, cudaStream_t s,
                            cudaEvent_t after_reduce = nullptr, uint32_t spin_limit = kSpinLimit,
                            bool wide = false, int64_t m_scan = -1, const uint32_t *hib = nullptr,
                            PackedRecs pk = PackedRecs{}) {
    const int64_t m_all = n_edges(n), m = m_scan >= 0 && m_scan < m_all ? m_scan : m_all;
    cudaError_t e = run_reduce(ws, L, n, m, val0, val1, sort_h, s, spin_limit, wide, 0, hib, m < m_all, pk.recs);
    if (e != cudaSuccess) return e;
    if (after_reduce) {
        e = cudaEventRecord(after_reduce, s);
        if (e != cudaSuccess) return e;
    }
    return order_and_emit(ws, L, n, m, val0, val1, key0, key1, sort_h, a, cpref, bars, inf, s, wide, hib, pk);
}

}  // namespace
int barcodes_whole(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_bar *bars_dev,
                   ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes, void *stream, const ph0_tuning *tuning,
                   bool fallback);

}  // namespace ph0

using namespace ph0;

extern "C" {

const char *ph0_strerror(int status) {
    switch (status) {
        case PH0_OK: return "ok";
        case PH0_EINVAL: return "invalid argument";
        case PH0_ENONFINITE: return "non-finite coordinate";
        case PH0_ETOOBIG: return "size above the supported maximum (n <= 131071 for ph0_barcodes, 92681 for the other whole-path calls, 65535 for the step calls; d <= 1024), or a cloud whose n-1 killing edges lie beyond the first 2^32 - 4096 sorted edges";
        case PH0_ENOMEM: return "workspace too small";
        case PH0_ETIMEOUT: return "a bounded device-side wait timed out";
        case PH0_ECUDA: return "CUDA runtime error";
        case PH0_EBUSY: return "busy";
        case PH0_EINTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

int32_t ph0_abi_version(void) { return 5; }

size_t ph0_workspace_bytes(int64_t n, int32_t d) {
    if (check_sizes(n, d, d, kMaxNHuge) != PH0_OK) return 0;
    return Layout(n, d).total;
}

int ph0_barcodes_tuned(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_bar *bars_dev,
                       ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes, void *stream,
                       const ph0_tuning *tuning) {
    return ph0::barcodes_whole(pts_dev, n, d, ld, bars_dev, inf_dev, ws, ws_bytes, stream, tuning, true);
}
}  // extern "C"

namespace ph0 {
// The whole path (ph0_barcodes_tuned); fallback = false leaves out the
// gated complete sort (see sort_whole): for a caller that waits for the call
// and reads h->fixup_fallback (the serving context).
int barcodes_whole(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_bar *bars_dev,
                   ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes, void *stream, const ph0_tuning *tuning,
                   bool fallback) {
    int rc = check_sizes(n, d, ld, kMaxNHuge);
    if (rc != PH0_OK) return rc;
    if (!pts_dev || !ws || (n > 1 && !bars_dev)) return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(pts_dev, 4) || !aligned(bars_dev, 8) || !aligned(inf_dev, 8))
        return PH0_EINVAL;
    const Layout L(n, d);
    if (ws_bytes < L.total) return PH0_ENOMEM;
    const Tune t(tuning, n, d);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Header *h = at<Header>(ws, L.hdr);
    uint64_t *k0 = at<uint64_t>(ws, L.key[0]), *k1 = at<uint64_t>(ws, L.key[1]);
    uint32_t *v0 = at<uint32_t>(ws, L.val[0]), *v1 = at<uint32_t>(ws, L.val[1]);
    uint32_t *cpref = at<uint32_t>(ws, L.cpref);
    cudaError_t e = begin_call(ws, L, s, t.top_bits);
    if (e == cudaSuccess)
        e = launch_dist(pts_dev, n, d, ld, k0, v0, h, s, t.split16, t.tile, nullptr, t.wide, t.packed);
    if (t.packed) {
        if (e == cudaSuccess) e = sort_packed(ws, L, pts_dev, n, d, ld, t, s, fallback);
        if (e == cudaSuccess) e = launch_dedupe_scan(cpref, L.m, at<uint64_t>(ws, L.dlook), h, s);
        if (e == cudaSuccess)
            e = reduce_and_emit(ws, L, n, v0, v1, k0, k1, h, nullptr, cpref, bars_dev, inf_dev, s, nullptr,
                                t.spin_limit, t.wide, -1, nullptr, packed_recs(ws, L));
        return cuda_status(e);
    }
    if (t.split) {  // two halves merged into buffer 0; positions scanned below 2^32
        const int64_t mscan = L.m < kMaxScanPos ? L.m : kMaxScanPos;
        const uint32_t *hib = n > kMaxN ? at<uint32_t>(ws, L.hib) : nullptr;
        if (e == cudaSuccess) e = sort_split(ws, L, t, s);
        if (e == cudaSuccess) e = launch_dedupe_count(k0, k0, nullptr, mscan, cpref, nullptr, s);
        if (e == cudaSuccess) e = launch_dedupe_scan(cpref, mscan, at<uint64_t>(ws, L.dlook), h, s);
        if (e == cudaSuccess)
            e = reduce_and_emit(ws, L, n, v0, v0, k0, k0, nullptr, nullptr, cpref, bars_dev, inf_dev, s, nullptr,
                                t.spin_limit, t.wide, mscan, hib);
        return cuda_status(e);
    }
    if (e == cudaSuccess) e = sort_whole(ws, L, pts_dev, n, d, ld, t, s, fallback);
    if (e == cudaSuccess) e = launch_dedupe_scan(cpref, L.m, at<uint64_t>(ws, L.dlook), h, s);
    if (e == cudaSuccess)
        e = reduce_and_emit(ws, L, n, v0, v1, k0, k1, h, nullptr, cpref, bars_dev, inf_dev, s, nullptr,
                            t.spin_limit, t.wide);
    return cuda_status(e);
}
}  // namespace ph0

extern "C" {

size_t ph0_status_offset(void) {
    static_assert(offsetof(Header, status) == 0, "the status word leads the header");
    return Layout(2, 1).hdr + offsetof(Header, status);  // the header is the first region for every size
}

int ph0_barcodes(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_bar *bars_dev,
                 ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes, void *stream) {
    return ph0_barcodes_tuned(pts_dev, n, d, ld, bars_dev, inf_dev, ws, ws_bytes, stream, nullptr);
}

int ph0_barcodes_early(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_bar *bars_dev,
                       ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes, void *stream) {
    return ph0_barcodes_early_tuned(pts_dev, n, d, ld, bars_dev, inf_dev, ws, ws_bytes, stream, nullptr, nullptr);
}

int ph0_barcodes_early_tuned(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_bar *bars_dev,
                             ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes, void *stream,
                             const ph0_tuning *tuning, ph0_stats *stats) {
    int rc = check_sizes(n, d, ld, kMaxNWide);
    if (rc != PH0_OK) return rc;
    if (!pts_dev || !ws || (n > 1 && !bars_dev)) return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(pts_dev, 4) || !aligned(bars_dev, 8) || !aligned(inf_dev, 8))
        return PH0_EINVAL;
    const Layout L(n, d);
    if (ws_bytes < L.total) return PH0_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto whole = [&]() {  // the whole path, then its device status
        const int r = ph0_barcodes_tuned(pts_dev, n, d, ld, bars_dev, inf_dev, ws, ws_bytes, stream, nullptr);
        return r != PH0_OK ? r : ph0_finish(ws, stream, stats);
    };
    // the whole path: tiny clouds and (built-in choice) clouds below
    // kEarlyMinEdges, where the rounds' fixed cost exceeds the saving
    const int rounds = tuning ? tuning->early_rounds : -1;
    if (n < 3 || rounds == 0 || (rounds != 1 && L.m < kEarlyMinEdges)) return whole();
    // edge-index records above 65,535 points (or when a test asks for them);
    // the rounds never split the sort (E < 2^32 up to 92,681 points)
    const Tune t(tuning, n);
    const int64_t m = L.m;
    Header *h = at<Header>(ws, L.hdr);
    Header *sh = at<Header>(ws, L.aux_hdr);  // header of the segment sorts
    uint64_t *k0 = at<uint64_t>(ws, L.key[0]), *k1 = at<uint64_t>(ws, L.key[1]);
    uint32_t *v0 = at<uint32_t>(ws, L.val[0]), *v1 = at<uint32_t>(ws, L.val[1]);
    uint64_t *look0 = at<uint64_t>(ws, L.look[0]), *look1 = at<uint64_t>(ws, L.look[1]);
    uint64_t *dlook = at<uint64_t>(ws, L.dlook);
    uint32_t *cpref = at<uint32_t>(ws, L.cpref), *bins = at<uint32_t>(ws, L.phist);

    // step 1, then the key histogram (read back: the host picks the rounds)
    cudaError_t e = begin_call(ws, L, s, t.top_bits);
    if (e == cudaSuccess) e = launch_dist(pts_dev, n, d, ld, k0, v0, h, s, t.split16, t.tile, nullptr, t.wide);
    if (e == cudaSuccess) e = launch_prefix_hist(k0, m, h, bins, s);
    std::vector<uint32_t> hb(kPrefixBins);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb.data(), bins, sizeof(uint32_t) * kPrefixBins, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    Header h0;
    if (e == cudaSuccess) e = cudaMemcpy(&h0, h, sizeof(Header), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return PH0_ECUDA;
    if (h0.status != PH0_OK) return h0.status;
    std::vector<int64_t> below(kPrefixBins + 1, 0);  // edges in the bins before bin i
    for (int i = 0; i < kPrefixBins; ++i) below[i + 1] = below[i] + hb[i];
    if (below[kPrefixBins] != m) return whole();  // inconsistent histogram: not expected

    // classes of consecutive bin ranges whose cumulative edge counts reach
    // these fractions of the edges (the last class takes the rest); one
    // stable radix pass with the class as digit puts them, class by class,
    // into buffer 1
    static const double kFractions[] = {0.02, 0.08, 0.25, 0.45};
    uint32_t bound[kPrefixClasses + 1];
    int64_t cstart[kPrefixClasses + 1];
    int nc = 0;
    bound[0] = 0;
    cstart[0] = 0;
    for (double f : kFractions) {
        const int64_t target = int64_t(f * double(m));
        uint32_t bnd = bound[nc] + 1;
        while (bnd < uint32_t(kPrefixBins) && below[bnd] < target) ++bnd;
        if (bnd >= uint32_t(kPrefixBins)) break;
        ++nc;
        bound[nc] = bnd;
        cstart[nc] = below[bnd];
    }
    ++nc;
    for (int c = nc; c <= kPrefixClasses; ++c) {
        bound[c] = kPrefixBins;
        cstart[c] = m;
    }
    e = cudaMemsetAsync(sh, 0, kHeaderBytes, s);
    if (e == cudaSuccess) e = launch_sort_init(sh, look0, L.tiles, s, t.top_bits);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        const uint64_t pk = h0.kmin;
        const int32_t ps = prefix_shift(h0.kmin, h0.kmax), pn = nc;
        uint32_t counts[kPrefixClasses];
        for (int c = 0; c < kPrefixClasses; ++c) counts[c] = uint32_t(c < nc ? cstart[c + 1] - cstart[c] : 0);
        e = cudaMemcpy(&sh->part_kmin, &pk, sizeof(pk), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(&sh->part_shift, &ps, sizeof(ps), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(&sh->part_nc, &pn, sizeof(pn), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(sh->part_bound, bound, sizeof(bound), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(&sh->hist[0][0], counts, sizeof(counts), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = prepare_sort_kernels();
    if (e == cudaSuccess) e = launch_sort_pass(k0, k1, v0, v1, m, kClassSlot, look0, look1, sh, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int32_t pst = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&pst, &sh->status, sizeof(pst), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return PH0_ECUDA;
    if (pst != PH0_OK) return pst;

    // rounds: sort the next class (in buffer 1, where the class pass put it)
    // into buffer 0, no longer needed otherwise, where the sorted prefix
    // grows; then run the reduction on the sorted prefix
    int64_t P = 0;
    bool done = false;
    for (int c = 0; c < nc && !done; ++c) {
        if (cstart[c + 1] == cstart[c]) continue;
        // the segment starts at the class start rounded down to 4 records, so
        // that its rows stay 16-byte aligned (bulk tile loads in every pass):
        // the at most 3 records before the class, already sorted into buffer
        // 0 with keys below every key of the class, are copied ahead of it in
        // buffer 1 and sort to where they are
        const int64_t c0 = cstart[c] & ~int64_t(3), seg = cstart[c + 1] - c0, lead = cstart[c] - c0;
        if (lead > 0) {
            e = cudaMemcpyAsync(k1 + c0, k0 + c0, size_t(lead) * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(v1 + c0, v0 + c0, size_t(lead) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return PH0_ECUDA;
        }
        const int64_t stiles = (seg + kSortTile - 1) / kSortTile;
        uint64_t *sk0 = k1 + c0, *sk1 = k0 + c0;  // the segment's buffers 0 and 1
        uint32_t *sv0 = v1 + c0, *sv1 = v0 + c0;
        e = cudaMemsetAsync(sh, 0, kHeaderBytes, s);
        if (e == cudaSuccess) e = launch_sort_init(sh, look0, stiles, s, t.top_bits, seg);
        if (e == cudaSuccess) e = launch_keystats(sk0, seg, sh, s);
        // the short sort of the whole path on the segment (it is in (u, v)
        // order within each class, the class pass being stable): the passes
        // from slot 2, the fix-up (its chunk counts go to cpref, scratch until
        // the prefix's de-duplication); the sorted prefix grows in buffer 0 of
        // the call, the segment's buffer 1, where an odd pass count (five
        // from slot 2, as a rule) leaves it: else one copy moves it there
        for (int p = kShortSortFirstSlot; p < kMaxPasses && e == cudaSuccess; ++p)
            e = launch_sort_pass(sk0, sk1, sv0, sv1, seg, p, look0, look1, sh, s, p == kMaxPasses - 1);
        if (e == cudaSuccess) e = launch_sort_fixup(sk0, sk1, sv0, sv1, seg, sh, cpref, look1, s);
        if (e == cudaSuccess) e = launch_copy_parity(sk1, sk0, sv1, sv0, seg, sh, 0, nullptr, s);
        // gated on sh->fixup_fallback (a long group out of order): the
        // complete sort of the segment as it stands, whose equal keys are
        // still in (u, v) order (the fix-up permutes within groups, stably),
        // from the segment's buffer 0 and back into its buffer 1
        const int32_t *fb = &sh->fixup_fallback;
        if (e == cudaSuccess) e = launch_copy_parity(sk0, sk1, sv0, sv1, seg, sh, -1, fb, s);
        if (e == cudaSuccess) e = launch_sort_init(sh, look0, stiles, s, t.top_bits, -1, fb);
        if (e == cudaSuccess) e = launch_keystats(sk0, seg, sh, s, fb);
        if (e == cudaSuccess) e = launch_sort_passes(sk0, sk1, sv0, sv1, seg, look0, look1, sh, s, true);
        if (e == cudaSuccess) e = launch_copy_parity(sk1, sk0, sv1, sv0, seg, sh, 0, fb, s);
        if (e != cudaSuccess) return PH0_ECUDA;
        const int64_t Pprev = P;
        P = c0 + seg;
        // steps 4-5 on the prefix, resumed where the last round stopped;
        // enough once it holds n-1 pivots
        e = run_reduce(ws, L, n, P, v0, v0, nullptr, s, kSpinLimit, t.wide, Pprev);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        Header hh;
        if (e == cudaSuccess) e = cudaMemcpy(&hh, h, sizeof(Header), cudaMemcpyDeviceToHost);
        int32_t sst = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&sst, &sh->status, sizeof(sst), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return PH0_ECUDA;
        if (hh.status != PH0_OK) return hh.status;
        if (sst != PH0_OK) return sst;
        done = int64_t(hh.npiv) >= n - 1;
    }
    if (!done) return PH0_EINTERNAL;  // all edges sorted: the reduction always completes

    // step 3 on the prefix (count mode) and the read-out; then the prefix length
    e = launch_dedupe(k0, k0, nullptr, P, nullptr, cpref, dlook, h, s);
    if (e == cudaSuccess)
        e = order_and_emit(ws, L, n, P, v0, v0, k0, k0, nullptr, nullptr, cpref, bars_dev, inf_dev, s, t.wide);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h->sorted_edges, &P, sizeof(P), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return PH0_ECUDA;
    return ph0_finish(ws, stream, stats);
}

int ph0_barcodes_profiled(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                          ph0_bar *bars_dev, ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes,
                          void *stream, const ph0_tuning *tuning, ph0_profile *prof) {
    int rc = check_sizes(n, d, ld, kMaxNWide);
    if (rc != PH0_OK) return rc;
    if (!pts_dev || !ws || !prof || (n > 1 && !bars_dev)) return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(pts_dev, 4) || !aligned(bars_dev, 8) || !aligned(inf_dev, 8))
        return PH0_EINVAL;
    const Layout L(n, d);
    if (ws_bytes < L.total) return PH0_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Header *h = at<Header>(ws, L.hdr);
    uint64_t *k0 = at<uint64_t>(ws, L.key[0]), *k1 = at<uint64_t>(ws, L.key[1]);
    uint32_t *v0 = at<uint32_t>(ws, L.val[0]), *v1 = at<uint32_t>(ws, L.val[1]);
    uint32_t *cpref = at<uint32_t>(ws, L.cpref);
    uint64_t *look0 = at<uint64_t>(ws, L.look[0]), *look1 = at<uint64_t>(ws, L.look[1]);
    constexpr int kEv = 6 + kMaxPasses;
    cudaEvent_t ev[kEv];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < kEv && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    if (e != cudaSuccess) {
        for (int i = 0; i < made - 1; ++i) cudaEventDestroy(ev[i]);
        return PH0_ECUDA;
    }
    // ev[0] | init, dist | ev[1] | pass p | ev[2+p] ... | fix-up, gated fallback | ev[2+P] |
    // dedupe | ev[3+P] | reduce | ev[4+P] | order pivots, emit | ev[5+P]
    // (P = kMaxPasses; the short sort launches the passes from slot 2 on;
    // passes that are not needed return at once.  The packed sort: its four
    // passes, then the fix-up, the short sort that runs only when the keys do
    // not pack, and the gated fallback)
    const Tune t(tuning, n, d);
    e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = begin_call(ws, L, s, t.top_bits);
    if (e == cudaSuccess)
        e = launch_dist(pts_dev, n, d, ld, k0, v0, h, s, t.split16, t.tile, nullptr, t.wide, t.packed);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess && L.m > 0) e = prepare_sort_kernels();
    if (t.packed) {
        if (e == cudaSuccess && L.m > 0) e = sort_packed(ws, L, pts_dev, n, d, ld, t, s, true, ev + 2);
        for (int p = 0; p < kMaxPasses && e == cudaSuccess && L.m <= 0; ++p) e = cudaEventRecord(ev[2 + p], s);
    } else {
        for (int p = 0; p < kMaxPasses && e == cudaSuccess; ++p) {
            if (L.m > 0 && p >= kShortSortFirstSlot)  // as launch_sort_short
                e = launch_sort_pass(k0, k1, v0, v1, L.m, p, look0, look1, h, s, p == kMaxPasses - 1);
            if (e == cudaSuccess) e = cudaEventRecord(ev[2 + p], s);
        }
        if (e == cudaSuccess && L.m > 0) e = launch_sort_fixup(k0, k1, v0, v1, L.m, h, cpref, look1, s);
        if (e == cudaSuccess && L.m > 0) e = sort_fallback(ws, L, pts_dev, n, d, ld, t, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 + kMaxPasses], s);
    if (e == cudaSuccess) e = launch_dedupe_scan(cpref, L.m, at<uint64_t>(ws, L.dlook), h, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3 + kMaxPasses], s);
    if (e == cudaSuccess)
        e = reduce_and_emit(ws, L, n, v0, v1, k0, k1, h, nullptr, cpref, bars_dev, inf_dev, s, ev[4 + kMaxPasses],
                            t.spin_limit, t.wide, -1, nullptr, t.packed ? packed_recs(ws, L) : PackedRecs{});
    if (e == cudaSuccess) e = cudaEventRecord(ev[5 + kMaxPasses], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[5 + kMaxPasses]);
    if (e == cudaSuccess) {
        auto span = [&](int i, int j) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[j]);
            return ms;
        };
        std::memset(prof, 0, sizeof(*prof));
        prof->total_ms = span(0, 5 + kMaxPasses);
        prof->dist_ms = span(0, 1);
        for (int p = 0; p < kMaxPasses; ++p) prof->pass_ms[p] = span(1 + p, 2 + p);
        prof->fixup_ms = span(1 + kMaxPasses, 2 + kMaxPasses);
        prof->sort_ms = span(1, 2 + kMaxPasses);
        prof->dedupe_ms = span(2 + kMaxPasses, 3 + kMaxPasses);
        prof->reduce_ms = span(3 + kMaxPasses, 4 + kMaxPasses);
        prof->emit_ms = span(4 + kMaxPasses, 5 + kMaxPasses);
    }
    for (int i = 0; i < kEv; ++i) cudaEventDestroy(ev[i]);
    return cuda_status(e);
}

int ph0_finish(const void *ws, void *stream, ph0_stats *stats) {
    if (!ws) return PH0_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return PH0_ECUDA;
    Header hh;  // the counters lead the header; its histograms are not read
    e = cudaMemcpy(&hh, ws, offsetof(Header, part_kmin), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return PH0_ECUDA;
    if (stats) {
        stats->status = hh.status;
        stats->sort_passes = hh.sort_passes;
        stats->key_bits = hh.key_bits;
        stats->windows = hh.windows;
        stats->n_distinct = hh.n_distinct;
        stats->edges_scanned = hh.edges_scanned;
        stats->candidates = hh.candidates;
        stats->rounds = hh.rounds;
        stats->n_bars = hh.n_bars;
        stats->dist_tiles = int64_t(hh.dist_tiles);
        stats->dist_tiles_int = int64_t(hh.dist_tiles_exact_int);
        stats->sorted_edges = hh.sorted_edges;
        stats->inf_vertex = hh.inf_vertex;
        stats->claim_rounds_max = int32_t(hh.claim_rounds_max);
        stats->claim_attempts = int64_t(hh.claim_attempts);
        stats->sort_form = hh.fixup_fallback ? 2 : (hh.packed ? 1 : 0);
        stats->_pad = 0;
    }
    return hh.status;
}

int ph0_trace_windows(const void *ws, int64_t n, int32_t d, void *stream, uint64_t *out,
                      int32_t max_windows) {
    int rc = check_sizes(n, d, d, kMaxNWide);
    if (rc != PH0_OK) return rc;
    if (!ws || !out || max_windows < 0) return PH0_EINVAL;
    const Layout L(n, d);
    const int w = max_windows < kTraceWindows ? max_windows : kTraceWindows;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess)
        e = cudaMemcpy(out, static_cast<const char *>(ws) + L.trace,
                       sizeof(uint64_t) * kTraceWords * size_t(w), cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

int ph0_distances(const float *pts_dev, int64_t n, int32_t d, int64_t ld, uint64_t *key_dev,
                  uint32_t *val_dev, void *ws, size_t ws_bytes, void *stream) {
    int rc = check_sizes(n, d, ld);
    if (rc != PH0_OK) return rc;
    if (!pts_dev || !ws || (n > 1 && (!key_dev || !val_dev))) return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(key_dev, 8) || !aligned(val_dev, 4)) return PH0_EINVAL;
    const Layout L(n, d);
    if (ws_bytes < L.total) return PH0_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = begin_call(ws, L, s);
    if (e == cudaSuccess) e = launch_dist(pts_dev, n, d, ld, key_dev, val_dev, at<Header>(ws, L.hdr), s);
    return cuda_status(e);
}

int ph0_sort(uint64_t *key_dev, uint32_t *val_dev, int64_t m, void *ws, size_t ws_bytes,
             void *stream) {
    if (m < 0 || m > int64_t(0x7fffffff)) return PH0_EINVAL;
    if (m == 0) return PH0_OK;
    if (!key_dev || !val_dev || !ws) return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(key_dev, 8) || !aligned(val_dev, 4)) return PH0_EINVAL;
    const int64_t n = n_for_edges(m);
    if (n > kMaxN) return PH0_ETOOBIG;
    const Layout L(n, 1);
    if (ws_bytes < L.total) return PH0_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Header *h = at<Header>(ws, L.hdr);
    uint64_t *k1 = at<uint64_t>(ws, L.key[1]);
    uint32_t *v1 = at<uint32_t>(ws, L.val[1]);
    const int64_t tiles = (m + kSortTile - 1) / kSortTile;
    cudaError_t e = cudaMemsetAsync(h, 0, kHeaderBytes, s);
    if (e == cudaSuccess) e = launch_sort_init(h, at<uint64_t>(ws, L.look[0]), tiles, s);
    if (e == cudaSuccess) e = launch_keystats(key_dev, m, h, s);
    if (e == cudaSuccess)
        e = launch_sort_passes(key_dev, k1, val_dev, v1, m, at<uint64_t>(ws, L.look[0]),
                               at<uint64_t>(ws, L.look[1]), h, s);
    if (e == cudaSuccess) e = launch_copy_if_odd(key_dev, k1, val_dev, v1, m, h, s);
    return cuda_status(e);
}

int ph0_dedupe(const uint64_t *key_sorted_dev, int64_t m, uint32_t *a_dev, void *ws,
               size_t ws_bytes, void *stream) {
    if (m < 0 || m > int64_t(0x7fffffff)) return PH0_EINVAL;
    if (!ws || (m > 0 && (!key_sorted_dev || !a_dev))) return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(key_sorted_dev, 8) || !aligned(a_dev, 4)) return PH0_EINVAL;
    const int64_t n = m > 0 ? n_for_edges(m) : 2;
    if (n > kMaxN) return PH0_ETOOBIG;
    const Layout L(n, 1);
    if (ws_bytes < L.total) return PH0_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Header *h = at<Header>(ws, L.hdr);
    cudaError_t e = cudaMemsetAsync(h, 0, kHeaderBytes, s);
    if (e == cudaSuccess)
        e = launch_dedupe(key_sorted_dev, key_sorted_dev, nullptr, m, a_dev, nullptr, at<uint64_t>(ws, L.dlook), h, s);
    return cuda_status(e);
}

int ph0_reduce(int64_t n, const uint32_t *val_sorted_dev, const uint32_t *a_dev,
               const uint64_t *key_sorted_dev, ph0_bar *bars_dev, void *ws, size_t ws_bytes,
               void *stream) {
    int rc = check_sizes(n, 1, 1);
    if (rc != PH0_OK) return rc;
    if (!ws || (n > 1 && (!val_sorted_dev || !a_dev || !key_sorted_dev || !bars_dev)))
        return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(bars_dev, 8)) return PH0_EINVAL;
    const Layout L(n, 1);
    if (ws_bytes < L.total) return PH0_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(at<Header>(ws, L.hdr), 0, kHeaderBytes, s);
    if (e == cudaSuccess)
        e = reduce_and_emit(ws, L, n, val_sorted_dev, val_sorted_dev, key_sorted_dev, key_sorted_dev,
                            nullptr, a_dev, nullptr, bars_dev, nullptr, s);
    return cuda_status(e);
}

int ph0_barcodes_backward(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                          const ph0_bar *bars_dev, int64_t n_bars, const double *dl_ddeath_dev,
                          float *grad_dev, void *ws, size_t ws_bytes, void *stream) {
    int rc = check_sizes(n, d, ld, kMaxNWide);
    if (rc != PH0_OK) return rc;
    if (n_bars < 0 || n_bars > n - 1) return PH0_EINVAL;
    if (!pts_dev || !grad_dev || !ws || (n_bars > 0 && (!bars_dev || !dl_ddeath_dev)))
        return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(bars_dev, 8) || !aligned(dl_ddeath_dev, 8)) return PH0_EINVAL;
    const Layout L(n, d);
    if (ws_bytes < L.total) return PH0_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return cuda_status(launch_backward(pts_dev, n, d, ld, bars_dev, n_bars, dl_ddeath_dev, grad_dev,
                                       at<double>(ws, L.grad), s));
}

size_t ph0_h1_workspace_bytes(int64_t n, int32_t d) {
    if (check_sizes(n, d, d, kH1MaxN) != PH0_OK) return 0;
    const Layout L(n, d);
    return H1Layout(n, L.total).total;
}

int ph0_h1(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_h1bar *bars_dev, void *ws,
           size_t ws_bytes, void *stream, ph0_h1_stats *stats) {
    int rc = check_sizes(n, d, ld, kH1MaxN);
    if (rc != PH0_OK) return rc;
    const int64_t m = n_edges(n), nbars = m - (n - 1);
    if (!pts_dev || !ws || (nbars > 0 && !bars_dev)) return PH0_EINVAL;
    if (!aligned(ws, 256) || !aligned(pts_dev, 4) || !aligned(bars_dev, 8)) return PH0_EINVAL;
    const Layout L(n, d);
    const H1Layout H(n, L.total);
    if (ws_bytes < H.total) return PH0_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Tune t(nullptr, n);
    Header *h = at<Header>(ws, L.hdr);
    uint64_t *k0 = at<uint64_t>(ws, L.key[0]), *k1 = at<uint64_t>(ws, L.key[1]);
    uint32_t *v0 = at<uint32_t>(ws, L.val[0]), *v1 = at<uint32_t>(ws, L.val[1]);
    uint32_t *cpref = at<uint32_t>(ws, L.cpref);
    // stage events: start | edges | triangles of each diameter | reduced | end
    cudaEvent_t ev[5] = {};
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < 5 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    if (e != cudaSuccess) {
        for (int i = 0; i < made - 1; ++i) cudaEventDestroy(ev[i]);
        return PH0_ECUDA;
    }
    // steps 1-3 of dimension 0: the edge order and the de-duplication
    e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = begin_call(ws, L, s, t.top_bits);
    if (e == cudaSuccess) e = launch_dist(pts_dev, n, d, ld, k0, v0, h, s, t.split16, t.tile);
    if (e == cudaSuccess) e = sort_whole(ws, L, pts_dev, n, d, ld, t, s);
    if (e == cudaSuccess) e = launch_dedupe_scan(cpref, L.m, at<uint64_t>(ws, L.dlook), h, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess && nbars > 0) e = run_h1(ws, H, n, k0, k1, v0, v1, h, cpref, h, bars_dev, s, ev[2], ev[3]);
    if (e == cudaSuccess && nbars <= 0) e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess && nbars <= 0) e = cudaEventRecord(ev[3], s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4], s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
    for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
    uint64_t cnt[7] = {0, 0, 0, 0, 0, 0, 0};
    int32_t status = PH0_OK;
    if (e == cudaSuccess) e = cudaMemcpy(&status, &h->status, sizeof(status), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nbars > 0) e = h1_counters(ws, H, n, cnt);
    if (e != cudaSuccess) return PH0_ECUDA;
    if (status == PH0_OK && nbars > 0 && (int64_t(cnt[0]) != nbars || int64_t(cnt[6]) != H.T))
        status = PH0_EINTERNAL;
    if (stats) {
        stats->n_bars = nbars > 0 ? int64_t(cnt[0]) : 0;
        stats->n_triangles = nbars > 0 ? int64_t(cnt[6]) : H.T;
        stats->apparent = int64_t(cnt[1]);
        stats->reduced = int64_t(cnt[2]);
        stats->additions = int64_t(cnt[3]);
        stats->max_column = int64_t(cnt[4]);
        stats->pool_entries = int64_t(cnt[5]);
        stats->edges_ms = ms[0];
        stats->scan_ms = ms[1];
        stats->reduce_ms = ms[2];
        stats->emit_ms = ms[3];
    }
    return status;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point.  Some callers cannot call cudaMalloc (or any
// allocator) at the point where they need barcodes: latency-critical loops
// where an allocation could synchronize the device or take a driver lock,
// and hosts that own all device memory through their own pool and forbid
// raw allocations.  For clouds small enough to fit, this entry point takes
// its workspace from a fixed array in the library's device memory instead of
// from the caller.  It waits for its stream before returning, so it is not
// meant for stream capture.
// ---------------------------------------------------------------------------
namespace ph0 {
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB, held by every GPU that loads the library
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
// Device address of the array per device, looked up once per device and
// process; a cudaDeviceReset() of the device makes it stale.
void *g_noalloc_addr[kNoAllocMaxDevices] = {};
}  // namespace
}  // namespace ph0

static __device__ __align__(256) unsigned char g_noalloc_scratch[ph0::kNoAllocScratchBytes];

extern "C" int ph0_barcodes_noalloc(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                                    ph0_bar *bars_dev, ph0_inf_bar *inf_dev, void *stream) {
    int rc = check_sizes(n, d, ld);
    if (rc != PH0_OK) return rc;
    if (!pts_dev || (n > 1 && !bars_dev)) return PH0_EINVAL;
    if (!aligned(pts_dev, 4) || !aligned(bars_dev, 8) || !aligned(inf_dev, 8)) return PH0_EINVAL;
    const Layout L(n, d);
    if (L.total > kNoAllocScratchBytes) return PH0_ETOOBIG;
    {  // it waits for its stream, which a capture forbids: refuse before queueing anything
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess) return PH0_ECUDA;
        if (cs != cudaStreamCaptureStatusNone) return PH0_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PH0_ECUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return PH0_EINVAL;
    void *ws = nullptr;
    {
        // once per device, with that device current: the device address of
        // the array (its host-side name is not a device pointer)
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PH0_ECUDA;
            g_noalloc_addr[dev] = p;
        }
        ws = g_noalloc_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Header *h = at<Header>(ws, L.hdr);
    uint64_t *k0 = at<uint64_t>(ws, L.key[0]), *k1 = at<uint64_t>(ws, L.key[1]);
    uint32_t *v0 = at<uint32_t>(ws, L.val[0]), *v1 = at<uint32_t>(ws, L.val[1]);
    uint32_t *cpref = at<uint32_t>(ws, L.cpref);
    // the array keeps the previous call's contents: begin_call zeroes the
    // header and the first look-back buffer, and every later stage clears or
    // overwrites what it reads before reading it
    const Tune t(nullptr);
    cudaError_t e = begin_call(ws, L, s);
    if (e == cudaSuccess) e = launch_dist(pts_dev, n, d, ld, k0, v0, h, s);
    if (e == cudaSuccess) e = sort_whole(ws, L, pts_dev, n, d, ld, t, s);
    if (e == cudaSuccess) e = launch_dedupe_scan(cpref, L.m, at<uint64_t>(ws, L.dlook), h, s);
    if (e == cudaSuccess) e = reduce_and_emit(ws, L, n, v0, v1, k0, k1, h, nullptr, cpref, bars_dev, inf_dev, s);
    // the status word is read on the caller's stream (a plain copy would go
    // through the legacy default stream and wait for other blocking streams)
    int32_t status = PH0_OK;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &h->status, sizeof(status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? status : PH0_ECUDA;
}
