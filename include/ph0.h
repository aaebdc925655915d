/*
 * ph0.h -- C ABI of the GB300 (sm_103a) 0th persistent homology barcode
 * library, libph0.so.
 *
 * Problem (Rawson, "Linear Run Time of Persistent Homology Computation with
 * GPU Parallelization", Sec. 2): given N data points X in E^d, compute the
 * barcodes of the Vietoris-Rips filtration in dimension 0.  Every vertex is
 * born at 0 (Sec. 1: near epsilon = 0 the complex has a vertex per point and
 * no edges); an edge that joins two disconnected subgraphs ends one class
 * (Sec. 1).  The path has the paper's five steps (Sec. 2; Sec. 4 steps 1-5):
 *   1. the N(N-1)/2 pairwise distances,
 *   2. a sort of the edges by distance,
 *   3. de-duplication into D and the 1-based index a of each edge in D,
 *   4. the vertex-by-edge boundary matrix M over F2[t], M(i,j) = t^a(j),
 *   5. column reduction of M; each remaining pivot entry t^b is a bar (0, b).
 *
 * Conventions fixed here where the paper is silent:
 *   - distances are computed squared, in binary64 from binary32 inputs, as
 *     s = 0; for k in 0..d-1: t = x[v,k] - x[u,k]; s = s + t*t, with every
 *     subtraction, product and sum rounded to nearest-even (no fused
 *     multiply-add); the distance is sqrt(s), a monotone map, so ties and
 *     order are those of s;
 *   - edges with equal distance are ordered by (u, v) lexicographically;
 *   - the pivot ("low") of a column is its largest row index; then the single
 *     bar that never dies sits on vertex 0.
 *
 * Memory: every pointer named *_dev is CUDA device memory (or managed memory)
 * owned by the caller.  The workspace entry points allocate nothing: `ws` is
 * a caller-owned device workspace of at least ph0_workspace_bytes() bytes,
 * 256-byte aligned; one workspace serves one call in flight at a time.  The
 * library keeps two kinds of state of its own: the 16 MiB device array of
 * ph0_barcodes_noalloc() (one per GPU that loads the library, held until the
 * process exits, plus a host-side cache of its device address), and the
 * device arena and pinned pool a serving context (ph0_ctx_create) allocates
 * and owns.  `stream` is a cudaStream_t passed as void* (NULL =
 * the legacy default stream).  All compute calls are asynchronous on
 * `stream`: they return host-detected errors immediately and leave
 * device-detected errors (non-finite input, a bounded wait that timed out) in
 * the workspace, where ph0_finish() reads them.
 *
 * Limits: 1 <= N <= 131071 for ph0_barcodes(), ph0_barcodes_tuned() and
 * ph0_workspace_bytes() (E = N(N-1)/2 < 2^33 edges: above 92,682 points the
 * records carry bit 32 of the edge index in the key's sign bit, the sort takes
 * two halves of fewer than 2^32 edges and merges them, and the reduction scans
 * at most the first 2^32 - 4096 sorted edges, enough for the n-1 killing edges
 * of any cloud whose last merge comes before that position: PH0_ETOOBIG
 * otherwise; the N = 100,000 workspace is about 132 GB), 1 <= N <= 92681 for
 * the other whole-path entry points (E < 2^32), 1 <= N <= 65535 for the step
 * entry points (whose edge records pack (u << 16) | v), 1 <= d <= 1024.
 */
#ifndef PH0_H
#define PH0_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PH0_OK = 0,
    PH0_EINVAL = 1,      /* bad argument: n < 1, d < 1, ld < d, null or misaligned pointer */
    PH0_ENONFINITE = 2,  /* a coordinate is NaN or +-Inf (detected on the device) */
    PH0_ETOOBIG = 3,     /* n above the entry point's limit (see Limits) or d > 1024 */
    PH0_ENOMEM = 4,      /* workspace smaller than ph0_workspace_bytes() */
    PH0_ETIMEOUT = 5,    /* a bounded device-side wait gave up (the kernel returned cleanly) */
    PH0_ECUDA = 6,       /* a CUDA runtime call failed */
    PH0_EBUSY = 7,       /* the resource is in use */
    PH0_EINTERNAL = 8    /* an internal consistency check failed */
} ph0_status;

/* One finite bar (birth 0).  40 bytes, naturally aligned. */
typedef struct {
    int32_t u, v;      /* killing edge, u < v                                   */
    uint32_t a;        /* 1-based index of its squared distance in D (the b of t^b) */
    int32_t low;       /* pivot row of its reduced column: the vertex whose class
                          this edge ends (max of the two component minima)       */
    int64_t order;     /* 0-based position of the edge in the sorted edge list  */
    double death_sq;   /* binary64 squared distance of the edge                 */
    double death;      /* sqrt(death_sq), IEEE round to nearest                 */
} ph0_bar;

/* The bar that never dies (birth 0, death +inf): the class of the vertex
 * that is the pivot row of no reduced column.  With the pivot convention
 * above (largest row) this is always vertex 0; the kernels derive it from
 * the pivot rows of the n-1 finite bars.  24 bytes. */
typedef struct {
    int32_t vertex;    /* representative vertex (the unpaired row)         */
    int32_t _pad;
    double birth;      /* 0                                                */
    double death;      /* +inf                                             */
} ph0_inf_bar;

/* Counters of the last call on a workspace, read back by ph0_finish(). */
typedef struct {
    int32_t status;          /* ph0_status of the device-side work            */
    int32_t sort_passes;     /* radix passes of the key range's plan (4 for
                              * the packed sort of sort_form 1; else the     *
                              * whole path runs those from slot 2 on)         */
    int32_t key_bits;        /* varying key bits sorted                       */
    int32_t windows;         /* reduction windows processed                   */
    int64_t n_distinct;      /* |D|                                           */
    int64_t edges_scanned;   /* sorted edges examined before the early exit   */
    int64_t candidates;      /* edges that reached the pivot-claiming rounds  */
    int64_t rounds;          /* pivot-claiming rounds over all windows        */
    int64_t n_bars;          /* finite bars written                           */
    int64_t dist_tiles;      /* distance tiles                                */
    int64_t dist_tiles_int;  /* ... of which computed on the integer path     */
    int64_t sorted_edges;    /* edges sorted: n(n-1)/2, or the prefix sorted by
                                ph0_barcodes_early (n_distinct then counts the
                                distinct values of that prefix)               */
    int32_t inf_vertex;      /* vertex of the bar that never dies (0)         */
    int32_t claim_rounds_max;/* most grid-wide claim rounds in one window     */
    int64_t claim_attempts;  /* atomic claims issued in the reduction (two per
                                candidate column and round)                   */
    int32_t sort_form;       /* which sort gave the whole path's order: 0 the
                                short sort of (key, value) records, 1 the packed
                                sort of 64-bit words, 2 the complete sort run
                                after a fix-up met a group it cannot order    */
    int32_t _pad;
} ph0_stats;

/* Human-readable name of a status code (static storage). */
const char *ph0_strerror(int status);

/* Library ABI version (incremented on any incompatible change). */
int32_t ph0_abi_version(void);

/* Bytes of workspace ph0_barcodes() and the step entry points need for a
 * cloud of n points in dimension d (0 on invalid sizes). */
size_t ph0_workspace_bytes(int64_t n, int32_t d);

/* Whole path, steps 1-5 (Sec. 2; Sec. 4 steps 1-5).
 *   pts_dev   float32 [n, ld] row-major, the first d columns are used
 *   bars_dev  ph0_bar [n-1] output, in filtration order (increasing `order`)
 *   inf_dev   ph0_inf_bar [1] output (device memory), the bar that never
 *             dies: (0, +inf) on the vertex that is no pivot row; may be
 *             NULL (ph0_finish() also reports the vertex)
 * Asynchronous; call ph0_finish() for the device status. */
int ph0_barcodes(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                 ph0_bar *bars_dev, ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes,
                 void *stream);

/* Tuning of the kernels (chosen per dimension by the autotuner in the Python
 * package; a NULL pointer or a field set to -1 selects the built-in choice).
 * None changes any result bit. */
typedef struct {
    int32_t dist_split16;   /* of every 16 rows of a distance tile, how many compute the
                               running sum on the binary64 units (the rest all in integers);
                               0..16, built-in 16                                        */
    int32_t dist_tile;      /* points per side of a distance tile: 32, 64 or 128; built-in
                               128 (smaller when the tile would not fit shared memory)    */
    int32_t sort_top_bits;  /* width of the single top radix pass: 8 or 9 (a wider top
                               part takes two passes of 8); built-in 9                   */
    int32_t reduce_spin_limit; /* test aid: polls before a grid-barrier wait of the
                               reduction gives up with PH0_ETIMEOUT (the kernel then
                               returns and the workspace stays usable); -1 = built-in
                               (2^24, about a second); 0 gives up at the first poll    */
    int32_t wide_ids;       /* 1: edge records hold the edge's lexicographic index
                               instead of (u << 16) | v, as they always do above 65535
                               points (test aid: runs the large-cloud form on any n);
                               -1 or 0: only above 65535 points                          */
    int32_t early_rounds;   /* ph0_barcodes_early_tuned: 1 always sorts the prefix in
                               rounds, 0 never (the whole path); -1 built-in: rounds
                               only for clouds of at least 2^27 edges (n >= 16385)     */
    int32_t split_sort;     /* 1: the whole path sorts the edges as two halves merged, as
                               it always does above 2^32 - 4096 edges (test aid: runs that
                               form on any n); -1 or 0: only above                       */
    int32_t packed_sort;    /* the whole path's packed sort (each edge one 64-bit word:
                               compact top part, key bits 22..47, (u << 15) | v; four
                               passes; clouds of at most 32768 points whose keys' top
                               part takes at most 256 values, else the short sort runs;
                               not with wide_ids = 1): 1 on any such cloud, 0 never,
                               -1 built-in: from 2^22 edges (n >= 2897) up to n = 32768
                               in dimension 4 and up                                   */
} ph0_tuning;

/* Early-terminating whole path (the paper has no counterpart; it exploits
 * that the reduction of Sec. 2 reads the sorted edges only up to the last
 * killing edge).  Same arguments and results as ph0_barcodes(), bit for bit:
 * the same n-1 bars (killing edges, positions `order` in the full sorted
 * edge list, indices a, deaths).  Instead of sorting all n(n-1)/2 edges it
 * sorts a prefix of the edge order: it histograms the squared distances,
 * partitions the edges stably into classes of consecutive distance ranges
 * (the first 2%, 8%, 25%, 45% of the edges, cumulative, then the rest), then
 * sorts one class after the other into the prefix and runs the reduction on
 * the prefix, until it holds n-1 pivots.  The prefix holds every killing
 * edge exactly when the reduction finds n-1 pivots in it, so the result
 * never differs.  Synchronous: waits for `stream` between rounds and returns the
 * device status (as ph0_finish() would); ph0_finish() reports the prefix
 * length in sorted_edges.  Fastest when the last killing edge comes early in
 * the edge order (clustered or uniform clouds). */
int ph0_barcodes_early(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                       ph0_bar *bars_dev, ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes,
                       void *stream);

/* ph0_barcodes_early() with a choice of path (tuning->early_rounds).  Built
 * in (NULL or -1): below 2^27 edges the whole path runs instead of the
 * rounds, because there the rounds' fixed cost (a host wait per round, the
 * histogram and the class pass) exceeds what skipping the sort of the
 * suffix saves (a 4096-point cloud: 3.2 ms in rounds against 1.2 ms whole);
 * above 65535 points the whole path always runs.  Same results either way.
 * stats (may be NULL) receives the counters, as from ph0_finish(). */
int ph0_barcodes_early_tuned(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                             ph0_bar *bars_dev, ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes,
                             void *stream, const ph0_tuning *tuning, ph0_stats *stats);

/* ph0_barcodes() with explicit tuning (NULL = built-in). */
int ph0_barcodes_tuned(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                       ph0_bar *bars_dev, ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes,
                       void *stream, const ph0_tuning *tuning);

/* Device time of each stage of one ph0_barcodes_profiled() call, from CUDA
 * events recorded on the caller's stream between the stages (milliseconds). */
typedef struct {
    float total_ms;          /* first to last event                          */
    float dist_ms;           /* step 1: distance kernel                       */
    float sort_ms;           /* step 2: all radix passes                      */
    float pass_ms[8];        /* step 2: each pass (0 for passes not needed; the
                                packed sort's four passes in slots 0-3)       */
    float dedupe_ms;         /* step 3                                        */
    float reduce_ms;         /* steps 4-5: pivot claiming                     */
    float emit_ms;           /* ordering of the pivot columns and bar output  */
    float fixup_ms;          /* step 2: the sort's fix-up of the groups its
                                passes leave (and the fallback, if taken; for
                                the packed sort also the short sort's gated
                                launches)                                     */
} ph0_profile;

/* ph0_barcodes() with a CUDA event between stages; waits for the stream and
 * fills `prof` (tracing aid: same kernels, same results). */
int ph0_barcodes_profiled(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                          ph0_bar *bars_dev, ph0_inf_bar *inf_dev, void *ws, size_t ws_bytes,
                          void *stream, const ph0_tuning *tuning, ph0_profile *prof);

/* Waits for `stream`, then returns the device status of the last call made
 * with `ws` and, when stats != NULL, its counters. */
int ph0_finish(const void *ws, void *stream, ph0_stats *stats);

/* Byte offset, within a workspace, of the int32 ph0_status of the last
 * call's device-side work (the word ph0_finish() reads; the same for every n
 * and d).  A caller that must not wait between calls, such as one replaying
 * a CUDA graph of many calls, can copy these words from all its workspaces
 * at once and check them afterwards.  No counterpart in the paper. */
size_t ph0_status_offset(void);

/* Tracing aid: copies to `out` (host, max_windows x 12 uint64) the per-window
 * records of the last reduction run on `ws` for a cloud of (n, d):
 * {first position, window size, candidates, grid-wide rounds, shared-memory
 *  rounds, pivots so far, then globaltimer stamps (ns): begin, filtered,
 *  grid rounds done, shared-memory rounds done, end}.  Unused records are 0.
 * Waits for `stream`. */
int ph0_trace_windows(const void *ws, int64_t n, int32_t d, void *stream, uint64_t *out,
                      int32_t max_windows);

/* ---- step entry points (each one step of the path, for testing and reuse) ---- */

/* Step 1 (Sec. 2: the distance of every pair of points; Sec. 4 step 1).
 * Writes, for every edge u<v at index e = u*(2n-u-1)/2 + (v-u-1)
 * (lexicographic order):
 *   key_dev[e] = bit pattern of the binary64 squared distance (uint64),
 *   val_dev[e] = (u << 16) | v.
 * key_dev: uint64 [E], val_dev: uint32 [E], E = n(n-1)/2, 16-byte aligned. */
int ph0_distances(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                  uint64_t *key_dev, uint32_t *val_dev,
                  void *ws, size_t ws_bytes, void *stream);

/* Step 2 (Sec. 2: the distances in increasing order; Sec. 4 step 2).  Stable sort
 * of the m (key, val) pairs by key, in place; keys are binary64 bit patterns
 * of non-negative numbers (unsigned order = numeric order).  Input in val
 * order gives the total order (distance, u, v).  m <= 2^31 - 1; `ws` must be
 * sized for some n with n(n-1)/2 >= m. */
int ph0_sort(uint64_t *key_dev, uint32_t *val_dev, int64_t m,
             void *ws, size_t ws_bytes, void *stream);

/* Step 3 (Sec. 2: D is the sorted distances without repeats, and a(j) is the
 * position, from 1 to |D|, of edge j's distance in D).
 *   key_sorted_dev  uint64 [m] sorted keys;  a_dev  uint32 [m] output. */
int ph0_dedupe(const uint64_t *key_sorted_dev, int64_t m, uint32_t *a_dev,
               void *ws, size_t ws_bytes, void *stream);

/* Steps 4-5 (Sec. 2: the matrix M of the edges and its column reduction; Sec. 4
 * steps 3-5).  Column p of M has the rows u_p, v_p of val_sorted_dev[p], both
 * t^a[p]; it is never materialised.  The columns are reduced in order with a
 * pivot table claimed by atomic priority (lower filtration position wins,
 * the loser retries), stopping once n-1 pivots exist.  Writes the n-1 bars
 * in filtration order.  Inputs: sorted val (uint32 [m]), a (uint32 [m]),
 * sorted key (uint64 [m]); m = n(n-1)/2. */
int ph0_reduce(int64_t n, const uint32_t *val_sorted_dev,
               const uint32_t *a_dev, const uint64_t *key_sorted_dev,
               ph0_bar *bars_dev, void *ws, size_t ws_bytes, void *stream);

/* ---- allocation-free variant (the paper has no counterpart) ----
 *
 * ph0_barcodes() for callers that cannot allocate device memory where they
 * need barcodes: latency-critical loops in which a cudaMalloc could
 * synchronize the device or take a driver lock, and hosts (frameworks with
 * their own caching allocator, embedded runtimes) whose device memory is all
 * owned by their own pool, so that a raw allocation would fail or fragment
 * it.  Instead of a caller workspace it uses a 16 MiB array in the library's
 * device memory (every GPU that loads the library holds it until the
 * process exits); the caller still passes the points and the outputs.
 * Clouds whose workspace would exceed 16 MiB (ph0_workspace_bytes(n, d) >
 * 16 MiB: n above 889 at d = 3, above 883 at d = 32) are rejected with
 * PH0_ETOOBIG before any work is queued.  It allocates nothing (no
 * cudaMalloc, cudaFree or allocating library call).
 *
 * Synchronous: it waits for `stream` and reads the device status back
 * before returning (as ph0_finish() would), so it cannot be recorded into a
 * CUDA graph: on a stream under capture it returns PH0_EINVAL before
 * anything is queued, and the caller's capture stays valid.  The first call on a device looks up the device address of the
 * array for that device (with that device current) and keeps it for the rest
 * of the process; after a cudaDeviceReset() of that device the kept address
 * is stale, so this entry point must not be called again in that process.
 * All calls share the one array per device, which keeps the last call's
 * contents (every stage clears what it needs zeroed): calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialized by
 * the caller. */
int ph0_barcodes_noalloc(const float *pts_dev, int64_t n, int32_t d, int64_t ld,
                         ph0_bar *bars_dev, ph0_inf_bar *inf_dev, void *stream);

/* ---- first homology (the extension the paper names, Sec. 1 and Sec. 4.2) ----
 *
 * The Vietoris-Rips 2-skeleton adds a triangle once its three edges are
 * present (Sec. 1, the recursive rule), at its diameter.  The edge-by-
 * triangle boundary matrix (entries t^a over F2[t], reducing like their F2
 * supports) is reduced left to right, triangles ordered by the position of
 * their diameter edge in the sorted edge order, then (u, v, w); each nonzero
 * reduced column pairs its low edge (a positive edge: one that closes a
 * cycle) with its triangle, the bar (a(edge), a(diameter)).  Every positive
 * edge is paired (the full simplex has no first homology): n(n-1)/2 - (n-1)
 * bars, zero-length ones included, in triangle order.  72 bytes. */
typedef struct {
    int32_t eu, ev;             /* birth edge, eu < ev                               */
    int32_t tu, tv, tw;         /* death triangle, tu < tv < tw                      */
    uint32_t birth_a, death_a;  /* 1-based indices in D of the birth edge and of the
                                   triangle's diameter edge                         */
    int32_t _pad;
    int64_t birth_order;        /* position of the birth edge in the sorted edge list */
    int64_t death_order;        /* position of the triangle's diameter edge          */
    int64_t death_rank;         /* position of the triangle in the triangle order    */
    double birth_sq, death_sq;  /* squared distances                                 */
} ph0_h1bar;

typedef struct {
    int64_t n_bars;             /* bars written: n(n-1)/2 - (n-1)                    */
    int64_t n_triangles;        /* n(n-1)(n-2)/6, from the per-edge triangle counts  */
    int64_t apparent;           /* bars of apparent pairs (no column addition)       */
    int64_t reduced;            /* columns reduced by additions (positive edges that
                                   are the diameter of no triangle)                 */
    int64_t additions;          /* column additions over all reduced columns         */
    int64_t max_column;         /* longest column met under reduction                */
    int64_t pool_entries;       /* triangle keys held by the reduced columns         */
    float edges_ms;             /* device time: steps 1-3 of dimension 0 (edge order) */
    float scan_ms;              /* ... positions, the triangles of each diameter     */
    float reduce_ms;            /* ... spanning forest and the reduced columns       */
    float emit_ms;              /* ... ranks in triangle order and the bars          */
} ph0_h1_stats;

/* Workspace bytes of ph0_h1() for n points in dimension d (0 on invalid sizes;
 * 3 <= n needs triangles, n <= 4096). */
size_t ph0_h1_workspace_bytes(int64_t n, int32_t d);

/* First-homology bars of the cloud (steps 1-3 of the dimension-0 path for the
 * edge order and a, then the pairs).  The pairs are computed through the
 * coboundary matrix, whose reduction has the same pairs: apparent pairs for
 * every edge that is the diameter of some triangle, the dimension-0 spanning
 * forest's columns cleared, the other columns reduced from the latest edge
 * down.  bars_dev: ph0_h1bar[n(n-1)/2 - (n-1)] (none for n <= 2), in triangle
 * order.  1 <= n <= 4096.  Synchronous: waits for `stream` and returns the
 * device status; PH0_ETOOBIG also when a column under reduction or the kept
 * reduced columns outgrow the workspace's room for them.  stats may be NULL. */
int ph0_h1(const float *pts_dev, int64_t n, int32_t d, int64_t ld, ph0_h1bar *bars_dev, void *ws,
           size_t ws_bytes, void *stream, ph0_h1_stats *stats);

/* ---- serving: a context that admits clouds as they arrive ----
 *
 * The paper computes one cloud at a time (Sec. 3.1, Sec. 4.1); this context
 * (no counterpart in the paper) keeps several clouds of any N and d on the GPU
 * at once.  It allocates one device arena (mem_budget) and one pinned host
 * pool (host_budget) when created, owns a worker thread, and admits queued
 * clouds in arrival order whenever their buffers fit and a slot is free.  Large
 * clouds run the same kernels as ph0_barcodes, each on its own stream; clouds
 * with n <= small_max_n (and d <= 64) are grouped into one launch of a fused
 * kernel that computes each cloud in one CTA (replayed from a captured CUDA
 * graph).  Every result equals what ph0_barcodes returns for that cloud. */
typedef struct ph0_ctx ph0_ctx;

typedef struct {
    size_t mem_budget;    /* device bytes for all clouds in flight (>= 1 MiB)       */
    size_t host_budget;   /* pinned host bytes for queued points and finished bars */
    int32_t streams;      /* large clouds in flight at once (1..64)                 */
    int32_t small_max_n;  /* batch clouds with n <= this (<= 180; 0 = never)        */
    int32_t batch_max;    /* clouds per fused launch                                */
    int32_t reserved;
} ph0_options;

typedef struct {
    uint64_t tag;         /* as submitted                                           */
    int32_t status;       /* ph0_status of this cloud                               */
    int32_t n, d;
    int32_t inf_vertex;   /* vertex of the bar that never dies (0)                  */
    int64_t n_bars;       /* n - 1                                                  */
    const ph0_bar *bars;  /* host memory owned by the context until ph0_release     */
    double submit_time;   /* steady-clock seconds at ph0_submit                     */
    double done_time;     /* steady-clock seconds when the worker saw it complete   */
} ph0_result;

/* Creates a context on the current device.  Returns PH0_ECUDA if the arena or
 * pool cannot be allocated. */
int ph0_ctx_create(const ph0_options *opt, ph0_ctx **ctx);

/* Queues a cloud (points copied from host memory at once, float32 [n, d]).
 * PH0_EBUSY: the host pool is full (poll and release first); PH0_ENOMEM: the
 * cloud can never fit mem_budget; PH0_EINVAL: the tag is still in use. */
int ph0_submit(ph0_ctx *ctx, const float *pts_host, int64_t n, int32_t d, uint64_t tag);

/* Returns up to `max` finished clouds (waiting up to wait_ms if none). */
int ph0_poll(ph0_ctx *ctx, ph0_result *out, int32_t max, int32_t *got, int32_t wait_ms);

/* Frees a returned result's host memory; the tag may then be reused. */
int ph0_release(ph0_ctx *ctx, uint64_t tag);

/* Waits for the work in flight and frees everything. */
int ph0_ctx_destroy(ph0_ctx *ctx);

/* ---- differentiation ---- */

/* Backward of death_i = |x_v - x_u| for fixed killing edges:
 *   grad[u] += g_i (x_u - x_v) / death_i,  grad[v] -= the same,
 * g_i = dl_ddeath_dev[i], in binary64, cast to float32 once at the end; a bar
 * of length 0 contributes 0.  grad_dev float32 [n, d] (dense, row-major) is
 * overwritten.  `ws` as for ph0_barcodes with the same n, d. */
int ph0_barcodes_backward(const float *pts_dev, int64_t n, int32_t d,
                          int64_t ld, const ph0_bar *bars_dev, int64_t n_bars,
                          const double *dl_ddeath_dev, float *grad_dev,
                          void *ws, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PH0_H */
