// k_small.cu -- the whole barcode path for a small cloud in one CTA, and many
// small clouds in one launch (Rawson, Sec. 2; Sec. 4 steps 1-5).
//
// A persistent kernel takes clouds from a task table (atomic counter); one
// CTA computes a cloud entirely in shared memory:
//   1. all E = n(n-1)/2 squared distances (the same rounded binary64 sequence
//      as k_dist: squares formed exactly with integers and sums on the
//      binary64 units when the cloud's coordinates fit 52 bits per dimension,
//      else all on the binary64 units),
//   2. a bitonic sort of (distance bits, edge id) -- the same total order
//      (distance, u, v) as the radix sort,
//   3. de-duplication: a = inclusive count of new distances (block scan),
//   4-5. the column reduction by component roots over chunks of the sorted
//      edges with the same claim rule as k_reduce (a column that holds the
//      claim of its larger root H is nonzero with pivot H), stopping at n-1
//      pivots, then the bars in filtration order.
// Results are bit-identical to the multi-kernel path.
#include "emu64.cuh"
#include "ph0_common.cuh"

namespace ph0 {

constexpr int kSmallThreads = 512;
constexpr int kSmallMaxN = 180;                       // E <= 16110
constexpr int kSmallSort = 16384;                     // power of two >= max E
constexpr int kSmallMaxD = 64;


struct SmallSmem {
    uint64_t key[kSmallSort];
    uint16_t idx[kSmallSort];
    uint16_t a[kSmallSort];
    uint16_t comp[256], parent[256];
    uint32_t res[256];
    uint32_t kpos[256];
    uint16_t klow[256];
    int32_t g[kSmallMaxD], lo[kSmallMaxD], hi[kSmallMaxD];
    uint32_t narrow[(kSmallMaxD + 31) / 32];
    uint32_t warp_sum[kSmallThreads / 32 + 1];
    uint32_t npiv, left, task, fixed_ok, bad;
};

__device__ __forceinline__ void edge_of(int e, int n, int &u, int &v) {
    // u = largest row with start(u) <= e, start(u) = u(2n-u-1)/2
    const double b = 2.0 * n - 1.0;
    int r = int((b - sqrt(b * b - 8.0 * double(e))) * 0.5);
    if (r < 0) r = 0;
    if (r > n - 2) r = n - 2;
    while (r > 0 && r * (2 * n - r - 1) / 2 > e) --r;
    while (r < n - 2 && (r + 1) * (2 * n - r - 2) / 2 <= e) ++r;
    u = r;
    v = e - r * (2 * n - r - 1) / 2 + r + 1;
}

__device__ __forceinline__ uint16_t small_find(uint16_t *par, uint16_t x) {
    for (;;) {
        const uint16_t p = par[x];
        if (p == x) return x;
        const uint16_t g = par[p];
        par[x] = g;
        x = g;
    }
}

__device__ void small_cloud(const SmallTask &T, SmallSmem &S) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = T.n, d = T.d;
    const int E = n * (n - 1) / 2;
    // ---- per dimension: bit range of the coordinates (fixed-point check) ----
    for (int k = tid; k < d; k += kSmallThreads) {
        S.lo[k] = 1 << 30;
        S.hi[k] = -(1 << 30);
    }
    if (tid == 0) S.bad = 0;
    __syncthreads();
    for (int i = tid; i < n * d; i += kSmallThreads) {
        const int p = i / d, k = i % d;
        const uint32_t b = __float_as_uint(T.pts[int64_t(p) * T.ld + k]);
        if ((b & 0x7f800000u) == 0x7f800000u) {
            S.bad = 1;
        } else if (b & 0x7fffffffu) {
            int32_t l, h;
            emu::bit_range_f32(b, l, h);
            atomicMin(&S.lo[k], l);
            atomicMax(&S.hi[k], h);
        }
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t ok = 1;
        for (int w = 0; w < (kSmallMaxD + 31) / 32; ++w) S.narrow[w] = 0;
        for (int k = 0; k < d; ++k) {
            const bool zero = S.lo[k] == (1 << 30);
            S.g[k] = zero ? 0 : S.lo[k];
            const int span = zero ? 0 : S.hi[k] + 1 - S.lo[k];
            if (span > 52) ok = 0;
            if (span <= 30) S.narrow[k >> 5] |= 1u << (k & 31);  // 32-bit differences
        }
        S.fixed_ok = ok;
    }
    __syncthreads();
    const bool fixed = S.fixed_ok != 0;
    if (fixed)
        for (int i = tid; i < n * d; i += kSmallThreads) {
            const int p = i / d, k = i % d;
            T.fixed[int64_t(k) * n + p] = emu::to_fixed(__float_as_uint(T.pts[int64_t(p) * T.ld + k]), S.g[k]);
        }
    __syncthreads();

    // ---- 1. distances (pad the sort array with the largest key) ----
    for (int e = tid; e < kSmallSort; e += kSmallThreads) {
        uint64_t kb = ~0ull;
        if (e < E) {
            int u, v;
            edge_of(e, n, u, v);
            if (fixed) {
                kb = emu::sq_dist_mixed(T.fixed + u, T.fixed + v, S.g, d, n, n, S.narrow);
            } else {
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double t = __dsub_rn(double(T.pts[int64_t(v) * T.ld + k]),
                                               double(T.pts[int64_t(u) * T.ld + k]));
                    s = __dadd_rn(s, __dmul_rn(t, t));
                }
                kb = uint64_t(__double_as_longlong(s));
            }
        }
        S.key[e] = kb;
        S.idx[e] = uint16_t(e < E ? e : 0xffff);
    }
    __syncthreads();

    // ---- 2. bitonic sort of (key, edge id) ----
    int M = 2;
    while (M < E) M <<= 1;
    for (int size = 2; size <= M; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < M / 2; i += kSmallThreads) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t ka = S.key[lo], kb = S.key[hi];
                const uint16_t ia = S.idx[lo], ib = S.idx[hi];
                const bool gt = ka > kb || (ka == kb && ia > ib);
                if (gt == up) {
                    S.key[lo] = kb;
                    S.key[hi] = ka;
                    S.idx[lo] = ib;
                    S.idx[hi] = ia;
                }
            }
            __syncthreads();
        }
    }

    // ---- 3. a = inclusive count of new distances (block scan over chunks) ----
    constexpr int IT = kSmallSort / kSmallThreads;  // 32 consecutive items per thread
    uint32_t cnt = 0;
    const int first = tid * IT;
    for (int j = 0; j < IT; ++j) {
        const int i = first + j;
        if (i < E && (i == 0 || S.key[i] != S.key[i - 1])) ++cnt;
    }
    uint32_t inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) S.warp_sum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = kSmallThreads / 32;
        const uint32_t w = lane < NW ? S.warp_sum[lane] : 0u;
        uint32_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) S.warp_sum[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = inc - cnt + S.warp_sum[warp];
    for (int j = 0; j < IT; ++j) {
        const int i = first + j;
        if (i < E) {
            if (i == 0 || S.key[i] != S.key[i - 1]) ++run;
            S.a[i] = uint16_t(run);
        }
    }
    // ---- 4-5. reduction over chunks of sorted edges ----
    for (int v = tid; v < 256; v += kSmallThreads) {
        S.comp[v] = uint16_t(v);
        S.parent[v] = uint16_t(v);
        S.res[v] = 0xffffffffu;
    }
    if (tid == 0) S.npiv = 0;
    __syncthreads();
    for (int c = 0; c < E && S.npiv < uint32_t(n - 1); c += kSmallThreads) {
        const int p = c + tid;
        int u = 0, v = 0;
        bool act = false;
        if (p < E) {
            edge_of(S.idx[p], n, u, v);
            act = S.comp[u] != S.comp[v];  // snapshot of the chunk start
        }
        for (;;) {
            uint16_t ra = 0, rb = 0;
            if (act) {
                ra = small_find(S.parent, S.comp[u]);
                rb = small_find(S.parent, S.comp[v]);
                if (ra == rb) {
                    act = false;
                } else {
                    atomicMin(&S.res[ra], uint32_t(p));
                    atomicMin(&S.res[rb], uint32_t(p));
                }
            }
            if (tid == 0) S.left = 0;
            __syncthreads();
            if (act) {
                const uint16_t lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
                if (S.res[hi] == uint32_t(p)) {  // holds its larger root: pivot hi
                    S.parent[hi] = lo;
                    const uint32_t j = atomicAdd(&S.npiv, 1u);
                    S.kpos[j] = uint32_t(p);
                    S.klow[j] = hi;
                    act = false;
                } else {
                    atomicAdd(&S.left, 1u);
                }
            }
            __syncthreads();
            for (int r = tid; r < 256; r += kSmallThreads) S.res[r] = 0xffffffffu;
            const uint32_t left = S.left;
            __syncthreads();
            if (left == 0) break;
        }
        for (int w = tid; w < n; w += kSmallThreads) S.comp[w] = small_find(S.parent, S.comp[w]);
        __syncthreads();
    }
    // ---- bars in filtration order ----
    const int nb = int(S.npiv);
    for (int j = tid; j < nb; j += kSmallThreads) {
        const uint32_t p = S.kpos[j];
        int rank = 0;
        for (int q = 0; q < nb; ++q) rank += S.kpos[q] < p;
        int u, v;
        edge_of(S.idx[p], n, u, v);
        ph0_bar b;
        b.u = u;
        b.v = v;
        b.a = S.a[p];
        b.low = S.klow[j];
        b.order = int64_t(p);
        b.death_sq = __longlong_as_double((long long)S.key[p]);
        b.death = __dsqrt_rn(b.death_sq);
        T.bars[rank] = b;
    }
    if (tid == 0) {
        // the bar that never dies: the vertex that is no pivot row (XOR of
        // 0..n-1 and of the n-1 pivot rows)
        uint32_t x = 0;
        for (int w = 0; w < n; ++w) x ^= uint32_t(w);
        for (int j = 0; j < nb; ++j) x ^= S.klow[j];
        const bool ok = nb == n - 1 && x < uint32_t(n);
        T.status[1] = ok ? int32_t(x) : 0;
        T.status[0] = S.bad ? PH0_ENONFINITE : (ok ? PH0_OK : PH0_EINTERNAL);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSmallThreads, 1)
k_small(const SmallTask *__restrict__ tasks, const int32_t *__restrict__ ntasks, uint32_t *counter) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    SmallSmem &S = *reinterpret_cast<SmallSmem *>(s_raw);
    for (;;) {
        if (threadIdx.x == 0) S.task = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t t = S.task;
        __syncthreads();
        if (t >= uint32_t(*ntasks)) break;
        const SmallTask task = tasks[t];
        if (task.n < 2) {
            if (threadIdx.x == 0) {
                task.status[0] = PH0_OK;
                task.status[1] = 0;
            }
            continue;
        }
        small_cloud(task, S);
    }
}

size_t small_smem() { return sizeof(SmallSmem); }

int small_max_n() { return kSmallMaxN; }
int small_max_d() { return kSmallMaxD; }

// One launch over the task table; `counter` must be zero (reset here).  The
// task count is read on the device so that a captured launch can be replayed
// for any batch.
cudaError_t prepare_small_kernel() {
    return cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(SmallSmem)));
}

cudaError_t launch_small(const SmallTask *tasks, const int32_t *ntasks_dev, uint32_t *counter, int grid,
                         cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_small<<<grid, kSmallThreads, sizeof(SmallSmem), s>>>(tasks, ntasks_dev, counter);
    return cudaGetLastError();
}

}  // namespace ph0
