// k_dist.cu -- step 1 of the barcode path: all pairwise squared distances
// (Rawson, Sec. 2 "calculate the distance between every pair of points";
// Sec. 3 notes the factor-2 saving from symmetry; Sec. 4 step 1).
//
// One CTA per tile of the upper triangle: a block of BT row points (u) by a
// block of BT column points (v), v-block >= u-block.  The binary32
// coordinates of both blocks are staged in shared memory as binary64,
// dimension-major, so that a warp reads 32 consecutive v (no bank conflicts)
// and the u coordinate is a broadcast.  A warp writes 32 consecutive edges of
// one row u, so the key (8 B) and val (4 B) stores are coalesced.
//
// Fused: the histogram of the low 8 key bits (radix pass 0), the min and max
// key (the sort's bit range), and the finiteness check of the input.
#include "ph0_common.cuh"

namespace ph0 {

constexpr int kDistThreads = 256;

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

__global__ void __launch_bounds__(kDistThreads)
k_dist(const float *__restrict__ pts, int n, int d, int64_t ld, int bt,
       uint64_t *__restrict__ key, uint32_t *__restrict__ val, Header *__restrict__ h) {
    extern __shared__ double s_coord[];  // [d][bt] for u block, then [d][bt] for v block
    __shared__ uint32_t s_hist[kRadix];
    __shared__ uint64_t s_min[kDistThreads / 32], s_max[kDistThreads / 32];

    const int64_t T = (n + bt - 1) / bt;
    int64_t bi, bj;
    tile_coords(blockIdx.x, T, bi, bj);
    const int u0 = int(bi) * bt, v0 = int(bj) * bt;
    double *su = s_coord;
    double *sv = s_coord + size_t(d) * bt;

    for (int b = threadIdx.x; b < kRadix; b += blockDim.x) s_hist[b] = 0;
    bool bad = false;
    for (int idx = threadIdx.x; idx < bt * d; idx += blockDim.x) {
        int p = idx / d, k = idx % d;
        float xu = (u0 + p < n) ? pts[int64_t(u0 + p) * ld + k] : 0.0f;
        float xv = (v0 + p < n) ? pts[int64_t(v0 + p) * ld + k] : 0.0f;
        bad |= !isfinite(xu) || !isfinite(xv);
        su[k * bt + p] = double(xu);
        sv[k * bt + p] = double(xv);
    }
    if (bad) set_status(h, PH0_ENONFINITE);
    __syncthreads();

    uint64_t kmin = ~0ull, kmax = 0;
    const int j = threadIdx.x % bt;                // column within the tile
    const int rows_per_pass = blockDim.x / bt;     // bt divides blockDim (bt <= 128)
    const int v = v0 + j;
    for (int i = threadIdx.x / bt; i < bt; i += rows_per_pass) {
        const int u = u0 + i;
        if (u < v && v < n) {
            double s = sq_dist_f64(su, sv, d, bt, i, j);
            uint64_t kb = uint64_t(__double_as_longlong(s));
            int64_t e = edge_index(n, u, v);
            key[e] = kb;
            val[e] = (uint32_t(u) << 16) | uint32_t(v);
            atomicAdd(&s_hist[kb & (kRadix - 1)], 1u);
            kmin = kb < kmin ? kb : kmin;
            kmax = kb > kmax ? kb : kmax;
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
    for (int b = threadIdx.x; b < kRadix; b += blockDim.x)
        if (s_hist[b]) atomicAdd(&h->hist[0][b], s_hist[b]);
}

// Tile edge for dimension d: the two staged blocks must fit in shared memory.
int dist_tile(int d) {
    int bt = 128;
    while (bt > 8 && size_t(2) * bt * d * sizeof(double) > 160 * 1024) bt /= 2;
    return bt;
}

cudaError_t launch_dist(const float *pts, int64_t n, int32_t d, int64_t ld, uint64_t *key,
                        uint32_t *val, Header *h, cudaStream_t s) {
    if (n < 2) return cudaSuccess;
    const int bt = dist_tile(d);
    const size_t smem = size_t(2) * bt * d * sizeof(double);
    if (smem > 160 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_dist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         160 * 1024);
    if (e != cudaSuccess) return e;
    const int64_t T = (n + bt - 1) / bt;
    const int64_t tiles = T * (T + 1) / 2;
    k_dist<<<unsigned(tiles), kDistThreads, smem, s>>>(pts, int(n), int(d), ld, bt, key, val, h);
    return cudaGetLastError();
}

}  // namespace ph0
