// k_prefix.cu -- the early-terminating path: sort only the prefix of the
// edge order that the reduction reads.
//
// The reduction walks the sorted edges in order and stops once n-1 pivots
// exist (Sec. 2: the bars are read off the reduced columns; a column after
// the last pivot cannot create one).  If the first P edges of the total order
// (d2, u, v) already give n-1 pivots, reducing them alone gives the same
// killing edges, positions, indices a (a counts distinct values from the
// bottom) and deaths as the whole path.  The first P edges are exactly the
// edges whose keys lie below a threshold, so the path
//   1. histograms the keys over their range (kPrefixBins bins, monotone),
//   2. partitions the edges stably (each class stays in (u, v) order) into a
//      few classes of consecutive bin ranges, which the host picks from the
//      histogram so that the first classes hold growing fractions of the
//      edges (ph0_barcodes_early); the partition is one radix pass whose
//      digit is the class (slot kClassSlot of k_sort.cu),
//   3. extends the sorted prefix class by class (the radix passes sort a
//      class in place) and runs the reduction on it, until it has n-1 pivots.
#include "ph0_common.cuh"

namespace ph0 {

struct PrefixBins {
    uint64_t kmin;
    int shift;
};

__device__ __forceinline__ PrefixBins prefix_bins(const Header *h) {
    return PrefixBins{h->kmin, prefix_shift(h->kmin, h->kmax)};
}

__device__ __forceinline__ uint32_t prefix_bin(uint64_t key, const PrefixBins &b) {
    return uint32_t(((key & kKeyBits) - b.kmin) >> b.shift);  // < kPrefixBins for kmin <= key <= kmax
}

// Step 1: bin counts of all m keys (grid-stride, shared-memory histogram).
__global__ void __launch_bounds__(256) k_prefix_hist(const uint64_t *__restrict__ keys, int64_t m,
                                                      const Header *h, uint32_t *__restrict__ bins) {
    __shared__ uint32_t s_bins[kPrefixBins];
    for (int i = threadIdx.x; i < kPrefixBins; i += blockDim.x) s_bins[i] = 0;
    __syncthreads();
    const PrefixBins b = prefix_bins(h);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint32_t bin = prefix_bin(keys[i], b);
        atomicAdd(&s_bins[bin < kPrefixBins ? bin : kPrefixBins - 1], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPrefixBins; i += blockDim.x)
        if (s_bins[i]) atomicAdd(&bins[i], s_bins[i]);
}

cudaError_t launch_prefix_hist(const uint64_t *keys, int64_t m, const Header *h, uint32_t *bins,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(uint32_t) * kPrefixBins, s);
    if (e != cudaSuccess || m <= 0) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (m + 255) / 256;
    const int64_t cap = int64_t(sms > 0 ? sms : 1) * 4;
    if (blocks > cap) blocks = cap;
    k_prefix_hist<<<unsigned(blocks), 256, 0, s>>>(keys, m, h, bins);
    return cudaGetLastError();
}

}  // namespace ph0
