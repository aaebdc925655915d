// k_backward.cu -- gradient of the finite death values with respect to the
// points, for fixed killing edges.  The paper has no counterpart; the
// forward map it defines (Sec. 2: death of bar i = distance of its killing
// edge) is piecewise smooth in the points, with
//   d death_i / d x_u =  (x_u - x_v) / death_i,
//   d death_i / d x_v = -(x_u - x_v) / death_i.
// The scatter is accumulated in binary64 and cast to binary32 once.
#include "ph0_common.cuh"

namespace ph0 {

__global__ void k_backward_scatter(const float *__restrict__ pts, int64_t n, int d, int64_t ld,
                                   const ph0_bar *__restrict__ bars, int64_t nb,
                                   const double *__restrict__ dl, double *__restrict__ acc) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t i = t / d;
    const int k = int(t % d);
    if (i >= nb) return;
    const ph0_bar b = bars[i];
    if (!(b.death > 0.0)) return;
    const double diff = __dsub_rn(double(pts[int64_t(b.u) * ld + k]), double(pts[int64_t(b.v) * ld + k]));
    const double g = __ddiv_rn(__dmul_rn(dl[i], diff), b.death);
    atomicAdd(acc + int64_t(b.u) * d + k, g);
    atomicAdd(acc + int64_t(b.v) * d + k, -g);
}

__global__ void k_backward_cast(const double *__restrict__ acc, float *__restrict__ grad, int64_t count) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x)
        grad[i] = __double2float_rn(acc[i]);
}

int sm_count();

cudaError_t launch_backward(const float *pts, int64_t n, int32_t d, int64_t ld, const ph0_bar *bars,
                            int64_t nb, const double *dl, float *grad, double *acc, cudaStream_t s) {
    const int64_t count = n * int64_t(d);
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * size_t(count), s);
    if (e != cudaSuccess) return e;
    const int64_t work = nb * int64_t(d);
    if (work > 0) {
        k_backward_scatter<<<unsigned((work + 255) / 256), 256, 0, s>>>(pts, n, d, ld, bars, nb, dl, acc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int64_t blocks = (count + 255) / 256;
    const int64_t cap = int64_t(sm_count()) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_backward_cast<<<unsigned(blocks), 256, 0, s>>>(acc, grad, count);
    return cudaGetLastError();
}

}  // namespace ph0
