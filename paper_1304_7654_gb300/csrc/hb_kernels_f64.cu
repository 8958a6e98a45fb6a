// FP64 instantiation of the tile, halo, init and force kernels, plus the
// precision-independent reduction and copy helpers.
#include "hb_kernels.cuh"
#define HB_T double
#include "hb_launch.inc"

namespace hbk {

// fixed-order FP64 finish of the per-tile norm partials: thread q < nv walks
// the tiles in order; the result is the RMS over cells and snapshots
__global__ void norm_finish_kernel(const double* partials, int ntiles, int nv, double inv_count,
                                   double* out, int* err) {
  __shared__ double acc[8][33];
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  if (q < nv) {
    double s = 0.0;
    for (int t = lane; t < ntiles; t += 32) s += partials[(int64_t)t * 8 + q];
    acc[q][lane] = s;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
    for (int l = 0; l < 32; ++l) s += acc[threadIdx.x][l];
    double r = sqrt(s * inv_count);
    if (out) out[threadIdx.x] = r;
    if (!(r == r) || r > 1.0e300) atomicExch(err, 4);
  }
}

cudaError_t launch_norm_finish(const double* partials, int ntiles, int nv, double inv_count,
                               double* out, int* err, cudaStream_t s) {
  norm_finish_kernel<<<1, 256, 0, s>>>(partials, ntiles, nv, inv_count, out, err);
  return cudaGetLastError();
}

__global__ void copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n16;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

cudaError_t launch_copy(void* dst, const void* src, int64_t bytes, cudaStream_t s) {
  if (bytes % 16 != 0) return cudaErrorInvalidValue;
  int64_t n16 = bytes / 16;
  if (n16 == 0) return cudaSuccess;
  int64_t nb = (n16 + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  copy_kernel<<<(unsigned)nb, 256, 0, s>>>((const uint4*)src, (uint4*)dst, n16);
  return cudaGetLastError();
}

}  // namespace hbk
