// FP64 instantiation of the tile, halo, init and force kernels, plus the
// precision-independent reduction and copy helpers.
#include "hb_kernels.cuh"
#define HB_T double
#include "hb_launch.inc"

namespace hbk {

// fixed-order FP64 finish of the per-tile norm partials: thread q < nv walks
// the tiles in order; the result is the RMS over cells and snapshots
__global__ void norm_finish_kernel(const double* partials, int ntiles, int nv, double inv_count,
                                   double* out, int* err, int raw) {
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
    double r = raw ? s : sqrt(s * inv_count);
    if (out) out[threadIdx.x] = r;
    if (!(r == r) || r > 1.0e300) atomicExch(err, 4);
  }
}

cudaError_t launch_norm_finish(const double* partials, int ntiles, int nv, double inv_count,
                               double* out, int* err, cudaStream_t s, int raw) {
  norm_finish_kernel<<<1, 256, 0, s>>>(partials, ntiles, nv, inv_count, out, err, raw);
  return cudaGetLastError();
}

// halo staging buffers of a block decomposition: buf[e] = U[idx[e]] (pack)
// and U[idx[e]] = buf[e] (unpack), e < n; idx are state offsets
template <typename T>
__global__ void halo_pack_kernel(const T* __restrict__ U, const int64_t* __restrict__ idx, int64_t n,
                                 T* __restrict__ buf) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    buf[e] = U[idx[e]];
}
template <typename T>
__global__ void halo_unpack_kernel(T* __restrict__ U, const int64_t* __restrict__ idx, int64_t n,
                                   const T* __restrict__ buf) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    U[idx[e]] = buf[e];
}

cudaError_t launch_halo_pack(const void* U, const int64_t* idx, int64_t n, void* buf, bool fp32, bool unpack,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t want = (n + 255) / 256;
  const unsigned grid = (unsigned)(want < 4096 ? want : 4096);
  if (fp32) {
    if (unpack) halo_unpack_kernel<float><<<grid, 256, 0, s>>>((float*)U, idx, n, (const float*)buf);
    else halo_pack_kernel<float><<<grid, 256, 0, s>>>((const float*)U, idx, n, (float*)buf);
  } else {
    if (unpack) halo_unpack_kernel<double><<<grid, 256, 0, s>>>((double*)U, idx, n, (const double*)buf);
    else halo_pack_kernel<double><<<grid, 256, 0, s>>>((const double*)U, idx, n, (double*)buf);
  }
  return cudaGetLastError();
}

__global__ void copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n16;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

__global__ void cast_down_kernel(const double* __restrict__ u64, float* __restrict__ u32, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    u32[e] = (float)u64[e];
}

__global__ void defect_source_kernel(const double* __restrict__ r64, const float* __restrict__ r32,
                                     float* __restrict__ src, double sigma, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    src[e] = (float)(sigma * r64[e] - (double)r32[e]);
}

__global__ void defect_update_kernel(double* __restrict__ u64, const float* __restrict__ v32,
                                     const float* __restrict__ u32, double inv_sigma, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    u64[e] += ((double)v32[e] - (double)u32[e]) * inv_sigma;
}

static unsigned elementwise_grid(int64_t n) {
  int64_t nb = (n + 255) / 256;
  return (unsigned)(nb > 152 * 16 ? 152 * 16 : (nb < 1 ? 1 : nb));
}

cudaError_t launch_cast_down(const double* u64, float* u32, int64_t n, cudaStream_t s) {
  cast_down_kernel<<<elementwise_grid(n), 256, 0, s>>>(u64, u32, n);
  return cudaGetLastError();
}

cudaError_t launch_defect_source(const double* r64, const float* r32, float* src, double sigma, int64_t n,
                                 cudaStream_t s) {
  defect_source_kernel<<<elementwise_grid(n), 256, 0, s>>>(r64, r32, src, sigma, n);
  return cudaGetLastError();
}

cudaError_t launch_defect_update(double* u64, const float* v32, const float* u32, double sigma, int64_t n,
                                 cudaStream_t s) {
  defect_update_kernel<<<elementwise_grid(n), 256, 0, s>>>(u64, v32, u32, 1.0 / sigma, n);
  return cudaGetLastError();
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
