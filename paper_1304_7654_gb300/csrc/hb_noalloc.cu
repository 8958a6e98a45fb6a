// Allocation-free residual-norm reduction (hb_residual_norms_noalloc).
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph
// capture, under a memory pool that forbids new allocations, or in a
// host runtime that only hands out pre-registered buffers.  This entry point
// needs no context (hb_create allocates) and allocates nothing: its per-CTA
// FP64 partial sums live in one file-scope __device__ array that every GPU
// loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/hb.h"

namespace {

// scratch: one FP64 partial per (CTA, variable), fixed CTA count
constexpr int kNoallocCtas = HB_NOALLOC_MAX_CTAS;
constexpr int kNoallocVars = HB_NOALLOC_MAX_VARS;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_norm_partials[kNoallocCtas * kNoallocVars];

// device address of g_norm_partials, looked up once per device
constexpr int kMaxDevices = 64;
double* g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// Phase 1: CTA b sums (R[n][v][c] / V[c])^2 over cells c = b, b + G, ... and
// all snapshots n, in a fixed order, and overwrites its own partial slots.
template <typename T>
__global__ void __launch_bounds__(kThreads) norm_partials_kernel(const T* __restrict__ R,
                                                                  const T* __restrict__ V,
                                                                  int64_t ncells, int ns, int nv,
                                                                  double* partials) {
  __shared__ double red[kThreads / 32][kNoallocVars];
  double acc[kNoallocVars];
  for (int v = 0; v < kNoallocVars; ++v) acc[v] = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < ncells;
       c += (int64_t)gridDim.x * kThreads) {
    const double iv = 1.0 / (double)V[c];
    for (int n = 0; n < ns; ++n)
      for (int v = 0; v < nv; ++v) {
        const double x = (double)R[((int64_t)n * nv + v) * ncells + c] * iv;
        acc[v] += x * x;
      }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = 0; v < nv; ++v) {
    double x = acc[v];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][v] = x;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * kNoallocVars + threadIdx.x] = s;
  }
}

// Phase 2: one CTA; thread v walks the partials of the G CTAs in order.
__global__ void norm_finish_noalloc_kernel(const double* partials, int G, int nv, double inv_count,
                                           double* out) {
  if (threadIdx.x < nv) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += partials[(int64_t)b * kNoallocVars + threadIdx.x];
    out[threadIdx.x] = sqrt(s * inv_count);
  }
}

// Resolve the device address of the scratch array for the current device.
// Host code may not pass g_norm_partials itself to a kernel: on the host that
// name is a stand-in object, not a device address.
hb_status scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_norm_partials) != cudaSuccess || !p) return HB_ERR_CUDA;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return HB_OK;
}

}  // namespace

extern "C" hb_status hb_residual_norms_noalloc(const void* R, const void* vol, int prec, int64_t ncells,
                                               int n_snap, int nv, double* norms, void* stream) {
  if (!R || !vol || !norms) return HB_ERR_INVALID_ARG;
  if (prec != HB_FP32 && prec != HB_FP64) return HB_ERR_INVALID_ARG;
  if (ncells < 1 || n_snap < 1 || nv < 1) return HB_ERR_INVALID_ARG;
  if (nv > HB_NOALLOC_MAX_VARS || ncells > HB_NOALLOC_MAX_CELLS ||
      (int64_t)n_snap * nv * ncells > HB_NOALLOC_MAX_VALUES)
    return HB_ERR_UNSUPPORTED;   // beyond the fixed scratch and index limits
  double* partials = nullptr;
  hb_status st = scratch_for_current_device(&partials);
  if (st != HB_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t G = (ncells + kThreads - 1) / kThreads;
  if (G > kNoallocCtas) G = kNoallocCtas;
  if (prec == HB_FP32)
    norm_partials_kernel<float><<<(unsigned)G, kThreads, 0, s>>>(
        static_cast<const float*>(R), static_cast<const float*>(vol), ncells, n_snap, nv, partials);
  else
    norm_partials_kernel<double><<<(unsigned)G, kThreads, 0, s>>>(
        static_cast<const double*>(R), static_cast<const double*>(vol), ncells, n_snap, nv, partials);
  if (cudaGetLastError() != cudaSuccess) return HB_ERR_CUDA;
  norm_finish_noalloc_kernel<<<1, 32, 0, s>>>(partials, (int)G, nv,
                                              1.0 / ((double)ncells * (double)n_snap), norms);
  if (cudaGetLastError() != cudaSuccess) return HB_ERR_CUDA;
  return HB_OK;
}
