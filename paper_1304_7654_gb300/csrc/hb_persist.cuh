// Persistent batched RK driver: one cooperative launch runs K iterations of
// every case of a batch (different grids, N_H, Mach and motion): per stage,
// all tiles, closed by a grid barrier.  The tiles fill the halos of their
// output themselves (fused ghost fill), so a stage needs one barrier; without
// the ghost tables each stage first runs the halo passes, one barrier each.
// The barrier spins with a wall-clock limit (globaltimer); on expiry it sets
// HB_ERR_TIMEOUT and an abort flag, every CTA leaves at its next barrier, and
// the kernel returns -- it never traps.  Tiles are claimed through an atomic
// counter in cost order (snapshots x cells, largest first); a tile's result
// does not depend on which CTA computes it, so the output is deterministic.
#pragma once

#include "hb_kernels.cuh"

namespace hbk {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
__device__ bool grid_barrier(const PersistParams<T>& P, int number) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* gen = P.bar + 1;
    volatile unsigned int* abort = P.bar + 2;
    const unsigned int g = *gen;
    __threadfence();
    const bool arrive = !(P.skip_cta == (int)blockIdx.x && number == 0);
    bool released = false;
    if (arrive) {
      const unsigned int prev = atomicAdd(P.bar, 1u);
      if (prev == gridDim.x - 1) {
        atomicExch(P.bar, 0u);
        __threadfence();
        atomicAdd((unsigned int*)(P.bar + 1), 1u);
        released = true;
      }
    }
    if (!released) {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (*abort) { ok = 0; break; }
        if ((long long)(global_ns() - t0) > P.timeout_ns) {
          atomicExch(P.err, 5);           // HB_ERR_TIMEOUT
          atomicExch((unsigned int*)(P.bar + 2), 1u);
          ok = 0;
          break;
        }
        __nanosleep(200);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// the persistent driver serves cases of every snapshot count with one
// shared-memory size: the tiles park their per-snapshot balances in global
// memory (sp.R), which leaves room for the snapshot pipeline at any N_s
template <typename T, bool VISC, int TI, int TJ>
__device__ __forceinline__ void tile_any_ns(const StageParams<T>& sp, int t, T* sm) {
  const int ns = sp.cases[sp.blocks[sp.tiles[t].x].cs].ns;
  switch (ns) {
    case 1: tile2d<T, 1, VISC, 1, TI, TJ, true, true>(sp, t, sm); break;
    case 3: tile2d<T, 3, VISC, 1, TI, TJ, true, true>(sp, t, sm); break;
    case 5: tile2d<T, 5, VISC, 1, TI, TJ, true, true>(sp, t, sm); break;
    case 7: tile2d<T, 7, VISC, 1, TI, TJ, true, true>(sp, t, sm); break;
    default: tile2d<T, 9, VISC, 1, TI, TJ, true, true>(sp, t, sm); break;
  }
}

// CTAs per SM the persistent kernel is compiled for: with its balances in
// global memory a 128-thread tile needs ~24 KB of shared memory, and seven
// FP32 CTAs (72 registers, a few spilled) outrun six (measured on the batch)
__host__ __device__ constexpr int persist_min_ctas(bool fp32, int NT) {
  return fp32 ? (NT == 128 ? 7 : 3 * (MAXNT / NT)) : MAXNT / NT;
}

template <typename T, bool VISC, int TI, int TJ>
__global__ void __launch_bounds__(TI * TJ, persist_min_ctas(sizeof(T) == 4, TI * TJ))
    persist_kernel(PersistParams<T> P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ int claim;
  int nbar = 0;
  for (int it = 0; it < P.K; ++it) {
    for (int s = 0; s < 4; ++s) {
      for (int pass = 0; pass < (P.fused ? 0 : P.dim); ++pass) {
        HaloParams<T> hp = P.halo[pass];
        hp.U = const_cast<T*>(P.st[s].Uprev);
        const int64_t tot = ((int64_t)hp.ncopy + hp.nbc) * hp.ns_max;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < tot;
             g += (int64_t)gridDim.x * blockDim.x)
          halo_item<T, 2>(hp, g);
        if (!grid_barrier(P, nbar++)) return;
      }
      // the next claim is issued when a tile starts and read when it ends,
      // so the atomic's latency hides behind the tile's work
      unsigned int* ctr = P.work + it * 4 + s;
      if (threadIdx.x == 0) claim = (int)atomicAdd(ctr, 1u);
      __syncthreads();
      int k = claim;
      while (k < P.ntiles) {
        __syncthreads();   // every thread has read the claim
        int next = 0;
        if (threadIdx.x == 0) next = (int)atomicAdd(ctr, 1u);
        tile_any_ns<T, VISC, TI, TJ>(P.st[s], P.order[k], sm);
        if (threadIdx.x == 0) claim = next;
        __syncthreads();
        k = claim;
      }
      if (!grid_barrier(P, nbar++)) return;
      if (s == 0 && P.norms) {
        // per-case RMS norms from the stage-1 partials, fixed order
        double* red = reinterpret_cast<double*>(sm);
        for (int c = blockIdx.x; c < P.ncases; c += gridDim.x) {
          const int t0 = P.case_tile0[c], nt = P.case_ntiles[c];
          double acc[4] = {0.0, 0.0, 0.0, 0.0};
          for (int t = threadIdx.x; t < nt; t += blockDim.x)
            for (int q = 0; q < 4; ++q) acc[q] += P.st[0].partials[(int64_t)(t0 + t) * 8 + q];
          block_sum8(acc, 4, red);
          if (threadIdx.x == 0) {
            for (int q = 0; q < 4; ++q) {
              const double r = sqrt(acc[q] * P.case_inv[c]);
              P.norms[((int64_t)it * P.ncases + c) * 8 + q] = r;
              if (!(r == r) || r > 1.0e300) atomicExch(P.err, 4);
            }
          }
          __syncthreads();
        }
      }
    }
  }
}

}  // namespace hbk
