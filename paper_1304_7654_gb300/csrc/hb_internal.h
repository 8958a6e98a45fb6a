// Internal structures shared by the host side (hb_api.cpp) and the CUDA
// kernels of libhb.so.  Not part of the public ABI (include/hb.h).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace hbk {

constexpr int MAXNS = 31;      // 2 * HB_MAX_HARMONICS + 1
constexpr int MAXNT = 256;     // threads per tile CTA
// compile-time snapshot counts of the 2D tile kernel go up to this; larger
// N_s run the runtime-count instantiation (NS = 0)
constexpr int kMaxStaticNS = 9;
// RK stages (MODE 1) whose 2D tile parks its per-snapshot flux balances in a
// global scratch instead of shared memory: one slice of kMaxStaticNS x nv x
// (TI x TJ) elements per tile, passed in StageParams::R by the host for
// exactly these stages (the kernel and the host both ask this function).
// At N_s = 9 this makes room for the snapshot pipeline; at N_s = 7 the tile
// measured slightly faster with the balances in L2 than in shared memory.
// k depth of a 3D tile (8 x 8 x tk cells, one thread per cell): 8 in FP32
// (512 threads, one CTA per SM, less halo work per cell: measured faster),
// 4 in FP64 (two 256-thread CTAs would not fit its registers at 512)
__host__ __device__ constexpr int tile3d_tk(bool fp32) { return fp32 ? 8 : 4; }
__host__ __device__ constexpr bool tile_balg(int NS, int MODE) { return (NS == kMaxStaticNS || NS == 7) && MODE == 1; }

// Per-case constants, in the kernel precision T.  Frames and freestream are
// tabulated per snapshot on the host in FP64 and rounded once.
template <typename T>
struct CaseDev {
  int dim, nv, ns, nh;
  int viscous, entropy_fix, motion, ubc;
  int n_bodies, functag;
  int block0, nblocks;
  int64_t interior_cells;
  T gamma, mu, kappa, prandtl, cfl, eps, ent_frac, omega, mach, pinf, ubc_amp, alpha0;
  T pivot[2];
  T cosa0, sina0;
  T D[MAXNS * MAXNS];                   // spectral derivative matrix (row n, column m)
  T cth[MAXNS], sth[MAXNS], thd[MAXNS]; // rotation and pitch rate at each snapshot
  T tn[MAXNS];                          // omega * t_n
  T winf[MAXNS][5];                     // freestream primitives (rho, u, v, w, p) per snapshot
};

// One block of the state: element (n, v, padded cell c) at off + (n*nv + v)*plane + c,
// padded cell c = ((k+gk)*P1 + (j+2))*P0 + (i+2).
struct BlockDev {
  int64_t off;
  int64_t plane;
  int64_t goff;       // offset of the block's padded cells in the geometry arrays
  int n[3];
  int P[3];
  int gk;
  int cs;             // case index
  int64_t noff;       // offset of the block's interior cells in compact [n][v][k][j][i] order
};

// geometry quantities, each an array over all padded cells of all blocks
enum {
  G_VOL = 0,
  G_XC = 1,            // 3 components
  G_S = 4,             // S[d][comp]: low face of the cell along d, 9 arrays
  G_XF = 13,           // face centroid [d][comp], 9 arrays
  G_DC = 22,           // centre minus centre of the low neighbour along d [d][comp], 9 arrays
  G_VG = 31,           // 2D rigid pitch: ((x_f - pivot) x S) / |S| of the low face along d, 2 arrays
  G_NQ = 33
};

struct CopyRec { int dst_blk, src_blk, dst_cell, src_cell; };
// physical-boundary ghost fill at one tangential position: both ghost layers
struct BcRec {
  int blk, type, p, sgn;   // sgn = +1 on the high face, -1 on the low face
  int gcell[2];            // ghost cells, layer 0 (adjacent) and 1
  int mcell[2];            // mirror cells, interior layer 0 and 1
  int fcell;               // owner of the boundary face (its low face along p)
  int body;
};

// A ghost cell whose value is a chain of at most three physical-boundary maps
// (op: index into the stage's BcRec table, applied in order) of one interior
// cell (root_cell, in the block of the tile that owns it).  Cut copies are the
// identity and leave no op.  After an RK stage the tile that wrote the root
// writes the ghost, so the next stage finds every halo filled.
struct GhostJob { int dst_blk, dst_cell, root_cell, nops, op[3], root_blk; };


template <typename T>
struct Geo {
  const T* q[G_NQ];
};

// one launch filling every ghost cell of dst from the interior cells of src
// (src == dst: an in-place halo fill; the roots are never ghosts)
template <typename T>
struct GhostFillParams {
  const CaseDev<T>* cases;
  const BlockDev* blocks;
  Geo<T> g;
  const T* src;
  T* dst;
  const GhostJob* jobs;
  int njobs;
  const BcRec* bcs;
  int ns_max;
};

template <typename T>
struct StageParams {
  const CaseDev<T>* cases;
  const BlockDev* blocks;
  const int4* tiles;       // (block, i0, j0, k0)
  int ntiles;
  Geo<T> g;
  const T* Uprev;          // halos filled
  const T* U0;             // iteration start state (RK mode)
  T* Unext;                // RK mode output
  T* R;                    // residual mode output
  double* partials;        // [ntiles][8] FP64 norm partials, or null
  T alpha;                 // RK stage coefficient
  int TI, TJ, ti_shift;    // tile shape; TI = 1 << ti_shift
  const T* H;              // N_s > 9: HB source V omega D Uprev; time-domain: the physical-time term
  T lam_v;                 // time-domain: added to the spectral radius per unit volume (a0 / dt)
  const T* src;            // RK mode: a fixed source added to the residual (defect correction), or null
  const int2* job_range;   // RK mode: [ntiles] (first, count) into jobs, or null (no fused ghost fill)
  const GhostJob* jobs;
  const BcRec* job_bcs;
};

template <typename T>
struct HaloParams {
  const CaseDev<T>* cases;
  const BlockDev* blocks;
  Geo<T> g;
  T* U;
  const CopyRec* copies;
  int ncopy;
  const BcRec* bcs;
  int nbc;
  int ns_max;
};

template <typename T>
struct ForceParams {
  const CaseDev<T>* cases;
  const BlockDev* blocks;
  Geo<T> g;
  const T* U;               // interior cells (and ghosts when G is null)
  const T* G;               // ghost cells (same layout), or null
  const BcRec* walls;
  int nwall;
  int ns;
  double* face_out;         // [ns][nwall][3]
  double* coef;             // [ns][nbodies][3] or null
  double* J;                // or null
  int nbodies;
  double* coef_scratch;     // [ns][nbodies][3] library-owned
  unsigned int* done;       // completion counter (zero between launches)
};

// One persistent launch advancing K RK iterations of every case: per stage,
// the halo passes then all tiles (claimed dynamically in cost order), each
// phase closed by a bounded-spin grid barrier.
template <typename T>
struct PersistParams {
  StageParams<T> st[4];     // per RK stage (tiles, Uprev, U0, Unext, alpha, partials)
  HaloParams<T> halo[3];    // per pass; the kernel points U at the stage input
  int dim;
  const int* order;         // tile indices in claim order
  int ntiles;
  unsigned int* work;       // [K * 4] claim counters, zero at launch
  unsigned int* bar;        // [0] arrivals, [1] generation, [2] abort flag; zero at launch
  int* err;                 // device error word
  int K;
  int ncases;
  const int* case_tile0;
  const int* case_ntiles;
  const double* case_inv;   // 1 / (cells * snapshots) per case
  double* norms;            // [K][ncases][8] or null
  long long timeout_ns;     // barrier wait limit
  int skip_cta;             // test hook: this CTA does not arrive at the first barrier (-1: none)
  int fused;                // 1: the stages fill the halos of their output (no halo phases)
  int ns_max;               // largest snapshot count of the cases (sizes the shared memory)
};

// launchers (defined per precision in hb_kernels_f32.cu / hb_kernels_f64.cu)
template <typename T>
cudaError_t launch_halo(const HaloParams<T>& p, cudaStream_t s);
template <typename T>
cudaError_t launch_stage(const StageParams<T>& p, int ns, int viscous, int mode, cudaStream_t s);
template <typename T>
cudaError_t launch_init(const CaseDev<T>* cases, const BlockDev* blocks, int nblocks, Geo<T> g,
                        T* U, const double* noise, double amp, int64_t total_interior,
                        const int64_t* block_noff, cudaStream_t s);
template <typename T>
cudaError_t launch_forces(const ForceParams<T>& p, cudaStream_t s);
template <typename T>
cudaError_t launch_ghost_fill(const GhostFillParams<T>& p, cudaStream_t s);
// time-domain physical-time term H = V (c0 U + c1 U_n + c2 U_nm1) over the
// chunks (U_nm1 may be null), c_k = a_k / dt
template <typename T>
cudaError_t launch_td_source(const BlockDev* blocks, Geo<T> g, const int2* chunks, int nchunks, int nv, T c0,
                             T c1, T c2, const T* U, const T* Un, const T* Unm1, T* H, cudaStream_t s);
// H = V omega D U over the chunks (block, first padded cell) of 128 cells of
// the blocks whose case has `ns` snapshots; D is that count's [ns][ns]
// derivative matrix (host, FP64)
template <typename T>
cudaError_t launch_hb_source(const CaseDev<T>* cases, const BlockDev* blocks, Geo<T> g, const int2* chunks,
                             int nchunks, int nv, int ns, const double* D, const T* U, T* H, cudaStream_t s);

// SMs x resident CTAs of the RK-stage tile kernel (one wave of tiles)
template <typename T>
cudaError_t stage_slots(int ns, int viscous, int TI, int TJ, int* slots);

template <typename T>
cudaError_t launch_stage3d(const StageParams<T>& p, int ns, int viscous, int mode, cudaStream_t s);
template <typename T>
cudaError_t launch_halo3d(const HaloParams<T>& p, cudaStream_t s);
template <typename T>
cudaError_t launch_init3d(const CaseDev<T>* cases, const BlockDev* blocks, int nblocks, Geo<T> g, T* U,
                          const double* noise, double amp, cudaStream_t s);
template <typename T>
cudaError_t launch_persist(const PersistParams<T>& p, int viscous, int TI, int TJ, cudaStream_t s,
                           int* grid_out);
template <typename T>
bool persist_available(int TI, int TJ);

// raw = 1: out = the fixed-order sum itself (no scaling, no square root)
cudaError_t launch_norm_finish(const double* partials, int ntiles, int nv, double inv_count,
                               double* out, int* err, cudaStream_t s, int raw = 0);
// gather (unpack = false: buf[e] = U[idx[e]]) or scatter (U[idx[e]] = buf[e])
// of state elements for the halo exchange of a block decomposition
cudaError_t launch_halo_pack(const void* U, const int64_t* idx, int64_t n, void* buf, bool fp32, bool unpack,
                             cudaStream_t s);
// defect correction, elementwise over n state entries: u32 = (float) u64;
// src = (float)(sigma r64 - r32); u64 += (v32 - u32) / sigma (in FP64)
cudaError_t launch_cast_down(const double* u64, float* u32, int64_t n, cudaStream_t s);
cudaError_t launch_defect_source(const double* r64, const float* r32, float* src, double sigma, int64_t n,
                                 cudaStream_t s);
cudaError_t launch_defect_update(double* u64, const float* v32, const float* u32, double sigma, int64_t n,
                                 cudaStream_t s);
cudaError_t launch_copy(void* dst, const void* src, int64_t bytes, cudaStream_t s);

}  // namespace hbk
