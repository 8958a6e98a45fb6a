/*
 * hb.h -- C ABI of the GB300 harmonic-balance (HB) residual library (libhb.so).
 *
 * The library evaluates and smooths the HB residual of the Navier-Stokes
 * equations on structured multi-block grids: for every cell and each of the
 * 2*N_H+1 time snapshots, the cell-centred finite-volume convective (MUSCL +
 * van Albada + Roe) and viscous (central) flux balance plus the HB source
 * V*omega*D*U that couples the snapshots through the spectral time-derivative
 * matrix D, driven by a 4-stage Runge-Kutta smoother with local time steps,
 * with block-interface ("cut") halos exchanged on the device.
 *
 * Paper anchors (Jackson & Campobasso, arXiv 1304.7654):
 *   - HB NS solver on structured multi-block grids, snapshot loop
 *     n = 0..2*nharms over the state q2(i,j,ipde,n): Sec. 1 and Sec. 3.1.
 *   - Cut (halo) exchange at every Runge-Kutta step, one aggregated exchange
 *     per process pair: Sec. 3.1 "MPI Optimisations" -> hb_exchange_halos.
 *   - Force coefficients cl, cd (and cm when functag == 3) per body and
 *     snapshot, aggregated into one reduction per RK step packed
 *     [snapshot][body][cl,cd,cm]: Sec. 3.1 -> hb_forces.
 *   - Restart file: Sec. 3.1 -> hb_save_state / hb_load_state (per-snapshot
 *     visualisation output is not part of this ABI).
 *   - The two test cases (31 and 17 snapshots, 512 and 2048 blocks):
 *     Sec. 4.1 -> HB_MAX_HARMONICS.
 * The scheme itself (flux, limiter, RK, time step, boundary conditions) is
 * not printed in the paper; the readings used are documented beside each
 * kernel in the sources.
 *
 * Conventions for every call:
 *   - Every function returns hb_status; nothing aborts, traps or throws.
 *   - Device pointers (U, R, psi, r_adj, norms, coeffs, J) are caller-owned
 *     CUDA device memory, in the layout reported by hb_state_layout.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream; host-side argument errors are returned
 *     immediately, device-side errors (non-finite norms, barrier timeouts)
 *     are latched in a device word and reported by hb_sync_status.
 *   - A context is not thread-safe: one host thread at a time per context.
 *   - Precision HB_FP32 computes fluxes, sources and updates in FP32 and keeps
 *     residual norms, force sums and conservation sums in FP64; HB_FP64
 *     computes everything in FP64.  The state element type follows it.
 */
#ifndef HB_H_
#define HB_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HB_OK = 0,
  HB_ERR_INVALID_ARG = 1,   /* malformed descriptor, table, pointer or size */
  HB_ERR_UNSUPPORTED = 2,   /* valid but not built (e.g. N_H above the maximum) */
  HB_ERR_CUDA = 3,          /* a CUDA runtime call failed; see hb_last_error */
  HB_ERR_NONFINITE = 4,     /* a residual norm became NaN or Inf */
  HB_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
  HB_ERR_OOM = 6            /* device allocation of library workspace failed */
} hb_status;

typedef enum { HB_FP64 = 0, HB_FP32 = 1 } hb_precision;
typedef enum { HB_BC_FARFIELD = 1, HB_BC_SLIP = 2, HB_BC_NOSLIP = 3 } hb_bc_type;
typedef enum { HB_MOTION_NONE = 0, HB_MOTION_PITCH = 1 } hb_motion;
typedef enum { HB_UBC_NONE = 0, HB_UBC_INLET_ANGLE = 1, HB_UBC_GUST = 2 } hb_unsteady_bc;

/* Largest supported number of harmonics N_H (snapshots 2*N_H+1): 15, i.e.
 * the 31 snapshots of the paper's first test case (Sec. 4.1).  Up to
 * HB_MAX_STATIC_HARMONICS the tile kernel is specialised on the snapshot
 * count and forms the HB source itself; above, a separate launch forms
 * H = V omega D U first, and 3D contexts and the persistent driver are not
 * available (HB_ERR_UNSUPPORTED). */
#define HB_MAX_HARMONICS 15
#define HB_MAX_STATIC_HARMONICS 4

/* One structured block of ni x nj (x nk) cells.  `nodes` is host memory, read
 * only during hb_create: (ni+5)*(nj+5)[*(nk+5)] points with `dim` coordinates
 * each, i fastest, including two ghost-node layers per direction (local node
 * index -2 .. n+2).  2D blocks pass nk = 1. */
typedef struct {
  int ni, nj, nk;
  const double* nodes;
} hb_block_desc;

/* One cut: fills the ghost box [lo, hi) (cell indices, hi exclusive) of block
 * dst_blk from block src_blk, src[a] = off[a] + sign[a] * dst[perm[a]].  The
 * box lies in the two ghost layers of one direction p (its pass); along
 * directions q < p it may extend over ghost cells (block corners), along
 * q > p it must stay inside the block.  Sources must be interior cells, or
 * ghost cells along directions q < p.  This is the device form of the
 * paper's per-RK-step cut exchange (Sec. 3.1).  src_blk = HB_EXTERNAL_BLOCK
 * marks a box whose source block lives in another process (a block
 * decomposition over several GPUs, the paper's MPI distribution of blocks,
 * Sec. 2-3): the library never writes it; the caller fills it between the
 * halo passes (hb_halo_pass, hb_pack_halo / hb_unpack_halo). */
#define HB_EXTERNAL_BLOCK (-1)
typedef struct {
  int dst_blk, src_blk;
  int lo[3], hi[3];
  int off[3], perm[3], sign[3];
} hb_cut_desc;

/* One physical boundary segment on face `face` = 2*p + side (side 0: low
 * index, 1: high index) of block `blk`, tangential cell range [lo, hi) (the
 * entry along p is ignored).  type: hb_bc_type.  body: index of the body whose
 * forces include this wall segment, or -1. */
typedef struct {
  int blk, face;
  int lo[3], hi[3];
  int type, body;
} hb_bc_desc;

/* One HB case.  Non-dimensionalisation: rho_inf = 1, c_inf = 1,
 * p_inf = 1/gamma, |u_inf| = mach, mu = mach/reynolds (constant),
 * heat conductivity mu/((gamma-1) prandtl), reference length 1. */
typedef struct {
  int dim;                    /* 2 or 3; 3D runs one launch per phase with 8x8x8 (FP32) or 8x8x4 (FP64) tiles and has no
                                 force integration or adjoint (HB_ERR_UNSUPPORTED) */
  int n_harm;                 /* N_H, 0 .. HB_MAX_HARMONICS (3D: .. HB_MAX_STATIC_HARMONICS) */
  double mach, reynolds, prandtl, gamma;
  double alpha0_deg;          /* mean incidence of the freestream */
  double omega;               /* fundamental angular frequency */
  double cfl;                 /* pseudo-time CFL number */
  double lim_eps;             /* van Albada epsilon (absolute) */
  double entropy_frac;        /* Harten fix width as a fraction of the Roe sound speed */
  int viscous, entropy_fix;
  int motion;                 /* hb_motion: rigid pitch A sin(omega t) about pivot */
  double pitch_amp_deg, pivot[2];
  int ubc;                    /* hb_unsteady_bc: periodic farfield variation */
  double ubc_amp;             /* inlet-angle amplitude (deg) or gust amplitude (fraction of mach) */
  int n_blocks;
  const hb_block_desc* blocks;
  int n_cuts;
  const hb_cut_desc* cuts;
  int n_bcs;
  const hb_bc_desc* bcs;
  int n_bodies;
  int functag;                /* 3: include cm in the force output (paper Sec. 3.1) */
  hb_precision prec;
} hb_case_desc;

typedef struct hb_ctx hb_ctx;   /* opaque, library-owned */

/* Create a context: validates and copies the descriptors, uploads geometry,
 * allocates library-owned workspace on the current CUDA device (two RK stage
 * buffers of the state's size, the precomputed metrics, and for 3D cases,
 * N_s 7 and 9 cases and the persistent driver a per-tile scratch of about the
 * state's size that holds each tile's per-snapshot flux balances during an RK
 * stage; hb_set_tuning and hb_autotune may grow it).  Errors:
 * HB_ERR_INVALID_ARG for malformed tables (cut boxes outside the ghost
 * layers, sources outside the allowed range, unknown BC types, block ids out
 * of range), HB_ERR_UNSUPPORTED for N_H > HB_MAX_HARMONICS, HB_ERR_OOM. */
hb_status hb_create(const hb_case_desc* desc, hb_ctx** out);

/* Create one context holding n independent cases (each with its own grid,
 * N_H, Mach and motion; all of the same dim, viscosity and precision).  The
 * state arrays of the cases are concatenated in case order; block indices in
 * hb_state_layout run over all blocks of all cases.  hb_rk_smooth on such a
 * context advances every case in one persistent launch per iteration. */
hb_status hb_create_batch(const hb_case_desc* cases, int n, hb_ctx** out);

hb_status hb_destroy(hb_ctx* ctx);

/* Total number of state elements (double for HB_FP64, float for HB_FP32). */
int64_t hb_state_size(const hb_ctx* ctx);

/* Layout of block `blk`: the element (n, v, k, j, i) with local cell indices
 * in [-g, n+g) sits at offset + n*strides[0] + v*strides[1] + (k+gk)*strides[2]
 * + (j+2)*strides[3] + (i+2)*strides[4]; ext[] receives the padded extents
 * (i, j, k) and gk = 2 in 3D, 0 in 2D.  Interior cells are i in [0, ni). */
hb_status hb_state_layout(const hb_ctx* ctx, int blk, int64_t* offset, int64_t strides[5],
                          int ext[3]);

/* U := freestream of each snapshot at the cell centre times (1 + amp*noise)
 * on interior cells, ghosts left unchanged.  noise_dev: device FP64 array
 * with one value per interior (block, snapshot, variable, cell), packed block
 * after block as [n][v][k][j][i].  noise_dev may be NULL (no noise). */
hb_status hb_init_state(hb_ctx* ctx, void* U, const double* noise_dev, double amp, void* stream);

/* Fill both ghost layers of every block and snapshot, in place: cut copies and
 * physical-BC ghost states (characteristic farfield, slip wall, no-slip
 * adiabatic wall), one pass per direction so block corners see their
 * diagonal neighbours. */
hb_status hb_exchange_halos(hb_ctx* ctx, void* U, void* stream);

/* R := R_HB(U), the HB residual of every interior cell and snapshot (flux
 * balance, outward-positive, plus V*omega*D*U).  U is not modified: the
 * library fills the halos of its own copy.  R has U's layout; its ghost
 * entries are left unchanged. */
hb_status hb_residual(hb_ctx* ctx, const void* U, void* R, void* stream);

/* n_iter iterations of the 4-stage Runge-Kutta smoother (coefficients 1/4,
 * 1/3, 1/2, 1) with local pseudo-time steps, in place on U.  norms_dev, if
 * not NULL: device FP64 [n_iter][n_cases][nv] (n_cases = 1 for hb_create),
 * the RMS over interior cells and snapshots of R/V per variable at the first
 * stage of each iteration, summed in a fixed order (bitwise reproducible).
 * Non-finite norms latch HB_ERR_NONFINITE (read with hb_sync_status).
 * Depending on the context's tuning, each chunk of up to 64 iterations runs
 * either as one launch per phase or as one persistent cooperative launch
 * (all cases, all phases, bounded-spin grid barriers: a barrier that waits
 * longer than HB_BARRIER_TIMEOUT_MS, default 2000, latches HB_ERR_TIMEOUT
 * and the launch returns); chunks are captured and replayed as CUDA graphs
 * where stream capture is available. */
hb_status hb_rk_smooth(hb_ctx* ctx, void* U, int n_iter, double* norms_dev, void* stream);

/* Block decomposition over processes (the paper's distribution of blocks
 * over MPI ranks with one aggregated cut exchange per RK step, Sec. 2-3).
 * A context whose cuts include HB_EXTERNAL_BLOCK boxes is one process's
 * share of a multi-block case; hb_rk_smooth and hb_autotune refuse it
 * (HB_ERR_UNSUPPORTED) and the caller advances it stage by stage:
 *   for each RK stage s = 0..3 and its input Uin:
 *     for each pass p (direction) = 0..dim-1:
 *       hb_pack_halo   -- the sources of the other processes' pass-p boxes
 *       (send / receive the packed buffers)
 *       hb_halo_pass(p)  -- this context's own cuts and boundary ghosts
 *       hb_unpack_halo -- the received pass-p boxes
 *     hb_rk_stage(Uin, U0, Uout, s)
 * so that corners see the same values as on one GPU.  hb_residual and
 * hb_forces fill only the context's own ghosts: the external boxes of their
 * U must have been filled by the caller.  The adjoint is not available on
 * such contexts (HB_ERR_UNSUPPORTED). */

/* The cut copies and physical-boundary ghosts of one pass (direction `pass`,
 * 0 .. dim-1) in place on U, external boxes untouched.  Asynchronous.
 * Errors: HB_ERR_INVALID_ARG (null U, pass out of range). */
hb_status hb_halo_pass(hb_ctx* ctx, void* U, int pass, void* stream);

/* One Runge-Kutta stage (coefficients 1/4, 1/3, 1/2, 1 for stage 0..3) with
 * local time steps from U0: Uout = U0 - alpha_stage dtau/V R_HB(Uin) on
 * interior cells (Uout's ghosts untouched); every ghost of Uin must be
 * filled.  norm_sums (device FP64 [n_cases][nv], may be NULL) receives at
 * stage 0 the fixed-order sums over the context's interior cells and
 * snapshots of (R/V)^2 per variable, the terms of the RMS norms of
 * hb_rk_smooth, so that processes can add theirs before the square root.
 * Uout may be U0 (each cell reads its own U0 entries before writing them)
 * but not Uin.  2D contexts.  Errors: HB_ERR_INVALID_ARG (null pointers,
 * stage out of range, Uout aliasing Uin), HB_ERR_UNSUPPORTED (3D).
 * Asynchronous. */
hb_status hb_rk_stage(hb_ctx* ctx, const void* Uin, const void* U0, void* Uout, int stage, double* norm_sums,
                      void* stream);

/* Staging buffers of the halo exchange: buf[e] = U[idx[e]] (pack) or
 * U[idx[e]] = buf[e] (unpack) for e < n.  idx: device int64 state offsets
 * (hb_state_layout); buf: device array of n elements of the context's
 * precision; both caller-owned.  n = 0 does nothing.  Errors:
 * HB_ERR_INVALID_ARG (n < 0, null pointers with n > 0).  Asynchronous. */
hb_status hb_pack_halo(hb_ctx* ctx, const void* U, const int64_t* idx, int64_t n, void* buf, void* stream);
hb_status hb_unpack_halo(hb_ctx* ctx, void* U, const int64_t* idx, int64_t n, const void* buf, void* stream);

/* Force coefficients of every body at every snapshot, packed
 * [snapshot][body][cl, cd, cm] in FP64 (cm is zero unless functag == 3), as
 * in the paper's aggregated force reduction (Sec. 3.1); J_dev receives the
 * time-averaged lift J = (1/N_s) sum_n sum_body cl.  Either output may be
 * NULL.  U is not modified. */
hb_status hb_forces(hb_ctx* ctx, const void* U, double* coeffs_dev, double* J_dev, void* stream);

/* Reverse-mode adjoint of the residual and lift functional:
 * r_adj := (dR_HB/dU)^T psi + J_seed * dJ/dU on interior entries (ghost
 * entries of r_adj are zeroed), the transpose including the halo/BC maps;
 * J_dev (may be NULL) receives J(U).  Limiter, Roe and viscous
 * intermediates are recomputed, not stored.  psi has U's layout (ghost
 * entries ignored).  Supported for HB_FP64 2D contexts. */
hb_status hb_adjoint_residual(hb_ctx* ctx, const void* U, const void* psi, double J_seed,
                              void* r_adj, double* J_dev, void* stream);

/* Autotuner: time `iters` RK iterations of every compiled combination of
 * driver (one launch per phase, or persistent) and tile shape (32x8, 32x4,
 * 16x8 cells) on a scratch copy of U, keep the fastest, and record it in the
 * cache file ($HB_TUNE_CACHE, default ~/.cache/hbgpu_autotune.txt) keyed by
 * the case signature, the device's SM count and the library build (a choice
 * timed with another build is not reused); hb_create reads that cache.  U is
 * not modified.
 * Synchronises `stream`.  hb_set_tuning forces a choice (mode 0: per-phase
 * launches, 1: persistent; + 2: separate halo passes before every stage
 * instead of the fused ghost fill, in which each 2D tile writes the ghost
 * cells whose value derives from its own cells right after its RK update);
 * hb_get_tuning reads it.  The two ghost-fill forms give the same state up to
 * rounding of the boundary maps' primitive/conservative conversions. */
hb_status hb_autotune(hb_ctx* ctx, const void* U, int iters, void* stream);
hb_status hb_set_tuning(hb_ctx* ctx, int mode, int TI, int TJ);
hb_status hb_get_tuning(const hb_ctx* ctx, int* mode, int* TI, int* TJ);

/* Benchmark timing.  While enabled, every launch of the tile kernels
 * (residual / RK stage: class 0) and of the halo kernels (class 1) made
 * outside a captured graph is bracketed by CUDA events recorded on the
 * launching stream.  hb_kernel_stats waits for those events and returns the
 * accumulated device time (ms) and launch count of class `which` since the
 * last reset; which = 2 returns the count of all library kernel launches
 * (graph replays included) and no time.  Paper counterpart: none (the paper
 * reports wall-clock runtimes only, Sec. 5). */
hb_status hb_set_timing(hb_ctx* ctx, int enable);
hb_status hb_kernel_stats(hb_ctx* ctx, int which, double* ms, int64_t* launches, int reset);

/* Which driver form hb_rk_smooth used.  *persist_captured: -1 while no
 * persistent chunk has run, 1 once a persistent chunk (one cooperative launch
 * for all cases and all stages of up to 64 iterations) was captured into a
 * CUDA graph, 0 if that capture failed and such chunks run as direct
 * cooperative launches.  counts (may be NULL): [0] RK chunks replayed from a
 * captured graph, [1] those that were persistent chunks, [2] persistent
 * chunks launched directly (capture refused, or timing enabled); cumulative
 * since hb_create.  Paper counterpart: none (the paper's drivers are MPI
 * processes; this reports how the batched single-GPU form was launched). */
hb_status hb_graph_info(const hb_ctx* ctx, int* persist_captured, int64_t counts[3]);

/* Limits of hb_residual_norms_noalloc's fixed scratch. */
#define HB_NOALLOC_MAX_CTAS 2048
#define HB_NOALLOC_MAX_VARS 8
#define HB_NOALLOC_MAX_CELLS ((int64_t)1 << 31)
#define HB_NOALLOC_MAX_VALUES ((int64_t)1 << 40)

/* Allocation-free residual norms, for callers that cannot allocate device
 * memory (inside a CUDA graph capture, under a pool that forbids growth, or
 * a host runtime that only hands out pre-registered buffers): no context is
 * needed and nothing is allocated -- no cudaMalloc/cudaFree, no allocating
 * library routine.  The paper has no counterpart; it is the norm reduction
 * of hb_rk_smooth offered without a context.
 *   norms[v] = sqrt( sum_{n,c} (R[n][v][c] / vol[c])^2 / (ncells * n_snap) )
 * R: device, [n_snap][nv][ncells] in `prec` (HB_FP32: float, HB_FP64:
 * double); vol: device, [ncells] in the same type; norms: device FP64 [nv].
 * Partial sums are FP64 and summed in a fixed order (bitwise reproducible
 * for a given ncells).  They live in one static device array of
 * HB_NOALLOC_MAX_CTAS x HB_NOALLOC_MAX_VARS doubles (128 KB) that every GPU
 * which loads the library holds until the process exits; every call
 * overwrites the slots it reads, so no clearing is needed, but calls that
 * overlap on the GPU (different streams, no ordering) race on that array.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * Errors: HB_ERR_INVALID_ARG for null pointers, a bad precision or a
 * non-positive size; HB_ERR_UNSUPPORTED for nv > HB_NOALLOC_MAX_VARS,
 * ncells > HB_NOALLOC_MAX_CELLS or n_snap*nv*ncells > HB_NOALLOC_MAX_VALUES;
 * HB_ERR_CUDA if a launch fails.  Asynchronous on `stream`. */
hb_status hb_residual_norms_noalloc(const void* R, const void* vol, int prec, int64_t ncells,
                                    int n_snap, int nv, double* norms, void* stream);

/* Restart files (the paper's restart file, Sec. 3.1): hb_save_state writes the
 * interior cells of the device state U, in the context's precision and in the
 * compact order [block][snapshot][variable][k][j][i], after a header with a
 * format version, the iteration number given by the caller and a signature
 * of the context (dimension, precision, cases, block sizes, snapshot counts
 * and flow parameters).  hb_load_state checks the signature and writes the
 * interior cells of U (ghost cells are not stored: every RK call fills
 * them), returning the stored iteration.  A run of n iterations, saved,
 * loaded and continued for m more, equals a run of n + m iterations bit for
 * bit.  Both synchronise `stream` (host file I/O).  Errors:
 * HB_ERR_INVALID_ARG for null arguments, an unreadable or unwritable file, a
 * truncated file, another format or a signature of another context;
 * HB_ERR_CUDA if a copy fails. */
hb_status hb_save_state(hb_ctx* ctx, const void* U, const char* path, int64_t iteration, void* stream);
hb_status hb_load_state(hb_ctx* ctx, void* U, const char* path, int64_t* iteration, void* stream);

/* Time-domain dual time stepping on the same kernels (contexts whose cases
 * all have n_harm = 0, 2D): one physical time step to time t of size dt,
 * i.e. n_inner pseudo-time RK iterations (4 stages, local time steps) in
 * place on U (device, state layout; start it from U_n) of
 *     R*(U) = R(U; t) + V (a0 U + a1 U_n + a2 U_nm1) / dt = 0,
 * (a0, a1, a2) = (3/2, -2, 1/2) (second-order backward differences), or
 * (1, -1, 0) when U_nm1 is NULL (first step); the pseudo time step adds
 * a0 V / dt to the spectral radius.  R(U; t) is the residual with the grid
 * pitched, moving and the inflow as at time t; the context keeps that frame
 * afterwards (hb_forces and hb_residual then refer to t).  norms (device,
 * may be NULL): [n_inner][n_cases][nv] FP64 RMS of R* / V at the first stage.
 * The HB residual's time-derivative source V omega D U is the periodic
 * counterpart of this term: a converged HB solution equals the periodic
 * limit of these steps up to the harmonics above N_H (Sec. 1: the HB solver
 * replaces the time-domain one for periodic flows).  Errors:
 * HB_ERR_INVALID_ARG (null U or U_n, dt <= 0, t < 0, n_inner < 0),
 * HB_ERR_UNSUPPORTED (3D, or a case with n_harm > 0).  Asynchronous on
 * `stream` after a short host synchronisation for the frame upload. */
hb_status hb_td_step(hb_ctx* ctx, void* U, const void* U_n, const void* U_nm1, double t, double dt,
                     int n_inner, double* norms, void* stream);

/* FP32 smoothing with an FP64 finish (defect correction): for an FP32 and an
 * FP64 context of the same 2D cases (N_H up to HB_MAX_STATIC_HARMONICS) and
 * an FP64 state U64 (device, ctx64's layout, e.g. a converged FP32 state cast
 * up), n_outer times: the FP64 residual r = R64(U64) and the FP32 residual of
 * u = (float) U64 are formed, the scaled correction equation
 *     R32(u + e) + (sigma r - R32(u)) = 0
 * is smoothed from e = 0 by n_inner FP32 RK iterations (one launch per
 * phase), and U64 += e / sigma in FP64.  The fixed point is R64(U64) = 0, so
 * the converged state and forces become the FP64 solution's (the FP32 target
 * on converged force coefficients).  sigma > 0 scales the correction so that
 * the FP32 state u + e resolves it: FP32 keeps about 7 digits of u, and the
 * FP32-converged state differs from the FP64 one by ~1e-6 |u|, so sigma of
 * order 1e4 is needed; each outer iteration then removes the defect down to
 * the linearisation error of e (sigma = 1 leaves the FP32 error in place).
 * norms (device, may be NULL): [n_outer][n_cases][nv] FP64 RMS over interior
 * cells and snapshots of (R32(u) + sigma r - R32(u)) / V at the first
 * correction iteration, i.e. sigma times the FP64 defect through FP32.
 * Errors: HB_ERR_INVALID_ARG (null pointers, negative counts, sigma <= 0,
 * contexts of other precisions or other cases), HB_ERR_UNSUPPORTED (N_H
 * above HB_MAX_STATIC_HARMONICS).  Asynchronous on `stream`. */
hb_status hb_defect_correction(hb_ctx* ctx32, hb_ctx* ctx64, void* U64, int n_outer, int n_inner, double sigma,
                               double* norms, void* stream);

/* Synchronise `stream`, then read and clear the device error word. */
hb_status hb_sync_status(hb_ctx* ctx, void* stream);

/* Message of the last error on this context (library-owned string). */
const char* hb_last_error(const hb_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HB_H_ */
