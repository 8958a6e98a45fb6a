// Host side of libhb.so: the C ABI declared in include/hb.h.
//
// hb_create validates the case descriptors, computes the static grid metrics
// from the nodes (FP64, rounded once to the kernel precision), expands the cut
// and boundary tables into per-ghost-cell records grouped by pass (direction
// i, then j, then k, so block corners take their diagonal neighbours), builds
// the tile work list and allocates the library-owned workspace.  Every entry
// point only enqueues kernels on the caller's stream.
#include <sys/stat.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <algorithm>
#include <tuple>

#include "../../include/hb.h"
#include "hb_adjoint.h"
#include "hb_internal.h"

using hbk::BcRec;
using hbk::BlockDev;
using hbk::CaseDev;
using hbk::CopyRec;

namespace {

struct CaseHost {
  hb_case_desc d;
  int ns, nv;
  int block0, nblocks;
  int tile0, ntiles;
  int64_t cells;
};

}  // namespace

struct hb_ctx {
  int dim = 2, nv = 4, prec = HB_FP64, viscous = 0;
  size_t tsize = 8;
  int device = 0;
  std::vector<CaseHost> cases;
  std::vector<BlockDev> blocks;
  int64_t state_size = 0;       // elements
  int64_t geo_cells = 0;
  int64_t interior_values = 0;  // sum over cases of cells * ns * nv
  int64_t total_cells = 0;
  int ns_max = 1;
  int TI = 32, TJ = 8, ti_shift = 5;
  int mode = 0;                 // 0: one launch per stage, 1: persistent driver
  std::vector<int4> tiles;
  int max_tiles = 0;            // capacity of the tile-sized device buffers
  int* d_order = nullptr;       // claim order for the persistent driver
  unsigned int* d_work = nullptr;   // [kMaxK * 4] claim counters
  unsigned int* d_bar = nullptr;    // barrier words
  int* d_case_tile0 = nullptr;
  int* d_case_ntiles = nullptr;
  double* d_case_inv = nullptr;
  long long timeout_ns = 2000000000LL;
  int skip_cta = -1;
  int persist_graph = -1;       // -1 untested, 0 capture unsupported, 1 captured
  int64_t n_graph_replays = 0;      // RK chunks replayed from a captured graph
  int64_t n_persist_replays = 0;    // ... of them persistent (one cooperative launch)
  int64_t n_persist_direct = 0;     // persistent chunks launched without a graph
  std::string tune_key;
  // device
  void* d_cases = nullptr;
  BlockDev* d_blocks = nullptr;
  int4* d_tiles = nullptr;
  void* d_geo = nullptr;        // G_NQ arrays of geo_cells elements
  CopyRec* d_copy[3] = {nullptr, nullptr, nullptr};
  BcRec* d_bc[3] = {nullptr, nullptr, nullptr};
  int ncopy[3] = {0, 0, 0}, nbc[3] = {0, 0, 0};
  BcRec* d_walls = nullptr;
  int nwall = 0;
  // fused ghost fill (2D): every ghost cell as a chain of boundary maps of one
  // interior root cell, grouped by the tile that owns the root
  bool jobs_ok = false;          // ghost jobs resolved (2D contexts)
  int64_t external_cells = 0;    // ghost cells of external cuts (filled by the caller: block decomposition)
  bool halo_phases = false;      // tuning: run the halo passes between stages instead
  bool fused() const { return jobs_ok && !halo_phases; }
  struct GhostJobHost { int root_blk, root_i, root_j; hbk::GhostJob job; };
  std::vector<GhostJobHost> gjobs;
  hbk::GhostJob* d_jobs = nullptr;
  int2* d_job_range = nullptr;   // [job_range_cap]
  int job_range_cap = 0;
  BcRec* d_job_bcs = nullptr;
  // large-N_s cases (N_s above the kernel's compile-time counts): the HB
  // source H = V omega D U is formed by its own launch over these chunks
  int2* d_chunks = nullptr;      // (block, first padded cell) of 128-cell chunks, grouped by N_s
  int nchunks = 0;
  struct SrcGroup { int ns, first, count; std::vector<double> D; };
  std::vector<SrcGroup> src_groups;
  void* d_H = nullptr;
  bool large_ns() const { return nchunks > 0; }
  // time-domain stepping: chunks over every block (built on first use)
  int2* d_td_chunks = nullptr;
  int n_td_chunks = 0;
  std::vector<unsigned char> td_case_buf;
  // defect correction workspace (FP32 context: u32, v32, r32, src; FP64 context: r64)
  void* d_dc[4] = {nullptr, nullptr, nullptr, nullptr};
  int n_bodies = 0;
  void* d_A = nullptr;          // RK ping-pong and residual scratch
  void* d_B = nullptr;
  void* d_bal = nullptr;        // 3D: per-snapshot flux balances of an RK stage, [tile][ns][nv][256]
  size_t bal_bytes = 0;
  double* d_partials = nullptr; // [ntiles][8]
  double* d_face = nullptr;     // [nwall][ns][3]
  double* d_coef = nullptr;     // [ns][nbodies][3]
  unsigned int* d_done = nullptr;
  double* d_ring = nullptr;     // [ring][8] norms ring for graph replays
  int ring = 0;
  int* d_err = nullptr;
  // adjoint (FP64 2D single case): face/cell offsets, wall tags, ghost CSR
  bool adj_ok = false;
  std::vector<int64_t> foff_h;
  int64_t nfaces = 0;
  int64_t* d_foff = nullptr;
  int64_t* d_coff = nullptr;
  int* d_wall = nullptr;
  double* d_adjbuf = nullptr;
  hbk::GhostAdjRow* d_grow[3] = {nullptr, nullptr, nullptr};
  hbk::GhostAdjEntry* d_gent[3] = {nullptr, nullptr, nullptr};
  int ngrow[3] = {0, 0, 0};
  cudaStream_t cap_stream = nullptr;
  std::map<std::pair<const void*, int>, cudaGraphExec_t> graphs;   // key: (U, K * 8 + mode)
  std::map<std::pair<const void*, int>, int64_t> graph_kernels;
  // benchmark timing
  int timing = 0;
  bool capturing = false;
  struct Timed { int cls; cudaEvent_t a, b; };
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> pool;
  double t_ms[2] = {0.0, 0.0};
  int64_t n_timed[2] = {0, 0};
  int64_t n_launch = 0;
  std::string err;
};

namespace {

hb_status fail(hb_ctx* c, hb_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

hb_status cuda_fail(hb_ctx* c, cudaError_t e, const char* where) {
  if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA;
}

#define HB_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

int round_up(int x, int m) { return (x + m - 1) / m * m; }

cudaEvent_t pool_event(hb_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// brackets one kernel launch with events when benchmark timing is on
struct TimedScope {
  hb_ctx* c;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  TimedScope(hb_ctx* c_, int cls_, cudaStream_t s_) : c(c_), cls(cls_), s(s_) {
    c->n_launch++;
    if (c->timing && !c->capturing) {
      a = pool_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~TimedScope() {
    if (a) {
      cudaEvent_t b = pool_event(c);
      cudaEventRecord(b, s);
      c->pending.push_back({cls, a, b});
    }
  }
};

// padded cell index of local cell (i,j,k) in the GPU layout
inline int64_t pcell(const BlockDev& B, int i, int j, int k) {
  return ((int64_t)(k + B.gk) * B.P[1] + (j + 2)) * B.P[0] + (i + 2);
}

// ------------------------------------------------------------ geometry --
// static metrics of every padded cell, FP64, from the nodes (2 ghost layers)
void compute_geometry(int dim, const hb_block_desc& bd, const BlockDev& B, std::vector<double>& G,
                      int64_t geo_cells, const double* pivot) {
  const int q0 = bd.ni + 5, q1 = bd.nj + 5;
  auto X = [&](int a, int b, int c, int comp) -> double {
    const int64_t idx = (dim == 3) ? (((int64_t)(c + 2) * q1 + (b + 2)) * q0 + (a + 2))
                                   : ((int64_t)(b + 2) * q0 + (a + 2));
    return bd.nodes[dim * idx + comp];
  };
  auto put = [&](int q, int64_t cell, double v) { G[(size_t)q * geo_cells + B.goff + cell] = v; };
  const int kg = (dim == 3) ? 2 : 0;
  for (int k = -kg; k < B.n[2] + kg; ++k)
    for (int j = -2; j < B.n[1] + 2; ++j)
      for (int i = -2; i < B.n[0] + 2; ++i) {
        const int64_t c = pcell(B, i, j, k);
        if (dim == 2) {
          const double x1 = X(i, j, 0, 0), y1 = X(i, j, 0, 1);
          const double x2 = X(i + 1, j, 0, 0), y2 = X(i + 1, j, 0, 1);
          const double x3 = X(i + 1, j + 1, 0, 0), y3 = X(i + 1, j + 1, 0, 1);
          const double x4 = X(i, j + 1, 0, 0), y4 = X(i, j + 1, 0, 1);
          put(hbk::G_VOL, c, 0.5 * ((x3 - x1) * (y4 - y2) - (y3 - y1) * (x4 - x2)));
          put(hbk::G_XC, c, 0.25 * (x1 + x2 + x3 + x4));
          put(hbk::G_XC + 1, c, 0.25 * (y1 + y2 + y3 + y4));
          // low i-face: edge (i,j)->(i,j+1), normal (dy, -dx); low j-face: (i,j)->(i+1,j), (-dy, dx)
          put(hbk::G_S + 0, c, y4 - y1);
          put(hbk::G_S + 1, c, -(x4 - x1));
          put(hbk::G_S + 3, c, -(y2 - y1));
          put(hbk::G_S + 4, c, x2 - x1);
          put(hbk::G_XF + 0, c, 0.5 * (x1 + x4));
          put(hbk::G_XF + 1, c, 0.5 * (y1 + y4));
          put(hbk::G_XF + 3, c, 0.5 * (x1 + x2));
          put(hbk::G_XF + 4, c, 0.5 * (y1 + y2));
        } else {
          // face d of the cell: quadrilateral with corners a,b,c,e; area vector
          // = 1/2 (diagonal 1) x (diagonal 2), oriented towards +d
          double sv = 0.0;
          auto face = [&](int d, int ii, int jj, int kk, double* S, double* xf) {
            int A[3], Bq[3], Cq[3], E[3];   // n00, n11, na, nb
            if (d == 0) {
              int a[3] = {ii, jj, kk}, b[3] = {ii, jj + 1, kk + 1}, c2[3] = {ii, jj, kk + 1}, e[3] = {ii, jj + 1, kk};
              memcpy(A, a, 12); memcpy(Bq, b, 12); memcpy(Cq, c2, 12); memcpy(E, e, 12);
            } else if (d == 1) {
              int a[3] = {ii, jj, kk}, b[3] = {ii + 1, jj, kk + 1}, c2[3] = {ii + 1, jj, kk}, e[3] = {ii, jj, kk + 1};
              memcpy(A, a, 12); memcpy(Bq, b, 12); memcpy(Cq, c2, 12); memcpy(E, e, 12);
            } else {
              int a[3] = {ii, jj, kk}, b[3] = {ii + 1, jj + 1, kk}, c2[3] = {ii, jj + 1, kk}, e[3] = {ii + 1, jj, kk};
              memcpy(A, a, 12); memcpy(Bq, b, 12); memcpy(Cq, c2, 12); memcpy(E, e, 12);
            }
            double d1[3], d2[3];
            for (int m = 0; m < 3; ++m) {
              d1[m] = X(Bq[0], Bq[1], Bq[2], m) - X(A[0], A[1], A[2], m);
              d2[m] = X(Cq[0], Cq[1], Cq[2], m) - X(E[0], E[1], E[2], m);
              xf[m] = 0.25 * (X(A[0], A[1], A[2], m) + X(Bq[0], Bq[1], Bq[2], m) +
                              X(Cq[0], Cq[1], Cq[2], m) + X(E[0], E[1], E[2], m));
            }
            S[0] = 0.5 * (d1[1] * d2[2] - d1[2] * d2[1]);
            S[1] = 0.5 * (d1[2] * d2[0] - d1[0] * d2[2]);
            S[2] = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0]);
          };
          for (int d = 0; d < 3; ++d) {
            double Sl[3], xl[3], Sh[3], xh[3];
            face(d, i, j, k, Sl, xl);
            face(d, i + (d == 0), j + (d == 1), k + (d == 2), Sh, xh);
            for (int m = 0; m < 3; ++m) {
              put(hbk::G_S + 3 * d + m, c, Sl[m]);
              put(hbk::G_XF + 3 * d + m, c, xl[m]);
              sv += xh[m] * Sh[m] - xl[m] * Sl[m];
            }
          }
          put(hbk::G_VOL, c, sv / 3.0);
          for (int m = 0; m < 3; ++m) {
            double s = 0.0;
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) s += X(i + a, j + b, k + e, m);
            put(hbk::G_XC + m, c, s / 8.0);
          }
        }
      }
  // rigid pitch about the pivot: the grid velocity through a face, thdot *
  // ((x_f - p) x S) / |S|, is frame independent (rotation keeps cross
  // products), so the face's static factor is stored once
  if (dim == 2)
    for (int j = -2; j < B.n[1] + 2; ++j)
      for (int i = -2; i < B.n[0] + 2; ++i) {
        const int64_t c = pcell(B, i, j, 0);
        for (int d = 0; d < 2; ++d) {
          auto at = [&](int q) { return G[(size_t)q * geo_cells + B.goff + c]; };
          const double sx = at(hbk::G_S + 3 * d), sy = at(hbk::G_S + 3 * d + 1);
          const double ax = at(hbk::G_XF + 3 * d) - pivot[0], ay = at(hbk::G_XF + 3 * d + 1) - pivot[1];
          const double a = std::sqrt(sx * sx + sy * sy);
          put(hbk::G_VG + d, c, a > 0.0 ? (ax * sy - ay * sx) / a : 0.0);
        }
      }
  // centre differences, FP64 (keeps the face-normal distance exact to the
  // kernel precision even when |x| is much larger than the cell size)
  const int64_t sd[3] = {1, B.P[0], (int64_t)B.P[0] * B.P[1]};
  for (int k = -kg; k < B.n[2] + kg; ++k)
    for (int j = -2; j < B.n[1] + 2; ++j)
      for (int i = -2; i < B.n[0] + 2; ++i) {
        const int64_t c = pcell(B, i, j, k);
        const int idx3[3] = {i, j, k};
        for (int d = 0; d < dim; ++d) {
          if (idx3[d] - 1 < ((d == 2) ? -kg : -2)) continue;
          for (int m = 0; m < dim; ++m)
            put(hbk::G_DC + 3 * d + m, c,
                G[(size_t)(hbk::G_XC + m) * geo_cells + B.goff + c] -
                    G[(size_t)(hbk::G_XC + m) * geo_cells + B.goff + c - sd[d]]);
        }
      }
}

// --------------------------------------------------------------- tables --
struct Tables {
  std::vector<CopyRec> copy[3];
  std::vector<BcRec> bc[3];
  std::vector<BcRec> walls;
};

hb_status build_tables(hb_ctx* ctx, const CaseHost& ch, Tables& T) {
  const hb_case_desc& d = ch.d;
  const int dim = d.dim;
  const int nb = d.n_blocks;
  auto blk = [&](int b) -> const BlockDev& { return ctx->blocks[ch.block0 + b]; };
  // ghost coverage count per padded cell
  std::vector<std::vector<unsigned char>> cover(nb);
  for (int b = 0; b < nb; ++b) cover[b].assign((size_t)blk(b).plane, 0);
  auto ghost_ok = [&](const BlockDev& B, int p, const int* c) {
    for (int a = 0; a < dim; ++a) {
      const int lo = (a < p) ? -2 : 0, hi = (a < p) ? B.n[a] + 2 : B.n[a];
      if (a == p) {
        if (!((c[a] >= -2 && c[a] < 0) || (c[a] >= B.n[a] && c[a] < B.n[a] + 2))) return false;
      } else if (c[a] < lo || c[a] >= hi) {
        return false;
      }
    }
    return true;
  };
  auto src_ok = [&](const BlockDev& B, int p, const int* c) {
    for (int a = 0; a < dim; ++a) {
      const int lo = (a < p) ? -2 : 0, hi = (a < p) ? B.n[a] + 2 : B.n[a];
      if (c[a] < lo || c[a] >= hi) return false;
    }
    return true;
  };
  for (int q = 0; q < d.n_cuts; ++q) {
    const hb_cut_desc& c = d.cuts[q];
    const bool external = c.src_blk == HB_EXTERNAL_BLOCK;
    if (c.dst_blk < 0 || c.dst_blk >= nb || (!external && (c.src_blk < 0 || c.src_blk >= nb)))
      return fail(ctx, HB_ERR_INVALID_ARG, "cut " + std::to_string(q) + ": block id out of range");
    const BlockDev& D = blk(c.dst_blk);
    const BlockDev& S = blk(external ? c.dst_blk : c.src_blk);
    int p = -1;
    for (int a = 0; a < dim; ++a)
      if (c.lo[a] < 0 || c.hi[a] > D.n[a]) p = a;
    if (p < 0) return fail(ctx, HB_ERR_INVALID_ARG, "cut " + std::to_string(q) + ": box is not in a ghost layer");
    bool permok = true;
    int seen = 0;
    for (int a = 0; a < 3; ++a) {
      if (c.perm[a] < 0 || c.perm[a] > 2 || (c.sign[a] != 1 && c.sign[a] != -1)) permok = false;
      else seen |= 1 << c.perm[a];
    }
    if (!permok || seen != 7)
      return fail(ctx, HB_ERR_INVALID_ARG, "cut " + std::to_string(q) + ": bad perm/sign");
    const int k0 = (dim == 3) ? c.lo[2] : 0, k1 = (dim == 3) ? c.hi[2] : 1;
    for (int k = k0; k < k1; ++k)
      for (int j = c.lo[1]; j < c.hi[1]; ++j)
        for (int i = c.lo[0]; i < c.hi[0]; ++i) {
          const int dc[3] = {i, j, k};
          int sc[3];
          for (int a = 0; a < 3; ++a) sc[a] = c.off[a] + c.sign[a] * dc[c.perm[a]];
          if (dim == 2) sc[2] = 0;
          if (!ghost_ok(D, p, dc))
            return fail(ctx, HB_ERR_INVALID_ARG, "cut " + std::to_string(q) + ": destination outside the ghost layers of its pass");
          if (external) {   // filled by the caller between halo passes: only coverage is recorded
            const int64_t dcell = pcell(D, dc[0], dc[1], dc[2]);
            if (cover[c.dst_blk][dcell]++)
              return fail(ctx, HB_ERR_INVALID_ARG, "cut " + std::to_string(q) + ": ghost cell filled twice");
            ctx->external_cells++;
            continue;
          }
          if (!src_ok(S, p, sc))
            return fail(ctx, HB_ERR_INVALID_ARG, "cut " + std::to_string(q) + ": source not interior or earlier-pass ghost");
          const int64_t dcell = pcell(D, dc[0], dc[1], dc[2]);
          if (cover[c.dst_blk][dcell]++)
            return fail(ctx, HB_ERR_INVALID_ARG, "cut " + std::to_string(q) + ": ghost cell filled twice");
          T.copy[p].push_back({ch.block0 + c.dst_blk, ch.block0 + c.src_blk, (int)dcell,
                               (int)pcell(S, sc[0], sc[1], sc[2])});
        }
  }
  for (int q = 0; q < d.n_bcs; ++q) {
    const hb_bc_desc& b = d.bcs[q];
    if (b.blk < 0 || b.blk >= nb || b.face < 0 || b.face >= 2 * dim ||
        b.type < HB_BC_FARFIELD || b.type > HB_BC_NOSLIP)
      return fail(ctx, HB_ERR_INVALID_ARG, "bc " + std::to_string(q) + ": bad block, face or type");
    const BlockDev& B = blk(b.blk);
    const int p = b.face / 2, side = b.face % 2;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = b.lo[a]; hi[a] = b.hi[a]; }
    if (dim == 2) { lo[2] = 0; hi[2] = 1; }
    lo[p] = 0;
    hi[p] = 1;
    for (int a = 0; a < dim; ++a) {
      if (a == p) continue;
      const int l = (a < p) ? -2 : 0, h = (a < p) ? B.n[a] + 2 : B.n[a];
      if (lo[a] < l || hi[a] > h || lo[a] >= hi[a])
        return fail(ctx, HB_ERR_INVALID_ARG, "bc " + std::to_string(q) + ": tangential range out of bounds");
    }
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int t[3] = {i, j, k};
          BcRec r;
          r.blk = ch.block0 + b.blk;
          r.type = b.type;
          r.p = p;
          r.sgn = side ? 1 : -1;
          r.body = b.body;
          for (int l = 0; l < 2; ++l) {
            int g[3] = {t[0], t[1], t[2]}, m[3] = {t[0], t[1], t[2]};
            g[p] = side ? B.n[p] + l : -1 - l;
            m[p] = side ? B.n[p] - 1 - l : l;
            r.gcell[l] = (int)pcell(B, g[0], g[1], g[2]);
            r.mcell[l] = (int)pcell(B, m[0], m[1], m[2]);
            if (cover[b.blk][r.gcell[l]]++)
              return fail(ctx, HB_ERR_INVALID_ARG, "bc " + std::to_string(q) + ": ghost cell filled twice");
          }
          int f[3] = {t[0], t[1], t[2]};
          f[p] = side ? B.n[p] : 0;
          r.fcell = (int)pcell(B, f[0], f[1], f[2]);
          T.bc[p].push_back(r);
          bool inside = true;
          for (int a = 0; a < dim; ++a)
            if (a != p && (t[a] < 0 || t[a] >= B.n[a])) inside = false;
          if (inside && (b.type == HB_BC_SLIP || b.type == HB_BC_NOSLIP) && b.body >= 0 &&
              b.body < d.n_bodies)
            T.walls.push_back(r);
        }
  }
  // every ghost cell of the standard pass boxes filled exactly once
  for (int b = 0; b < nb; ++b) {
    const BlockDev& B = blk(b);
    const int kg = (dim == 3) ? 2 : 0;
    for (int k = -kg; k < B.n[2] + kg; ++k)
      for (int j = -2; j < B.n[1] + 2; ++j)
        for (int i = -2; i < B.n[0] + 2; ++i) {
          const bool in = i >= 0 && i < B.n[0] && j >= 0 && j < B.n[1] && k >= 0 && k < B.n[2];
          if (in) continue;
          if (cover[b][pcell(B, i, j, k)] != 1)
            return fail(ctx, HB_ERR_INVALID_ARG,
                        "block " + std::to_string(b) + ": ghost cell (" + std::to_string(i) + "," +
                            std::to_string(j) + "," + std::to_string(k) + ") not filled by any cut or BC");
        }
  }
  return HB_OK;
}

// Resolve every ghost cell into (root interior cell, chain of boundary maps)
// by replaying the pass-ordered fill symbolically: a cut copy passes its
// source's chain on unchanged, a boundary record appends itself to the chain
// of its mirror (walls) or first interior (farfield) cell.  bc_index[p] is the
// position of Tables::bc[p][0] in the concatenated table the ops refer to.
hb_status resolve_ghost_jobs(hb_ctx* ctx, const Tables& T, const int* bc_index) {
  struct Res { int blk, cell, nops, op[3]; };
  const int nb = (int)ctx->blocks.size();
  std::vector<std::vector<Res>> res(nb);
  for (int b = 0; b < nb; ++b) {
    const BlockDev& B = ctx->blocks[b];
    res[b].assign((size_t)B.plane, Res{-1, -1, 0, {-1, -1, -1}});
    for (int j = 0; j < B.n[1]; ++j)
      for (int i = 0; i < B.n[0]; ++i) {
        const int c = (int)pcell(B, i, j, 0);
        res[b][c] = Res{b, c, 0, {-1, -1, -1}};
      }
  }
  for (int p = 0; p < ctx->dim; ++p) {
    for (const CopyRec& r : T.copy[p]) {
      const Res& src = res[r.src_blk][r.src_cell];
      if (src.blk < 0) return fail(ctx, HB_ERR_INVALID_ARG, "ghost chain: copy from an unfilled cell");
      res[r.dst_blk][r.dst_cell] = src;
    }
    for (size_t q = 0; q < T.bc[p].size(); ++q) {
      const BcRec& r = T.bc[p][q];
      for (int l = 0; l < 2; ++l) {
        Res x = res[r.blk][r.type == HB_BC_FARFIELD ? r.mcell[0] : r.mcell[l]];
        if (x.blk < 0 || x.nops >= 3) return fail(ctx, HB_ERR_INVALID_ARG, "ghost chain: unresolved boundary source");
        x.op[x.nops++] = bc_index[p] + (int)q;
        res[r.blk][r.gcell[l]] = x;
      }
    }
  }
  ctx->gjobs.clear();
  for (int b = 0; b < nb; ++b) {
    const BlockDev& B = ctx->blocks[b];
    for (int j = -2; j < B.n[1] + 2; ++j)
      for (int i = -2; i < B.n[0] + 2; ++i) {
        if (i >= 0 && i < B.n[0] && j >= 0 && j < B.n[1]) continue;
        const int c = (int)pcell(B, i, j, 0);
        const Res& x = res[b][c];
        if (x.blk < 0) return fail(ctx, HB_ERR_INVALID_ARG, "ghost chain: ghost cell without a root");
        const BlockDev& R = ctx->blocks[x.blk];
        hb_ctx::GhostJobHost g;
        g.root_blk = x.blk;
        g.root_i = x.cell % R.P[0] - 2;
        g.root_j = x.cell / R.P[0] - 2;
        g.job = hbk::GhostJob{b, c, x.cell, x.nops, {x.op[0], x.op[1], x.op[2]}, x.blk};
        ctx->gjobs.push_back(g);
      }
  }
  return HB_OK;
}

// per-case constants; td_time >= 0: one snapshot at that physical time
// (time-domain stepping) instead of the HB snapshot times
template <typename T>
void fill_case_dev(const CaseHost& ch, CaseDev<T>& C, double td_time = -1.0) {
  const hb_case_desc& d = ch.d;
  memset(&C, 0, sizeof(C));
  C.dim = d.dim;
  C.nv = d.dim + 2;
  C.ns = ch.ns;
  C.nh = d.n_harm;
  C.viscous = d.viscous;
  C.entropy_fix = d.entropy_fix;
  C.motion = d.motion;
  C.ubc = d.ubc;
  C.n_bodies = d.n_bodies;
  C.functag = d.functag;
  C.block0 = ch.block0;
  C.nblocks = ch.nblocks;
  C.interior_cells = ch.cells;
  const double mu = d.mach / d.reynolds;
  C.gamma = (T)d.gamma;
  C.mu = (T)mu;
  C.kappa = (T)(mu / ((d.gamma - 1.0) * d.prandtl));
  C.prandtl = (T)d.prandtl;
  C.cfl = (T)d.cfl;
  C.eps = (T)d.lim_eps;
  C.ent_frac = (T)d.entropy_frac;
  C.omega = (T)d.omega;
  C.mach = (T)d.mach;
  C.pinf = (T)(1.0 / d.gamma);
  C.ubc_amp = (T)d.ubc_amp;
  const double a0 = d.alpha0_deg * M_PI / 180.0;
  C.alpha0 = (T)a0;
  C.cosa0 = (T)std::cos(a0);
  C.sina0 = (T)std::sin(a0);
  C.pivot[0] = (T)d.pivot[0];
  C.pivot[1] = (T)d.pivot[1];
  const int ns = ch.ns;
  for (int n = 0; n < ns; ++n)
    for (int m = 0; m < ns; ++m) {
      double v = 0.0;
      if (n != m) {
        const int k = n - m;
        const double sg = (k % 2 == 0) ? 1.0 : -1.0;
        v = 0.5 * sg / std::sin(M_PI * (double)k / (double)ns);
      }
      C.D[n * ns + m] = (T)v;
    }
  const double amp = d.pitch_amp_deg * M_PI / 180.0;
  for (int n = 0; n < ns; ++n) {
    const double t = (td_time >= 0.0) ? td_time : (d.omega > 0.0) ? 2.0 * M_PI * n / (ns * d.omega) : 0.0;
    double th = 0.0, thd = 0.0;
    if (d.motion == HB_MOTION_PITCH) {
      th = amp * std::sin(d.omega * t);
      thd = amp * d.omega * std::cos(d.omega * t);
    }
    C.cth[n] = (T)std::cos(th);
    C.sth[n] = (T)std::sin(th);
    C.thd[n] = (T)thd;
    C.tn[n] = (T)(d.omega * t);
    double alpha = a0;
    if (d.ubc == HB_UBC_INLET_ANGLE) alpha += d.ubc_amp * M_PI / 180.0 * std::sin(d.omega * t);
    C.winf[n][0] = (T)1.0;
    C.winf[n][1] = (T)(d.mach * std::cos(alpha));
    C.winf[n][2] = (T)(d.mach * std::sin(alpha));
    C.winf[n][3] = (T)0.0;
    C.winf[n][4] = (T)(1.0 / d.gamma);
  }
}

template <typename T>
hbk::Geo<T> geo_of(const hb_ctx* c) {
  hbk::Geo<T> g;
  const T* base = static_cast<const T*>(c->d_geo);
  for (int q = 0; q < hbk::G_NQ; ++q) g.q[q] = base + (size_t)q * c->geo_cells;
  return g;
}

void free_ctx(hb_ctx* c) {
  for (auto& t : c->pending) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  for (auto e : c->pool) cudaEventDestroy(e);
  c->pending.clear();
  c->pool.clear();
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  cudaFree(c->d_cases);
  cudaFree(c->d_blocks);
  cudaFree(c->d_tiles);
  cudaFree(c->d_geo);
  for (int p = 0; p < 3; ++p) { cudaFree(c->d_copy[p]); cudaFree(c->d_bc[p]); }
  cudaFree(c->d_walls);
  cudaFree(c->d_jobs);
  cudaFree(c->d_job_range);
  cudaFree(c->d_job_bcs);
  cudaFree(c->d_chunks);
  cudaFree(c->d_H);
  cudaFree(c->d_td_chunks);
  for (int k = 0; k < 4; ++k) cudaFree(c->d_dc[k]);
  cudaFree(c->d_A);
  cudaFree(c->d_B);
  cudaFree(c->d_bal);
  cudaFree(c->d_partials);
  cudaFree(c->d_face);
  cudaFree(c->d_coef);
  cudaFree(c->d_done);
  cudaFree(c->d_ring);
  cudaFree(c->d_err);
  cudaFree(c->d_order);
  cudaFree(c->d_work);
  cudaFree(c->d_bar);
  cudaFree(c->d_case_tile0);
  cudaFree(c->d_case_ntiles);
  cudaFree(c->d_case_inv);
  cudaFree(c->d_foff);
  cudaFree(c->d_coff);
  cudaFree(c->d_wall);
  cudaFree(c->d_adjbuf);
  for (int p = 0; p < 3; ++p) { cudaFree(c->d_grow[p]); cudaFree(c->d_gent[p]); }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
}

constexpr int kMaxK = 64;   // iterations per persistent launch / graph

// Concurrent CTAs of the RK-stage work for a case (mode 0: its own launch)
// or for the whole batch (mode 1: the persistent grid); 0 if unknown.
int wave_slots(hb_ctx* c, int mode, int ns, int TI, int TJ) {
  int slots = 0;
  cudaError_t e;
  if (mode == 1) {
    if (!(c->prec == HB_FP32 ? hbk::persist_available<float>(TI, TJ) : hbk::persist_available<double>(TI, TJ)))
      return 0;
    if (c->prec == HB_FP32) {
      hbk::PersistParams<float> p{};
      p.ns_max = c->ns_max;   // K = 0: query only
      e = hbk::launch_persist<float>(p, c->viscous, TI, TJ, nullptr, &slots);
    } else {
      hbk::PersistParams<double> p{};
      p.ns_max = c->ns_max;
      e = hbk::launch_persist<double>(p, c->viscous, TI, TJ, nullptr, &slots);
    }
  } else {
    e = c->prec == HB_FP32 ? hbk::stage_slots<float>(ns, c->viscous, TI, TJ, &slots)
                           : hbk::stage_slots<double>(ns, c->viscous, TI, TJ, &slots);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return slots;
}

// Split the tiles that would run in a final partial wave into row strips.
// With N tiles in dispatch order and S concurrent CTAs, the last N mod S
// tiles run alone after the full waves, each taking a full tile time; as q
// strips of TJ/q rows (q * (N mod S) <= S) they finish in a fraction of it.
// Strips of at least two rows: thinner ones cost as much as two-row strips.
void split_tail(std::vector<int4>& tl, const std::vector<int>& dispatch, int S, int TJ) {
  const int N = (int)dispatch.size();
  if (S <= 0 || N == 0) return;
  const int r = N % S;
  if (r == 0) return;
  int q = 1;
  while (q * 2 <= TJ / 2 && (long long)r * q * 2 <= S) q *= 2;
  if (q == 1) return;
  std::vector<char> cut(tl.size(), 0);
  for (int k = N - r; k < N; ++k) cut[dispatch[k]] = 1;
  std::vector<int4> out;
  out.reserve(tl.size() + (size_t)r * (q - 1));
  for (size_t k = 0; k < tl.size(); ++k) {
    const int4 t = tl[k];
    if (!cut[k] || t.w < 2) {
      out.push_back(t);
      continue;
    }
    const int h = (t.w + q - 1) / q;
    for (int j = 0; j < t.w; j += h) out.push_back(make_int4(t.x, t.y, t.z + j, std::min(h, t.w - j)));
  }
  tl.swap(out);
}

// Tile work list for shape TI x TJ: tiles of every case in case order (2D
// tiles carry their row count in .w; the tail of a wave is split into row
// strips for the driver `mode`), the claim order (cost = snapshots x cells,
// largest first) and per-case ranges.
hb_status rebuild_tiles(hb_ctx* c, int TI, int TJ, int mode) {
  std::vector<int4> tiles;
  std::vector<int> t0(c->cases.size()), nt(c->cases.size());
  std::vector<double> inv(c->cases.size());
  std::vector<long long> tcost;
  auto cells_of = [&](const int4& t) -> long long {
    const BlockDev& B = c->blocks[t.x];
    if (c->dim == 3)
      return (long long)std::min(8, B.n[0] - t.y) * std::min(8, B.n[1] - t.z) *
             std::min(hbk::tile3d_tk(c->prec == HB_FP32), B.n[2] - t.w);
    return (long long)std::min(TI, B.n[0] - t.y) * t.w;
  };
  for (size_t k = 0; k < c->cases.size(); ++k) {
    CaseHost& ch = c->cases[k];
    ch.tile0 = (int)tiles.size();
    std::vector<int4> ct;
    for (int b = 0; b < ch.nblocks; ++b) {
      const BlockDev& B = c->blocks[ch.block0 + b];
      if (c->dim == 3) {   // fixed 8 x 8 x tk tiles
        for (int k = 0; k < B.n[2]; k += hbk::tile3d_tk(c->prec == HB_FP32))
          for (int j = 0; j < B.n[1]; j += 8)
            for (int i = 0; i < B.n[0]; i += 8) ct.push_back(make_int4(ch.block0 + b, i, j, k));
        continue;
      }
      for (int j = 0; j < B.n[1]; j += TJ)
        for (int i = 0; i < B.n[0]; i += TI) ct.push_back(make_int4(ch.block0 + b, i, j, std::min(TJ, B.n[1] - j)));
    }
    if (c->dim == 2 && mode == 0) {   // this case's launch dispatches its tiles in list order
      std::vector<int> disp(ct.size());
      for (size_t q = 0; q < ct.size(); ++q) disp[q] = (int)q;
      split_tail(ct, disp, wave_slots(c, 0, ch.ns, TI, TJ), TJ);
    }
    tiles.insert(tiles.end(), ct.begin(), ct.end());
    for (const int4& t : ct) tcost.push_back(cells_of(t) * ch.ns);
    ch.ntiles = (int)tiles.size() - ch.tile0;
    t0[k] = ch.tile0;
    nt[k] = ch.ntiles;
    inv[k] = 1.0 / ((double)ch.cells * ch.ns);
  }
  auto claim_order = [&]() {
    std::vector<std::pair<long long, int>> cost(tiles.size());
    for (size_t q = 0; q < tiles.size(); ++q) cost[q] = {-tcost[q], (int)q};
    std::stable_sort(cost.begin(), cost.end());
    std::vector<int> order(cost.size());
    for (size_t q = 0; q < cost.size(); ++q) order[q] = cost[q].second;
    return order;
  };
  std::vector<int> order = claim_order();
  if (c->dim == 2 && mode == 1) {   // one persistent grid claims all tiles in cost order
    const size_t before = tiles.size();
    split_tail(tiles, order, wave_slots(c, 1, c->ns_max, TI, TJ), TJ);
    if (tiles.size() != before) {   // per-case ranges and costs of the new list
      tcost.clear();
      size_t q = 0;
      for (size_t k = 0; k < c->cases.size(); ++k) {
        CaseHost& ch = c->cases[k];
        ch.tile0 = (int)q;
        while (q < tiles.size() && c->blocks[tiles[q].x].cs == (int)k) tcost.push_back(cells_of(tiles[q++]) * ch.ns);
        ch.ntiles = (int)q - ch.tile0;
        t0[k] = ch.tile0;
        nt[k] = ch.ntiles;
      }
      order = claim_order();
    }
  }
  const int n = (int)tiles.size();
  if (n > c->max_tiles) {
    cudaFree(c->d_tiles);
    cudaFree(c->d_order);
    cudaFree(c->d_partials);
    c->d_tiles = nullptr; c->d_order = nullptr; c->d_partials = nullptr;
    HB_CUDA(c, cudaMalloc(&c->d_tiles, sizeof(int4) * std::max(1, n)));
    HB_CUDA(c, cudaMalloc(&c->d_order, sizeof(int) * std::max(1, n)));
    HB_CUDA(c, cudaMalloc(&c->d_partials, sizeof(double) * 8 * std::max(1, n)));
    c->max_tiles = n;
  }
  // balance scratch of the RK stages: 3D tiles (256 cells x ns x nv each) and
  // the 2D tiles of the persistent driver or of a case at the largest static
  // N_s (TI x TJ cells x that N_s x nv)
  bool balg = false;
  for (const auto& ch : c->cases) balg = balg || hbk::tile_balg(ch.ns, 1);
  if (c->dim == 3 || mode == 1 || balg) {
    const size_t per_tile = (c->dim == 3) ? (size_t)c->ns_max * c->nv * (8 * 8 * hbk::tile3d_tk(c->prec == HB_FP32))
                                          : (size_t)hbk::kMaxStaticNS * c->nv * TI * TJ;
    const size_t need = (size_t)std::max(1, n) * per_tile * c->tsize;
    if (need > c->bal_bytes) {
      cudaFree(c->d_bal);
      c->d_bal = nullptr;
      c->bal_bytes = 0;
      HB_CUDA(c, cudaMalloc(&c->d_bal, need));
      c->bal_bytes = need;
    }
  }
  HB_CUDA(c, cudaMemcpy(c->d_tiles, tiles.data(), sizeof(int4) * n, cudaMemcpyHostToDevice));
  HB_CUDA(c, cudaMemcpy(c->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  if (c->jobs_ok) {
    // ghost jobs grouped by the tile owning the root, in destination order
    // within a tile; owner[b][j * columns + i / TI] = tile of row j, column i
    std::vector<std::vector<int>> owner(c->blocks.size());
    std::vector<int> cols(c->blocks.size(), 1);
    for (size_t b = 0; b < c->blocks.size(); ++b) {
      cols[b] = (c->blocks[b].n[0] + TI - 1) / TI;
      owner[b].assign((size_t)cols[b] * c->blocks[b].n[1], -1);
    }
    for (int q = 0; q < n; ++q)
      for (int j = tiles[q].z; j < tiles[q].z + tiles[q].w; ++j)
        owner[tiles[q].x][(size_t)j * cols[tiles[q].x] + tiles[q].y / TI] = q;
    std::vector<std::pair<int, int>> key(c->gjobs.size());
    for (size_t q = 0; q < c->gjobs.size(); ++q) {
      const auto& g = c->gjobs[q];
      key[q] = {owner[g.root_blk][(size_t)g.root_j * cols[g.root_blk] + g.root_i / TI], (int)q};
    }
    std::stable_sort(key.begin(), key.end());
    std::vector<hbk::GhostJob> jobs(key.size());
    std::vector<int2> range(std::max(1, n), make_int2(0, 0));
    for (size_t q = 0; q < key.size(); ++q) {
      jobs[q] = c->gjobs[key[q].second].job;
      int2& r = range[key[q].first];
      if (r.y == 0) r.x = (int)q;
      r.y++;
    }
    if (!c->d_jobs && !jobs.empty()) HB_CUDA(c, cudaMalloc(&c->d_jobs, sizeof(hbk::GhostJob) * jobs.size()));
    if (n > c->job_range_cap) {
      cudaFree(c->d_job_range);
      c->d_job_range = nullptr;
      HB_CUDA(c, cudaMalloc(&c->d_job_range, sizeof(int2) * std::max(1, n)));
      c->job_range_cap = n;
    }
    if (!jobs.empty())
      HB_CUDA(c, cudaMemcpy(c->d_jobs, jobs.data(), sizeof(hbk::GhostJob) * jobs.size(), cudaMemcpyHostToDevice));
    HB_CUDA(c, cudaMemcpy(c->d_job_range, range.data(), sizeof(int2) * std::max(1, n), cudaMemcpyHostToDevice));
  }
  if (!c->d_case_tile0) {
    HB_CUDA(c, cudaMalloc(&c->d_case_tile0, sizeof(int) * c->cases.size()));
    HB_CUDA(c, cudaMalloc(&c->d_case_ntiles, sizeof(int) * c->cases.size()));
    HB_CUDA(c, cudaMalloc(&c->d_case_inv, sizeof(double) * c->cases.size()));
  }
  HB_CUDA(c, cudaMemcpy(c->d_case_tile0, t0.data(), sizeof(int) * t0.size(), cudaMemcpyHostToDevice));
  HB_CUDA(c, cudaMemcpy(c->d_case_ntiles, nt.data(), sizeof(int) * nt.size(), cudaMemcpyHostToDevice));
  HB_CUDA(c, cudaMemcpy(c->d_case_inv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice));
  c->tiles = tiles;
  c->TI = TI;
  c->TJ = TJ;
  c->ti_shift = 0;
  while ((1 << c->ti_shift) < TI) ++c->ti_shift;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  c->graph_kernels.clear();
  return HB_OK;
}

// autotune cache: one line per signature, "key mode TI TJ"
std::string tune_cache_path() {
  const char* e = getenv("HB_TUNE_CACHE");
  if (e && *e) return e;
  const char* h = getenv("HOME");
  return std::string(h && *h ? h : "/tmp") + "/.cache/hbgpu_autotune.txt";
}

bool tune_lookup(const std::string& key, int* mode, int* TI, int* TJ) {
  FILE* f = fopen(tune_cache_path().c_str(), "r");
  if (!f) return false;
  char k[512];
  int m, a, b;
  bool found = false;
  while (fscanf(f, "%511s %d %d %d", k, &m, &a, &b) == 4)
    if (key == k) { *mode = m; *TI = a; *TJ = b; found = true; }
  fclose(f);
  return found;
}

void tune_store(const std::string& key, int mode, int TI, int TJ) {
  const std::string path = tune_cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    std::string dir = path.substr(0, slash);
    for (size_t q = 1; q <= dir.size(); ++q)
      if (q == dir.size() || dir[q] == '/') mkdir(dir.substr(0, q).c_str(), 0755);
  }
  FILE* f = fopen(path.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d\n", key.c_str(), mode, TI, TJ);
  fclose(f);
}

hb_status create_impl(const hb_case_desc* descs, int n, hb_ctx** out) {
  if (!out) return HB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!descs || n <= 0) return HB_ERR_INVALID_ARG;
  hb_ctx* ctx = new hb_ctx();
  auto bad = [&](hb_status s, const std::string& m) {
    ctx->err = m;
    fprintf(stderr, "hb_create: %s\n", m.c_str());
    free_ctx(ctx);
    delete ctx;
    return s;
  };
  const hb_case_desc& d0 = descs[0];
  ctx->dim = d0.dim;
  ctx->nv = d0.dim + 2;
  ctx->prec = d0.prec;
  ctx->viscous = d0.viscous;
  ctx->tsize = (d0.prec == HB_FP32) ? sizeof(float) : sizeof(double);
  if (d0.dim != 2 && d0.dim != 3) return bad(HB_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (d0.prec != HB_FP32 && d0.prec != HB_FP64) return bad(HB_ERR_INVALID_ARG, "bad precision");
  int64_t off = 0, goff = 0, noff = 0;
  for (int c = 0; c < n; ++c) {
    const hb_case_desc& d = descs[c];
    if (d.dim != d0.dim || d.prec != d0.prec || d.viscous != d0.viscous)
      return bad(HB_ERR_INVALID_ARG, "batched cases must share dim, precision and viscosity");
    if (d.n_harm < 0) return bad(HB_ERR_INVALID_ARG, "n_harm < 0");
    if (d.n_harm > HB_MAX_HARMONICS) return bad(HB_ERR_UNSUPPORTED, "n_harm above HB_MAX_HARMONICS");
    if (d.dim == 3 && d.n_harm > HB_MAX_STATIC_HARMONICS)
      return bad(HB_ERR_UNSUPPORTED, "3D contexts support n_harm up to HB_MAX_STATIC_HARMONICS");
    if (d.n_blocks <= 0 || !d.blocks) return bad(HB_ERR_INVALID_ARG, "no blocks");
    if ((d.n_cuts > 0 && !d.cuts) || (d.n_bcs > 0 && !d.bcs) || d.n_cuts < 0 || d.n_bcs < 0)
      return bad(HB_ERR_INVALID_ARG, "null table");
    if (!(d.gamma > 1.0) || !(d.mach > 0.0) || !(d.reynolds > 0.0) || !(d.prandtl > 0.0) ||
        !(d.cfl > 0.0) || !(d.omega >= 0.0) || d.n_bodies < 0)
      return bad(HB_ERR_INVALID_ARG, "bad flow parameters");
    CaseHost ch;
    ch.d = d;
    ch.ns = 2 * d.n_harm + 1;
    ch.nv = d.dim + 2;
    ch.block0 = (int)ctx->blocks.size();
    ch.nblocks = d.n_blocks;
    ch.cells = 0;
    ctx->ns_max = std::max(ctx->ns_max, ch.ns);
    ctx->n_bodies = std::max(ctx->n_bodies, d.n_bodies);
    for (int b = 0; b < d.n_blocks; ++b) {
      const hb_block_desc& bd = d.blocks[b];
      if (bd.ni < 1 || bd.nj < 1 || bd.nk < 1 || (d.dim == 2 && bd.nk != 1) || !bd.nodes)
        return bad(HB_ERR_INVALID_ARG, "bad block " + std::to_string(b));
      BlockDev B;
      memset(&B, 0, sizeof(B));
      B.n[0] = bd.ni; B.n[1] = bd.nj; B.n[2] = bd.nk;
      B.gk = (d.dim == 3) ? 2 : 0;
      B.P[0] = round_up(bd.ni + 4, 8);
      B.P[1] = bd.nj + 4;
      B.P[2] = (d.dim == 3) ? bd.nk + 4 : 1;
      B.plane = (int64_t)B.P[0] * B.P[1] * B.P[2];
      B.plane = (B.plane + 31) / 32 * 32;
      B.off = off;
      B.goff = goff;
      B.noff = noff;
      B.cs = c;
      off += B.plane * ch.ns * ch.nv;
      goff += B.plane;
      const int64_t cells = (int64_t)bd.ni * bd.nj * bd.nk;
      noff += cells * ch.ns * ch.nv;
      ch.cells += cells;
      ctx->blocks.push_back(B);
    }
    ctx->total_cells += ch.cells;
    ctx->interior_values += ch.cells * ch.ns * ch.nv;
    ctx->cases.push_back(ch);
  }
  ctx->state_size = off;
  ctx->geo_cells = goff;
  // tables
  Tables Tb;
  for (auto& ch : ctx->cases) {
    hb_status s = build_tables(ctx, ch, Tb);
    if (s != HB_OK) return bad(s, ctx->err);
  }
  // geometry (FP64 on the host, rounded once)
  std::vector<double> G((size_t)hbk::G_NQ * ctx->geo_cells, 0.0);
  for (auto& ch : ctx->cases)
    for (int b = 0; b < ch.nblocks; ++b)
      compute_geometry(ctx->dim, ch.d.blocks[b], ctx->blocks[ch.block0 + b], G, ctx->geo_cells, ch.d.pivot);
  for (auto& ch : ctx->cases)
    for (int b = 0; b < ch.nblocks; ++b) {
      const BlockDev& B = ctx->blocks[ch.block0 + b];
      // interior cells must be right-handed; ghost cells reflected through a
      // sharp corner may be inverted but must not be degenerate
      const int kg = B.gk;
      for (int k = -kg; k < B.n[2] + kg; ++k)
      for (int j = -2; j < B.n[1] + 2; ++j)
        for (int i = -2; i < B.n[0] + 2; ++i) {
          const double v = G[(size_t)hbk::G_VOL * ctx->geo_cells + B.goff + pcell(B, i, j, k)];
          const bool in = i >= 0 && i < B.n[0] && j >= 0 && j < B.n[1] && k >= 0 && k < B.n[2];
          if (in ? !(v > 0.0) : !(v != 0.0 && std::isfinite(v)))
            return bad(HB_ERR_INVALID_ARG, in ? "non-positive interior cell volume (left-handed block)"
                                              : "degenerate ghost cell (zero volume)");
        }
    }
  cudaError_t e;
#define CK(call)                                        \
  do {                                                  \
    e = (call);                                         \
    if (e != cudaSuccess) {                             \
      return bad(e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA, \
                 std::string(#call) + ": " + cudaGetErrorString(e)); \
    }                                                   \
  } while (0)
  CK(cudaGetDevice(&ctx->device));
  const size_t ts = ctx->tsize;
  CK(cudaMalloc(&ctx->d_geo, ts * hbk::G_NQ * ctx->geo_cells));
  if (ctx->prec == HB_FP32) {
    std::vector<float> Gf(G.size());
    for (size_t q = 0; q < G.size(); ++q) Gf[q] = (float)G[q];
    CK(cudaMemcpy(ctx->d_geo, Gf.data(), ts * Gf.size(), cudaMemcpyHostToDevice));
  } else {
    CK(cudaMemcpy(ctx->d_geo, G.data(), ts * G.size(), cudaMemcpyHostToDevice));
  }
  const size_t csz = (ctx->prec == HB_FP32) ? sizeof(CaseDev<float>) : sizeof(CaseDev<double>);
  std::vector<unsigned char> cbuf(csz * ctx->cases.size());
  for (size_t c = 0; c < ctx->cases.size(); ++c) {
    if (ctx->prec == HB_FP32) fill_case_dev<float>(ctx->cases[c], *(CaseDev<float>*)(cbuf.data() + csz * c));
    else fill_case_dev<double>(ctx->cases[c], *(CaseDev<double>*)(cbuf.data() + csz * c));
  }
  CK(cudaMalloc(&ctx->d_cases, cbuf.size()));
  CK(cudaMemcpy(ctx->d_cases, cbuf.data(), cbuf.size(), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ctx->d_blocks, sizeof(BlockDev) * ctx->blocks.size()));
  CK(cudaMemcpy(ctx->d_blocks, ctx->blocks.data(), sizeof(BlockDev) * ctx->blocks.size(), cudaMemcpyHostToDevice));
  for (int p = 0; p < 3; ++p) {
    ctx->ncopy[p] = (int)Tb.copy[p].size();
    ctx->nbc[p] = (int)Tb.bc[p].size();
    if (ctx->ncopy[p]) {
      CK(cudaMalloc(&ctx->d_copy[p], sizeof(CopyRec) * ctx->ncopy[p]));
      CK(cudaMemcpy(ctx->d_copy[p], Tb.copy[p].data(), sizeof(CopyRec) * ctx->ncopy[p], cudaMemcpyHostToDevice));
    }
    if (ctx->nbc[p]) {
      CK(cudaMalloc(&ctx->d_bc[p], sizeof(BcRec) * ctx->nbc[p]));
      CK(cudaMemcpy(ctx->d_bc[p], Tb.bc[p].data(), sizeof(BcRec) * ctx->nbc[p], cudaMemcpyHostToDevice));
    }
  }
  if (ctx->dim == 2 && ctx->external_cells == 0) {
    int bc_index[3] = {0, 0, 0};
    std::vector<BcRec> all;
    for (int p = 0; p < 3; ++p) {
      bc_index[p] = (int)all.size();
      all.insert(all.end(), Tb.bc[p].begin(), Tb.bc[p].end());
    }
    hb_status s = resolve_ghost_jobs(ctx, Tb, bc_index);
    if (s != HB_OK) return bad(s, ctx->err);
    if (!all.empty()) {
      CK(cudaMalloc(&ctx->d_job_bcs, sizeof(BcRec) * all.size()));
      CK(cudaMemcpy(ctx->d_job_bcs, all.data(), sizeof(BcRec) * all.size(), cudaMemcpyHostToDevice));
    }
    ctx->jobs_ok = true;
  }
  {   // chunks of the large-N_s blocks for the HB source launches, one group per N_s
    std::vector<int2> ch;
    for (int ns = 2 * HB_MAX_STATIC_HARMONICS + 3; ns <= 2 * HB_MAX_HARMONICS + 1; ns += 2) {
      hb_ctx::SrcGroup grp;
      grp.ns = ns;
      grp.first = (int)ch.size();
      for (const CaseHost& cs : ctx->cases) {
        if (cs.ns != ns) continue;
        for (int b = cs.block0; b < cs.block0 + cs.nblocks; ++b)
          for (int64_t c0 = 0; c0 < ctx->blocks[b].plane; c0 += 128) ch.push_back(make_int2(b, (int)c0));
      }
      grp.count = (int)ch.size() - grp.first;
      if (grp.count == 0) continue;
      grp.D.assign((size_t)ns * ns, 0.0);
      for (int n = 0; n < ns; ++n)
        for (int m = 0; m < ns; ++m)
          if (n != m) {
            const int k = n - m;
            grp.D[(size_t)n * ns + m] = 0.5 * ((k % 2 == 0) ? 1.0 : -1.0) / std::sin(M_PI * (double)k / (double)ns);
          }
      ctx->src_groups.push_back(grp);
    }
    ctx->nchunks = (int)ch.size();
    if (ctx->nchunks) {
      CK(cudaMalloc(&ctx->d_chunks, sizeof(int2) * ch.size()));
      CK(cudaMemcpy(ctx->d_chunks, ch.data(), sizeof(int2) * ch.size(), cudaMemcpyHostToDevice));
      CK(cudaMalloc(&ctx->d_H, ts * ctx->state_size));
      CK(cudaMemset(ctx->d_H, 0, ts * ctx->state_size));
    }
  }
  ctx->nwall = (int)Tb.walls.size();
  if (ctx->nwall) {
    CK(cudaMalloc(&ctx->d_walls, sizeof(BcRec) * ctx->nwall));
    CK(cudaMemcpy(ctx->d_walls, Tb.walls.data(), sizeof(BcRec) * ctx->nwall, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_face, sizeof(double) * 3 * ctx->nwall * ctx->ns_max));
  }
  CK(cudaMalloc(&ctx->d_coef, sizeof(double) * 3 * ctx->ns_max * std::max(1, ctx->n_bodies)));
  CK(cudaMalloc(&ctx->d_done, sizeof(unsigned int)));
  CK(cudaMemset(ctx->d_done, 0, sizeof(unsigned int)));
  CK(cudaMalloc(&ctx->d_A, ts * ctx->state_size));
  CK(cudaMalloc(&ctx->d_B, ts * ctx->state_size));
  CK(cudaMemset(ctx->d_A, 0, ts * ctx->state_size));
  CK(cudaMemset(ctx->d_B, 0, ts * ctx->state_size));
  ctx->ring = kMaxK;
  CK(cudaMalloc(&ctx->d_ring, sizeof(double) * 8 * ctx->ring * ctx->cases.size()));
  CK(cudaMalloc(&ctx->d_work, sizeof(unsigned int) * 4 * kMaxK));
  CK(cudaMalloc(&ctx->d_bar, sizeof(unsigned int) * 4));
  CK(cudaMemset(ctx->d_bar, 0, sizeof(unsigned int) * 4));
  {
    const char* e = getenv("HB_BARRIER_TIMEOUT_MS");
    if (e && *e) ctx->timeout_ns = (long long)(atof(e) * 1.0e6);
    e = getenv("HB_TEST_SKIP_BARRIER_CTA");
    if (e && *e) ctx->skip_cta = atoi(e);
  }
  // tuning: cached choice for this signature, else the defaults
  {
    std::string key = "d" + std::to_string(ctx->dim) + "_p" + std::to_string(ctx->prec) + "_v" +
                      std::to_string(ctx->viscous) + "_c" + std::to_string(ctx->cases.size()) + "_n" +
                      std::to_string(ctx->total_cells) + "_b" + std::to_string(ctx->blocks.size()) + "_s";
    for (auto& ch : ctx->cases) key += std::to_string(ch.ns);
    key += "_g2";   // drivers with the fused ghost fill and split wave tails
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    key += "_sm" + std::to_string(sms);
    // a choice timed with another build of the kernels is not reused
    key += std::string("_built ") + __DATE__ + " " + __TIME__;
    for (char& ch : key)
      if (ch == ' ') ch = '_';
    ctx->tune_key = key.substr(0, 500);
    int m = (ctx->cases.size() > 1 && ctx->prec == HB_FP32 && ctx->dim == 2 && !ctx->large_ns()) ? 1 : 0;
    int a = 32, b = 8;
    int mm, aa, bb;
    if (ctx->dim == 2 && tune_lookup(ctx->tune_key, &mm, &aa, &bb)) { m = mm; a = aa; b = bb; }
    ctx->mode = m;
    hb_status st = rebuild_tiles(ctx, a, b, m);
    if (st != HB_OK) return bad(st, ctx->err);
  }
  CK(cudaMalloc(&ctx->d_err, sizeof(int)));
  CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
  CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  // adjoint tables (FP64, 2D, single case)
  if (ctx->prec == HB_FP64 && ctx->dim == 2 && ctx->cases.size() == 1 && ctx->external_cells == 0) {
    const int nb = (int)ctx->blocks.size();
    std::vector<int64_t> foff(nb + 1, 0), coff(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
      const BlockDev& B = ctx->blocks[b];
      foff[b + 1] = foff[b] + (int64_t)(B.n[0] + 1) * B.n[1] + (int64_t)B.n[0] * (B.n[1] + 1);
      coff[b] = B.goff;
    }
    coff[nb] = ctx->geo_cells;
    ctx->nfaces = foff[nb];
    ctx->foff_h = foff;
    std::vector<int> wall((size_t)ctx->nfaces, 0);
    for (const BcRec& r : Tb.walls) {
      const BlockDev& B = ctx->blocks[r.blk];
      const int fi = r.fcell % B.P[0] - 2, fj = r.fcell / B.P[0] - 2;
      const int64_t nfi = (int64_t)(B.n[0] + 1) * B.n[1];
      const int64_t f = (r.p == 0) ? foff[r.blk] + (int64_t)fj * (B.n[0] + 1) + fi
                                   : foff[r.blk] + nfi + (int64_t)fj * B.n[0] + fi;
      wall[f] = r.sgn * (r.body + 1);
    }
    CK(cudaMalloc(&ctx->d_foff, sizeof(int64_t) * (nb + 1)));
    CK(cudaMemcpy(ctx->d_foff, foff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_coff, sizeof(int64_t) * (nb + 1)));
    CK(cudaMemcpy(ctx->d_coff, coff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_wall, sizeof(int) * std::max<int64_t>(1, ctx->nfaces)));
    CK(cudaMemcpy(ctx->d_wall, wall.data(), sizeof(int) * ctx->nfaces, cudaMemcpyHostToDevice));
    for (int p = 0; p < ctx->dim; ++p) {
      // (source block, source cell, kind, record, layer), sorted: a fixed gather order
      std::vector<std::tuple<int, int, int, int, int>> ge;
      for (int k = 0; k < (int)Tb.copy[p].size(); ++k)
        ge.emplace_back(Tb.copy[p][k].src_blk, Tb.copy[p][k].src_cell, 0, k, 0);
      for (int k = 0; k < (int)Tb.bc[p].size(); ++k) {
        const BcRec& r = Tb.bc[p][k];
        if (r.type == HB_BC_FARFIELD) ge.emplace_back(r.blk, r.mcell[0], 1, k, 0);
        else for (int l = 0; l < 2; ++l) ge.emplace_back(r.blk, r.mcell[l], 2, k, l);
      }
      std::sort(ge.begin(), ge.end());
      std::vector<hbk::GhostAdjRow> rows;
      std::vector<hbk::GhostAdjEntry> ent;
      for (size_t q = 0; q < ge.size(); ++q) {
        const int sb = std::get<0>(ge[q]), sc = std::get<1>(ge[q]);
        if (rows.empty() || rows.back().src_blk != sb || rows.back().src_cell != sc)
          rows.push_back({sb, sc, (int)q, (int)q});
        rows.back().end = (int)q + 1;
        ent.push_back({std::get<2>(ge[q]), std::get<3>(ge[q]), std::get<4>(ge[q]), 0});
      }
      ctx->ngrow[p] = (int)rows.size();
      if (!rows.empty()) {
        CK(cudaMalloc(&ctx->d_grow[p], sizeof(hbk::GhostAdjRow) * rows.size()));
        CK(cudaMemcpy(ctx->d_grow[p], rows.data(), sizeof(hbk::GhostAdjRow) * rows.size(), cudaMemcpyHostToDevice));
        CK(cudaMalloc(&ctx->d_gent[p], sizeof(hbk::GhostAdjEntry) * ent.size()));
        CK(cudaMemcpy(ctx->d_gent[p], ent.data(), sizeof(hbk::GhostAdjEntry) * ent.size(), cudaMemcpyHostToDevice));
      }
    }
    ctx->adj_ok = true;
  }
#undef CK
  *out = ctx;
  return HB_OK;
}

// ------------------------------------------------------------ launches --
// every ghost cell of dst from the interior of src in one launch (2D)
template <typename T>
hb_status ghost_fill(hb_ctx* c, const T* src, T* dst, cudaStream_t s) {
  hbk::GhostFillParams<T> p;
  p.cases = (const CaseDev<T>*)c->d_cases;
  p.blocks = c->d_blocks;
  p.g = geo_of<T>(c);
  p.src = src;
  p.dst = dst;
  p.jobs = c->d_jobs;
  p.njobs = (int)c->gjobs.size();
  p.bcs = c->d_job_bcs;
  p.ns_max = c->ns_max;
  if (p.njobs == 0) return HB_OK;
  TimedScope ts(c, 1, s);
  HB_CUDA(c, hbk::launch_ghost_fill<T>(p, s));
  return HB_OK;
}

// halo fill in place: 2D one launch over the resolved ghost chains, 3D the
// pass-ordered cut copies and boundary records (one launch per pass)
template <typename T>
hb_status halos(hb_ctx* c, T* U, cudaStream_t s) {
  if (c->jobs_ok) return ghost_fill<T>(c, U, U, s);
  hbk::HaloParams<T> p;
  p.cases = (const CaseDev<T>*)c->d_cases;
  p.blocks = c->d_blocks;
  p.g = geo_of<T>(c);
  p.U = U;
  p.ns_max = c->ns_max;
  for (int pass = 0; pass < c->dim; ++pass) {
    p.copies = c->d_copy[pass];
    p.ncopy = c->ncopy[pass];
    p.bcs = c->d_bc[pass];
    p.nbc = c->nbc[pass];
    if ((int64_t)(p.ncopy + p.nbc) == 0) continue;
    TimedScope ts(c, 1, s);
    if (c->dim == 3) HB_CUDA(c, hbk::launch_halo3d<T>(p, s));
    else HB_CUDA(c, hbk::launch_halo<T>(p, s));
  }
  return HB_OK;
}

template <typename T>
hbk::StageParams<T> stage_params(hb_ctx* c) {
  hbk::StageParams<T> p;
  memset(&p, 0, sizeof(p));
  p.cases = (const CaseDev<T>*)c->d_cases;
  p.blocks = c->d_blocks;
  p.g = geo_of<T>(c);
  p.TI = c->TI;
  p.TJ = c->TJ;
  p.ti_shift = c->ti_shift;
  return p;
}

// one launch per case (each case has its own snapshot count)
template <typename T>
hb_status stage_all(hb_ctx* c, hbk::StageParams<T> p, int mode, cudaStream_t s) {
  for (auto& ch : c->cases) {
    p.tiles = c->d_tiles + ch.tile0;
    p.ntiles = ch.ntiles;
    double* part = p.partials;
    if (part) p.partials = part + (size_t)8 * ch.tile0;
    const int2* jr = p.job_range;
    if (jr) p.job_range = jr + ch.tile0;
    // the precomputed source serves the large-N_s cases (and time-domain
    // steps); the other cases of a batch form their HB source in the tile
    const T* H = p.H;
    if (p.lam_v == T(0) && ch.ns <= 2 * HB_MAX_STATIC_HARMONICS + 1) p.H = nullptr;
    TimedScope ts(c, 0, s);
    // the 3D tile parks each snapshot's flux balance in R until its epilogue
    if (c->dim == 3 && mode == 1)
      p.R = (T*)c->d_bal + (size_t)ch.tile0 * c->ns_max * c->nv * (8 * 8 * hbk::tile3d_tk(sizeof(T) == 4));
    // (and so does a 2D tile where tile_balg says so)
    if (c->dim == 2 && hbk::tile_balg(ch.ns, mode)) {
      if (!c->d_bal) return fail(c, HB_ERR_OOM, "stage: balance scratch not allocated");
      p.R = (T*)c->d_bal + (size_t)ch.tile0 * hbk::kMaxStaticNS * c->nv * c->TI * c->TJ;
    }
    if (c->dim == 3) HB_CUDA(c, hbk::launch_stage3d<T>(p, ch.ns, c->viscous, mode, s));
    else HB_CUDA(c, hbk::launch_stage<T>(p, ch.ns, c->viscous, mode, s));
    p.partials = part;
    p.job_range = jr;
    p.H = H;
  }
  return HB_OK;
}

// H = V omega D W for the large-N_s cases
template <typename T>
hb_status hb_source(hb_ctx* c, const T* W, cudaStream_t s) {
  for (const auto& grp : c->src_groups) {
    TimedScope ts(c, 1, s);
    HB_CUDA(c, hbk::launch_hb_source<T>((const CaseDev<T>*)c->d_cases, c->d_blocks, geo_of<T>(c),
                                        c->d_chunks + grp.first, grp.count, c->nv, grp.ns, grp.D.data(), W,
                                        (T*)c->d_H, s));
  }
  return HB_OK;
}

template <typename T>
hb_status residual_impl(hb_ctx* c, const T* U, T* R, cudaStream_t s) {
  T* W = (T*)c->d_A;
  c->n_launch++;
  HB_CUDA(c, hbk::launch_copy(W, U, (int64_t)c->tsize * c->state_size, s));
  hb_status st = halos<T>(c, W, s);
  if (st != HB_OK) return st;
  auto p = stage_params<T>(c);
  p.Uprev = W;
  p.R = R;
  st = hb_source<T>(c, W, s);
  if (st != HB_OK) return st;
  if (c->large_ns()) p.H = (const T*)c->d_H;
  return stage_all<T>(c, p, 0, s);
}

// one RK iteration; norms (nv doubles per case block of 8) written to `norm_out`
template <typename T>
hb_status rk_iteration(hb_ctx* c, T* U, double* norm_out, cudaStream_t s, const T* src = nullptr) {
  static const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  T* A = (T*)c->d_A;
  T* Bf = (T*)c->d_B;
  T* in[4] = {U, A, Bf, A};
  T* out[4] = {A, Bf, A, U};
  const bool fused = c->fused();
  for (int st = 0; st < 4; ++st) {
    hb_status r = fused ? HB_OK : halos<T>(c, in[st], s);   // fused: the previous stage filled them
    if (r != HB_OK) return r;
    auto p = stage_params<T>(c);
    if (fused) {
      p.job_range = c->d_job_range;
      p.jobs = c->d_jobs;
      p.job_bcs = c->d_job_bcs;
    }
    p.Uprev = in[st];
    p.U0 = U;
    p.Unext = out[st];
    p.alpha = (T)alpha[st];
    p.partials = (st == 0) ? c->d_partials : nullptr;
    r = hb_source<T>(c, in[st], s);
    if (r != HB_OK) return r;
    if (c->large_ns()) p.H = (const T*)c->d_H;
    p.src = src;
    r = stage_all<T>(c, p, 1, s);
    if (r != HB_OK) return r;
    if (st == 0) {
      // norms per case, fixed order, into norm_out[case][8]
      for (size_t k = 0; k < c->cases.size(); ++k) {
        const CaseHost& ch = c->cases[k];
        c->n_launch++;
        HB_CUDA(c, hbk::launch_norm_finish(c->d_partials + (size_t)8 * ch.tile0, ch.ntiles, c->nv,
                                           1.0 / ((double)ch.cells * ch.ns), norm_out + 8 * k, c->d_err, s));
      }
    }
  }
  return HB_OK;
}

// the cut copies and boundary ghosts of one pass (direction), in place
template <typename T>
hb_status halo_pass(hb_ctx* c, T* U, int pass, cudaStream_t s) {
  hbk::HaloParams<T> p;
  p.cases = (const CaseDev<T>*)c->d_cases;
  p.blocks = c->d_blocks;
  p.g = geo_of<T>(c);
  p.U = U;
  p.ns_max = c->ns_max;
  p.copies = c->d_copy[pass];
  p.ncopy = c->ncopy[pass];
  p.bcs = c->d_bc[pass];
  p.nbc = c->nbc[pass];
  if ((int64_t)(p.ncopy + p.nbc) == 0) return HB_OK;
  TimedScope ts(c, 1, s);
  if (c->dim == 3) HB_CUDA(c, hbk::launch_halo3d<T>(p, s));
  else HB_CUDA(c, hbk::launch_halo<T>(p, s));
  return HB_OK;
}

// one RK stage Uout = U0 - alpha_stage dtau/V R(Uin), the halos of Uin filled
// by the caller; at stage 0 the per-case sums of (R/V)^2 into sums[case][nv]
template <typename T>
hb_status rk_stage_impl(hb_ctx* c, const T* Uin, const T* U0, T* Uout, int stage, double* sums, cudaStream_t s) {
  static const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  auto p = stage_params<T>(c);
  p.Uprev = Uin;
  p.U0 = U0;
  p.Unext = Uout;
  p.alpha = (T)alpha[stage];
  p.partials = (stage == 0 && sums) ? c->d_partials : nullptr;
  hb_status r = hb_source<T>(c, Uin, s);
  if (r != HB_OK) return r;
  if (c->large_ns()) p.H = (const T*)c->d_H;
  r = stage_all<T>(c, p, 1, s);
  if (r != HB_OK) return r;
  if (p.partials)
    for (size_t k = 0; k < c->cases.size(); ++k) {
      const CaseHost& ch = c->cases[k];
      c->n_launch++;
      HB_CUDA(c, hbk::launch_norm_finish(c->d_partials + (size_t)8 * ch.tile0, ch.ntiles, c->nv, 1.0,
                                         sums + (size_t)c->nv * k, c->d_err, s, 1));
    }
  return HB_OK;
}

// one persistent launch of K iterations (norms into the ring)
template <typename T>
hb_status persist_chunk(hb_ctx* c, T* U, int K, cudaStream_t s) {
  static const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  HB_CUDA(c, cudaMemsetAsync(c->d_work, 0, sizeof(unsigned int) * 4 * K, s));
  HB_CUDA(c, cudaMemsetAsync(c->d_bar, 0, sizeof(unsigned int) * 4, s));
  hbk::PersistParams<T> p;
  memset(&p, 0, sizeof(p));
  T* A = (T*)c->d_A;
  T* Bf = (T*)c->d_B;
  T* in[4] = {U, A, Bf, A};
  T* out[4] = {A, Bf, A, U};
  for (int st = 0; st < 4; ++st) {
    p.st[st] = stage_params<T>(c);
    p.st[st].tiles = c->d_tiles;
    p.st[st].ntiles = (int)c->tiles.size();
    p.st[st].Uprev = in[st];
    p.st[st].U0 = U;
    p.st[st].Unext = out[st];
    p.st[st].R = (T*)c->d_bal;   // the tiles' parked balances
    p.st[st].alpha = (T)alpha[st];
    p.st[st].partials = (st == 0) ? c->d_partials : nullptr;
    if (c->fused()) {
      p.st[st].job_range = c->d_job_range;
      p.st[st].jobs = c->d_jobs;
      p.st[st].job_bcs = c->d_job_bcs;
    }
  }
  p.fused = c->fused() ? 1 : 0;
  p.ns_max = c->ns_max;
  for (int pass = 0; pass < c->dim; ++pass) {
    hbk::HaloParams<T>& h = p.halo[pass];
    h.cases = (const CaseDev<T>*)c->d_cases;
    h.blocks = c->d_blocks;
    h.g = geo_of<T>(c);
    h.U = nullptr;
    h.copies = c->d_copy[pass];
    h.ncopy = c->ncopy[pass];
    h.bcs = c->d_bc[pass];
    h.nbc = c->nbc[pass];
    h.ns_max = c->ns_max;
  }
  p.dim = c->dim;
  p.order = c->d_order;
  p.ntiles = (int)c->tiles.size();
  p.work = c->d_work;
  p.bar = c->d_bar;
  p.err = c->d_err;
  p.K = K;
  p.ncases = (int)c->cases.size();
  p.case_tile0 = c->d_case_tile0;
  p.case_ntiles = c->d_case_ntiles;
  p.case_inv = c->d_case_inv;
  p.norms = c->d_ring;
  p.timeout_ns = c->timeout_ns;
  p.skip_cta = c->skip_cta;
  TimedScope ts(c, 0, s);
  int grid = 0;
  HB_CUDA(c, hbk::launch_persist<T>(p, c->viscous, c->TI, c->TJ, s, &grid));
  return HB_OK;
}

// ring [K][ncases][8] -> user norms [K][ncases][nv]
hb_status copy_norms(hb_ctx* c, double* norms, int done, int K, cudaStream_t s) {
  if (!norms) return HB_OK;
  const size_t nc = c->cases.size();
  HB_CUDA(c, cudaMemcpy2DAsync(norms + (size_t)done * nc * c->nv, sizeof(double) * c->nv, c->d_ring,
                               sizeof(double) * 8, sizeof(double) * c->nv, (size_t)K * nc,
                               cudaMemcpyDeviceToDevice, s));
  return HB_OK;
}

// ---- time-domain dual time stepping: one-snapshot cases at physical time t
template <typename T>
hb_status td_iteration(hb_ctx* c, T* U, const T* Un, const T* Unm1, double dt, double* norm_out,
                       cudaStream_t s) {
  static const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  // BDF2, or backward Euler on the first step
  const double a0 = Unm1 ? 1.5 : 1.0, a1 = Unm1 ? -2.0 : -1.0, a2 = Unm1 ? 0.5 : 0.0;
  T* A = (T*)c->d_A;
  T* Bf = (T*)c->d_B;
  T* in[4] = {U, A, Bf, A};
  T* out[4] = {A, Bf, A, U};
  for (int st = 0; st < 4; ++st) {
    {
      TimedScope ts(c, 1, s);
      HB_CUDA(c, hbk::launch_td_source<T>(c->d_blocks, geo_of<T>(c), c->d_td_chunks, c->n_td_chunks, c->nv,
                                          (T)(a0 / dt), (T)(a1 / dt), (T)(a2 / dt), in[st], Un, Unm1,
                                          (T*)c->d_H, s));
    }
    auto p = stage_params<T>(c);
    p.job_range = c->d_job_range;
    p.jobs = c->d_jobs;
    p.job_bcs = c->d_job_bcs;
    p.Uprev = in[st];
    p.U0 = U;
    p.Unext = out[st];
    p.alpha = (T)alpha[st];
    p.partials = (st == 0) ? c->d_partials : nullptr;
    p.H = (const T*)c->d_H;
    p.lam_v = (T)(a0 / dt);
    hb_status r = stage_all<T>(c, p, 1, s);
    if (r != HB_OK) return r;
    if (st == 0)
      for (size_t k = 0; k < c->cases.size(); ++k) {
        const CaseHost& ch = c->cases[k];
        c->n_launch++;
        HB_CUDA(c, hbk::launch_norm_finish(c->d_partials + (size_t)8 * ch.tile0, ch.ntiles, c->nv,
                                           1.0 / (double)ch.cells, norm_out + 8 * k, c->d_err, s));
      }
  }
  return HB_OK;
}

template <typename T>
hb_status td_step_impl(hb_ctx* c, T* U, const T* Un, const T* Unm1, double t, double dt, int n_inner,
                       double* norms, cudaStream_t s) {
  if (!c->d_td_chunks) {   // chunks of 128 padded cells over every block; H buffer
    std::vector<int2> ch;
    for (size_t b = 0; b < c->blocks.size(); ++b)
      for (int64_t c0 = 0; c0 < c->blocks[b].plane; c0 += 128) ch.push_back(make_int2((int)b, (int)c0));
    HB_CUDA(c, cudaMalloc(&c->d_td_chunks, sizeof(int2) * ch.size()));
    HB_CUDA(c, cudaMemcpy(c->d_td_chunks, ch.data(), sizeof(int2) * ch.size(), cudaMemcpyHostToDevice));
    c->n_td_chunks = (int)ch.size();
    if (!c->d_H) HB_CUDA(c, cudaMalloc(&c->d_H, c->tsize * c->state_size));
  }
  // the cases' frame, grid velocity and inflow at time t
  const size_t csz = sizeof(CaseDev<T>);
  c->td_case_buf.resize(csz * c->cases.size());
  for (size_t k = 0; k < c->cases.size(); ++k)
    fill_case_dev<T>(c->cases[k], *(CaseDev<T>*)(c->td_case_buf.data() + csz * k), t);
  HB_CUDA(c, cudaMemcpyAsync(c->d_cases, c->td_case_buf.data(), c->td_case_buf.size(), cudaMemcpyHostToDevice, s));
  HB_CUDA(c, cudaStreamSynchronize(s));   // the host buffer is reused by the next step
  hb_status r = halos<T>(c, U, s);
  if (r != HB_OK) return r;
  const size_t nc = c->cases.size();
  int done = 0;
  while (done < n_inner) {
    const int K = std::min(n_inner - done, c->ring);
    for (int k = 0; k < K; ++k) {
      r = td_iteration<T>(c, U, Un, Unm1, dt, c->d_ring + 8 * nc * k, s);
      if (r != HB_OK) return r;
    }
    r = copy_norms(c, norms, done, K, s);
    if (r != HB_OK) return r;
    done += K;
  }
  return HB_OK;
}

template <typename T>
hb_status rk_chunk_direct(hb_ctx* c, T* U, int K, cudaStream_t s) {
  if (c->fused()) {   // the stages keep the halos filled from here on
    hb_status r = halos<T>(c, U, s);
    if (r != HB_OK) return r;
  }
  if (c->mode == 1 && hbk::persist_available<T>(c->TI, c->TJ)) return persist_chunk<T>(c, U, K, s);
  const size_t nc = c->cases.size();
  for (int k = 0; k < K; ++k) {
    hb_status r = rk_iteration<T>(c, U, c->d_ring + 8 * nc * k, s);
    if (r != HB_OK) return r;
  }
  return HB_OK;
}

template <typename T>
hb_status rk_smooth_impl(hb_ctx* c, T* U, int n_iter, double* norms, cudaStream_t s) {
  int done = 0;
  while (done < n_iter) {
    const int K = std::min(n_iter - done, c->ring);
    const bool persist = c->mode == 1 && hbk::persist_available<T>(c->TI, c->TJ);
    // chunks of two or more iterations (or any persistent chunk) replay a
    // captured graph; a persistent chunk runs directly if capture fails
    // (benchmark timing brackets individual launches, so it runs without graphs)
    bool use_graph = (K >= 2 || persist) && !(persist && c->persist_graph == 0) && !c->timing;
    if (use_graph) {
      auto key = std::make_pair((const void*)U, K * 8 + c->mode);
      auto it = c->graphs.find(key);
      if (it == c->graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        HB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
        c->capturing = true;
        const int64_t n0 = c->n_launch;
        hb_status r = rk_chunk_direct<T>(c, U, K, c->cap_stream);
        c->capturing = false;
        const int64_t nk = c->n_launch - n0;
        c->n_launch = n0;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (r == HB_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        if (r != HB_OK || e != cudaSuccess) {
          cudaGetLastError();
          if (!persist) return r != HB_OK ? r : cuda_fail(c, e, "graph capture");
          c->persist_graph = 0;      // cooperative launch not capturable here
          use_graph = false;
        } else {
          if (persist) c->persist_graph = 1;
          it = c->graphs.emplace(key, ex).first;
          c->graph_kernels[key] = nk;
        }
      }
      if (use_graph) {
        c->n_launch += c->graph_kernels[key];
        HB_CUDA(c, cudaGraphLaunch(it->second, s));
        c->n_graph_replays += 1;
        if (persist) c->n_persist_replays += 1;
      }
    }
    if (!use_graph) {
      hb_status r = rk_chunk_direct<T>(c, U, K, s);
      if (r != HB_OK) return r;
      if (persist) c->n_persist_direct += 1;
    }
    hb_status r = copy_norms(c, norms, done, K, s);
    if (r != HB_OK) return r;
    done += K;
  }
  return HB_OK;
}

// autotuner: time every compiled (driver, tile shape) on a copy of U
template <typename T>
hb_status autotune_impl(hb_ctx* c, const T* U, int iters, cudaStream_t s) {
  void* tmp = nullptr;
  HB_CUDA(c, cudaMalloc(&tmp, c->tsize * c->state_size));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  c->halo_phases = false;
  int bm = c->mode, bi = c->TI, bj = c->TJ;
  hb_status st = HB_OK;
  const int shapes[3][2] = {{32, 8}, {32, 4}, {16, 8}};
  for (int m = 0; m < 2 && st == HB_OK; ++m)
    for (int q = 0; q < 3 && st == HB_OK; ++q) {
      if (m == 1 && (c->large_ns() || !hbk::persist_available<T>(shapes[q][0], shapes[q][1]))) continue;
      if ((st = rebuild_tiles(c, shapes[q][0], shapes[q][1], m)) != HB_OK) break;
      c->mode = m;
      cudaMemcpyAsync(tmp, U, c->tsize * c->state_size, cudaMemcpyDeviceToDevice, s);
      if ((st = rk_smooth_impl<T>(c, (T*)tmp, iters, nullptr, s)) != HB_OK) break;   // warm-up, graphs
      cudaEventRecord(e0, s);
      if ((st = rk_smooth_impl<T>(c, (T*)tmp, iters, nullptr, s)) != HB_OK) break;
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bm = m; bi = shapes[q][0]; bj = shapes[q][1]; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (st != HB_OK) return st;
  st = rebuild_tiles(c, bi, bj, bm);
  c->mode = bm;
  if (st == HB_OK) tune_store(c->tune_key, bm, bi, bj);
  return st;
}

template <typename T>
hb_status forces_filled(hb_ctx* c, const T* W, const T* G, double* coef, double* J, cudaStream_t s);

// U is the caller's (not written): 2D fills the ghosts into the workspace and
// the force kernel reads interior cells from U and ghosts from there
template <typename T>
hb_status forces_impl(hb_ctx* c, const T* U, double* coef, double* J, cudaStream_t s) {
  T* W = (T*)c->d_A;
  if (c->jobs_ok) {
    hb_status st = ghost_fill<T>(c, U, W, s);
    if (st != HB_OK) return st;
    return forces_filled<T>(c, U, W, coef, J, s);
  }
  c->n_launch++;
  HB_CUDA(c, hbk::launch_copy(W, U, (int64_t)c->tsize * c->state_size, s));
  hb_status st = halos<T>(c, W, s);
  if (st != HB_OK) return st;
  return forces_filled<T>(c, W, nullptr, coef, J, s);
}

// forces of a state W whose ghosts are filled (in W, or in G when not null)
template <typename T>
hb_status forces_filled(hb_ctx* c, const T* W, const T* G, double* coef, double* J, cudaStream_t s) {
  hbk::ForceParams<T> p;
  p.cases = (const CaseDev<T>*)c->d_cases;
  p.blocks = c->d_blocks;
  p.g = geo_of<T>(c);
  p.U = W;
  p.G = G;
  p.walls = c->d_walls;
  p.nwall = c->nwall;
  p.ns = c->cases[0].ns;
  p.face_out = c->d_face;
  p.coef = coef;
  p.J = J;
  p.nbodies = c->cases[0].d.n_bodies;
  p.coef_scratch = c->d_coef;
  p.done = c->d_done;
  if (p.nbodies == 0) {
    if (J) HB_CUDA(c, cudaMemsetAsync(J, 0, sizeof(double), s));
    return HB_OK;
  }
  c->n_launch += (p.nwall * p.ns > 0) ? 2 : 1;
  HB_CUDA(c, hbk::launch_forces<T>(p, s));
  return HB_OK;
}

template <typename T>
hb_status init_impl(hb_ctx* c, T* U, const double* noise, double amp, cudaStream_t s) {
  c->n_launch += (int64_t)c->blocks.size();
  if (c->dim == 3) {
    HB_CUDA(c, hbk::launch_init3d<T>((const CaseDev<T>*)c->d_cases, c->d_blocks, (int)c->blocks.size(),
                                     geo_of<T>(c), U, noise, amp, s));
    return HB_OK;
  }
  HB_CUDA(c, hbk::launch_init<T>((const CaseDev<T>*)c->d_cases, c->d_blocks, (int)c->blocks.size(),
                                 geo_of<T>(c), U, noise, amp, c->interior_values, nullptr, s));
  return HB_OK;
}

}  // namespace

// ================================================================== C ABI
// ---- restart files
namespace {
constexpr char kCkptMagic[8] = {'H', 'B', 'R', 'E', 'S', 'T', 'R', '1'};

// FNV-1a over the context's defining integers and flow parameters
uint64_t ctx_signature(const hb_ctx* c) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t k = 0; k < n; ++k) { h ^= b[k]; h *= 1099511628211ull; }
  };
  mix(&c->dim, sizeof(int));
  mix(&c->prec, sizeof(int));
  const int nc = (int)c->cases.size();
  mix(&nc, sizeof(int));
  for (const CaseHost& ch : c->cases) {
    const hb_case_desc& d = ch.d;
    mix(&d.n_harm, sizeof(int));
    mix(&d.n_blocks, sizeof(int));
    mix(&d.viscous, sizeof(int));
    const double prm[6] = {d.mach, d.reynolds, d.gamma, d.omega, d.alpha0_deg, d.pitch_amp_deg};
    mix(prm, sizeof(prm));
  }
  for (const BlockDev& B : c->blocks) mix(B.n, sizeof(B.n));
  return h;
}

struct CkptHeader {
  char magic[8];
  uint64_t signature;
  int64_t values;       // interior values stored
  int64_t iteration;
  int32_t prec, pad;
};

// host copy of the interior of every block in compact order, or the reverse
template <typename T>
void interior_copy(const hb_ctx* c, std::vector<T>& full, std::vector<T>& compact, bool to_compact) {
  int64_t q = 0;
  for (const CaseHost& ch : c->cases)
    for (int b = ch.block0; b < ch.block0 + ch.nblocks; ++b) {
      const BlockDev& B = c->blocks[b];
      for (int n = 0; n < ch.ns; ++n)
        for (int v = 0; v < c->nv; ++v)
          for (int k = 0; k < B.n[2]; ++k)
            for (int j = 0; j < B.n[1]; ++j)
              for (int i = 0; i < B.n[0]; ++i, ++q) {
                const int64_t e = B.off + ((int64_t)n * c->nv + v) * B.plane + pcell(B, i, j, k);
                if (to_compact) compact[q] = full[e];
                else full[e] = compact[q];
              }
    }
}

template <typename T>
hb_status save_impl(hb_ctx* c, const T* U, const char* path, int64_t it, cudaStream_t s) {
  std::vector<T> full((size_t)c->state_size), comp((size_t)c->interior_values);
  HB_CUDA(c, cudaMemcpyAsync(full.data(), U, sizeof(T) * full.size(), cudaMemcpyDeviceToHost, s));
  HB_CUDA(c, cudaStreamSynchronize(s));
  interior_copy<T>(c, full, comp, true);
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kCkptMagic, 8);
  h.signature = ctx_signature(c);
  h.values = c->interior_values;
  h.iteration = it;
  h.prec = c->prec;
  FILE* f = fopen(path, "wb");
  if (!f) return fail(c, HB_ERR_INVALID_ARG, std::string("cannot write ") + path);
  const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(comp.data(), sizeof(T), comp.size(), f) == comp.size();
  if (fclose(f) != 0 || !ok) return fail(c, HB_ERR_INVALID_ARG, std::string("write failed: ") + path);
  return HB_OK;
}

template <typename T>
hb_status load_impl(hb_ctx* c, T* U, const char* path, int64_t* it, cudaStream_t s) {
  FILE* f = fopen(path, "rb");
  if (!f) return fail(c, HB_ERR_INVALID_ARG, std::string("cannot read ") + path);
  CkptHeader h;
  std::vector<T> comp((size_t)c->interior_values);
  bool ok = fread(&h, sizeof(h), 1, f) == 1;
  if (ok && (memcmp(h.magic, kCkptMagic, 8) != 0 || h.prec != c->prec || h.values != c->interior_values ||
             h.signature != ctx_signature(c))) {
    fclose(f);
    return fail(c, HB_ERR_INVALID_ARG, std::string("restart file of another format or context: ") + path);
  }
  ok = ok && fread(comp.data(), sizeof(T), comp.size(), f) == comp.size();
  fclose(f);
  if (!ok) return fail(c, HB_ERR_INVALID_ARG, std::string("truncated restart file: ") + path);
  std::vector<T> full((size_t)c->state_size);
  HB_CUDA(c, cudaMemcpyAsync(full.data(), U, sizeof(T) * full.size(), cudaMemcpyDeviceToHost, s));
  HB_CUDA(c, cudaStreamSynchronize(s));
  interior_copy<T>(c, full, comp, false);
  HB_CUDA(c, cudaMemcpyAsync(U, full.data(), sizeof(T) * full.size(), cudaMemcpyHostToDevice, s));
  HB_CUDA(c, cudaStreamSynchronize(s));
  if (it) *it = h.iteration;
  return HB_OK;
}
}  // namespace

// ---- FP32 smoothing with an FP64 finish (defect correction)
namespace {
uint64_t ctx_signature_any_precision(const hb_ctx* c) {
  hb_ctx tmp;   // only the fields the signature reads
  tmp.dim = c->dim;
  tmp.prec = 0;
  tmp.cases = c->cases;
  tmp.blocks = c->blocks;
  return ctx_signature(&tmp);
}

hb_status defect_impl(hb_ctx* c32, hb_ctx* c64, double* U64, int n_outer, int n_inner, double sigma,
                      double* norms, cudaStream_t s) {
  const int64_t n = c32->state_size;
  for (int k = 0; k < 4; ++k)
    if (!c32->d_dc[k]) HB_CUDA(c32, cudaMalloc(&c32->d_dc[k], sizeof(float) * n));
  if (!c64->d_dc[0]) HB_CUDA(c64, cudaMalloc(&c64->d_dc[0], sizeof(double) * n));
  float* u32 = (float*)c32->d_dc[0];
  float* v32 = (float*)c32->d_dc[1];
  float* r32 = (float*)c32->d_dc[2];
  float* src = (float*)c32->d_dc[3];
  double* r64 = (double*)c64->d_dc[0];
  const size_t nc = c32->cases.size();
  HB_CUDA(c32, cudaMemsetAsync(r32, 0, sizeof(float) * n, s));
  HB_CUDA(c64, cudaMemsetAsync(r64, 0, sizeof(double) * n, s));
  for (int it = 0; it < n_outer; ++it) {
    // the FP64 defect of the current state and the FP32 residual of its rounding
    hb_status r = residual_impl<double>(c64, U64, r64, s);
    if (r != HB_OK) return r;
    HB_CUDA(c32, hbk::launch_cast_down(U64, u32, n, s));
    r = residual_impl<float>(c32, u32, r32, s);
    if (r != HB_OK) return r;
    HB_CUDA(c32, hbk::launch_defect_source(r64, r32, src, sigma, n, s));
    // smooth R32(u32 + d) + (r64 - R32(u32)) = 0 from d = 0 in FP32, then u64 += d
    HB_CUDA(c32, cudaMemcpyAsync(v32, u32, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    r = halos<float>(c32, v32, s);
    if (r != HB_OK) return r;
    for (int k = 0; k < n_inner; ++k) {
      r = rk_iteration<float>(c32, v32, c32->d_ring + (k == 0 ? 0 : 8 * nc), s, src);
      if (r != HB_OK) return r;
    }
    HB_CUDA(c32, hbk::launch_defect_update(U64, v32, u32, sigma, n, s));
    if (norms && n_inner > 0)
      HB_CUDA(c32, cudaMemcpy2DAsync(norms + (size_t)it * nc * c32->nv, sizeof(double) * c32->nv, c32->d_ring,
                                     sizeof(double) * 8, sizeof(double) * c32->nv, nc, cudaMemcpyDeviceToDevice, s));
  }
  return HB_OK;
}
}  // namespace

extern "C" {

hb_status hb_create(const hb_case_desc* desc, hb_ctx** out) { return create_impl(desc, 1, out); }

hb_status hb_create_batch(const hb_case_desc* cases, int n, hb_ctx** out) {
  return create_impl(cases, n, out);
}

hb_status hb_destroy(hb_ctx* ctx) {
  if (!ctx) return HB_ERR_INVALID_ARG;
  free_ctx(ctx);
  delete ctx;
  return HB_OK;
}

int64_t hb_state_size(const hb_ctx* ctx) { return ctx ? ctx->state_size : -1; }

hb_status hb_state_layout(const hb_ctx* ctx, int blk, int64_t* offset, int64_t strides[5], int ext[3]) {
  if (!ctx || blk < 0 || blk >= (int)ctx->blocks.size() || !offset || !strides) return HB_ERR_INVALID_ARG;
  const BlockDev& B = ctx->blocks[blk];
  *offset = B.off;
  strides[0] = B.plane * ctx->nv;
  strides[1] = B.plane;
  strides[2] = (int64_t)B.P[0] * B.P[1];
  strides[3] = B.P[0];
  strides[4] = 1;
  if (ext) { ext[0] = B.P[0]; ext[1] = B.P[1]; ext[2] = B.P[2]; }
  return HB_OK;
}

hb_status hb_init_state(hb_ctx* ctx, void* U, const double* noise, double amp, void* stream) {
  if (!ctx || !U) return fail(ctx, HB_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? init_impl<float>(ctx, (float*)U, noise, amp, s)
                              : init_impl<double>(ctx, (double*)U, noise, amp, s);
}

hb_status hb_halo_pass(hb_ctx* ctx, void* U, int pass, void* stream) {
  if (!ctx || !U || pass < 0 || pass >= ctx->dim) return fail(ctx, HB_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? halo_pass<float>(ctx, (float*)U, pass, s) : halo_pass<double>(ctx, (double*)U, pass, s);
}

hb_status hb_rk_stage(hb_ctx* ctx, const void* Uin, const void* U0, void* Uout, int stage, double* norm_sums,
                      void* stream) {
  if (!ctx || !Uin || !U0 || !Uout || stage < 0 || stage > 3) return fail(ctx, HB_ERR_INVALID_ARG, "bad argument");
  if (Uin == Uout) return fail(ctx, HB_ERR_INVALID_ARG, "Uout must not alias Uin");
  if (ctx->dim != 2) return fail(ctx, HB_ERR_UNSUPPORTED, "hb_rk_stage: 2D contexts");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32
             ? rk_stage_impl<float>(ctx, (const float*)Uin, (const float*)U0, (float*)Uout, stage, norm_sums, s)
             : rk_stage_impl<double>(ctx, (const double*)Uin, (const double*)U0, (double*)Uout, stage, norm_sums, s);
}

hb_status hb_pack_halo(hb_ctx* ctx, const void* U, const int64_t* idx, int64_t n, void* buf, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!U || !idx || !buf))) return fail(ctx, HB_ERR_INVALID_ARG, "bad argument");
  ctx->n_launch += n > 0;
  HB_CUDA(ctx, hbk::launch_halo_pack(U, idx, n, buf, ctx->prec == HB_FP32, false, (cudaStream_t)stream));
  return HB_OK;
}

hb_status hb_unpack_halo(hb_ctx* ctx, void* U, const int64_t* idx, int64_t n, const void* buf, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!U || !idx || !buf))) return fail(ctx, HB_ERR_INVALID_ARG, "bad argument");
  ctx->n_launch += n > 0;
  HB_CUDA(ctx, hbk::launch_halo_pack(U, idx, n, const_cast<void*>(buf), ctx->prec == HB_FP32, true,
                                     (cudaStream_t)stream));
  return HB_OK;
}

hb_status hb_exchange_halos(hb_ctx* ctx, void* U, void* stream) {
  if (!ctx || !U) return fail(ctx, HB_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? halos<float>(ctx, (float*)U, s) : halos<double>(ctx, (double*)U, s);
}

hb_status hb_residual(hb_ctx* ctx, const void* U, void* R, void* stream) {
  if (!ctx || !U || !R) return fail(ctx, HB_ERR_INVALID_ARG, "null argument");
  if (U == R) return fail(ctx, HB_ERR_INVALID_ARG, "U and R must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? residual_impl<float>(ctx, (const float*)U, (float*)R, s)
                              : residual_impl<double>(ctx, (const double*)U, (double*)R, s);
}

hb_status hb_rk_smooth(hb_ctx* ctx, void* U, int n_iter, double* norms, void* stream) {
  if (!ctx || !U || n_iter < 0) return fail(ctx, HB_ERR_INVALID_ARG, "bad argument");
  if (ctx->external_cells)
    return fail(ctx, HB_ERR_UNSUPPORTED, "external cuts: advance with hb_halo_pass / hb_rk_stage and the caller's exchange");
  if (n_iter == 0) return HB_OK;
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? rk_smooth_impl<float>(ctx, (float*)U, n_iter, norms, s)
                              : rk_smooth_impl<double>(ctx, (double*)U, n_iter, norms, s);
}

hb_status hb_forces(hb_ctx* ctx, const void* U, double* coef, double* J, void* stream) {
  if (!ctx || !U) return fail(ctx, HB_ERR_INVALID_ARG, "null argument");
  if (ctx->cases.size() != 1) return fail(ctx, HB_ERR_UNSUPPORTED, "hb_forces needs a single-case context");
  if (ctx->dim == 3 && ctx->cases[0].d.n_bodies > 0)
    return fail(ctx, HB_ERR_UNSUPPORTED, "3D force integration is not built");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? forces_impl<float>(ctx, (const float*)U, coef, J, s)
                              : forces_impl<double>(ctx, (const double*)U, coef, J, s);
}

hb_status hb_adjoint_residual(hb_ctx* ctx, const void* U, const void* psi, double J_seed, void* r_adj,
                              double* J_dev, void* stream) {
  if (!ctx || !U || !psi || !r_adj) return fail(ctx, HB_ERR_INVALID_ARG, "null argument");
  if (!ctx->adj_ok) return fail(ctx, HB_ERR_UNSUPPORTED, "the adjoint needs a single-case FP64 2D context");
  if (r_adj == U || r_adj == psi) return fail(ctx, HB_ERR_INVALID_ARG, "r_adj must not alias U or psi");
  cudaStream_t s = (cudaStream_t)stream;
  const int ns = ctx->cases[0].ns;
  if (!ctx->d_adjbuf) {
    cudaError_t e = cudaMalloc(&ctx->d_adjbuf, sizeof(double) * 32 * ctx->nfaces * ns);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(adjoint face buffer)");
  }
  double* W = (double*)ctx->d_A;
  ctx->n_launch++;
  HB_CUDA(ctx, hbk::launch_copy(W, U, (int64_t)sizeof(double) * ctx->state_size, s));
  hb_status st = halos<double>(ctx, W, s);
  if (st != HB_OK) return st;
  hbk::AdjParams p;
  p.cases = (const CaseDev<double>*)ctx->d_cases;
  p.blocks = ctx->d_blocks;
  p.g = geo_of<double>(ctx);
  p.nblocks = (int)ctx->blocks.size();
  p.ns = ns;
  p.foff = ctx->d_foff;
  p.coff = ctx->d_coff;
  p.nfaces = ctx->nfaces;
  p.ncells_padded = ctx->geo_cells;
  p.U = W;
  p.psi = (const double*)psi;
  p.J_seed = J_seed;
  p.wall = ctx->d_wall;
  p.buf = ctx->d_adjbuf;
  p.out = (double*)ctx->d_B;
  hbk::AdjGhostPass gp[3];
  for (int q = 0; q < ctx->dim; ++q) {
    gp[q].rows = ctx->d_grow[q];
    gp[q].nrows = ctx->ngrow[q];
    gp[q].ent = ctx->d_gent[q];
    gp[q].copies = ctx->d_copy[q];
    gp[q].bcs = ctx->d_bc[q];
  }
  ctx->n_launch += 3 + ctx->dim;
  HB_CUDA(ctx, hbk::launch_adjoint(p, gp, ctx->dim, (double*)r_adj, s));
  if (J_dev) return forces_filled<double>(ctx, W, nullptr, nullptr, J_dev, s);
  return HB_OK;
}

hb_status hb_autotune(hb_ctx* ctx, const void* U, int iters, void* stream) {
  if (!ctx || !U || iters < 1) return fail(ctx, HB_ERR_INVALID_ARG, "bad argument");
  if (ctx->dim == 3) return HB_OK;   // one 3D tile shape and driver: nothing to choose
  if (ctx->external_cells) return fail(ctx, HB_ERR_UNSUPPORTED, "external cuts: the autotuner times hb_rk_smooth");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? autotune_impl<float>(ctx, (const float*)U, iters, s)
                              : autotune_impl<double>(ctx, (const double*)U, iters, s);
}

hb_status hb_set_tuning(hb_ctx* ctx, int mode, int TI, int TJ) {
  if (!ctx || mode < 0 || mode > 3) return fail(ctx, HB_ERR_INVALID_ARG, "bad tuning");
  const bool phases = (mode & 2) != 0;
  mode &= 1;
  if (ctx->dim == 3) return fail(ctx, HB_ERR_UNSUPPORTED, "3D contexts use fixed 8x8x8 (FP32) or 8x8x4 (FP64) tiles, one launch per phase");
  const bool ok = (TI == 32 && TJ == 8) || (TI == 32 && TJ == 4) || (TI == 16 && TJ == 8);
  if (!ok) return fail(ctx, HB_ERR_UNSUPPORTED, "tile shape not built");
  const bool pok = ctx->prec == HB_FP32 ? hbk::persist_available<float>(TI, TJ)
                                        : hbk::persist_available<double>(TI, TJ);
  if (mode == 1 && !pok) return fail(ctx, HB_ERR_UNSUPPORTED, "persistent driver not built for this shape");
  if (mode == 1 && ctx->large_ns())
    return fail(ctx, HB_ERR_UNSUPPORTED, "persistent driver: n_harm above HB_MAX_STATIC_HARMONICS");
  hb_status st = rebuild_tiles(ctx, TI, TJ, mode);
  if (st != HB_OK) return st;
  ctx->mode = mode;
  ctx->halo_phases = phases;
  return HB_OK;
}

hb_status hb_get_tuning(const hb_ctx* ctx, int* mode, int* TI, int* TJ) {
  if (!ctx) return HB_ERR_INVALID_ARG;
  if (mode) *mode = ctx->mode | (ctx->halo_phases ? 2 : 0);
  if (TI) *TI = ctx->TI;
  if (TJ) *TJ = ctx->TJ;
  return HB_OK;
}

hb_status hb_set_timing(hb_ctx* ctx, int enable) {
  if (!ctx) return HB_ERR_INVALID_ARG;
  ctx->timing = enable ? 1 : 0;
  return HB_OK;
}

hb_status hb_kernel_stats(hb_ctx* ctx, int which, double* ms, int64_t* launches, int reset) {
  if (!ctx || which < 0 || which > 2) return HB_ERR_INVALID_ARG;
  for (auto& t : ctx->pending) {
    HB_CUDA(ctx, cudaEventSynchronize(t.b));
    float e = 0.0f;
    HB_CUDA(ctx, cudaEventElapsedTime(&e, t.a, t.b));
    ctx->t_ms[t.cls] += e;
    ctx->n_timed[t.cls] += 1;
    ctx->pool.push_back(t.a);
    ctx->pool.push_back(t.b);
  }
  ctx->pending.clear();
  if (ms) *ms = (which < 2) ? ctx->t_ms[which] : 0.0;
  if (launches) *launches = (which < 2) ? ctx->n_timed[which] : ctx->n_launch;
  if (reset) {
    ctx->t_ms[0] = ctx->t_ms[1] = 0.0;
    ctx->n_timed[0] = ctx->n_timed[1] = 0;
    ctx->n_launch = 0;
  }
  return HB_OK;
}

hb_status hb_graph_info(const hb_ctx* ctx, int* persist_captured, int64_t counts[3]) {
  if (!ctx) return HB_ERR_INVALID_ARG;
  if (persist_captured) *persist_captured = ctx->persist_graph;
  if (counts) {
    counts[0] = ctx->n_graph_replays;
    counts[1] = ctx->n_persist_replays;
    counts[2] = ctx->n_persist_direct;
  }
  return HB_OK;
}

hb_status hb_save_state(hb_ctx* ctx, const void* U, const char* path, int64_t iteration, void* stream) {
  if (!ctx || !U || !path) return fail(ctx, HB_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? save_impl<float>(ctx, (const float*)U, path, iteration, s)
                              : save_impl<double>(ctx, (const double*)U, path, iteration, s);
}

hb_status hb_load_state(hb_ctx* ctx, void* U, const char* path, int64_t* iteration, void* stream) {
  if (!ctx || !U || !path) return fail(ctx, HB_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32 ? load_impl<float>(ctx, (float*)U, path, iteration, s)
                              : load_impl<double>(ctx, (double*)U, path, iteration, s);
}

hb_status hb_td_step(hb_ctx* ctx, void* U, const void* U_n, const void* U_nm1, double t, double dt,
                     int n_inner, double* norms, void* stream) {
  if (!ctx || !U || !U_n || n_inner < 0 || !(dt > 0.0) || !(t >= 0.0))
    return fail(ctx, HB_ERR_INVALID_ARG, "bad argument");
  if (ctx->dim != 2 || ctx->ns_max != 1 || !ctx->jobs_ok)
    return fail(ctx, HB_ERR_UNSUPPORTED, "time-domain stepping needs 2D cases with n_harm = 0");
  if (n_inner == 0) return HB_OK;
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->prec == HB_FP32
             ? td_step_impl<float>(ctx, (float*)U, (const float*)U_n, (const float*)U_nm1, t, dt, n_inner, norms, s)
             : td_step_impl<double>(ctx, (double*)U, (const double*)U_n, (const double*)U_nm1, t, dt, n_inner,
                                    norms, s);
}

hb_status hb_defect_correction(hb_ctx* ctx32, hb_ctx* ctx64, void* U64, int n_outer, int n_inner, double sigma,
                               double* norms, void* stream) {
  if (!ctx32 || !ctx64 || !U64 || n_outer < 0 || n_inner < 0 || !(sigma > 0.0))
    return fail(ctx32, HB_ERR_INVALID_ARG, "bad argument");
  if (ctx32->prec != HB_FP32 || ctx64->prec != HB_FP64 || ctx32->dim != 2 ||
      ctx32->state_size != ctx64->state_size ||
      ctx_signature_any_precision(ctx32) != ctx_signature_any_precision(ctx64))
    return fail(ctx32, HB_ERR_INVALID_ARG, "defect correction needs an FP32 and an FP64 context of the same 2D cases");
  if (ctx32->large_ns()) return fail(ctx32, HB_ERR_UNSUPPORTED, "defect correction: n_harm above HB_MAX_STATIC_HARMONICS");
  return defect_impl(ctx32, ctx64, (double*)U64, n_outer, n_inner, sigma, norms, (cudaStream_t)stream);
}

hb_status hb_sync_status(hb_ctx* ctx, void* stream) {
  if (!ctx) return HB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  HB_CUDA(ctx, cudaStreamSynchronize(s));
  int e = 0;
  HB_CUDA(ctx, cudaMemcpy(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  HB_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
  if (e == HB_ERR_NONFINITE) return fail(ctx, HB_ERR_NONFINITE, "non-finite residual norm");
  if (e == HB_ERR_TIMEOUT) return fail(ctx, HB_ERR_TIMEOUT, "device wait timed out");
  if (e != 0) return fail(ctx, HB_ERR_CUDA, "device error word " + std::to_string(e));
  return HB_OK;
}

const char* hb_last_error(const hb_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

}  // extern "C"
