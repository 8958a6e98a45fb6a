// Internal interface of the FP64 2D adjoint kernels (hb_adjoint.cu).
#pragma once

#include <cstdint>

#include "hb_internal.h"

namespace hbk {

struct AdjParams {
  const CaseDev<double>* cases;
  const BlockDev* blocks;
  Geo<double> g;
  int nblocks, ns;
  const int64_t* foff;      // [nblocks+1] face offsets: i-faces (n0+1)*n1 then j-faces n0*(n1+1)
  const int64_t* coff;      // [nblocks+1] padded-cell offsets (one plane per block)
  int64_t nfaces, ncells_padded;
  const double* U;          // primal state with ghosts filled
  const double* psi;        // residual adjoint, state layout (ghost entries ignored)
  double J_seed;
  const int* wall;          // [nfaces]: 0, or +-(body+1) with the sign of the wall's outward side
  double* buf;              // [nfaces][ns][8 slots][4]
  double* out;              // adjoint over all padded cells, state layout
};

// ghost-map transpose: one row per source cell, entries in a fixed order
struct GhostAdjRow { int src_blk, src_cell, begin, end; };
struct GhostAdjEntry { int kind, rec, layer, pad; };   // kind 0 copy, 1 farfield, 2 wall layer

struct AdjGhostPass {
  const GhostAdjRow* rows;
  int nrows;
  const GhostAdjEntry* ent;
  const CopyRec* copies;
  const BcRec* bcs;
};

cudaError_t launch_adjoint(const AdjParams& p, const AdjGhostPass* passes, int npass, double* r_adj,
                           cudaStream_t s);

}  // namespace hbk
