// 3D tile kernel of the HB residual path: the same method and readings as the
// 2D kernel (hb_kernels.cuh) with five conservative variables, three face
// directions and the full 3x3 Stokes stress.
//
// One CTA owns an 8 x 8 x 8 (FP32) or 8 x 8 x 4 (FP64) tile of one block and
// loops over all snapshots.
// Once per stage it stages the static geometry in shared memory: 1/V of the
// region, the low-face vectors of every face the gradient ring and the tile
// close over, and the centre differences of the tile's faces.  Per snapshot
// it stages primitives (rho, u, v, w, p) and T of the tile plus a 2-cell halo,
// computes Green-Gauss gradients of (u, v, w, T) on the 1-cell ring, then
// every face of the tile once (MUSCL + van Albada, Roe, viscous), and parks
// the flux balance of each own cell in global memory (the residual output, or
// a balance scratch in an RK stage); the HB source and the RK update run in
// the epilogue.
#pragma once

#include "hb_kernels.cuh"

namespace hbk {

constexpr int T3I = 8, T3J = 8;

// Roe flux of the 3D path, written as roe2d with a third velocity component
template <typename T>
__device__ __forceinline__ void roe3d(const T* WL, const T* WR, T Sx, T Sy, T Sz, T vgn, T gm1, T gg1,
                                      int efix, T efrac, T hef, T* F) {
  const T A2 = Sx * Sx + Sy * Sy + Sz * Sz;
  const T iA = Ar<T>::rsq(A2);
  const T hA = T(0.5) * (A2 * iA);
  const T nx = Sx * iA, ny = Sy * iA, nz = Sz * iA;
  T irL, irR;
  Ar<T>::rcp2(WL[0], WR[0], irL, irR);
  const T qL = WL[1] * nx + WL[2] * ny + WL[3] * nz;
  const T qR = WR[1] * nx + WR[2] * ny + WR[3] * nz;
  const T kL = T(0.5) * (WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3]);
  const T kR = T(0.5) * (WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3]);
  const T HL = gg1 * WL[4] * irL + kL;
  const T HR = gg1 * WR[4] * irR + kR;
  const T rr = WR[0] * irL;
  const T r = rr * Ar<T>::rsq(rr);
  const T rt = r * WL[0];
  const T inv1r = Ar<T>::rcp(T(1) + r);
  const T ut = (WL[1] + r * WR[1]) * inv1r;
  const T vt = (WL[2] + r * WR[2]) * inv1r;
  const T wt = (WL[3] + r * WR[3]) * inv1r;
  const T Ht = (HL + r * HR) * inv1r;
  const T kt = T(0.5) * (ut * ut + vt * vt + wt * wt);
  const T ct2 = gm1 * (Ht - kt);
  const T ict = Ar<T>::rsq(ct2);
  const T ct = ct2 * ict;
  const T ict2 = ict * ict;
  const T qt = ut * nx + vt * ny + wt * nz;
  const T qtr = qt - vgn;
  T l1 = fabs(qtr - ct), l2 = fabs(qtr), l3 = fabs(qtr + ct);
  if (efix) {
    const T del = efrac * ct, d2 = del * del, hid = hef * ict;
    l1 = l1 < del ? (l1 * l1 + d2) * hid : l1;
    l3 = l3 < del ? (l3 * l3 + d2) * hid : l3;
  }
  const T dp = WR[4] - WL[4], drho = WR[0] - WL[0], dq = qR - qL;
  const T m = rt * ct * dq, h = T(0.5) * ict2;
  const T w1 = l1 * ((dp - m) * h), w3 = l3 * ((dp + m) * h);
  const T l2a2 = l2 * (drho - dp * ict2), l2rt = l2 * rt;
  const T dux = (WR[1] - WL[1]) - dq * nx;
  const T duy = (WR[2] - WL[2]) - dq * ny;
  const T duz = (WR[3] - WL[3]) - dq * nz;
  const T s13 = w1 + w3, dw = ct * (w3 - w1);
  const T D0 = s13 + l2a2;
  const T D1 = ut * D0 + nx * dw + l2rt * dux;
  const T D2 = vt * D0 + ny * dw + l2rt * duy;
  const T D3 = wt * D0 + nz * dw + l2rt * duz;
  const T D4 = Ht * s13 + qt * dw + l2a2 * kt + l2rt * (ut * dux + vt * duy + wt * duz);
  const T mL = WL[0] * (qL - vgn), mR = WR[0] * (qR - vgn);
  const T ps = WL[4] + WR[4];
  F[0] = hA * (mL + mR - D0);
  F[1] = hA * (mL * WL[1] + mR * WR[1] + ps * nx - D1);
  F[2] = hA * (mL * WL[2] + mR * WR[2] + ps * ny - D2);
  F[3] = hA * (mL * WL[3] + mR * WR[3] + ps * nz - D3);
  F[4] = hA * (mL * HL + mR * HR + ps * vgn - D4);
}

// viscous flux through S from gradients gL, gR [4 quantities][3] (u, v, w, T),
// cell values phiL, phiR (u, v, w, T) and the centre difference t = x_R - x_L
template <typename T>
__device__ __forceinline__ void visc3d(const T* gL, const T* gR, const T* pL, const T* pR, T tx, T ty, T tz,
                                       T Sx, T Sy, T Sz, T mu, T kap, T* Fv) {
  const T il = Ar<T>::rsq(tx * tx + ty * ty + tz * tz);
  const T e[3] = {tx * il, ty * il, tz * il};
  T g[12];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) b[a] = T(0.5) * (gL[3 * q + a] + gR[3 * q + a]);
    const T corr = (pR[q] - pL[q]) * il - (b[0] * e[0] + b[1] * e[1] + b[2] * e[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) g[3 * q + a] = b[a] + corr * e[a];
  }
  const T div = g[0] + g[4] + g[8];
  const T S[3] = {Sx, Sy, Sz};
  T f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T tau = mu * (g[3 * a + c] + g[3 * c + a]);
      if (a == c) tau -= T(2.0 / 3.0) * mu * div;
      s += tau * S[c];
    }
    f[a] = s;
  }
  Fv[0] = T(0);
  Fv[1] = f[0];
  Fv[2] = f[1];
  Fv[3] = f[2];
  Fv[4] = T(0.5) * ((pL[0] + pR[0]) * f[0] + (pL[1] + pR[1]) * f[1] + (pL[2] + pR[2]) * f[2]) +
          kap * (g[9] * Sx + g[10] * Sy + g[11] * Sz);
}

// region (tile + 2-cell halo), gradient ring (tile + 1 cell), faces of the
// tile; tk the tile's k depth (tile3d_tk)
constexpr int R3I = T3I + 4, R3J = T3J + 4;
constexpr int G3I = T3I + 2, G3J = T3J + 2;
__host__ __device__ constexpr int nr3(int tk) { return R3I * R3J * (tk + 4); }
__host__ __device__ constexpr int ng3(int tk) { return G3I * G3J * (tk + 2); }
__host__ __device__ constexpr int nf3(int tk) { return (T3I + 1) * T3J * tk + T3I * (T3J + 1) * tk + T3I * T3J * (tk + 1); }
// low-face vectors along d of the ring box extended by one cell on the high
// side along d: every face a ring cell closes over, and every face of the tile
__host__ __device__ constexpr int sbox3_i(int d) { return G3I + (d == 0); }
__host__ __device__ constexpr int sbox3_j(int d) { return G3J + (d == 1); }
__host__ __device__ constexpr int sbox3_n(int d, int tk) { return sbox3_i(d) * sbox3_j(d) * (tk + 2 + (d == 2)); }
__host__ __device__ constexpr int sbox3_off(int d, int tk) {
  return d == 0 ? 0 : (d == 1 ? 3 * sbox3_n(0, tk) : 3 * (sbox3_n(0, tk) + sbox3_n(1, tk)));
}
__host__ __device__ constexpr int nsb3(int tk) { return 3 * (sbox3_n(0, tk) + sbox3_n(1, tk) + sbox3_n(2, tk)); }

__host__ __device__ constexpr size_t tile3d_smem_elems(int NS, int tk) {
  return (size_t)7 * nr3(tk) + (size_t)12 * ng3(tk) + (size_t)5 * nf3(tk) + (size_t)nsb3(tk) + (size_t)3 * nf3(tk) +
         (size_t)NS * NS;
}

template <typename T, int NS, bool VISC, int MODE>
__device__ __forceinline__ void tile3d(const StageParams<T>& P, int t, T* sm) {
  constexpr int NV = 5;
  constexpr int TI = T3I, TJ = T3J, TK = tile3d_tk(sizeof(T) == 4), NT = TI * TJ * TK;
  constexpr int RI = R3I, RJ = R3J, R3K = TK + 4, NR = nr3(TK);
  constexpr int GI = G3I, GJ = G3J, GK = TK + 2, NG = ng3(TK);
  constexpr int NGU = TI * TJ * TK + 2 * (TJ * TK + TI * TK + TI * TJ);
  constexpr int NFI = (TI + 1) * TJ * TK, NFJ = TI * (TJ + 1) * TK, NF = nf3(TK);
  const int4 tl = P.tiles[t];
  const BlockDev B = P.blocks[tl.x];
  const CaseDev<T>* C = P.cases + B.cs;
  const int i0 = tl.y, j0 = tl.z, k0 = tl.w;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int P0 = B.P[0], P1 = B.P[1];
  const int n0 = B.n[0], n1 = B.n[1], n2 = B.n[2];
  const int64_t sJ = P0, sK = (int64_t)P0 * P1;

  T* sW = sm;              // [NR][4] (u, v, w, p) of each cell
  T* sRT = sW + 4 * NR;    // [NR][2] (rho, T = gamma p / rho)
  T* sIV = sRT + 2 * NR;   // [NR]
  T* sG = sIV + NR;        // [NG][12] gradients of (u, v, w, T), (x, y, z) each, ring box order
  T* sF = sG + 12 * NG;    // [NV][NF]
  T* sSb = sF + NV * NF;   // [d][3][box of d] static low-face vectors
  T* sDC = sSb + nsb3(TK);     // [3][NF] static centre differences of the tile's faces
  T* sD = sDC + 3 * NF;    // [NS][NS]

  const T gam = C->gamma, gm1 = C->gamma - T(1), eps = C->eps, efrac = C->ent_frac;
  const T gg1 = gam / gm1, hef = T(0.5) / efrac;
  const T mu = C->mu, kap = C->kappa, omega = C->omega;
  const int efix = C->entropy_fix;
  const bool moving = C->motion != 0;

  auto rcell = [&](int ri, int rj, int rk) { return (rk * RJ + rj) * RI + ri; };
  auto pcell = [&](int i, int j, int k) -> int64_t { return (int64_t)(k + 2) * sK + (int64_t)(j + 2) * sJ + (i + 2); };
  auto inpad = [&](int i, int j, int k) { return i <= n0 + 1 && j <= n1 + 1 && k <= n2 + 1; };
  // storage index of ring-box position (gi, gj, gk) (cell i0-1+gi, ...) in the face-vector box of d
  auto sbidx = [&](int d, int gi, int gj, int gk) { return (gk * sbox3_j(d) + gj) * sbox3_i(d) + gi; };
  // face work item fq -> direction and the tile position of the cell whose low face it is
  auto face_of = [&](int fq, int& d, int& fi, int& fj, int& fk) {
    if (fq < NFI) { d = 0; fi = fq % (TI + 1); fj = (fq / (TI + 1)) % TJ; fk = fq / ((TI + 1) * TJ); }
    else if (fq < NFI + NFJ) { const int q2 = fq - NFI; d = 1; fi = q2 % TI; fj = (q2 / TI) % (TJ + 1); fk = q2 / (TI * (TJ + 1)); }
    else { const int q3 = fq - NFI - NFJ; d = 2; fi = q3 % TI; fj = (q3 / TI) % TJ; fk = q3 / (TI * TJ); }
  };
  auto face_used = [&](int d, int Ri, int Rj, int Rk) {
    return !(Ri > n0 - (d != 0) || Rj > n1 - (d != 1) || Rk > n2 - (d != 2));
  };

  // ---- static geometry, once per stage: 1/V of the region, the low-face
  // vectors of the ring boxes and the centre differences of the tile's faces
  // (every load of a thread issued before the first is used; blockDim.x = NT)
  {
    constexpr int ITR = (NR + NT - 1) / NT;
    constexpr int ITS = (sbox3_n(2, TK) + NT - 1) / NT;   // the largest of the three boxes
    T vq[ITR], sq[3][ITS][3];
#pragma unroll
    for (int it = 0; it < ITR; ++it) {
      const int r = tid + it * NT;
      const int ri = r % RI, rj = (r / RI) % RJ, rk = r / (RI * RJ);
      const int i = i0 - 2 + ri, j = j0 - 2 + rj, k = k0 - 2 + rk;
      vq[it] = (r < NR && inpad(i, j, k)) ? P.g.q[G_VOL][B.goff + pcell(i, j, k)] : T(1);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int it = 0; it < ITS; ++it) {
        const int e = tid + it * NT;
        const int EI = sbox3_i(d), EJ = sbox3_j(d);
        const int gi = e % EI, gj = (e / EI) % EJ, gk = e / (EI * EJ);
        const int i = i0 - 1 + gi, j = j0 - 1 + gj, k = k0 - 1 + gk;
        const bool in = e < sbox3_n(d, TK) && inpad(i, j, k);
        const int64_t c = B.goff + pcell(i, j, k);
#pragma unroll
        for (int a = 0; a < 3; ++a) sq[d][it][a] = in ? P.g.q[G_S + 3 * d + a][c] : T(0);
      }
#pragma unroll
    for (int it = 0; it < ITR; ++it)
      if (tid + it * NT < NR) sIV[tid + it * NT] = Ar<T>::rcp(vq[it]);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int it = 0; it < ITS; ++it) {
        const int e = tid + it * NT;
        if (e < sbox3_n(d, TK))
#pragma unroll
          for (int a = 0; a < 3; ++a) sSb[sbox3_off(d, TK) + a * sbox3_n(d, TK) + e] = sq[d][it][a];
      }
  }
  if (VISC) {
    constexpr int ITF = (NF + NT - 1) / NT;
    T dq[ITF][3];
#pragma unroll
    for (int it = 0; it < ITF; ++it) {
      const int fq = tid + it * NT;
      int d, fi, fj, fk;
      face_of(fq, d, fi, fj, fk);
      const bool use = fq < NF && face_used(d, i0 + fi, j0 + fj, k0 + fk);
      const int64_t c = B.goff + pcell(i0 + fi, j0 + fj, k0 + fk);
#pragma unroll
      for (int a = 0; a < 3; ++a) dq[it][a] = use ? P.g.q[G_DC + 3 * d + a][c] : T(1);
    }
#pragma unroll
    for (int it = 0; it < ITF; ++it)
      if (tid + it * NT < NF)
#pragma unroll
        for (int a = 0; a < 3; ++a) sDC[a * NF + tid + it * NT] = dq[it][a];
  }
  for (int e = tid; e < NS * NS; e += nt) sD[e] = C->D[e];

  const int ti = tid % TI, tj = (tid / TI) % TJ, tk = tid / (TI * TJ);
  const int ci = i0 + ti, cj = j0 + tj, ck = k0 + tk;
  const bool own = (tid < NT) && ci < n0 && cj < n1 && ck < n2;
  const int rown = rcell(ti + 2, tj + 2, tk + 2);
  const int64_t cown = pcell(ci, cj, ck);
  // where the flux balance of the own cell at snapshot n waits for the
  // epilogue: in the residual output itself, or (RK stage) in this tile's
  // slice of the balance scratch, [n][q][thread], whose 128-byte lines belong
  // to one warp each and are discarded from L2 once read back
  T* const bal = (MODE == 1) ? P.R + (int64_t)t * NS * NV * NT : P.R;
  auto bal_at = [&](int n, int q) -> T& {
    if constexpr (MODE == 1) return bal[(n * NV + q) * NT + tid];
    else return P.R[B.off + ((int64_t)n * NV + q) * B.plane + cown];
  };

  for (int n = 0; n < NS; ++n) {
    const Fr<T> f = frame_at(C, n);
    __syncthreads();
    // the region at snapshot n: every load of a thread's cells issued before
    // the first is used (one L2 latency per snapshot instead of one per cell)
    {
      constexpr int NRT = (NR + NT - 1) / NT;   // cells per thread (blockDim.x = NT)
      T uq[NRT][5];
#pragma unroll
      for (int it = 0; it < NRT; ++it) {
        const int r = tid + it * NT;
        const int ri = r % RI, rj = (r / RI) % RJ, rk = r / (RI * RJ);
        const int i = i0 - 2 + ri, j = j0 - 2 + rj, k = k0 - 2 + rk;
        if (r < NR && inpad(i, j, k)) {
          const T* u = P.Uprev + B.off + (int64_t)n * NV * B.plane + pcell(i, j, k);
#pragma unroll
          for (int q = 0; q < 5; ++q) uq[it][q] = u[q * B.plane];
        } else {   // outside the padded block: a benign state, never used by own cells
          uq[it][0] = T(1);
          uq[it][1] = uq[it][2] = uq[it][3] = T(0);
          uq[it][4] = T(1) / gm1;
        }
      }
#pragma unroll
      for (int it = 0; it < NRT; ++it) {
        const int r = tid + it * NT;
        if (r < NR) {
          const T rho = uq[it][0], ir = Ar<T>::rcp(rho);
          const T u = uq[it][1] * ir, v = uq[it][2] * ir, w = uq[it][3] * ir;
          const T p = gm1 * (uq[it][4] - T(0.5) * rho * (u * u + v * v + w * w));
          sts4(sW + 4 * r, u, v, w, p);
          sts2(sRT + 2 * r, rho, gam * p * ir);
        }
      }
    }
    __syncthreads();
    if (VISC) {
      // Green-Gauss gradients of (u, v, w, T) on the ring, as the closed-cell
      // sum of (phi_nb - phi_c)/2 S with the static face vectors, rotated once
      // per quantity into the frame of snapshot n (the sum is linear in S)
      // only the ring cells that are L or R of a tile face: the tile and its
      // six face-adjacent slabs (the ring's edges and corners are never read),
      // NGU work items (896 for an 8x8x8 tile on 512 threads, 512 for an 8x8x4
      // tile on 256: two full rounds)
      for (int w = tid; w < NGU; w += nt) {
        int gi, gj, gk;
        if (w < NT) {
          gi = w % TI + 1; gj = (w / TI) % TJ + 1; gk = w / (TI * TJ) + 1;
        } else if (w < NT + 2 * TJ * TK) {
          const int s2 = w - NT, e = s2 % (TJ * TK);
          gi = (s2 < TJ * TK) ? 0 : GI - 1; gj = e % TJ + 1; gk = e / TJ + 1;
        } else if (w < NT + 2 * TJ * TK + 2 * TI * TK) {
          const int s2 = w - NT - 2 * TJ * TK, e = s2 % (TI * TK);
          gj = (s2 < TI * TK) ? 0 : GJ - 1; gi = e % TI + 1; gk = e / TI + 1;
        } else {
          const int s2 = w - NT - 2 * TJ * TK - 2 * TI * TK, e = s2 % (TI * TJ);
          gk = (s2 < TI * TJ) ? 0 : GK - 1; gi = e % TI + 1; gj = e / TI + 1;
        }
        const int gq = (gk * GJ + gj) * GI + gi;
        const int r = rcell(gi + 1, gj + 1, gk + 1);
        const int i = i0 - 1 + gi, j = j0 - 1 + gj, k = k0 - 1 + gk;
        // ring cells beyond index n are never L or R of a computed face; their
        // high faces would lie outside the padded block
        if (i > n0 || j > n1 || k > n2) {
#pragma unroll
          for (int q = 0; q < 3; ++q) sts4(sG + 12 * gq + 4 * q, T(0), T(0), T(0), T(0));
          continue;
        }
        T g[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) g[q] = T(0);
        T pc[4], pdum;
        lds4(sW + 4 * r, pc[0], pc[1], pc[2], pdum);
        pc[3] = sRT[2 * r + 1];
        const int rs[3] = {1, RI, RI * RJ};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T* Sd = sSb + sbox3_off(d, TK);
          const int NB = sbox3_n(d, TK);
          const int lo = sbidx(d, gi, gj, gk);
          const int hi = lo + (d == 0 ? 1 : (d == 1 ? sbox3_i(1) : sbox3_i(2) * sbox3_j(2)));
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            const int o = side ? r + rs[d] : r - rs[d];
            const int e = side ? hi : lo;
            const T sv[3] = {Sd[e], Sd[NB + e], Sd[2 * NB + e]};
            T po[4];
            lds4(sW + 4 * o, po[0], po[1], po[2], po[3]);
            const T dphi[4] = {po[0] - pc[0], po[1] - pc[1], po[2] - pc[2], sRT[2 * o + 1] - pc[3]};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int a = 0; a < 3; ++a) g[3 * q + a] = side ? g[3 * q + a] + dphi[q] * sv[a] : g[3 * q + a] - dphi[q] * sv[a];
          }
        }
        const T hiv = T(0.5) * sIV[r];
        T go[12];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T gx = g[3 * q], gy = g[3 * q + 1];
          if (moving) rotv(f, g[3 * q], g[3 * q + 1], gx, gy);
          go[3 * q] = gx * hiv;
          go[3 * q + 1] = gy * hiv;
          go[3 * q + 2] = g[3 * q + 2] * hiv;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) sts4(sG + 12 * gq + 4 * q, go[4 * q], go[4 * q + 1], go[4 * q + 2], go[4 * q + 3]);
      }
      __syncthreads();
    }
    for (int fq = tid; fq < NF; fq += nt) {
      int d, fi, fj, fk;
      face_of(fq, d, fi, fj, fk);
      // the face is the low face of cell R = (i0+fi, j0+fj, k0+fk) along d
      const int Ri = i0 + fi, Rj = j0 + fj, Rk = k0 + fk;
      if (!face_used(d, Ri, Rj, Rk)) continue;
      const int st = (d == 0) ? 1 : (d == 1 ? RI : RI * RJ);
      const int rR = rcell(fi + 2, fj + 2, fk + 2);
      const int rL = rR - st;
      // (u, v) and (w, p) limited two at a time, rho alone
      using M = Two<T>;
      const T* Wa = sW + 4 * (rL - st);
      const T* Wb = sW + 4 * rL;
      const T* Wc = sW + 4 * rR;
      const T* Wd = sW + 4 * (rR + st);
      typename M::v uvL, uvR, wpL, wpR;
      const typename M::v uvb = M::ld(Wb), uvc = M::ld(Wc), wpb = M::ld(Wb + 2), wpc = M::ld(Wc + 2);
      muscl2<T>(M::ld(Wa), uvb, uvc, M::ld(Wd), eps, uvL, uvR);
      muscl2<T>(M::ld(Wa + 2), wpb, wpc, M::ld(Wd + 2), eps, wpL, wpR);
      T rhoL, rhoR;
      {
        const T a = sRT[2 * (rL - st)], b = sRT[2 * rL], c = sRT[2 * rR], dd = sRT[2 * (rR + st)];
        const T d0 = b - a, d1 = c - b, d2 = dd - c;
        const T w1 = va_weight(d1, eps);
        rhoL = b + T(0.5) * van_albada_w(d0, d1, va_weight(d0, eps), w1);
        rhoR = c - T(0.5) * van_albada_w(d1, d2, w1, va_weight(d2, eps));
      }
      const T WL[5] = {rhoL, uvL.x, uvL.y, wpL.x, wpL.y}, WR[5] = {rhoR, uvR.x, uvR.y, wpR.x, wpR.y};
      const T* Sd = sSb + sbox3_off(d, TK);
      const int NB = (d == 0) ? sbox3_n(0, TK) : (d == 1 ? sbox3_n(1, TK) : sbox3_n(2, TK));
      const int eR = (d == 0) ? sbidx(0, fi + 1, fj + 1, fk + 1)
                              : (d == 1 ? sbidx(1, fi + 1, fj + 1, fk + 1) : sbidx(2, fi + 1, fj + 1, fk + 1));
      T sx, sy;
      rotv(f, Sd[eR], Sd[NB + eR], sx, sy);
      const T sz = Sd[2 * NB + eR];
      T vgn = T(0);
      if (moving) {
        const int64_t gR = pcell(Ri, Rj, Rk);
        T xf, yf;
        rotp(f, __ldg(P.g.q[G_XF + 3 * d] + B.goff + gR), __ldg(P.g.q[G_XF + 3 * d + 1] + B.goff + gR), xf, yf);
        const T vgx = -f.thd * (yf - f.py), vgy = f.thd * (xf - f.px);
        vgn = (vgx * sx + vgy * sy) * Ar<T>::rsq(sx * sx + sy * sy + sz * sz);
      }
      T F[5];
      roe3d(WL, WR, sx, sy, sz, vgn, gm1, gg1, efix, efrac, hef, F);
      if (VISC) {
        // ring index of L and R
        const int gRi = ((fk + 1) * GJ + (fj + 1)) * GI + (fi + 1);
        const int gs = (d == 0) ? 1 : (d == 1 ? GI : GI * GJ);
        const int gLi = gRi - gs;
        T gl[12], gr[12];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          lds4(sG + 12 * gLi + 4 * q, gl[4 * q], gl[4 * q + 1], gl[4 * q + 2], gl[4 * q + 3]);
          lds4(sG + 12 * gRi + 4 * q, gr[4 * q], gr[4 * q + 1], gr[4 * q + 2], gr[4 * q + 3]);
        }
        T tx, ty;
        rotv(f, sDC[fq], sDC[NF + fq], tx, ty);
        const T tz = sDC[2 * NF + fq];
        const T pL[4] = {uvb.x, uvb.y, wpb.x, sRT[2 * rL + 1]};
        const T pR[4] = {uvc.x, uvc.y, wpc.x, sRT[2 * rR + 1]};
        T Fv[5];
        visc3d(gl, gr, pL, pR, tx, ty, tz, sx, sy, sz, mu, kap, Fv);
#pragma unroll
        for (int q = 0; q < 5; ++q) F[q] -= Fv[q];
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) sF[q * NF + fq] = F[q];
    }
    __syncthreads();
    // flux balance of the own cell at snapshot n, parked in global memory
    // until the epilogue adds the HB source (the shared memory goes to the
    // static face geometry)
    if (own) {
      const int fi0 = (tk * TJ + tj) * (TI + 1) + ti;
      const int fj0 = NFI + (tk * (TJ + 1) + tj) * TI + ti;
      const int fk0 = NFI + NFJ + (tk * TJ + tj) * TI + ti;
#pragma unroll
      for (int q = 0; q < NV; ++q)
        bal_at(n, q) = (sF[q * NF + fi0 + 1] - sF[q * NF + fi0]) + (sF[q * NF + fj0 + TI] - sF[q * NF + fj0]) +
                       (sF[q * NF + fk0 + TI * TJ] - sF[q * NF + fk0]);
    }
  }

  T tacc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) tacc[q] = T(0);
  double nacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (own) {
    const T V = P.g.q[G_VOL][B.goff + cown];
    const T vw = V * omega;
    const T iV = sIV[rown];
    T uu[NS][NV];
#pragma unroll
    for (int m = 0; m < NS; ++m)
#pragma unroll
      for (int q = 0; q < NV; ++q) uu[m][q] = P.Uprev[B.off + ((int64_t)m * NV + q) * B.plane + cown];
    T Sb[3][3], m2[3], mg[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T* Sd = sSb + sbox3_off(d, TK);
      const int NB = sbox3_n(d, TK);
      const int lo = sbidx(d, ti + 1, tj + 1, tk + 1);
      const int hi = lo + (d == 0 ? 1 : (d == 1 ? sbox3_i(1) : sbox3_i(2) * sbox3_j(2)));
#pragma unroll
      for (int a = 0; a < 3; ++a) Sb[d][a] = T(0.5) * (Sd[a * NB + lo] + Sd[a * NB + hi]);
      m2[d] = Sb[d][0] * Sb[d][0] + Sb[d][1] * Sb[d][1] + Sb[d][2] * Sb[d][2];
      mg[d] = m2[d] * Ar<T>::rsq(m2[d]);
    }
    for (int n = 0; n < NS; ++n) {
      const int64_t base = B.off + (int64_t)n * NV * B.plane + cown;
      T Rn[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        T h = T(0);
#pragma unroll
        for (int m = 0; m < NS; ++m) h += sD[n * NS + m] * uu[m][q];
        Rn[q] = bal_at(n, q) + vw * h;
      }
      if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) P.R[base + q * B.plane] = Rn[q];
      } else {
        T u0[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) u0[q] = P.U0[base + q * B.plane];
        const Fr<T> f = frame_at(C, n);
        const T rho = u0[0], irho = Ar<T>::rcp(rho);
        const T uv = u0[1] * irho, vv = u0[2] * irho, wv = u0[3] * irho;
        const T pp = gm1 * (u0[4] - T(0.5) * rho * (uv * uv + vv * vv + wv * wv));
        const T c2 = gam * pp * irho;
        const T cs_ = c2 * Ar<T>::rsq(c2);
        T ur[3] = {uv, vv, wv};
        if (moving) {
          T xc, yc;
          rotp(f, P.g.q[G_XC][B.goff + cown], P.g.q[G_XC + 1][B.goff + cown], xc, yc);
          ur[0] -= -f.thd * (yc - f.py);
          ur[1] -= f.thd * (xc - f.px);
        }
        T lam = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          T ax, ay;
          rotv(f, Sb[d][0], Sb[d][1], ax, ay);
          lam += fabs(ur[0] * ax + ur[1] * ay + ur[2] * Sb[d][2]) + cs_ * mg[d];
        }
        if (VISC) {
          const T cv = (gam / C->prandtl > T(4.0 / 3.0)) ? gam / C->prandtl : T(4.0 / 3.0);
          lam += T(4) * cv * (mu * irho) * (m2[0] + m2[1] + m2[2]) * iV;
        }
        lam += omega * T(C->nh) * V;
        const T fac = P.alpha * C->cfl * Ar<T>::rcp(lam);
#pragma unroll
        for (int q = 0; q < NV; ++q) P.Unext[base + q * B.plane] = u0[q] - fac * Rn[q];
        if (P.partials) {
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            const T x = Rn[q] * iV;
            tacc[q] += x * x;
          }
        }
      }
    }
  }
  if constexpr (MODE == 1) {
    // the parked balances are dead: drop their L2 lines unwritten (every lane
    // of the warp has read its values before the barrier)
    __syncwarp();
    constexpr int LPP = (32 * (int)sizeof(T)) / 128;   // 128-byte lines per warp and (n, q)
    const int lane = tid & 31;
    for (int e = lane; e < NS * NV * LPP; e += 32) {
      const T* line = bal + (e / LPP) * NT + (tid & ~31) + (e % LPP) * (128 / (int)sizeof(T));
      asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
    }
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) nacc[q] = (double)tacc[q];
  if (MODE == 1 && P.partials) {
    __syncthreads();
    double* scratch = reinterpret_cast<double*>(sm);
    block_sum8(nacc, NV, scratch);
    if (threadIdx.x == 0)
      for (int q = 0; q < NV; ++q) P.partials[(int64_t)t * 8 + q] = nacc[q];
  }
}

template <typename T, int NS, bool VISC, int MODE>
__global__ void __launch_bounds__(T3I * T3J * tile3d_tk(sizeof(T) == 4), 1) tile3d_kernel(StageParams<T> P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  tile3d<T, NS, VISC, MODE>(P, blockIdx.x, reinterpret_cast<T*>(smraw));
}

}  // namespace hbk
