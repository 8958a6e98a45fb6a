// CUDA kernels of the HB residual path (sm_103a), templated on the
// arithmetic type T (float or double).
//
// Method (the paper's HB NS solver, Sec. 1; per-RK-step cut exchange and
// force reduction, Sec. 3.1), with the scheme readings:
//   * primitives W = (rho, u, v, p); MUSCL W_L = W_{i-1} + s_{i-1}/2,
//     W_R = W_i - s_i/2, slopes s = va(backward, forward) with the van Albada
//     limiter va(a,b) = ((b^2+eps) a + (a^2+eps) b) / (a^2 + b^2 + 2 eps);
//   * Roe flux with the grid velocity of a rigid pitch (relative normal
//     velocity in the convective terms), Harten fix on the acoustic waves;
//   * viscous flux: Green-Gauss cell gradients of (u, v, T), face gradient =
//     mean + edge-normal correction, Stokes stress, Fourier heat flux;
//   * HB source V * omega * sum_m D[n][m] U_m;
//   * local time step CFL V / (sum_d (|u_rel . S_d| + c|S_d|) + viscous
//     + omega N_H V), 4-stage RK U^(s) = U^(0) - alpha_s dtau/V R(U^(s-1)).
//
// Tile kernel layout: one CTA owns a TI x TJ tile (or a row strip of one) of
// one block and loops over all snapshots; per snapshot it stages the
// primitives of the tile plus a 2-cell halo in shared memory (double-buffered:
// the next snapshot is staged while this one's faces run), computes
// Green-Gauss gradients on a 1-cell ring, then every face flux of the tile
// exactly once, and keeps the flux balance of each own cell per snapshot in
// shared memory.  The epilogue adds the HB source, which needs the own cell
// at all snapshots (read once per stage), and updates every snapshot; the
// tile then writes the ghost cells its own cells feed (fused halo fill).  With
// more than 9 snapshots the HB source comes precomputed from its own launch
// and each snapshot is updated as soon as its fluxes are known.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hb_internal.h"

namespace hbk {

template <typename T>
struct Fr {
  T c, s, thd, px, py;
};

template <typename T>
__device__ __forceinline__ Fr<T> frame_at(const CaseDev<T>* C, int n) {
  Fr<T> f;
  f.c = C->cth[n];
  f.s = C->sth[n];
  f.thd = C->thd[n];
  f.px = C->pivot[0];
  f.py = C->pivot[1];
  return f;
}

template <typename T>
__device__ __forceinline__ void rotv(const Fr<T>& f, T x, T y, T& ox, T& oy) {
  ox = f.c * x - f.s * y;
  oy = f.s * x + f.c * y;
}

template <typename T>
__device__ __forceinline__ void rotp(const Fr<T>& f, T x, T y, T& ox, T& oy) {
  T rx = x - f.px, ry = y - f.py;
  ox = f.c * rx - f.s * ry + f.px;
  oy = f.s * rx + f.c * ry + f.py;
}

// Precision-specific arithmetic.  The FP32 path uses the hardware reciprocal
// and reciprocal-square-root forms (a few ulp each, well inside the FP32
// error budget of the residual); the FP64 path keeps correctly rounded
// division and takes the 1-ulp reciprocal square root (one FP64 sequence
// instead of a square root followed by a division).
template <typename T>
struct Ar;
template <>
struct Ar<float> {
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float rcp(float b) { return __fdividef(1.0f, b); }
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ void rcp2(float a, float b, float& ia, float& ib) {
    ia = __fdividef(1.0f, a);
    ib = __fdividef(1.0f, b);
  }
};
template <>
struct Ar<double> {
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double rcp(double b) { return 1.0 / b; }
  static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
  // 1/a and 1/b through one division, 1/(a b) (within 1.5 ulp); a, b are
  // positive quantities of moderate range (densities, limiter weights)
  static __device__ __forceinline__ void rcp2(double a, double b, double& ia, double& ib) {
    const double r = 1.0 / (a * b);
    ia = b * r;
    ib = a * r;
  }
};

// van Albada limiter in the form ((b^2+eps) a + (a^2+eps) b) / ((b^2+eps) +
// (a^2+eps)): the two weights also make the denominator, and the weight of a
// difference is shared by the two faces that limit with it
// two or four consecutive shared-memory values of a cell in one access
__device__ __forceinline__ void lds4(const float* p, float& a, float& b, float& c, float& d) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void lds4(const double* p, double& a, double& b, double& c, double& d) {
  const double2 v = reinterpret_cast<const double2*>(p)[0], w = reinterpret_cast<const double2*>(p)[1];
  a = v.x; b = v.y; c = w.x; d = w.y;
}
__device__ __forceinline__ void lds2(const float* p, float& a, float& b) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  a = v.x; b = v.y;
}
__device__ __forceinline__ void lds2(const double* p, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = v.x; b = v.y;
}
__device__ __forceinline__ void sts2(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void sts2(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void sts4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void sts4(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// Two-lane arithmetic: on sm_100+ one packed FP32 instruction does both
// lanes (the same rounding per lane as the scalar instruction); the FP64
// form is the plain per-lane arithmetic.
template <typename T>
struct Two;
template <>
struct Two<float> {
  using v = float2;
  static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  // a - b as one packed fma: b * (-1) is exact, so the single rounding is that of a - b
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
  // c - h * x as one packed fma (h a power of two: h * x exact)
  static __device__ __forceinline__ float2 fnma(float2 h, float2 x, float2 c) {
    return __ffma2_rn(make_float2(-h.x, -h.y), x, c);
  }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ float2 rcp(float2 a) {
    return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
  }
  static __device__ __forceinline__ float2 ld(const float* p) { return *reinterpret_cast<const float2*>(p); }
};
template <>
struct Two<double> {
  using v = double2;
  static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ double2 mul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
  static __device__ __forceinline__ double2 fma(double2 a, double2 b, double2 c) {
    return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
  }
  static __device__ __forceinline__ double2 fnma(double2 h, double2 x, double2 c) {
    return make_double2(c.x - h.x * x.x, c.y - h.y * x.y);
  }
  static __device__ __forceinline__ double2 rcp(double2 a) {
    double2 r;
    Ar<double>::rcp2(a.x, a.y, r.x, r.y);
    return r;
  }
  static __device__ __forceinline__ double2 ld(const double* p) { return *reinterpret_cast<const double2*>(p); }
};

// an int index descriptor (fields below bit 30) carried in a slot of a
// floating-point record; in FP32 bit 30 is set so that the pattern is a
// normal number (never a denormal that a flush-to-zero path could clear, nor a
// NaN); the decoder masks its fields and ignores that bit
__device__ __forceinline__ float int_in(float, int v) { return __int_as_float(v | 0x40000000); }
__device__ __forceinline__ double int_in(double, int v) { return (double)v; }
__device__ __forceinline__ int int_of(float x) { return __float_as_int(x); }
__device__ __forceinline__ int int_of(double x) { return (int)x; }

// MUSCL face states of two variables at once from the stencil a | b || c | d
// (face between b and c): WL = b + va(b-a, c-b)/2, WR = c - va(c-b, d-c)/2
template <typename T>
__device__ __forceinline__ void muscl2(typename Two<T>::v a, typename Two<T>::v b, typename Two<T>::v c,
                                       typename Two<T>::v d, T eps, typename Two<T>::v& wl,
                                       typename Two<T>::v& wr) {
  using M = Two<T>;
  const auto e = M::make(eps, eps), h = M::make(T(0.5), T(0.5));
  const auto d0 = M::sub(b, a), d1 = M::sub(c, b), d2 = M::sub(d, c);
  const auto w0 = M::fma(d0, d0, e), w1 = M::fma(d1, d1, e), w2 = M::fma(d2, d2, e);
  const auto sl = M::mul(M::fma(w1, d0, M::mul(w0, d1)), M::rcp(M::add(w0, w1)));
  const auto sr = M::mul(M::fma(w2, d1, M::mul(w1, d2)), M::rcp(M::add(w1, w2)));
  wl = M::fma(h, sl, b);
  wr = M::fnma(h, sr, c);
}

template <typename T>
__device__ __forceinline__ T va_weight(T a, T eps) { return a * a + eps; }
template <typename T>
__device__ __forceinline__ T van_albada_w(T a, T b, T wa, T wb) {
  return Ar<T>::div(wb * a + wa * b, wa + wb);
}

// Roe flux through area vector (Sx, Sy) of a face moving with normal speed
// vgn (grid velocity . unit normal).  W = (rho, u, v, p).  F = (mass, mx, my, E).
// gg1 = gamma/(gamma-1); hef = 1/(2 efrac) for the entropy fix.
// Written with the mass fluxes m = rho (q - vgn), the energy flux in the form
// m H + p vgn (= E (q - vgn) + p q), and the wave sum factored as
// D = s (1, u, v, H) + l2 a2 (1, u, v, k) + ct (w3 - w1) (0, nx, ny, q)
//     + l2 rho~ (0, du, dv, u.du), s = w1 + w3 (the same sum as the textbook
// form of the three waves).
template <typename T>
__device__ __forceinline__ void roe2d(const T* WL, const T* WR, T Sx, T Sy, T vgn, T gm1, T gg1,
                                      int efix, T efrac, T hef, T* F) {
  const T A2 = Sx * Sx + Sy * Sy;
  const T iA = Ar<T>::rsq(A2);
  const T hA = T(0.5) * (A2 * iA);
  const T nx = Sx * iA, ny = Sy * iA;
  T irL, irR;
  Ar<T>::rcp2(WL[0], WR[0], irL, irR);
  const T qL = WL[1] * nx + WL[2] * ny;
  const T qR = WR[1] * nx + WR[2] * ny;
  const T kL = T(0.5) * (WL[1] * WL[1] + WL[2] * WL[2]);
  const T kR = T(0.5) * (WR[1] * WR[1] + WR[2] * WR[2]);
  const T HL = gg1 * WL[3] * irL + kL;
  const T HR = gg1 * WR[3] * irR + kR;
  const T rr = WR[0] * irL;
  const T r = rr * Ar<T>::rsq(rr);          // sqrt(rho_R / rho_L)
  const T rt = r * WL[0];
  const T inv1r = Ar<T>::rcp(T(1) + r);
  const T ut = (WL[1] + r * WR[1]) * inv1r;
  const T vt = (WL[2] + r * WR[2]) * inv1r;
  const T Ht = (HL + r * HR) * inv1r;
  const T kt = T(0.5) * (ut * ut + vt * vt);
  const T ct2 = gm1 * (Ht - kt);
  const T ict = Ar<T>::rsq(ct2);
  const T ct = ct2 * ict;
  const T ict2 = ict * ict;
  const T qt = ut * nx + vt * ny;
  const T qtr = qt - vgn;
  T l1 = fabs(qtr - ct), l2 = fabs(qtr), l3 = fabs(qtr + ct);
  if (efix) {   // (l^2 + del^2) / (2 del) below del = efrac c~
    const T del = efrac * ct, d2 = del * del, hid = hef * ict;
    l1 = l1 < del ? (l1 * l1 + d2) * hid : l1;
    l3 = l3 < del ? (l3 * l3 + d2) * hid : l3;
  }
  const T dp = WR[3] - WL[3], drho = WR[0] - WL[0], dq = qR - qL;
  const T m = rt * ct * dq, h = T(0.5) * ict2;
  const T w1 = l1 * ((dp - m) * h), w3 = l3 * ((dp + m) * h);
  const T l2a2 = l2 * (drho - dp * ict2), l2rt = l2 * rt;
  const T dux = (WR[1] - WL[1]) - dq * nx;
  const T duy = (WR[2] - WL[2]) - dq * ny;
  const T s13 = w1 + w3, dw = ct * (w3 - w1);
  const T D0 = s13 + l2a2;
  const T D1 = ut * D0 + nx * dw + l2rt * dux;
  const T D2 = vt * D0 + ny * dw + l2rt * duy;
  const T D3 = Ht * s13 + qt * dw + l2a2 * kt + l2rt * (ut * dux + vt * duy);
  const T mL = WL[0] * (qL - vgn), mR = WR[0] * (qR - vgn);
  const T ps = WL[3] + WR[3];
  F[0] = hA * (mL + mR - D0);
  F[1] = hA * (mL * WL[1] + mR * WR[1] + ps * nx - D1);
  F[2] = hA * (mL * WL[2] + mR * WR[2] + ps * ny - D2);
  F[3] = hA * (mL * HL + mR * HR + ps * vgn - D3);
}

// Viscous flux through (Sx, Sy) from cell gradients gL, gR = (ux,uy,vx,vy,Tx,Ty),
// cell values (u, v, T) and the rotated centre difference (tx, ty) = x_R - x_L.
template <typename T>
__device__ __forceinline__ void visc2d(const T* gL, const T* gR, T uL, T vL, T TL, T uR, T vR,
                                       T TR, T tx, T ty, T Sx, T Sy, T mu, T kap, T* Fv) {
  const T il = Ar<T>::rsq(tx * tx + ty * ty);
  const T ex = tx * il, ey = ty * il;
  T g[6];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    using M = Two<T>;
    const auto bq = M::mul(M::make(T(0.5), T(0.5)),
                           M::add(M::make(gL[2 * q], gL[2 * q + 1]), M::make(gR[2 * q], gR[2 * q + 1])));
    const T bx = bq.x, by = bq.y;
    const T dphi = (q == 0) ? (uR - uL) : (q == 1) ? (vR - vL) : (TR - TL);
    const T corr = dphi * il - (bx * ex + by * ey);
    g[2 * q] = bx + corr * ex;
    g[2 * q + 1] = by + corr * ey;
  }
  // mu (2 u_x - 2/3 div) = 4/3 mu u_x - 2/3 mu v_y, and alike
  const T m43 = T(4.0 / 3.0) * mu, m23 = T(2.0 / 3.0) * mu;
  const T txx = m43 * g[0] - m23 * g[3];
  const T tyy = m43 * g[3] - m23 * g[0];
  const T txy = mu * (g[1] + g[2]);
  const T fx = txx * Sx + txy * Sy;
  const T fy = txy * Sx + tyy * Sy;
  const T uf = T(0.5) * (uL + uR), vf = T(0.5) * (vL + vR);
  Fv[0] = T(0);
  Fv[1] = fx;
  Fv[2] = fy;
  Fv[3] = uf * fx + vf * fy + kap * (g[4] * Sx + g[5] * Sy);
}

// shared-memory elements of one tile CTA
// The snapshot loop of a tile is pipelined (primitives double-buffered)
// where the extra shared memory keeps the occupancy: up to 7 snapshots.
// A tile whose per-snapshot balances wait in global memory (tile_park) has
// the room for the pipeline at any static N_s: an RK stage where tile_balg
// says so (a scratch slice per tile), and every residual evaluation (the
// residual output itself holds them until the epilogue adds the HB source)
__host__ __device__ constexpr bool tile_park(int NS, int MODE) { return tile_balg(NS, MODE) || (MODE == 0 && NS > 0); }
__host__ __device__ constexpr bool tile_pipelined(int NS, int MODE) { return NS <= 7 || tile_park(NS, MODE); }


// (NS = 0: the runtime snapshot count of the large-N_s path, whose HB
// source comes precomputed, so it keeps no per-snapshot balances)
// (balg: the per-snapshot balances are parked in global memory instead)
// (face records of tile2d_face_words elements per face work item)
__host__ __device__ constexpr int tile2d_face_words(bool visc) { return visc ? 4 : 2; }
__host__ __device__ constexpr size_t tile2d_smem_elems(int TI, int TJ, int NS, bool pipe, bool balg, bool visc) {
  return (size_t)(pipe ? 15 : 10) * (TI + 4) * (TJ + 4) + (size_t)6 * (TI + 2) * (TJ + 2) +
         (size_t)(4 + tile2d_face_words(visc)) * ((TI + 1) * TJ + TI * (TJ + 1)) +
         (size_t)(balg ? 0 : NS * 4 * TI * TJ) + (size_t)NS * NS;
}

// block-wide FP64 sum of up to 8 values, fixed order; result valid in thread 0
__device__ __forceinline__ void block_sum8(double* v, int nv, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
  for (int q = 0; q < nv; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) scratch[warp * 8 + q] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < nv; ++q) {
      double s = 0.0;
      for (int w = 0; w < nwarp; ++w) s += scratch[w * 8 + q];
      v[q] = s;
    }
  }
}

// ------------------------------------------------------------- halos/BCs --
template <typename T>
__device__ __forceinline__ void freestream_at(const CaseDev<T>* C, int n, T x, T* W) {
  W[0] = C->winf[n][0];
  W[1] = C->winf[n][1];
  W[2] = C->winf[n][2];
  W[3] = C->winf[n][3];
  W[4] = C->winf[n][4];
  if (C->ubc == 2) W[2] += C->ubc_amp * C->mach * sin(C->tn[n] - C->omega * x / C->mach);
}

// conservative <-> primitive (rho, u, v, w, p); w = 0 in 2D
template <typename T, int DIM>
__device__ __forceinline__ void prim_of(const T* Q, T gm1, T* W) {
  constexpr int NV = DIM + 2;
  const T rho = Q[0];
  W[0] = rho;
  W[1] = Q[1] / rho;
  W[2] = Q[2] / rho;
  W[3] = (DIM == 3) ? Q[3] / rho : T(0);
  W[4] = gm1 * (Q[NV - 1] - T(0.5) * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]));
}

template <typename T, int DIM>
__device__ __forceinline__ void cons_of(const T* W, T gm1, T* Q) {
  constexpr int NV = DIM + 2;
  Q[0] = W[0];
  Q[1] = W[0] * W[1];
  Q[2] = W[0] * W[2];
  if (DIM == 3) Q[3] = W[0] * W[3];
  Q[NV - 1] = W[4] / gm1 + T(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

// primitives of a padded cell of a block at one snapshot (Ub: snapshot base)
template <typename T, int DIM>
__device__ __forceinline__ void load_prim(const T* Ub, int64_t plane, int64_t cell, T gm1, T* W) {
  constexpr int NV = DIM + 2;
  T Q[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Q[v] = Ub[v * plane + cell];
  prim_of<T, DIM>(Q, gm1, W);
}

template <typename T, int DIM>
__device__ __forceinline__ void store_cons(T* Ub, int64_t plane, int64_t cell, T gm1, const T* W) {
  constexpr int NV = DIM + 2;
  T Q[NV];
  cons_of<T, DIM>(W, gm1, Q);
#pragma unroll
  for (int v = 0; v < NV; ++v) Ub[v * plane + cell] = Q[v];
}

// Physical-boundary ghost state at snapshot n from Wi: type 1 characteristic
// farfield (Wi = first interior cell; Riemann invariants normal to the face,
// entropy and tangential velocity from inside on outflow, from the freestream
// on inflow), type 2 slip wall (Wi = mirror cell; relative normal velocity
// reflected), type 3 no-slip adiabatic wall (u_g = 2 v_wall - u).  The
// boundary face is the low face along p of padded cell fcell; sgn = +1 on a
// high face, -1 on a low face.
template <typename T, int DIM>
__device__ __forceinline__ void bc_map(const CaseDev<T>* C, const Geo<T>& g, const BlockDev& B, int type, int p,
                                       int sgn, int fcell, int n, const T* Wi, T* Wg) {
  const Fr<T> f = frame_at(C, n);
  const T gam = C->gamma, gm1 = gam - T(1);
  const int64_t fc = B.goff + fcell;
  T S[3] = {g.q[G_S + 3 * p][fc], g.q[G_S + 3 * p + 1][fc], T(0)};
  T X[3] = {g.q[G_XF + 3 * p][fc], g.q[G_XF + 3 * p + 1][fc], T(0)};
  if (DIM == 3) {
    S[2] = g.q[G_S + 3 * p + 2][fc];
    X[2] = g.q[G_XF + 3 * p + 2][fc];
  }
  T sr[3], xr[3];
  rotv(f, S[0], S[1], sr[0], sr[1]);
  sr[2] = S[2];
  rotp(f, X[0], X[1], xr[0], xr[1]);
  xr[2] = X[2];
  const T vg[3] = {-f.thd * (xr[1] - f.py), f.thd * (xr[0] - f.px), T(0)};
  const T A = sqrt(sr[0] * sr[0] + sr[1] * sr[1] + sr[2] * sr[2]);
  const T sg = T(sgn);
  const T nr[3] = {sg * sr[0] / A, sg * sr[1] / A, sg * sr[2] / A};
  if (type == 1) {
    T Wf[5];
    freestream_at(C, n, xr[0], Wf);
    const T qi = (Wi[1] - vg[0]) * nr[0] + (Wi[2] - vg[1]) * nr[1] + (Wi[3] - vg[2]) * nr[2];
    const T qf = (Wf[1] - vg[0]) * nr[0] + (Wf[2] - vg[1]) * nr[1] + (Wf[3] - vg[2]) * nr[2];
    const T ci = sqrt(gam * Wi[4] / Wi[0]), cf = sqrt(gam * Wf[4] / Wf[0]);
    const T Rp = qi + T(2) * ci / gm1, Rm = qf - T(2) * cf / gm1;
    const T qb = T(0.5) * (Rp + Rm);
    const T cb = T(0.25) * gm1 * (Rp - Rm);
    const bool outflow = qb > T(0);
    T Wr[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) Wr[a] = outflow ? Wi[a] : Wf[a];
    const T qr = outflow ? qi : qf;
    const T ent = Wr[4] / pow(Wr[0], gam);
    Wg[0] = pow(cb * cb / (gam * ent), T(1) / gm1);
#pragma unroll
    for (int a = 0; a < 3; ++a) Wg[1 + a] = vg[a] + ((Wr[1 + a] - vg[a]) - qr * nr[a]) + qb * nr[a];
    Wg[4] = Wg[0] * cb * cb / gam;
  } else {
    Wg[0] = Wi[0];
    Wg[4] = Wi[4];
    if (type == 2) {
      const T qn = (Wi[1] - vg[0]) * nr[0] + (Wi[2] - vg[1]) * nr[1] + (Wi[3] - vg[2]) * nr[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) Wg[1 + a] = Wi[1 + a] - T(2) * qn * nr[a];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) Wg[1 + a] = T(2) * vg[a] - Wi[1 + a];
    }
  }
  if (DIM == 2) Wg[3] = T(0);
}

// One 2D ghost cell at snapshot n: its root cell of src (in block R) taken
// through the job's chain of boundary maps, written to dst.
template <typename T>
__device__ __forceinline__ void ghost_job(const CaseDev<T>* C, const Geo<T>& g, const BlockDev* blocks,
                                          const BcRec* bcs, const GhostJob* J, const BlockDev& R, int n,
                                          const T* src, T* dst) {
  constexpr int NV = 4;
  const T gm1 = C->gamma - T(1);
  const T* s = src + R.off + (int64_t)n * NV * R.plane + J->root_cell;
  T Q[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Q[v] = s[v * R.plane];
  const int nops = J->nops;
  for (int k = 0; k < nops; ++k) {
    const BcRec& r = bcs[J->op[k]];
    T Wi[5], Wg[5];
    prim_of<T, 2>(Q, gm1, Wi);
    bc_map<T, 2>(C, g, blocks[r.blk], r.type, r.p, r.sgn, r.fcell, n, Wi, Wg);
    cons_of<T, 2>(Wg, gm1, Q);
  }
  const BlockDev& D = blocks[J->dst_blk];
  T* d = dst + D.off + (int64_t)n * NV * D.plane + J->dst_cell;
#pragma unroll
  for (int v = 0; v < NV; ++v) d[v * D.plane] = Q[v];
}

// Fused ghost fill after an RK stage: the ghost cells whose root is an own
// cell of tile t, at every snapshot, from the stage output just written.
template <typename T, int NS>
__device__ __forceinline__ void fill_tile_ghosts(const StageParams<T>& P, int t, const BlockDev& B,
                                                 const CaseDev<T>* C) {
  const int2 jr = P.job_range[t];
  if (jr.y <= 0) return;
  __syncthreads();   // own-cell outputs of every thread of the CTA are visible
  const int nitem = jr.y * (NS ? NS : C->ns);
  for (int w = threadIdx.x; w < nitem; w += blockDim.x) {
    const int n = w / jr.y;
    ghost_job<T>(C, P.g, P.blocks, P.job_bcs, P.jobs + jr.x + (w - n * jr.y), B, n, P.Unext, P.Unext);
  }
}

// Every 2D ghost cell in one launch: one item per (job, snapshot),
// snapshot-major so that neighbouring threads write neighbouring ghosts.
template <typename T>
__global__ void ghost_fill_kernel(GhostFillParams<T> p) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)p.njobs * p.ns_max) return;
  const int n = (int)(gid / p.njobs), q = (int)(gid - (int64_t)n * p.njobs);
  const GhostJob* J = p.jobs + q;
  const BlockDev& R = p.blocks[J->root_blk];
  const CaseDev<T>* C = p.cases + R.cs;
  if (n >= C->ns) return;
  ghost_job<T>(C, p.g, p.blocks, p.bcs, J, R, n, p.src, p.dst);
}

// HB source of the large-N_s path, H = V omega D U (the harmonic balance
// operator of the HB solver, Sec. 1, couples every snapshot of a cell).  D depends on N_s
// only; it travels as a kernel parameter, so every product takes its
// coefficient from the constant bank while the cell's N_s values sit in
// registers.  One thread per (padded cell, variable) of 128-cell chunks of
// the blocks whose case has this N_s.
constexpr int kSrcCells = 128;
template <typename T, int NS>
struct DMat {
  T d[NS * NS];
};

template <typename T, int NS>
__global__ void __launch_bounds__(kSrcCells) hb_source_kernel(const CaseDev<T>* cases, const BlockDev* blocks,
                                                              Geo<T> g, const int2* chunks, int nv, DMat<T, NS> D,
                                                              const T* U, T* H) {
  const int2 ck = chunks[blockIdx.x];           // (block, first cell)
  const int q = blockIdx.y;
  const BlockDev& B = blocks[ck.x];
  const int64_t c = (int64_t)ck.y + threadIdx.x;
  if (c >= B.plane) return;
  const T vw = g.q[G_VOL][B.goff + c] * cases[B.cs].omega;
  const T* u = U + B.off + (int64_t)q * B.plane + c;
  T x[NS];
#pragma unroll
  for (int m = 0; m < NS; ++m) x[m] = u[(int64_t)m * nv * B.plane];
  T* h = H + B.off + (int64_t)q * B.plane + c;
#pragma unroll
  for (int n = 0; n < NS; ++n) {
    T acc = T(0);
#pragma unroll
    for (int m = 0; m < NS; ++m) acc += D.d[n * NS + m] * x[m];
    h[(int64_t)n * nv * B.plane] = vw * acc;
  }
}

// Physical-time term of time-domain dual time stepping (second-order
// backward differences): H = V (c0 U + c1 U_n + c2 U_nm1), per padded cell
// and variable of one-snapshot blocks.
template <typename T>
__global__ void __launch_bounds__(kSrcCells) td_source_kernel(const BlockDev* blocks, Geo<T> g, const int2* chunks,
                                                              T c0, T c1, T c2, const T* U, const T* Un,
                                                              const T* Unm1, T* H) {
  const int2 ck = chunks[blockIdx.x];
  const BlockDev& B = blocks[ck.x];
  const int64_t c = (int64_t)ck.y + threadIdx.x;
  if (c >= B.plane) return;
  const int64_t e = B.off + (int64_t)blockIdx.y * B.plane + c;
  T u = c0 * U[e] + c1 * Un[e];
  if (Unm1) u += c2 * Unm1[e];
  H[e] = g.q[G_VOL][B.goff + c] * u;
}

// MODE 0: R := residual.  MODE 1: RK stage update (+ norm partials if set).
// NS = 0: the snapshot count is the case's (large N_s); the HB source comes
// from P.H and each snapshot is updated as soon as its face fluxes are known.
// The tile shape TI x TJ (TI a power of two) is a compile-time constant so that
// every flat-index decomposition is a multiply-shift.
// BALG: the per-snapshot flux balances wait for the epilogue in global memory
// instead of shared memory: in an RK stage in this tile's slice of a scratch
// (P.R, [tile][kMaxStaticNS][NV][NT]), whose L2 lines are discarded once read;
// in a residual evaluation in the residual output P.R itself
template <typename T, int NS, bool VISC, int MODE, int TI, int TJ, bool PIPE, bool BALG = false>
__device__ __forceinline__ void tile2d(const StageParams<T>& P, int t, T* sm) {
  constexpr int NV = 4;
  const int4 tl = P.tiles[t];
  const BlockDev B = P.blocks[tl.x];
  const CaseDev<T>* C = P.cases + B.cs;
  constexpr int NT = TI * TJ;
  constexpr int RI = TI + 4, RJ = TJ + 4, NR = RI * RJ;
  constexpr int GI = TI + 2, NG = GI * (TJ + 2);
  constexpr int NFI = (TI + 1) * TJ, NF = NFI + TI * (TJ + 1);
  static_assert((TI & (TI - 1)) == 0 && NT <= MAXNT, "tile shape");
  const int i0 = tl.y, j0 = tl.z;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int P0 = B.P[0];
  const int n0 = B.n[0], n1 = B.n[1];
  // own rows j0 .. je-1 (a row strip of a tile has fewer than TJ); the
  // region and the gradient ring are only needed two and one rows beyond
  const int je = j0 + tl.w;
  const int NRt = RI * (tl.w + 4), NGt = GI * (tl.w + 2);

  // PIPE: primitives and temperature double-buffered over snapshots, so
  // that the region of snapshot n+1 is staged while the faces of n run
  constexpr int NB = PIPE ? 2 : 1;
  T* sW = sm;              // [NB][NR][4] primitives (u, v, rho, p) of each cell
  T* sT = sW + NB * 4 * NR;   // [NB][NR] temperature gamma p / rho
  T* sIV = sT + NB * NR;   // [NR] 1 / volume
  T* sS = sIV + NR;        // [d*2+comp][NR] low-face vectors
  T* sG = sS + 4 * NR;     // [3][NG][2] gradients (x, y) of u, v, T on the 1-cell ring
  T* sF = sG + 6 * NG;     // [NV][NF] face fluxes
  T* sAcc = sF + 4 * NF;   // [NS][NV][NT] flux balance per snapshot of each own cell
  constexpr int FRW = tile2d_face_words(VISC);
  T* sFR = sAcc + (BALG ? 0 : NS * NV * NT);   // [NF][FRW] per face work item: (vg, dcx, dcy, descriptor), or (vg, descriptor) inviscid
  T* sD = sFR + FRW * NF;   // [NS][NS]
  static_assert(RI * (TJ + 4) <= 512 && NF <= 1024 && GI * (TJ + 2) <= 508, "face descriptor fields");
  static_assert(!BALG || (NS > 0 && NS <= kMaxStaticNS), "global balances: static N_s");
  T* const bal = (BALG && MODE == 1) ? P.R + (int64_t)t * kMaxStaticNS * NV * NT : nullptr;
  if (BALG && P.R == nullptr) return;   // no scratch passed (the host refuses such a launch first)
  constexpr bool DYN = NS == 0;
  const int ns = DYN ? C->ns : NS;

  const T gam = C->gamma, gm1 = C->gamma - T(1), eps = C->eps, efrac = C->ent_frac;
  const T gg1 = gam / gm1, hef = T(0.5) / efrac;
  const T mu = C->mu, kap = C->kappa, omega = C->omega;
  const int efix = C->entropy_fix;
  const bool moving = C->motion != 0;

  // ---- static geometry of the region (tile + 2-cell halo), once per stage
  // (every load of a thread issued before the first is used)
  {
    constexpr int NGEO = (NR + NT - 1) / NT;
    T gq[NGEO][5];
#pragma unroll
    for (int it = 0; it < NGEO; ++it) {
      const int r = tid + it * nt;
      const int ri = r % RI, rj = r / RI;
      const int i = i0 - 2 + ri, j = j0 - 2 + rj;
      if (r < NRt && i <= n0 + 1 && j <= n1 + 1) {
        const int64_t c = B.goff + (int64_t)(j + 2) * P0 + (i + 2);
        gq[it][0] = P.g.q[G_VOL][c];
        gq[it][1] = P.g.q[G_S + 0][c];
        gq[it][2] = P.g.q[G_S + 1][c];
        gq[it][3] = P.g.q[G_S + 3][c];
        gq[it][4] = P.g.q[G_S + 4][c];
      } else {   // outside the padded block: a benign unit cell, never used by own cells
        gq[it][0] = T(1);
        gq[it][1] = T(1);
        gq[it][2] = T(0);
        gq[it][3] = T(0);
        gq[it][4] = T(1);
      }
    }
#pragma unroll
    for (int it = 0; it < NGEO; ++it) {
      const int r = tid + it * nt;
      if (r < NRt) {
        sIV[r] = Ar<T>::rcp(gq[it][0]);
        sS[r] = gq[it][1];
        sS[NR + r] = gq[it][2];
        sS[2 * NR + r] = gq[it][3];
        sS[3 * NR + r] = gq[it][4];
      }
    }
  }
  for (int e = tid; e < NS * NS; e += nt) sD[e] = C->D[e];
  // the face work items, decoded once per stage (they are the same for every
  // snapshot): work item w -> bit 0 used, bit 1 direction d, bits 2-10 region
  // index of L, bits 11-20 flux storage index, bits 21-29 ring index of L;
  // with the static grid-velocity factor and centre difference of the face.
  // Order of w: the first TI x TJ i-faces row by row, TI to a row (a warp
  // reads one region row: no bank conflicts), then the TJ faces of column TI,
  // then the j-faces
  for (int w = tid; w < NF; w += nt) {
    int d, fi, fj, fq, rL, gLi;
    bool used;
    if (w < NFI) {
      if (w < TI * TJ) {
        fi = w % TI;
        fj = w / TI;
      } else {
        fi = TI;
        fj = w - TI * TJ;
      }
      fq = fj * (TI + 1) + fi;
      used = !(i0 + fi > n0 || j0 + fj >= je);
      rL = (fj + 2) * RI + (fi + 1);
      d = 0;
      gLi = (fj + 1) * GI + fi;
    } else {
      const int g2 = w - NFI;
      fi = g2 % TI;
      fj = g2 / TI;
      fq = w;
      used = !(i0 + fi >= n0 || j0 + fj > je);
      rL = (fj + 1) * RI + (fi + 2);
      d = 1;
      gLi = fj * GI + fi + 1;
    }
    // the face is the low face of cell R = (i0 + fi, j0 + fj) along d
    const int64_t gR = B.goff + (int64_t)(j0 + fj + 2) * P0 + (i0 + fi + 2);
    const T vg = (used && moving) ? P.g.q[G_VG + d][gR] : T(0);
    const int desc = (used ? 1 : 0) | (d << 1) | (rL << 2) | (fq << 11) | (gLi << 21);
    if constexpr (VISC) {
      const T dx = used ? P.g.q[G_DC + 3 * d][gR] : T(1);
      const T dy = used ? P.g.q[G_DC + 3 * d + 1][gR] : T(0);
      sts4(sFR + 4 * w, vg, dx, dy, int_in(T(0), desc));
    } else {
      sts2(sFR + 2 * w, vg, int_in(T(0), desc));
    }
  }

  const int ti = tid % TI, tj = tid / TI;
  const int ci = i0 + ti, cj = j0 + tj;
  const bool own = (tid < NT) && ci < n0 && cj < je;
  const int rown = (tj + 2) * RI + (ti + 2);
  const int64_t cown = (int64_t)(cj + 2) * P0 + (ci + 2);

  // primitives of region cell r at snapshot n into buffer b (the limiter
  // acts on the Cartesian velocity components of the inertial frame, so the
  // velocity is staged in that frame and the metrics are rotated instead)
  struct Q4 { T x, y, z, w; };   // conservative variables of one cell
  auto load_cell = [&](int r, int n) -> Q4 {
    const int ri = r % RI, rj = r / RI;
    const int i = i0 - 2 + ri, j = j0 - 2 + rj;
    Q4 q;
    if (r < NRt && i <= n0 + 1 && j <= n1 + 1) {
      const T* u = P.Uprev + B.off + (int64_t)n * NV * B.plane + (int64_t)(j + 2) * P0 + (i + 2);
      q.x = u[0];
      q.y = u[B.plane];
      q.z = u[2 * B.plane];
      q.w = u[3 * B.plane];
    } else {   // outside the padded block: a benign state, never used by own cells
      q.x = T(1);
      q.y = q.z = T(0);
      q.w = T(1) / gm1;
    }
    return q;
  };
  auto store_cell = [&](int r, int b, Q4 q) {
    const T rho = q.x;
    const T ir = Ar<T>::rcp(rho);
    const T w1 = q.y * ir, w2 = q.z * ir;
    const T w3 = gm1 * (q.w - T(0.5) * rho * (w1 * w1 + w2 * w2));
    sts4(sW + (b * NR + r) * 4, w1, w2, rho, w3);
    sT[b * NR + r] = gam * w3 * ir;
  };
  // region cells r0, r0 + nt, ... (< NRt) at snapshot n into buffer b: every
  // load of the thread issued before the first is used
  constexpr int NSTG = (NR + NT - 1) / NT;
  auto stage_cells = [&](int r0, int n, int b) {
    Q4 q[NSTG];
#pragma unroll
    for (int it = 0; it < NSTG; ++it) q[it] = load_cell(r0 + it * nt, n);
#pragma unroll
    for (int it = 0; it < NSTG; ++it)
      if (r0 + it * nt < NRt) store_cell(r0 + it * nt, b, q[it]);
  };

  // Green-Gauss gradients of (u, v, T) at ring cell gq from buffer b, written
  // as sum (phi_nb - phi_c)/2 S over the closed cell (the faces sum to zero),
  // which keeps the rounding of large face vectors out of small cells
  // work item w over the ring rows 0 .. rows-1: the TI inner columns of each
  // row first (a warp reads one region row), then the two edge columns;
  // gq is the ring cell's storage index in sG
  const int ring_rows = tl.w + 2;
  auto grad_cell = [&](int w, const Fr<T>& f, int b) {
    const T* W = sW + b * 4 * NR;
    const T* TT = sT + b * NR;
    int gi, gj;
    if (w < TI * ring_rows) {
      gi = w % TI + 1;
      gj = w / TI;
    } else {
      const int k = w - TI * ring_rows;
      gi = (k & 1) ? TI + 1 : 0;
      gj = k >> 1;
    }
    const int gq = gj * GI + gi;
    const int r = (gj + 1) * RI + (gi + 1);
    T uc, vc;
    lds2(W + 4 * r, uc, vc);
    const T Tc = TT[r];
    // summed with the static face vectors (the low face enters with -S,
    // the high one with +S) and rotated once per quantity into the frame
    // of snapshot n: the sum is linear in S
    T g[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    const int nb[4] = {r - 1, r + 1, r - RI, r + RI};
    const int fo[4] = {r, r + 1, r, r + RI};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int d = k >> 1;
      const T sx = sS[(2 * d) * NR + fo[k]], sy = sS[(2 * d + 1) * NR + fo[k]];
      const int o = nb[k];
      T uo, vo;
      lds2(W + 4 * o, uo, vo);
      const T du = uo - uc, dv = vo - vc, dT = TT[o] - Tc;
      if (k & 1) {
        g[0] += du * sx; g[1] += du * sy;
        g[2] += dv * sx; g[3] += dv * sy;
        g[4] += dT * sx; g[5] += dT * sy;
      } else {
        g[0] -= du * sx; g[1] -= du * sy;
        g[2] -= dv * sx; g[3] -= dv * sy;
        g[4] -= dT * sx; g[5] -= dT * sy;
      }
    }
    const T hiv = T(0.5) * sIV[r];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T gx = g[2 * q], gy = g[2 * q + 1];
      if (moving) rotv(f, g[2 * q], g[2 * q + 1], gx, gy);
      sts2(sG + 2 * (q * NG + gq), gx * hiv, gy * hiv);
    }
  };

  // one face of the tile from buffer b (faces no own cell uses are skipped)
  // work item w: the first TI x TJ i-faces row by row, TI to a row (a warp
  // reads one region row: no bank conflicts), then the TJ faces of column
  // TI, then the j-faces; fq is the face's storage index in sF
  auto face = [&](int w, const Fr<T>& f, int b) {
    const T* W = sW + b * 4 * NR;
    const T* TT = sT + b * NR;
    T vgf, dcx = T(1), dcy = T(0), dsc;
    if constexpr (VISC) lds4(sFR + 4 * w, vgf, dcx, dcy, dsc);
    else lds2(sFR + 2 * w, vgf, dsc);
    const int desc = int_of(dsc);
    if (!(desc & 1)) return;
    const int d = (desc >> 1) & 1, rL = (desc >> 2) & 511, fq = (desc >> 11) & 1023, gLi = (desc >> 21) & 511;
    const int st = d ? RI : 1;
    const int gRi = gLi + (d ? GI : 1);
    const int rR = rL + st;
    // the four cells of the stencil, (u, v) and (rho, p) of each, limited
    // two variables at a time
    using M = Two<T>;
    const T* Wa = W + 4 * (rL - st);
    const T* Wb = W + 4 * rL;
    const T* Wc = W + 4 * rR;
    const T* Wd = W + 4 * (rR + st);
    typename M::v uvL, uvR, rpL, rpR;
    const typename M::v uvb = M::ld(Wb), uvc = M::ld(Wc);
    muscl2<T>(M::ld(Wa), uvb, uvc, M::ld(Wd), eps, uvL, uvR);
    muscl2<T>(M::ld(Wa + 2), M::ld(Wb + 2), M::ld(Wc + 2), M::ld(Wd + 2), eps, rpL, rpR);
    const T WL[4] = {rpL.x, uvL.x, uvL.y, rpL.y}, WR[4] = {rpR.x, uvR.x, uvR.y, rpR.y};   // (rho, u, v, p)
    T sx, sy;
    rotv(f, sS[(2 * d) * NR + rR], sS[(2 * d + 1) * NR + rR], sx, sy);
    // normal grid velocity of the pitching face: thdot times its static factor
    const T vgn = moving ? f.thd * vgf : T(0);
    T F[4];
    roe2d(WL, WR, sx, sy, vgn, gm1, gg1, efix, efrac, hef, F);
    if (VISC) {
      T gl[6], gr[6];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        lds2(sG + 2 * (q * NG + gLi), gl[2 * q], gl[2 * q + 1]);
        lds2(sG + 2 * (q * NG + gRi), gr[2 * q], gr[2 * q + 1]);
      }
      T tx, ty;
      rotv(f, dcx, dcy, tx, ty);
      T Fv[4];
      visc2d(gl, gr, uvb.x, uvb.y, TT[rL], uvc.x, uvc.y, TT[rR], tx, ty, sx,
             sy, mu, kap, Fv);
#pragma unroll
      for (int q = 0; q < 4; ++q) F[q] -= Fv[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) sF[q * NF + fq] = F[q];
  };

  // ---- own-cell geometry that does not change with the snapshot (filled
  // once the region's metrics are staged) and the RK update of one snapshot
  T V = T(1), iV = T(1), a0x = T(0), a0y = T(0), b0x = T(0), b0y = T(0), ma2 = T(1), mb2 = T(1);
  auto own_static = [&]() {
    V = P.g.q[G_VOL][B.goff + cown];
    iV = sIV[rown];
    a0x = T(0.5) * (sS[rown] + sS[rown + 1]);
    a0y = T(0.5) * (sS[NR + rown] + sS[NR + rown + 1]);
    b0x = T(0.5) * (sS[2 * NR + rown] + sS[2 * NR + rown + RI]);
    b0y = T(0.5) * (sS[3 * NR + rown] + sS[3 * NR + rown + RI]);
    ma2 = a0x * a0x + a0y * a0y;
    mb2 = b0x * b0x + b0y * b0y;
  };
  T tacc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) tacc[q] = T(0);
  // residual Rn of the own cell at snapshot n -> R, or the RK update of U0
  // with the local time step (and the norm partial)
  auto finish = [&](int n, T* Rn) {
    const int64_t base = B.off + (int64_t)n * NV * B.plane + cown;
    if (MODE == 1 && P.src) {
#pragma unroll
      for (int q = 0; q < NV; ++q) Rn[q] += P.src[base + q * B.plane];
    }
    if constexpr (MODE == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) P.R[base + q * B.plane] = Rn[q];
    } else {
      T u0[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) u0[q] = P.U0[base + q * B.plane];
      const T rho = u0[0], irho = Ar<T>::rcp(rho);
      const T uv = u0[1] * irho, vv = u0[2] * irho;
      const T pp = gm1 * (u0[3] - T(0.5) * rho * (uv * uv + vv * vv));
      const T c2 = gam * pp * irho;
      const T cs = c2 * Ar<T>::rsq(c2);
      // velocity relative to the pitching grid, in the static frame:
      // R^T u - thdot z x (x_static - pivot)
      T urx = uv, ury = vv;
      if (moving) {
        const Fr<T> f = frame_at(C, n);
        const T xc = P.g.q[G_XC][B.goff + cown], yc = P.g.q[G_XC + 1][B.goff + cown];
        urx = f.c * uv + f.s * vv + f.thd * (yc - f.py);
        ury = f.c * vv - f.s * uv - f.thd * (xc - f.px);
      }
      const T ma = ma2 * Ar<T>::rsq(ma2), mb = mb2 * Ar<T>::rsq(mb2);
      T lam = fabs(urx * a0x + ury * a0y) + cs * ma + fabs(urx * b0x + ury * b0y) + cs * mb;
      if (VISC) {
        const T cv = (gam / C->prandtl > T(4.0 / 3.0)) ? gam / C->prandtl : T(4.0 / 3.0);
        lam += T(4) * cv * (mu * irho) * (ma2 + mb2) * iV;
      }
      lam += (omega * T(C->nh) + P.lam_v) * V;
      // dtau / V = cfl / lambda
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
  };

  // flux balance of the own cell at snapshot n from the face fluxes: kept
  // for the epilogue, or (NS = 0) finished at once with the given HB source
  auto accumulate = [&](int n) {
    if (own) {
      const int fi0 = tj * (TI + 1) + ti;
      const int fj0 = NFI + tj * TI + ti;
      T Rn[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q)
        Rn[q] = (sF[q * NF + fi0 + 1] - sF[q * NF + fi0]) + (sF[q * NF + fj0 + TI] - sF[q * NF + fj0]);
      if constexpr (DYN) {
        if (n == 0) own_static();
        const int64_t base = B.off + (int64_t)n * NV * B.plane + cown;
#pragma unroll
        for (int q = 0; q < NV; ++q) Rn[q] += P.H[base + q * B.plane];
        finish(n, Rn);
      } else {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          if constexpr (BALG && MODE == 1) bal[(n * NV + q) * NT + tid] = Rn[q];
          else if constexpr (BALG) P.R[B.off + ((int64_t)n * NV + q) * B.plane + cown] = Rn[q];
          else sAcc[(n * NV + q) * NT + tid] = Rn[q];
        }
      }
    }
  };

  if constexpr (PIPE) {
    // prologue: snapshot 0 staged (and its gradients); then per snapshot two
    // phases: (A) faces of n + staging of n+1, (B) balance of n + gradients
    // of n+1
    stage_cells(tid, 0, 0);
    __syncthreads();
    if (VISC) {
      const Fr<T> f0 = frame_at(C, 0);
      for (int gq = tid; gq < NGt; gq += nt) grad_cell(gq, f0, 0);
      __syncthreads();
    }
    for (int n = 0; n < ns; ++n) {
      const int b = n & 1;
      const bool next = n + 1 < ns;
      const Fr<T> f = frame_at(C, n);
      // one round-robin over faces then region cells: a thread with one face
      // fewer takes a region cell first
      int w = tid;
      for (; w < NF; w += nt) face(w, f, b);
      if (next) stage_cells(w - NF, n + 1, b ^ 1);
      __syncthreads();
      accumulate(n);
      if (VISC && next) {
        const Fr<T> f1 = frame_at(C, n + 1);
        for (int gq = tid; gq < NGt; gq += nt) grad_cell(gq, f1, b ^ 1);
      }
      __syncthreads();
    }
  } else {
    // per snapshot: staging, gradients, faces, balance; the staging of n+1
    // needs no barrier after the balance of n (which reads only the fluxes)
    for (int n = 0; n < ns; ++n) {
      const Fr<T> f = frame_at(C, n);
      stage_cells(tid, n, 0);
      __syncthreads();
      if (VISC) {
        for (int gq = tid; gq < NGt; gq += nt) grad_cell(gq, f, 0);
        __syncthreads();
      }
      for (int fq = tid; fq < NF; fq += nt) face(fq, f, 0);
      __syncthreads();
      accumulate(n);
    }
    __syncthreads();
  }

  // ---- epilogue: HB source and residual or RK update (compile-time N_s)
  double nacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if constexpr (!DYN) {
    if (own) {
      own_static();
      const T vw = V * omega;
      // the own cell at every snapshot (recently staged, served from cache)
      T uu[DYN ? 1 : NS][NV];
#pragma unroll
      for (int m = 0; m < NS; ++m)
#pragma unroll
        for (int q = 0; q < NV; ++q)
          uu[m][q] = P.Uprev[B.off + ((int64_t)m * NV + q) * B.plane + cown];
      for (int n = 0; n < NS; ++n) {
        T Rn[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          T h = T(0);
#pragma unroll
          for (int m = 0; m < NS; ++m) h += sD[n * NS + m] * uu[m][q];
          T bq;
          if constexpr (BALG && MODE == 1) bq = bal[(n * NV + q) * NT + tid];
          else if constexpr (BALG) bq = P.R[B.off + ((int64_t)n * NV + q) * B.plane + cown];
          else bq = sAcc[(n * NV + q) * NT + tid];
          Rn[q] = bq + vw * h;
        }
        finish(n, Rn);
      }
    }
  }
  if constexpr (BALG && MODE == 1) {
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
    double* scratch = reinterpret_cast<double*>(sm);   // primitives are dead here
    block_sum8(nacc, NV, scratch);
    if (threadIdx.x == 0)
      for (int q = 0; q < NV; ++q) P.partials[(int64_t)t * 8 + q] = nacc[q];
  }
  if (MODE == 1 && P.job_range) fill_tile_ghosts<T, NS>(P, t, B, C);
}

// CTAs per SM a tile kernel is compiled for: 24 warps in FP32, 8 in FP64;
// the inviscid runtime-N_s tile of 128 threads (no balance array: 25 KB of
// shared memory) runs seven CTAs (28 warps) within 72 registers (eight
// spilled and measured slower)
__host__ __device__ constexpr int tile2d_min_ctas(bool fp32, int NS, bool VISC, int NT) {
  return fp32 ? ((NS == 0 && !VISC && NT == 128) ? 7 : 3 * (MAXNT / NT)) : MAXNT / NT;
}

template <typename T, int NS, bool VISC, int MODE, int TI, int TJ>
__global__ void __launch_bounds__(TI * TJ, tile2d_min_ctas(sizeof(T) == 4, NS, VISC, TI * TJ))
    tile2d_kernel(StageParams<T> P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  tile2d<T, NS, VISC, MODE, TI, TJ, tile_pipelined(NS, MODE), tile_park(NS, MODE)>(
      P, blockIdx.x, reinterpret_cast<T*>(smraw));
}

// tile shapes built into the library (index = StageParams shape id)
constexpr int kTileShapes = 3;
__host__ __device__ constexpr int tile_ti(int id) { return id == 0 ? 32 : (id == 1 ? 32 : 16); }
__host__ __device__ constexpr int tile_tj(int id) { return id == 0 ? 8 : (id == 1 ? 4 : 8); }

// ------------------------------------------------------------- halo kernel --
// one work item per (record, snapshot), snapshot-major so that neighbouring
// threads touch neighbouring cells
template <typename T, int DIM>
__device__ __forceinline__ void halo_item(const HaloParams<T>& p, int64_t gid) {
  constexpr int NV = DIM + 2;
  const int64_t nc = (int64_t)p.ncopy * p.ns_max;
  if (gid < nc) {
    const int n = (int)(gid / p.ncopy), rec = (int)(gid % p.ncopy);
    const CopyRec r = p.copies[rec];
    const BlockDev& D = p.blocks[r.dst_blk];
    const BlockDev& S = p.blocks[r.src_blk];
    if (n >= p.cases[D.cs].ns) return;
    const T* src = p.U + S.off + (int64_t)n * NV * S.plane + r.src_cell;
    T* dst = p.U + D.off + (int64_t)n * NV * D.plane + r.dst_cell;
#pragma unroll
    for (int v = 0; v < NV; ++v) dst[v * D.plane] = src[v * S.plane];
    return;
  }
  const int64_t gb = gid - nc;
  if (gb >= (int64_t)p.nbc * p.ns_max) return;
  const int n = (int)(gb / p.nbc), rec = (int)(gb % p.nbc);
  const BcRec r = p.bcs[rec];
  const BlockDev& B = p.blocks[r.blk];
  const CaseDev<T>* C = p.cases + B.cs;
  if (n >= C->ns) return;
  const T gm1 = C->gamma - T(1);
  T* Ub = p.U + B.off + (int64_t)n * NV * B.plane;
  T Wi[5], Wg[5];
  if (r.type == 1) {   // farfield: both ghost layers from the first interior cell
    load_prim<T, DIM>(Ub, B.plane, r.mcell[0], gm1, Wi);
    bc_map<T, DIM>(C, p.g, B, r.type, r.p, r.sgn, r.fcell, n, Wi, Wg);
    store_cons<T, DIM>(Ub, B.plane, r.gcell[0], gm1, Wg);
    store_cons<T, DIM>(Ub, B.plane, r.gcell[1], gm1, Wg);
  } else {             // walls: each ghost layer mirrors its own interior layer
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      load_prim<T, DIM>(Ub, B.plane, r.mcell[l], gm1, Wi);
      bc_map<T, DIM>(C, p.g, B, r.type, r.p, r.sgn, r.fcell, n, Wi, Wg);
      store_cons<T, DIM>(Ub, B.plane, r.gcell[l], gm1, Wg);
    }
  }
}

template <typename T, int DIM>
__global__ void halo_kernel(HaloParams<T> p) {
  halo_item<T, DIM>(p, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------- initial state --
template <typename T, int DIM>
__global__ void init_kernel(const CaseDev<T>* cases, const BlockDev* blocks, Geo<T> g, T* U,
                            const double* noise, double amp, int blk) {
  constexpr int NV = DIM + 2;
  const BlockDev B = blocks[blk];
  const CaseDev<T>* C = cases + B.cs;
  const int64_t ncell = (int64_t)B.n[0] * B.n[1] * B.n[2];
  const int64_t tot = ncell * C->ns * NV;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cellid = e % ncell;
    const int v = (int)((e / ncell) % NV);
    const int n = (int)(e / (ncell * NV));
    const int i = (int)(cellid % B.n[0]);
    const int j = (int)((cellid / B.n[0]) % B.n[1]);
    const int k = (int)(cellid / ((int64_t)B.n[0] * B.n[1]));
    const int64_t c = ((int64_t)(k + B.gk) * B.P[1] + (j + 2)) * B.P[0] + (i + 2);
    T W[5];
    freestream_at(C, n, g.q[G_XC][B.goff + c], W);
    T val;
    if (v == 0) val = W[0];
    else if (v <= DIM) val = W[0] * W[v];
    else val = W[4] / (C->gamma - T(1)) + T(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
    const double z = noise ? noise[B.noff + e] : 0.0;
    U[B.off + ((int64_t)n * NV + v) * B.plane + c] = (T)((double)val * (1.0 + amp * z));
  }
}

// ----------------------------------------------------------------- forces --
// Green-Gauss gradient of (u, v, T) at padded cell c from global memory (2D)
// snapshot base of padded cell cc: Ub for interior cells, Gb for ghosts
template <typename T>
__device__ __forceinline__ const T* cell_src(const BlockDev& B, const T* Ub, const T* Gb, int cc) {
  const int i = cc % B.P[0] - 2, j = cc / B.P[0] - 2;
  return (i >= 0 && i < B.n[0] && j >= 0 && j < B.n[1]) ? Ub : Gb;
}

template <typename T>
__device__ void grad_global2d(const BlockDev& B, const CaseDev<T>* C, const Geo<T>& g,
                              const T* Ub, const T* Gb, const Fr<T>& f, int c, T* out) {
  const T gam = C->gamma, gm1 = gam - T(1);
  auto prim = [&](int cc, T& u, T& v, T& Tt) {
    const T* X = cell_src(B, Ub, Gb, cc);
    const T rho = X[cc];
    u = X[B.plane + cc] / rho;
    v = X[2 * B.plane + cc] / rho;
    const T p = gm1 * (X[3 * B.plane + cc] - T(0.5) * rho * (u * u + v * v));
    Tt = gam * p / rho;
  };
  T uc, vc, Tc;
  prim(c, uc, vc, Tc);
  const int P0 = B.P[0];
  const int nb[4] = {c - 1, c + 1, c - P0, c + P0};
  const int fo[4] = {c, c + 1, c, c + P0};
  for (int q = 0; q < 6; ++q) out[q] = T(0);
  for (int k = 0; k < 4; ++k) {
    const int d = k >> 1;
    const T sg = (k & 1) ? T(1) : T(-1);
    T sx, sy;
    rotv(f, g.q[G_S + 3 * d][B.goff + fo[k]], g.q[G_S + 3 * d + 1][B.goff + fo[k]], sx, sy);
    T un, vn, Tn;
    prim(nb[k], un, vn, Tn);
    const T fu = T(0.5) * (un - uc), fv = T(0.5) * (vn - vc), fT = T(0.5) * (Tn - Tc);
    out[0] += sg * fu * sx; out[1] += sg * fu * sy;
    out[2] += sg * fv * sx; out[3] += sg * fv * sy;
    out[4] += sg * fT * sx; out[5] += sg * fT * sy;
  }
  const T iv = T(1) / g.q[G_VOL][B.goff + c];
  for (int q = 0; q < 6; ++q) out[q] *= iv;
}

// per wall face and snapshot: pressure and viscous force, moment about the pivot
template <typename T>
__global__ void force_faces_kernel(ForceParams<T> p) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= p.nwall * p.ns) return;
  // consecutive threads take consecutive wall faces of one snapshot
  const int n = gid / p.nwall, rec = gid % p.nwall;
  const BcRec r = p.walls[rec];
  const BlockDev B = p.blocks[r.blk];
  const CaseDev<T>* C = p.cases + B.cs;
  const Fr<T> f = frame_at(C, n);
  const T gam = C->gamma, gm1 = gam - T(1);
  const T* Ub = p.U + B.off + (int64_t)n * 4 * B.plane;
  const T* Gb = (p.G ? p.G : p.U) + B.off + (int64_t)n * 4 * B.plane;
  const int64_t fc = B.goff + r.fcell;
  T sx, sy, xf, yf;
  rotv(f, p.g.q[G_S + 3 * r.p][fc], p.g.q[G_S + 3 * r.p + 1][fc], sx, sy);
  rotp(f, p.g.q[G_XF + 3 * r.p][fc], p.g.q[G_XF + 3 * r.p + 1][fc], xf, yf);
  const T sg = T(r.sgn);
  const T sbx = sg * sx, sby = sg * sy;   // into the body
  const int ic = r.mcell[0], gc = r.gcell[0];
  const T rho = Ub[ic], u = Ub[B.plane + ic] / rho, v = Ub[2 * B.plane + ic] / rho;
  const T pw = gm1 * (Ub[3 * B.plane + ic] - T(0.5) * rho * (u * u + v * v));
  T Fx = (pw - C->pinf) * sbx, Fy = (pw - C->pinf) * sby;
  if (C->viscous) {
    const int cl = (r.sgn > 0) ? ic : gc, cr = (r.sgn > 0) ? gc : ic;
    T gL[6], gR[6];
    grad_global2d(B, C, p.g, Ub, Gb, f, cl, gL);
    grad_global2d(B, C, p.g, Ub, Gb, f, cr, gR);
    T tx, ty;   // centre difference x_R - x_L, stored with the high cell cr = cl + e_p
    rotv(f, p.g.q[G_DC + 3 * r.p][B.goff + cr], p.g.q[G_DC + 3 * r.p + 1][B.goff + cr], tx, ty);
    auto prim = [&](int cc, T& uu, T& vv, T& Tt) {
      const T* X = cell_src(B, Ub, Gb, cc);
      const T rr = X[cc];
      uu = X[B.plane + cc] / rr;
      vv = X[2 * B.plane + cc] / rr;
      Tt = gam * gm1 * (X[3 * B.plane + cc] - T(0.5) * rr * (uu * uu + vv * vv)) / rr;
    };
    T uL, vL, TL, uR, vR, TR;
    prim(cl, uL, vL, TL);
    prim(cr, uR, vR, TR);
    // traction through the face vector (pointing L -> R): reuse the flux routine
    T Fv[4];
    visc2d(gL, gR, uL, vL, TL, uR, vR, TR, tx, ty, sx, sy, C->mu, C->kappa, Fv);
    // Fv[1..2] = tau . S with S = sgn * S_b; tau . S_b = sgn * Fv
    Fx -= sg * Fv[1];
    Fy -= sg * Fv[2];
  }
  const double q = 0.5 * (double)C->mach * (double)C->mach;
  double* o = p.face_out + ((int64_t)n * p.nwall + rec) * 3;
  o[0] = ((double)Fx * (double)-C->sina0 + (double)Fy * (double)C->cosa0) / q;
  o[1] = ((double)Fx * (double)C->cosa0 + (double)Fy * (double)C->sina0) / q;
  o[2] = (C->functag == 3)
             ? (((double)xf - (double)C->pivot[0]) * (double)Fy - ((double)yf - (double)C->pivot[1]) * (double)Fx) / q
             : 0.0;
}

// fixed-order FP64 sums per (snapshot, body): CTA (n, b) strides over the
// wall faces, then a fixed warp/tree order; the last CTA to finish forms J
template <typename T>
__global__ void force_finish_kernel(ForceParams<T> p, unsigned int* done) {
  __shared__ double red[32][3];
  const int n = blockIdx.x / p.nbodies, b = blockIdx.x % p.nbodies;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int rec = threadIdx.x; rec < p.nwall; rec += blockDim.x)
    if (p.walls[rec].body == b)
      for (int k = 0; k < 3; ++k) acc[k] += p.face_out[((int64_t)n * p.nwall + rec) * 3 + k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 3; ++k) {
    double x = acc[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w][threadIdx.x];
    p.coef_scratch[(n * p.nbodies + b) * 3 + threadIdx.x] = sum;
    if (p.coef) p.coef[(n * p.nbodies + b) * 3 + threadIdx.x] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int ticket = atomicAdd(done, 1u);
    if (ticket == gridDim.x - 1) {      // last CTA: every partial is visible
      __threadfence();
      if (p.J) {
        double j = 0.0;
        for (int nn = 0; nn < p.ns; ++nn)
          for (int bb = 0; bb < p.nbodies; ++bb)
            j += ((volatile double*)p.coef_scratch)[(nn * p.nbodies + bb) * 3];
        *p.J = j / (double)p.ns;
      }
      *done = 0u;                       // ready for the next launch
    }
  }
}

}  // namespace hbk
