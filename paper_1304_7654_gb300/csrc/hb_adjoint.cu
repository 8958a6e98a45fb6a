// Reverse-mode adjoint of the 2D HB residual and the time-averaged lift
// (hb_adjoint_residual), FP64.
//
//   r_adj = (dR_HB/dU)^T psi + J_seed dJ/dU
//
// R_HB(U) = F(G(U)) + V omega D U, with G the ghost fill (cuts and physical
// boundary ghosts, pass by pass) and F the flux balance; J = (1/N_s) sum cl.
// Hand-written reverse of every step, recomputing the primal intermediates
// (reconstruction, limiter, Roe averages, gradients) instead of storing them:
//   A. per face and snapshot: Fbar = psi_L - psi_R (interior sides only), plus
//      the lift seed on wall faces; reverse through Roe, MUSCL/van Albada,
//      the viscous flux and the two Green-Gauss gradients to the 8 cells of
//      the face stencil; the 8 x nv contributions go to a face buffer;
//   B. per padded cell and snapshot: gather the 16 (face, slot) contributions
//      in a fixed order, add the HB transpose V omega D^T psi (D^T = -D);
//   C. ghost transpose, last pass first: every source cell gathers, in a
//      fixed order, the adjoint of the ghost cells it fills (copy, or the
//      Jacobian-transpose of the farfield / wall map at the primal state);
//   D. r_adj = interior part.
// No atomics: every sum has one owner thread and a fixed order.
#include <cuda_runtime.h>

#include <cstdint>

#include "hb_adjoint.h"
#include "hb_kernels.cuh"

namespace hbk {

namespace {

using T = double;
constexpr int NV = 4;

__device__ __forceinline__ T sgnf(T x) { return x < 0.0 ? -1.0 : 1.0; }

// primitives (rho, u, v, p) and T from conservative U
__device__ __forceinline__ void prim4(const T* U, T gm1, T gam, T* W, T& Tt) {
  const T ir = 1.0 / U[0];
  W[0] = U[0];
  W[1] = U[1] * ir;
  W[2] = U[2] * ir;
  W[3] = gm1 * (U[3] - 0.5 * U[0] * (W[1] * W[1] + W[2] * W[2]));
  Tt = gam * W[3] * ir;
}

// Wbar (rho, u, v, p) and Tbar -> Ubar
__device__ __forceinline__ void prim4_adj(const T* W, T Tbar, const T* Wb_in, T gm1, T gam, T* Ub) {
  T Wb[4] = {Wb_in[0], Wb_in[1], Wb_in[2], Wb_in[3]};
  const T rho = W[0], u = W[1], v = W[2], ir = 1.0 / rho;
  // T = gam p / rho
  const T tg = Tbar * gam * ir;
  Wb[3] += tg;
  Wb[0] -= tg * W[3] * ir;
  Ub[0] = Wb[0] - (Wb[1] * u + Wb[2] * v) * ir + Wb[3] * gm1 * 0.5 * (u * u + v * v);
  Ub[1] = Wb[1] * ir - Wb[3] * gm1 * u;
  Ub[2] = Wb[2] * ir - Wb[3] * gm1 * v;
  Ub[3] = Wb[3] * gm1;
}

// adjoint of conservative-from-primitive (Ubar -> Wbar)
__device__ __forceinline__ void cons4_adj(const T* W, const T* Ub, T ig1, T* Wb) {
  const T k = 0.5 * (W[1] * W[1] + W[2] * W[2]);
  Wb[0] = Ub[0] + Ub[1] * W[1] + Ub[2] * W[2] + Ub[3] * k;
  Wb[1] = Ub[1] * W[0] + Ub[3] * W[0] * W[1];
  Wb[2] = Ub[2] * W[0] + Ub[3] * W[0] * W[2];
  Wb[3] = Ub[3] * ig1;
}

// van Albada va(a, b) = N / Dn, returned, and its partial derivatives
__device__ __forceinline__ T va_d(T a, T b, T eps, T& da, T& db) {
  const T N = (b * b + eps) * a + (a * a + eps) * b;
  const T iD = 1.0 / (a * a + b * b + 2.0 * eps);
  const T v = N * iD;
  da = (b * b + eps + 2.0 * a * b - v * 2.0 * a) * iD;
  db = (2.0 * a * b + a * a + eps - v * 2.0 * b) * iD;
  return v;
}

// Reverse of roe2d (plain FP64 forms): Fb -> WLb, WRb (accumulated)
__device__ void roe2d_adj(const T* WL, const T* WR, T Sx, T Sy, T vgn, T gam, int efix, T efrac,
                          const T* Fb, T* WLb, T* WRb) {
  const T gm1 = gam - 1.0, gg1 = gam / gm1, ig1 = 1.0 / gm1;
  // each quotient below multiplies by one reciprocal taken once
  const T A = sqrt(Sx * Sx + Sy * Sy), iA = 1.0 / A;
  const T nx = Sx * iA, ny = Sy * iA;
  // ---- forward
  const T rL = WL[0], uL = WL[1], vL = WL[2], pL = WL[3];
  const T rR = WR[0], uR = WR[1], vR = WR[2], pR = WR[3];
  const T irL = 1.0 / rL, irR = 1.0 / rR;
  const T qL = uL * nx + vL * ny, qR = uR * nx + vR * ny;
  const T kL = 0.5 * (uL * uL + vL * vL), kR = 0.5 * (uR * uR + vR * vR);
  const T HL = gg1 * pL * irL + kL, HR = gg1 * pR * irR + kR;
  const T rr = rR * irL;
  const T r = sqrt(rr);
  const T ir = r * rL * irR;   // 1 / r = r / rr
  const T rt = r * rL;
  const T den = 1.0 + r, iden = 1.0 / den;
  const T ut = (uL + r * uR) * iden, vt = (vL + r * vR) * iden, Ht = (HL + r * HR) * iden;
  const T kt = 0.5 * (ut * ut + vt * vt);
  const T ct2 = gm1 * (Ht - kt);
  const T ct = sqrt(ct2), ict2 = 1.0 / ct2, ict = ct * ict2;
  const T qt = ut * nx + vt * ny;
  const T qtr = qt - vgn;
  const T x1 = qtr - ct, x3 = qtr + ct;
  T l1 = fabs(x1), l2 = fabs(qtr), l3 = fabs(x3);
  const T del = efrac * ct;
  const T idel = efix ? 1.0 / del : 0.0;
  bool f1 = false, f3 = false;
  if (efix) {
    if (l1 < del) { l1 = (l1 * l1 + del * del) * (0.5 * idel); f1 = true; }
    if (l3 < del) { l3 = (l3 * l3 + del * del) * (0.5 * idel); f3 = true; }
  }
  const T dp = pR - pL, drho = rR - rL, dq = qR - qL;
  const T h2 = 0.5 * ict2;   // 1 / (2 ct2)
  const T a1 = (dp - rt * ct * dq) * h2;
  const T a3 = (dp + rt * ct * dq) * h2;
  const T a2 = drho - dp * ict2;
  const T dux = (uR - uL) - dq * nx, duy = (vR - vL) - dq * ny;
  const T udu = ut * dux + vt * duy;
  const T w1 = l1 * a1, w3 = l3 * a3;
  const T qLr = qL - vgn, qRr = qR - vgn;
  const T EL = pL * ig1 + rL * kL, ER = pR * ig1 + rR * kR;
  // ---- reverse
  const T hA = 0.5 * A;
  const T t0 = hA * Fb[0], t1 = hA * Fb[1], t2 = hA * Fb[2], t3 = hA * Fb[3];
  T rLb = 0, uLb = 0, vLb = 0, pLb = 0, rRb = 0, uRb = 0, vRb = 0, pRb = 0;
  T qLrb = 0, qRrb = 0, qLb = 0, qRb = 0, ELb = 0, ERb = 0;
  // F0 = hA (rL qLr + rR qRr - D0)
  rLb += t0 * qLr; qLrb += t0 * rL; rRb += t0 * qRr; qRrb += t0 * rR;
  T D0b = -t0;
  // F1 = hA (rL uL qLr + pL nx + rR uR qRr + pR nx - D1)
  rLb += t1 * uL * qLr; uLb += t1 * rL * qLr; qLrb += t1 * rL * uL; pLb += t1 * nx;
  rRb += t1 * uR * qRr; uRb += t1 * rR * qRr; qRrb += t1 * rR * uR; pRb += t1 * nx;
  T D1b = -t1;
  // F2
  rLb += t2 * vL * qLr; vLb += t2 * rL * qLr; qLrb += t2 * rL * vL; pLb += t2 * ny;
  rRb += t2 * vR * qRr; vRb += t2 * rR * qRr; qRrb += t2 * rR * vR; pRb += t2 * ny;
  T D2b = -t2;
  // F3 = hA (EL qLr + pL qL + ER qRr + pR qR - D3)
  ELb += t3 * qLr; qLrb += t3 * EL; pLb += t3 * qL; qLb += t3 * pL;
  ERb += t3 * qRr; qRrb += t3 * ER; pRb += t3 * qR; qRb += t3 * pR;
  T D3b = -t3;
  // E = p ig1 + rho k
  T kLb = 0, kRb = 0;
  pLb += ELb * ig1; rLb += ELb * kL; kLb += ELb * rL;
  pRb += ERb * ig1; rRb += ERb * kR; kRb += ERb * rR;
  qLb += qLrb;
  qRb += qRrb;
  // dissipation terms
  T w1b = 0, w3b = 0, l2b = 0, a2b = 0, Htb = 0, ctb = 0, qtb = 0, ktb = 0, rtb = 0, udub = 0;
  T utb = 0, vtb = 0, duxb = 0, duyb = 0;
  // D3 = w1 (Ht - ct qt) + l2 (a2 kt + rt udu) + w3 (Ht + ct qt)
  w1b += D3b * (Ht - ct * qt);
  w3b += D3b * (Ht + ct * qt);
  Htb += D3b * (w1 + w3);
  ctb += D3b * (w3 - w1) * qt;
  qtb += D3b * (w3 - w1) * ct;
  l2b += D3b * (a2 * kt + rt * udu);
  a2b += D3b * l2 * kt;
  ktb += D3b * l2 * a2;
  rtb += D3b * l2 * udu;
  udub += D3b * l2 * rt;
  // D2 = w1 (vt - ct ny) + l2 (a2 vt + rt duy) + w3 (vt + ct ny)
  w1b += D2b * (vt - ct * ny);
  w3b += D2b * (vt + ct * ny);
  vtb += D2b * (w1 + l2 * a2 + w3);
  ctb += D2b * (w3 - w1) * ny;
  l2b += D2b * (a2 * vt + rt * duy);
  a2b += D2b * l2 * vt;
  rtb += D2b * l2 * duy;
  duyb += D2b * l2 * rt;
  // D1
  w1b += D1b * (ut - ct * nx);
  w3b += D1b * (ut + ct * nx);
  utb += D1b * (w1 + l2 * a2 + w3);
  ctb += D1b * (w3 - w1) * nx;
  l2b += D1b * (a2 * ut + rt * dux);
  a2b += D1b * l2 * ut;
  rtb += D1b * l2 * dux;
  duxb += D1b * l2 * rt;
  // D0 = w1 + l2 a2 + w3
  w1b += D0b;
  w3b += D0b;
  l2b += D0b * a2;
  a2b += D0b * l2;
  // w1 = l1 a1, w3 = l3 a3
  T l1b = w1b * a1, a1b = w1b * l1, l3b = w3b * a3, a3b = w3b * l3;
  // udu = ut dux + vt duy
  utb += udub * dux; duxb += udub * ut; vtb += udub * duy; duyb += udub * vt;
  // dux = (uR - uL) - dq nx, duy = (vR - vL) - dq ny
  T dqb = 0, dpb = 0, drhob = 0, ct2b = 0;
  uRb += duxb; uLb -= duxb; dqb -= duxb * nx;
  vRb += duyb; vLb -= duyb; dqb -= duyb * ny;
  // a2 = drho - dp / ct2
  drhob += a2b; dpb -= a2b * ict2; ct2b += a2b * dp * ict2 * ict2;
  // a3 = (dp + rt ct dq) / (2 ct2)
  dpb += a3b * h2; rtb += a3b * ct * dq * h2; ctb += a3b * rt * dq * h2;
  dqb += a3b * rt * ct * h2; ct2b -= a3b * a3 * ict2;
  // a1 = (dp - rt ct dq) / (2 ct2)
  dpb += a1b * h2; rtb -= a1b * ct * dq * h2; ctb -= a1b * rt * dq * h2;
  dqb -= a1b * rt * ct * h2; ct2b -= a1b * a1 * ict2;
  pRb += dpb; pLb -= dpb; rRb += drhob; rLb -= drhob; qRb += dqb; qLb -= dqb;
  // wave speeds
  T qtrb = 0, delb = 0;
  {
    const T ax = fabs(x1);
    T x1b;
    if (f1) { x1b = l1b * (ax * idel) * sgnf(x1); delb += l1b * (0.5 - 0.5 * ax * ax * idel * idel); }
    else x1b = l1b * sgnf(x1);
    qtrb += x1b; ctb -= x1b;
  }
  {
    const T ax = fabs(x3);
    T x3b;
    if (f3) { x3b = l3b * (ax * idel) * sgnf(x3); delb += l3b * (0.5 - 0.5 * ax * ax * idel * idel); }
    else x3b = l3b * sgnf(x3);
    qtrb += x3b; ctb += x3b;
  }
  qtrb += l2b * sgnf(qtr);
  ctb += delb * efrac;
  qtb += qtrb;
  utb += qtb * nx; vtb += qtb * ny;
  ct2b += ctb * (0.5 * ict);
  Htb += gm1 * ct2b; ktb -= gm1 * ct2b;
  utb += ktb * ut; vtb += ktb * vt;
  // Roe averages
  T HLb = 0, HRb = 0, rb = 0, denb = 0;
  HLb += Htb * iden; HRb += Htb * r * iden; rb += Htb * HR * iden; denb -= Htb * Ht * iden;
  uLb += utb * iden; uRb += utb * r * iden; rb += utb * uR * iden; denb -= utb * ut * iden;
  vLb += vtb * iden; vRb += vtb * r * iden; rb += vtb * vR * iden; denb -= vtb * vt * iden;
  rb += denb;
  rb += rtb * rL; rLb += rtb * r;
  const T rrb = rb * (0.5 * ir);
  rRb += rrb * irL; rLb -= rrb * rr * irL;
  // H = gg1 p / rho + k
  pLb += HLb * gg1 * irL; rLb -= HLb * gg1 * pL * irL * irL; kLb += HLb;
  pRb += HRb * gg1 * irR; rRb -= HRb * gg1 * pR * irR * irR; kRb += HRb;
  uLb += kLb * uL; vLb += kLb * vL; uRb += kRb * uR; vRb += kRb * vR;
  uLb += qLb * nx; vLb += qLb * ny; uRb += qRb * nx; vRb += qRb * ny;
  WLb[0] += rLb; WLb[1] += uLb; WLb[2] += vLb; WLb[3] += pLb;
  WRb[0] += rRb; WRb[1] += uRb; WRb[2] += vRb; WRb[3] += pRb;
}

// Reverse of visc2d: Fvb (Fv[1..3]) -> gLb, gRb (6 each), phi bars at L, R
__device__ void visc2d_adj(const T* gL, const T* gR, T uL, T vL, T TL, T uR, T vR, T TR, T tx, T ty,
                           T Sx, T Sy, T mu, T kap, const T* Fvb, T* gLb, T* gRb, T* phiLb,
                           T* phiRb) {
  const T len = sqrt(tx * tx + ty * ty);
  const T il = 1.0 / len;
  const T ex = tx * il, ey = ty * il;
  T g[6];
  for (int q = 0; q < 3; ++q) {
    const T bx = 0.5 * (gL[2 * q] + gR[2 * q]);
    const T by = 0.5 * (gL[2 * q + 1] + gR[2 * q + 1]);
    const T dphi = (q == 0) ? (uR - uL) : (q == 1) ? (vR - vL) : (TR - TL);
    const T corr = dphi * il - (bx * ex + by * ey);
    g[2 * q] = bx + corr * ex;
    g[2 * q + 1] = by + corr * ey;
  }
  const T div = g[0] + g[3];
  const T txx = 2.0 * mu * g[0] - (2.0 / 3.0) * mu * div;
  const T tyy = 2.0 * mu * g[3] - (2.0 / 3.0) * mu * div;
  const T txy = mu * (g[1] + g[2]);
  const T fx = txx * Sx + txy * Sy;
  const T fy = txy * Sx + tyy * Sy;
  const T uf = 0.5 * (uL + uR), vf = 0.5 * (vL + vR);
  // reverse
  const T fxb = Fvb[1] + Fvb[3] * uf, fyb = Fvb[2] + Fvb[3] * vf;
  const T ufb = Fvb[3] * fx, vfb = Fvb[3] * fy;
  T gb[6] = {0, 0, 0, 0, Fvb[3] * kap * Sx, Fvb[3] * kap * Sy};
  const T txxb = fxb * Sx, txyb = fxb * Sy + fyb * Sx, tyyb = fyb * Sy;
  const T divb = -(2.0 / 3.0) * mu * (txxb + tyyb);
  gb[0] += 2.0 * mu * txxb + divb;
  gb[3] += 2.0 * mu * tyyb + divb;
  gb[1] += mu * txyb;
  gb[2] += mu * txyb;
  phiLb[0] += 0.5 * ufb; phiRb[0] += 0.5 * ufb;
  phiLb[1] += 0.5 * vfb; phiRb[1] += 0.5 * vfb;
  for (int q = 0; q < 3; ++q) {
    const T gxb = gb[2 * q], gyb = gb[2 * q + 1];
    const T corrb = gxb * ex + gyb * ey;
    const T bxb = gxb - corrb * ex, byb = gyb - corrb * ey;
    const T dphib = corrb * il;
    gLb[2 * q] += 0.5 * bxb; gRb[2 * q] += 0.5 * bxb;
    gLb[2 * q + 1] += 0.5 * byb; gRb[2 * q + 1] += 0.5 * byb;
    phiRb[q] += dphib; phiLb[q] -= dphib;
  }
}

struct FaceCtx {
  const BlockDev* B;
  const Geo<T>* g;
  Fr<T> f;
};

// rotated low-face vector of padded cell c along d
__device__ __forceinline__ void face_S(const BlockDev& B, const Geo<T>& g, const Fr<T>& f, int d,
                                       int64_t c, T& sx, T& sy) {
  rotv(f, g.q[G_S + 3 * d][B.goff + c], g.q[G_S + 3 * d + 1][B.goff + c], sx, sy);
}

// Green-Gauss gradient of (u, v, T) at cell c whose 4 neighbours are given
// (order: -d, +d, -t, +t with d = 0 the i direction): returns g[6]
__device__ void gg_grad(const BlockDev& B, const Geo<T>& g, const Fr<T>& f, int64_t c,
                        const int64_t* nb, const T (*phi_c), const T (*phi_nb)[3], T* out) {
  const int64_t fo[4] = {c, nb[1], c, nb[3]};
  const int dirs[4] = {0, 0, 1, 1};
  for (int q = 0; q < 6; ++q) out[q] = 0.0;
  for (int k = 0; k < 4; ++k) {
    T sx, sy;
    face_S(B, g, f, dirs[k], fo[k], sx, sy);
    const T sg = (k & 1) ? 0.5 : -0.5;
    for (int q = 0; q < 3; ++q) {
      const T dphi = phi_nb[k][q] - phi_c[q];
      out[2 * q] += sg * dphi * sx;
      out[2 * q + 1] += sg * dphi * sy;
    }
  }
  const T iv = 1.0 / g.q[G_VOL][B.goff + c];
  for (int q = 0; q < 6; ++q) out[q] *= iv;
}

__device__ void gg_grad_adj(const BlockDev& B, const Geo<T>& g, const Fr<T>& f, int64_t c,
                            const int64_t* nb, const T* gb, T* phicb, T (*phinbb)[3]) {
  const int64_t fo[4] = {c, nb[1], c, nb[3]};
  const int dirs[4] = {0, 0, 1, 1};
  const T iv = 1.0 / g.q[G_VOL][B.goff + c];
  for (int k = 0; k < 4; ++k) {
    T sx, sy;
    face_S(B, g, f, dirs[k], fo[k], sx, sy);
    const T sg = (k & 1) ? 0.5 : -0.5;
    for (int q = 0; q < 3; ++q) {
      const T db = (gb[2 * q] * sx + gb[2 * q + 1] * sy) * sg * iv;
      phinbb[k][q] += db;
      phicb[q] -= db;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- phase A --
__global__ void adj_faces_kernel(AdjParams p) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= p.nfaces * (int64_t)p.ns) return;
  const int n = (int)(gid % p.ns);
  const int64_t face = gid / p.ns;
  int b = 0;
  while (b + 1 < p.nblocks && p.foff[b + 1] <= face) ++b;
  const BlockDev B = p.blocks[b];
  const CaseDev<T>* C = p.cases + B.cs;
  const int64_t lf = face - p.foff[b];
  const int n0 = B.n[0], n1 = B.n[1];
  const int64_t nfi = (int64_t)(n0 + 1) * n1;
  int d, fi, fj;
  if (lf < nfi) { d = 0; fi = (int)(lf % (n0 + 1)); fj = (int)(lf / (n0 + 1)); }
  else { d = 1; const int64_t q = lf - nfi; fi = (int)(q % n0); fj = (int)(q / n0); }
  const int P0 = B.P[0];
  auto pc = [&](int i, int j) -> int64_t { return (int64_t)(j + 2) * P0 + (i + 2); };
  const int ed[2] = {d == 0 ? 1 : 0, d == 0 ? 0 : 1};   // e_d
  const int et[2] = {d == 0 ? 0 : 1, d == 0 ? 1 : 0};   // e_t
  const int Ri = fi, Rj = fj, Li = fi - ed[0], Lj = fj - ed[1];
  // stencil: 0 LL, 1 L, 2 R, 3 RR, 4 L-t, 5 L+t, 6 R-t, 7 R+t
  int si[8], sj[8];
  si[0] = Li - ed[0]; sj[0] = Lj - ed[1];
  si[1] = Li; sj[1] = Lj;
  si[2] = Ri; sj[2] = Rj;
  si[3] = Ri + ed[0]; sj[3] = Rj + ed[1];
  si[4] = Li - et[0]; sj[4] = Lj - et[1];
  si[5] = Li + et[0]; sj[5] = Lj + et[1];
  si[6] = Ri - et[0]; sj[6] = Rj - et[1];
  si[7] = Ri + et[0]; sj[7] = Rj + et[1];
  int64_t sc[8];
  for (int k = 0; k < 8; ++k) sc[k] = pc(si[k], sj[k]);
  const T gam = C->gamma, gm1 = gam - 1.0;
  const T* Ub = p.U + B.off + (int64_t)n * NV * B.plane;
  T W[8][4], Tt[8];
  for (int k = 0; k < 8; ++k) {
    T u[4];
    for (int v = 0; v < NV; ++v) u[v] = Ub[v * B.plane + sc[k]];
    prim4(u, gm1, gam, W[k], Tt[k]);
  }
  const Fr<T> f = frame_at(C, n);
  // face residual adjoint: F enters R_L with +, R_R with -
  const bool Lin = Li >= 0 && Li < n0 && Lj >= 0 && Lj < n1;
  const bool Rin = Ri >= 0 && Ri < n0 && Rj >= 0 && Rj < n1;
  const T* Pb = p.psi + B.off + (int64_t)n * NV * B.plane;
  T Fb[4];
  for (int v = 0; v < NV; ++v)
    Fb[v] = (Lin ? Pb[v * B.plane + sc[1]] : 0.0) - (Rin ? Pb[v * B.plane + sc[2]] : 0.0);
  // face geometry (low face of R along d)
  T sx, sy;
  face_S(B, p.g, f, d, sc[2], sx, sy);
  T vgn = 0.0;
  if (C->motion) {
    T xf, yf;
    rotp(f, p.g.q[G_XF + 3 * d][B.goff + sc[2]], p.g.q[G_XF + 3 * d + 1][B.goff + sc[2]], xf, yf);
    const T vgx = -f.thd * (yf - f.py), vgy = f.thd * (xf - f.px);
    vgn = (vgx * sx + vgy * sy) / sqrt(sx * sx + sy * sy);
  }
  T Wb[8][4], Tb[8];
  for (int k = 0; k < 8; ++k) { Tb[k] = 0.0; for (int v = 0; v < 4; ++v) Wb[k][v] = 0.0; }
  // lift seed on wall faces: J_f = s [(p_w - p_inf) Sb.eL - sgn (Fv1, Fv2).eL]
  T Fvb_force[4] = {0.0, 0.0, 0.0, 0.0};
  const int wtag = p.wall ? p.wall[face] : 0;   // 0: none, +-(body+1): wall, sign = outward side
  if (wtag != 0 && p.J_seed != 0.0) {
    const T wsg = wtag > 0 ? 1.0 : -1.0;
    const T s = p.J_seed / (0.5 * C->mach * C->mach * (T)p.ns);
    const T eLx = -C->sina0, eLy = C->cosa0;
    const int ic = (wsg > 0) ? 1 : 2;            // interior cell of the wall face: L if high wall
    Wb[ic][3] += s * wsg * (sx * eLx + sy * eLy);
    Fvb_force[1] = -s * wsg * eLx;
    Fvb_force[2] = -s * wsg * eLy;
  }
  // ---- convective part: MUSCL on primitives + Roe
  {
    T WL[4], WR[4];
    T dL[4][2], dR[4][2];
    for (int q = 0; q < 4; ++q) {
      const T a = W[1][q] - W[0][q], bq = W[2][q] - W[1][q], cq = W[3][q] - W[2][q];
      WL[q] = W[1][q] + 0.5 * va_d(a, bq, C->eps, dL[q][0], dL[q][1]);
      WR[q] = W[2][q] - 0.5 * va_d(bq, cq, C->eps, dR[q][0], dR[q][1]);
    }
    T WLb[4] = {0, 0, 0, 0}, WRb[4] = {0, 0, 0, 0};
    roe2d_adj(WL, WR, sx, sy, vgn, gam, C->entropy_fix, C->ent_frac, Fb, WLb, WRb);
    for (int q = 0; q < 4; ++q) {
      // WL = W1 + va(W1 - W0, W2 - W1)/2
      Wb[1][q] += WLb[q];
      const T ab = 0.5 * WLb[q] * dL[q][0], bb = 0.5 * WLb[q] * dL[q][1];
      Wb[1][q] += ab - bb; Wb[0][q] -= ab; Wb[2][q] += bb;
      // WR = W2 - va(W2 - W1, W3 - W2)/2
      Wb[2][q] += WRb[q];
      const T ab2 = -0.5 * WRb[q] * dR[q][0], bb2 = -0.5 * WRb[q] * dR[q][1];
      Wb[2][q] += ab2 - bb2; Wb[1][q] -= ab2; Wb[3][q] += bb2;
    }
  }
  // ---- viscous part (F = Fc - Fv, so Fv receives -Fb)
  if (C->viscous) {
    // neighbours of L (order -i,+i,-j,+j) and R, as stencil slots
    int nbL[4], nbR[4];
    if (d == 0) { nbL[0] = 0; nbL[1] = 2; nbL[2] = 4; nbL[3] = 5; nbR[0] = 1; nbR[1] = 3; nbR[2] = 6; nbR[3] = 7; }
    else { nbL[0] = 4; nbL[1] = 5; nbL[2] = 0; nbL[3] = 2; nbR[0] = 6; nbR[1] = 7; nbR[2] = 1; nbR[3] = 3; }
    T phi[8][3];
    for (int k = 0; k < 8; ++k) { phi[k][0] = W[k][1]; phi[k][1] = W[k][2]; phi[k][2] = Tt[k]; }
    int64_t cnL[4], cnR[4];
    T pnL[4][3], pnR[4][3];
    for (int k = 0; k < 4; ++k) {
      cnL[k] = sc[nbL[k]]; cnR[k] = sc[nbR[k]];
      for (int q = 0; q < 3; ++q) { pnL[k][q] = phi[nbL[k]][q]; pnR[k][q] = phi[nbR[k]][q]; }
    }
    T gL[6], gR[6];
    gg_grad(B, p.g, f, sc[1], cnL, phi[1], pnL, gL);
    gg_grad(B, p.g, f, sc[2], cnR, phi[2], pnR, gR);
    T tx, ty;
    rotv(f, p.g.q[G_DC + 3 * d][B.goff + sc[2]], p.g.q[G_DC + 3 * d + 1][B.goff + sc[2]], tx, ty);
    T Fvb[4];
    for (int v = 0; v < 4; ++v) Fvb[v] = -Fb[v] + Fvb_force[v];
    T gLb[6] = {0, 0, 0, 0, 0, 0}, gRb[6] = {0, 0, 0, 0, 0, 0};
    T phLb[3] = {0, 0, 0}, phRb[3] = {0, 0, 0};
    visc2d_adj(gL, gR, phi[1][0], phi[1][1], phi[1][2], phi[2][0], phi[2][1], phi[2][2], tx, ty, sx, sy,
               C->mu, C->kappa, Fvb, gLb, gRb, phLb, phRb);
    T pcb[8][3];
    for (int k = 0; k < 8; ++k) for (int q = 0; q < 3; ++q) pcb[k][q] = 0.0;
    for (int q = 0; q < 3; ++q) { pcb[1][q] += phLb[q]; pcb[2][q] += phRb[q]; }
    T pnLb[4][3], pnRb[4][3];
    for (int k = 0; k < 4; ++k) for (int q = 0; q < 3; ++q) { pnLb[k][q] = 0.0; pnRb[k][q] = 0.0; }
    gg_grad_adj(B, p.g, f, sc[1], cnL, gLb, pcb[1], pnLb);
    gg_grad_adj(B, p.g, f, sc[2], cnR, gRb, pcb[2], pnRb);
    for (int k = 0; k < 4; ++k)
      for (int q = 0; q < 3; ++q) { pcb[nbL[k]][q] += pnLb[k][q]; pcb[nbR[k]][q] += pnRb[k][q]; }
    for (int k = 0; k < 8; ++k) { Wb[k][1] += pcb[k][0]; Wb[k][2] += pcb[k][1]; Tb[k] += pcb[k][2]; }
  }
  double* out = p.buf + (face * p.ns + n) * 32;
  for (int k = 0; k < 8; ++k) {
    T Ubk[4];
    prim4_adj(W[k], Tb[k], Wb[k], gm1, gam, Ubk);
    for (int v = 0; v < NV; ++v) out[k * 4 + v] = Ubk[v];
  }
}

// ---------------------------------------------------------------- phase B --
__global__ void adj_cells_kernel(AdjParams p) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= p.ncells_padded * (int64_t)p.ns) return;
  const int n = (int)(gid % p.ns);
  const int64_t cell = gid / p.ns;
  int b = 0;
  while (b + 1 < p.nblocks && p.coff[b + 1] <= cell) ++b;
  const BlockDev B = p.blocks[b];
  const CaseDev<T>* C = p.cases + B.cs;
  const int64_t lc = cell - p.coff[b];
  const int P0 = B.P[0], n0 = B.n[0], n1 = B.n[1];
  const int ci = (int)(lc % P0) - 2, cj = (int)(lc / P0) - 2;
  if (ci > n0 + 1 || cj > n1 + 1) return;   // row and plane padding
  const int64_t pcell = lc;
  T acc[4] = {0, 0, 0, 0};
  const int64_t nfi = (int64_t)(n0 + 1) * n1;
  // i-faces with this cell in slot k: face R position
  const int ifi[8] = {ci + 2, ci + 1, ci, ci - 1, ci + 1, ci + 1, ci, ci};
  const int ifj[8] = {cj, cj, cj, cj, cj + 1, cj - 1, cj + 1, cj - 1};
  for (int k = 0; k < 8; ++k) {
    const int fi = ifi[k], fj = ifj[k];
    if (fi < 0 || fi > n0 || fj < 0 || fj >= n1) continue;
    const int64_t face = p.foff[b] + (int64_t)fj * (n0 + 1) + fi;
    const double* src = p.buf + (face * p.ns + n) * 32 + k * 4;
    for (int v = 0; v < 4; ++v) acc[v] += src[v];
  }
  const int jfi[8] = {ci, ci, ci, ci, ci + 1, ci - 1, ci + 1, ci - 1};
  const int jfj[8] = {cj + 2, cj + 1, cj, cj - 1, cj + 1, cj + 1, cj, cj};
  for (int k = 0; k < 8; ++k) {
    const int fi = jfi[k], fj = jfj[k];
    if (fi < 0 || fi >= n0 || fj < 0 || fj > n1) continue;
    const int64_t face = p.foff[b] + nfi + (int64_t)fj * n0 + fi;
    const double* src = p.buf + (face * p.ns + n) * 32 + k * 4;
    for (int v = 0; v < 4; ++v) acc[v] += src[v];
  }
  // HB source transpose on interior cells: d/dU_m of sum_n psi_n V omega D[n][m] U_m
  if (ci >= 0 && ci < n0 && cj >= 0 && cj < n1) {
    const T vw = p.g.q[G_VOL][B.goff + pcell] * C->omega;
    for (int v = 0; v < 4; ++v) {
      T h = 0.0;
      for (int m = 0; m < p.ns; ++m)
        h += C->D[m * p.ns + n] * p.psi[B.off + ((int64_t)m * NV + v) * B.plane + pcell];
      acc[v] += vw * h;
    }
  }
  for (int v = 0; v < 4; ++v) p.out[B.off + ((int64_t)n * NV + v) * B.plane + pcell] = acc[v];
}

// ---------------------------------------------------------------- phase C --
// Jacobian-transpose of the ghost maps, gathered per source cell
__global__ void adj_ghost_kernel(AdjParams p, const GhostAdjRow* rows, int nrows,
                                 const GhostAdjEntry* ent, const CopyRec* copies, const BcRec* bcs) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)nrows * p.ns) return;
  const int n = (int)(gid / nrows), row = (int)(gid % nrows);
  const GhostAdjRow R = rows[row];
  const BlockDev SB = p.blocks[R.src_blk];
  const CaseDev<T>* C = p.cases + SB.cs;
  const T gam = C->gamma, gm1 = gam - 1.0, ig1 = 1.0 / gm1;
  T acc[4] = {0, 0, 0, 0};
  const T* Us = p.U + SB.off + (int64_t)n * NV * SB.plane;
  T* As = p.out + SB.off + (int64_t)n * NV * SB.plane;
  for (int e = R.begin; e < R.end; ++e) {
    const GhostAdjEntry E = ent[e];
    if (E.kind == 0) {   // copy
      const CopyRec cr = copies[E.rec];
      const BlockDev DB = p.blocks[cr.dst_blk];
      const T* Ad = p.out + DB.off + (int64_t)n * NV * DB.plane;
      for (int v = 0; v < 4; ++v) acc[v] += Ad[v * DB.plane + cr.dst_cell];
      continue;
    }
    const BcRec r = bcs[E.rec];
    const Fr<T> f = frame_at(C, n);
    const int64_t fc = SB.goff + r.fcell;
    T sx, sy, xf, yf;
    rotv(f, p.g.q[G_S + 3 * r.p][fc], p.g.q[G_S + 3 * r.p + 1][fc], sx, sy);
    rotp(f, p.g.q[G_XF + 3 * r.p][fc], p.g.q[G_XF + 3 * r.p + 1][fc], xf, yf);
    const T vgx = -f.thd * (yf - f.py), vgy = f.thd * (xf - f.px);
    const T A = sqrt(sx * sx + sy * sy);
    const T nx = r.sgn * sx / A, ny = r.sgn * sy / A;
    if (E.kind == 1) {   // farfield: both ghost layers from the first interior cell
      T u[4], Wi[4], Tt;
      for (int v = 0; v < 4; ++v) u[v] = Us[v * SB.plane + r.mcell[0]];
      prim4(u, gm1, gam, Wi, Tt);
      const T* Wf = C->winf[n];
      T wf2 = Wf[2];
      if (C->ubc == 2) wf2 += C->ubc_amp * C->mach * sin(C->tn[n] - C->omega * xf / C->mach);
      const T qi = (Wi[1] - vgx) * nx + (Wi[2] - vgy) * ny;
      const T qf = (Wf[1] - vgx) * nx + (wf2 - vgy) * ny;
      const T ci = sqrt(gam * Wi[3] / Wi[0]), cf = sqrt(gam * Wf[4] / Wf[0]);
      const T Rp = qi + 2.0 * ci / gm1, Rm = qf - 2.0 * cf / gm1;
      const T qb = 0.5 * (Rp + Rm), cb = 0.25 * gm1 * (Rp - Rm);
      const bool out = qb > 0.0;
      const T ent = out ? Wi[3] / pow(Wi[0], gam) : Wf[4] / pow(Wf[0], gam);
      const T utx = out ? (Wi[1] - vgx) - qi * nx : (Wf[1] - vgx) - qf * nx;
      const T uty = out ? (Wi[2] - vgy) - qi * ny : (wf2 - vgy) - qf * ny;
      const T X = cb * cb / (gam * ent);
      const T rb = pow(X, 1.0 / gm1);
      T Wg[4] = {rb, vgx + utx + qb * nx, vgy + uty + qb * ny, rb * cb * cb / gam};
      // ghost adjoints of both layers, through the conservative map
      const BlockDev& GB = SB;
      T Ugb[4];
      for (int v = 0; v < 4; ++v)
        Ugb[v] = As[v * GB.plane + r.gcell[0]] + As[v * GB.plane + r.gcell[1]];
      T Wgb[4];
      cons4_adj(Wg, Ugb, ig1, Wgb);
      // reverse of the characteristic construction
      T cbb = Wgb[3] * rb * 2.0 * cb / gam;
      T rbb = Wgb[0] + Wgb[3] * cb * cb / gam;
      const T utxb = Wgb[1], utyb = Wgb[2];
      T qbb = Wgb[1] * nx + Wgb[2] * ny;
      const T Xb = rbb * rb / (gm1 * X);
      cbb += Xb * 2.0 * cb / (gam * ent);
      const T entb = -Xb * X / ent;
      T Wib[4] = {0, 0, 0, 0};
      T qib = 0.0;
      if (out) {
        Wib[3] += entb / pow(Wi[0], gam);
        Wib[0] -= entb * gam * ent / Wi[0];
        Wib[1] += utxb; Wib[2] += utyb;
        qib -= utxb * nx + utyb * ny;
      }
      const T Rpb = 0.5 * qbb + 0.25 * gm1 * cbb;
      qib += Rpb;
      const T cib = 2.0 * Rpb / gm1;
      Wib[3] += cib * gam / (2.0 * ci * Wi[0]);
      Wib[0] -= cib * ci / (2.0 * Wi[0]);
      Wib[1] += qib * nx; Wib[2] += qib * ny;
      T Uib[4];
      prim4_adj(Wi, 0.0, Wib, gm1, gam, Uib);
      for (int v = 0; v < 4; ++v) acc[v] += Uib[v];
    } else {             // wall layer E.layer: ghost = reflection of the mirror cell
      const int l = E.layer;
      T u[4], Wm[4], Tt;
      for (int v = 0; v < 4; ++v) u[v] = Us[v * SB.plane + r.mcell[l]];
      prim4(u, gm1, gam, Wm, Tt);
      T Wg[4];
      Wg[0] = Wm[0];
      Wg[3] = Wm[3];
      T Wmb[4];
      T Ugb[4];
      for (int v = 0; v < 4; ++v) Ugb[v] = As[v * SB.plane + r.gcell[l]];
      if (r.type == 2) {
        const T qn = (Wm[1] - vgx) * nx + (Wm[2] - vgy) * ny;
        Wg[1] = Wm[1] - 2.0 * qn * nx;
        Wg[2] = Wm[2] - 2.0 * qn * ny;
        T Wgb[4];
        cons4_adj(Wg, Ugb, ig1, Wgb);
        const T dn = Wgb[1] * nx + Wgb[2] * ny;
        Wmb[0] = Wgb[0];
        Wmb[3] = Wgb[3];
        Wmb[1] = Wgb[1] - 2.0 * dn * nx;
        Wmb[2] = Wgb[2] - 2.0 * dn * ny;
      } else {
        Wg[1] = 2.0 * vgx - Wm[1];
        Wg[2] = 2.0 * vgy - Wm[2];
        T Wgb[4];
        cons4_adj(Wg, Ugb, ig1, Wgb);
        Wmb[0] = Wgb[0];
        Wmb[3] = Wgb[3];
        Wmb[1] = -Wgb[1];
        Wmb[2] = -Wgb[2];
      }
      T Umb[4];
      prim4_adj(Wm, 0.0, Wmb, gm1, gam, Umb);
      for (int v = 0; v < 4; ++v) acc[v] += Umb[v];
    }
  }
  for (int v = 0; v < 4; ++v) As[v * SB.plane + R.src_cell] += acc[v];
}

// ---------------------------------------------------------------- phase D --
__global__ void adj_final_kernel(AdjParams p, double* r_adj) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= p.ncells_padded * (int64_t)p.ns) return;
  const int n = (int)(gid % p.ns);
  const int64_t cell = gid / p.ns;
  int b = 0;
  while (b + 1 < p.nblocks && p.coff[b + 1] <= cell) ++b;
  const BlockDev B = p.blocks[b];
  const int64_t lc = cell - p.coff[b];
  const int ci = (int)(lc % B.P[0]) - 2, cj = (int)(lc / B.P[0]) - 2;
  if (ci > B.n[0] + 1 || cj > B.n[1] + 1) return;
  const bool in = ci >= 0 && ci < B.n[0] && cj >= 0 && cj < B.n[1];
  for (int v = 0; v < 4; ++v) {
    const int64_t a = B.off + ((int64_t)n * NV + v) * B.plane + lc;
    r_adj[a] = in ? p.out[a] : 0.0;
  }
}

cudaError_t launch_adjoint(const AdjParams& p, const AdjGhostPass* passes, int npass, double* r_adj,
                           cudaStream_t s) {
  const int bs = 128;
  int64_t tot = p.nfaces * (int64_t)p.ns;
  adj_faces_kernel<<<(unsigned)((tot + bs - 1) / bs), bs, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tot = p.ncells_padded * (int64_t)p.ns;
  adj_cells_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int q = npass - 1; q >= 0; --q) {
    const AdjGhostPass& gp = passes[q];
    if (gp.nrows == 0) continue;
    const int64_t t2 = (int64_t)gp.nrows * p.ns;
    adj_ghost_kernel<<<(unsigned)((t2 + 127) / 128), 128, 0, s>>>(p, gp.rows, gp.nrows, gp.ent, gp.copies,
                                                                 gp.bcs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  adj_final_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p, r_adj);
  return cudaGetLastError();
}

}  // namespace hbk
