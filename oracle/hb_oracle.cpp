// FP64 CPU oracle of the harmonic-balance (HB) residual path.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline of the benchmark may load this library; the product path never
// does.  It shares no code, header, table or helper with the CUDA library.
//
// It restates, step by step and in plain loops, what the HB Navier-Stokes
// method computes for every cell of a structured multi-block grid and every
// one of the 2*N_H+1 time snapshots (paper, Sec. 1: HB solver on structured
// multi-block grids; snapshot loop n = 0..2*nharms and state q2(i,j,ipde,n),
// Sec. 3.1 "MPI Optimisations"):
//   * cut exchange and physical boundary ghosts (Sec. 3.1, per RK step),
//   * MUSCL reconstruction of primitives with the van Albada limiter,
//   * Roe's approximate Riemann flux with a Harten fix on acoustic waves and
//     the grid-velocity (ALE) term of rigid pitching,
//   * central viscous fluxes from Green-Gauss cell gradients,
//   * the HB source V*omega*D*U with the closed-form spectral derivative D,
//   * local pseudo-time steps and the 4-stage Runge-Kutta smoother,
//   * FP64 residual norms and force coefficients cl, cd, cm per body and
//     snapshot (Sec. 3.1, the aggregated force reduction; cm when functag==3),
//   * Jacobian-transpose columns of the residual plus lift functional, by
//     forward-mode dual numbers (exact) or central finite differences.
// The residual of a cell sums the fluxes of its own faces; every face is
// recomputed from both sides, every gradient from scratch: slow and plain.
#include <algorithm>
#include <array>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------- duals --
struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double a) : v(a), d(0.0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual& operator/=(Dual& a, Dual b) { a = a / b; return a; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }
inline Dual pow(Dual a, double e) {
  double p = std::pow(a.v, e);
  return Dual(p, e * std::pow(a.v, e - 1.0) * a.d);
}
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::sqrt;
using std::fabs;
using std::pow;

// ---------------------------------------------------------------- case --
enum { BC_FARFIELD = 1, BC_SLIP = 2, BC_NOSLIP = 3 };
enum { UBC_NONE = 0, UBC_INLET_ANGLE = 1, UBC_GUST = 2 };

struct Block {
  int n[3], g[3], p[3];   // cells, ghost layers, padded extent per direction
  int q[3];               // node extent per direction
  int64_t ncell;
  int64_t stride[3];
  std::vector<double> X;  // nodes, 3 components each (z = 0 in 2D)
  std::vector<double> vol, xc;
  std::vector<double> S[3], xf[3];  // low face of each padded cell along d
  int64_t cell(int i, int j, int k) const {
    return ((int64_t)(k + g[2]) * p[1] + (j + g[1])) * p[0] + (i + g[0]);
  }
  const double* node(int a, int b, int c) const {
    return &X[3 * (((int64_t)(c + g[2]) * q[1] + (b + g[1])) * q[0] + (a + g[0]))];
  }
  bool interior(int i, int j, int k) const {
    return i >= 0 && i < n[0] && j >= 0 && j < n[1] && k >= 0 && k < n[2];
  }
};

struct Cut { int dst, src, lo[3], hi[3], off[3], perm[3], sign[3], pass; };
struct Bc { int blk, face, lo[3], hi[3], type, body; };

struct Case {
  int dim, nv, nh, ns;
  double gamma, prandtl, mach, reynolds, alpha0, omega, cfl, lim_eps, ent_frac;
  int viscous, entropy_fix, motion;
  double pitch_amp, pivot[2];
  int ubc;
  double ubc_amp;
  int n_bodies, functag;
  std::vector<Block> B;
  std::vector<Cut> cuts;
  std::vector<Bc> bcs;
  std::vector<int64_t> boff;
  int64_t total;
  std::vector<double> D;  // ns x ns
  double mu, kappa, pinf;
  // time-domain mode (one snapshot at physical time td_t): the frame, grid
  // velocity and unsteady inflow are those of td_t instead of t_0 = 0
  int td = 0;
  double td_t = 0.0;
  double td_lam = 0.0;    // a0 / dt: the physical-time term's share of the pseudo-time step
  int64_t at(int b, int n, int v, int64_t c) const {
    return boff[b] + ((int64_t)n * nv + v) * B[b].ncell + c;
  }
};

// spectral time-derivative matrix on ns = 2*nh+1 equispaced snapshots over one
// period 2*pi (trigonometric interpolation): D[n][m] = (-1)^(n-m) / (2 sin(pi (n-m)/ns))
void d_matrix(int ns, double* D) {
  for (int n = 0; n < ns; ++n)
    for (int m = 0; m < ns; ++m) {
      if (n == m) { D[n * ns + m] = 0.0; continue; }
      int k = n - m;
      double sgn = (((k % 2) + 2) % 2 == 0) ? 1.0 : -1.0;
      D[n * ns + m] = 0.5 * sgn / std::sin(M_PI * (double)k / (double)ns);
    }
}

void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// face vector (oriented towards +d) and centroid of the low face of cell (i,j,k)
void face_geom(const Case& C, const Block& B, int d, int i, int j, int k, double* S, double* xf) {
  if (C.dim == 2) {
    const double* a = B.node(i, j, 0);
    const double* b = (d == 0) ? B.node(i, j + 1, 0) : B.node(i + 1, j, 0);
    double e[2] = {b[0] - a[0], b[1] - a[1]};
    if (d == 0) { S[0] = e[1]; S[1] = -e[0]; } else { S[0] = -e[1]; S[1] = e[0]; }
    S[2] = 0.0;
    for (int c = 0; c < 3; ++c) xf[c] = 0.5 * (a[c] + b[c]);
    return;
  }
  const double *n00, *n11, *na, *nb;  // d1 = n11 - n00, d2 = na - nb
  const double *c1, *c2;
  if (d == 0) {
    n00 = B.node(i, j, k); n11 = B.node(i, j + 1, k + 1);
    na = B.node(i, j, k + 1); nb = B.node(i, j + 1, k);
  } else if (d == 1) {
    n00 = B.node(i, j, k); n11 = B.node(i + 1, j, k + 1);
    na = B.node(i + 1, j, k); nb = B.node(i, j, k + 1);
  } else {
    n00 = B.node(i, j, k); n11 = B.node(i + 1, j + 1, k);
    na = B.node(i, j + 1, k); nb = B.node(i + 1, j, k);
  }
  c1 = na; c2 = nb;
  double d1[3], d2[3], cr[3];
  for (int c = 0; c < 3; ++c) { d1[c] = n11[c] - n00[c]; d2[c] = c1[c] - c2[c]; }
  cross(d1, d2, cr);
  for (int c = 0; c < 3; ++c) {
    S[c] = 0.5 * cr[c];
    xf[c] = 0.25 * (n00[c] + n11[c] + c1[c] + c2[c]);
  }
}

void build_geometry(const Case& C, Block& B) {
  B.vol.assign(B.ncell, 0.0);
  B.xc.assign(3 * B.ncell, 0.0);
  for (int d = 0; d < 3; ++d) { B.S[d].assign(3 * B.ncell, 0.0); B.xf[d].assign(3 * B.ncell, 0.0); }
  int k0 = -B.g[2], k1 = B.n[2] + B.g[2];
  for (int k = k0; k < k1; ++k)
    for (int j = -B.g[1]; j < B.n[1] + B.g[1]; ++j)
      for (int i = -B.g[0]; i < B.n[0] + B.g[0]; ++i) {
        int64_t c = B.cell(i, j, k);
        for (int d = 0; d < C.dim; ++d) face_geom(C, B, d, i, j, k, &B.S[d][3 * c], &B.xf[d][3 * c]);
        if (C.dim == 2) {
          const double* x1 = B.node(i, j, 0);
          const double* x2 = B.node(i + 1, j, 0);
          const double* x3 = B.node(i + 1, j + 1, 0);
          const double* x4 = B.node(i, j + 1, 0);
          double a[2] = {x3[0] - x1[0], x3[1] - x1[1]}, b[2] = {x4[0] - x2[0], x4[1] - x2[1]};
          B.vol[c] = 0.5 * (a[0] * b[1] - a[1] * b[0]);
          for (int q = 0; q < 3; ++q) B.xc[3 * c + q] = 0.25 * (x1[q] + x2[q] + x3[q] + x4[q]);
        } else {
          double v = 0.0;
          for (int d = 0; d < 3; ++d) {
            double Sl[3], xl[3], Sh[3], xh[3];
            face_geom(C, B, d, i, j, k, Sl, xl);
            face_geom(C, B, d, i + (d == 0), j + (d == 1), k + (d == 2), Sh, xh);
            for (int q = 0; q < 3; ++q) v += xh[q] * Sh[q] - xl[q] * Sl[q];
          }
          B.vol[c] = v / 3.0;
          for (int q = 0; q < 3; ++q) {
            double s = 0.0;
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b)
                for (int cc = 0; cc < 2; ++cc) s += B.node(i + a, j + b, k + cc)[q];
            B.xc[3 * c + q] = s / 8.0;
          }
        }
      }
}

// ----------------------------------------------------- snapshot frame --
// rigid pitch theta(t) = A sin(omega t) about the pivot, t_n = 2 pi n/(ns omega)
struct Frame { double c, s, thdot, t, px, py; };

Frame frame(const Case& C, int n) {
  Frame f;
  f.t = (C.omega > 0.0) ? 2.0 * M_PI * n / (C.ns * C.omega) : 0.0;
  if (C.td) f.t = C.td_t;
  double th = 0.0, thd = 0.0;
  if (C.motion == 1) {
    th = C.pitch_amp * std::sin(C.omega * f.t);
    thd = C.pitch_amp * C.omega * std::cos(C.omega * f.t);
  }
  f.c = std::cos(th); f.s = std::sin(th); f.thdot = thd;
  f.px = C.pivot[0]; f.py = C.pivot[1];
  return f;
}
void rotv(const Frame& f, const double* a, double* b) {
  b[0] = f.c * a[0] - f.s * a[1];
  b[1] = f.s * a[0] + f.c * a[1];
  b[2] = a[2];
}
void rotp(const Frame& f, const double* a, double* b) {
  double r[3] = {a[0] - f.px, a[1] - f.py, a[2]}, o[3];
  rotv(f, r, o);
  b[0] = o[0] + f.px; b[1] = o[1] + f.py; b[2] = o[2];
}
// grid velocity of a (rotated) point: thdot * z x (x - pivot)
void gridvel(const Frame& f, const double* x, double* vg) {
  vg[0] = -f.thdot * (x[1] - f.py);
  vg[1] = f.thdot * (x[0] - f.px);
  vg[2] = 0.0;
}

// freestream primitives (rho, u, v, w, p) at snapshot n and point x:
// rho = 1, c = 1, p = 1/gamma, |u| = M
void freestream(const Case& C, const Frame& f, const double* x, double* W) {
  double alpha = C.alpha0;
  if (C.ubc == UBC_INLET_ANGLE) alpha += C.ubc_amp * M_PI / 180.0 * std::sin(C.omega * f.t);
  W[0] = 1.0;
  W[1] = C.mach * std::cos(alpha);
  W[2] = C.mach * std::sin(alpha);
  W[3] = 0.0;
  W[4] = 1.0 / C.gamma;
  if (C.ubc == UBC_GUST)
    W[2] += C.ubc_amp * C.mach * std::sin(C.omega * f.t - C.omega * x[0] / C.mach);
}

// ------------------------------------------------ state conversions --
template <class S>
void prim(const Case& C, const S* U, S* W) {  // U has nv comps
  S rho = U[0];
  S u = U[1] / rho, v = U[2] / rho, w = (C.dim == 3) ? U[3] / rho : S(0.0);
  S E = U[C.nv - 1];
  W[0] = rho; W[1] = u; W[2] = v; W[3] = w;
  W[4] = (C.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w));
}
template <class S>
void cons(const Case& C, const S* W, S* U) {
  U[0] = W[0];
  U[1] = W[0] * W[1];
  U[2] = W[0] * W[2];
  if (C.dim == 3) U[3] = W[0] * W[3];
  U[C.nv - 1] = W[4] / (C.gamma - 1.0) + 0.5 * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}
template <class S>
void load_prim(const Case& C, const S* U, int b, int n, int64_t c, S* W) {
  S u[5];
  for (int v = 0; v < C.nv; ++v) u[v] = U[C.at(b, n, v, c)];
  prim(C, u, W);
}
// index of the 5-component flux (mass, mx, my, mz, energy) for variable v
inline int comp5(const Case& C, int v) { return (C.dim == 3 || v < 3) ? v : 4; }

// --------------------------------------------------- van Albada limiter --
template <class S>
S van_albada(S a, S b, double eps) {
  return ((b * b + eps) * a + (a * a + eps) * b) / (a * a + b * b + 2.0 * eps);
}

// ------------------------------------------------------------ Roe flux --
// mode 0: flux; mode 1: sum_k lambda_k alpha_k r_k (signed, no fix);
// mode 2: sum_k alpha_k r_k.  W = (rho,u,v,w,p); Svec area vector; vg grid velocity.
template <class S>
void roe(const Case& C, const S* WL, const S* WR, const double* Svec, const double* vg, int mode,
         S* F) {
  const double g = C.gamma;
  double A = std::sqrt(Svec[0] * Svec[0] + Svec[1] * Svec[1] + Svec[2] * Svec[2]);
  double nx[3] = {Svec[0] / A, Svec[1] / A, Svec[2] / A};
  double vgn = vg[0] * nx[0] + vg[1] * nx[1] + vg[2] * nx[2];
  S qL = WL[1] * nx[0] + WL[2] * nx[1] + WL[3] * nx[2];
  S qR = WR[1] * nx[0] + WR[2] * nx[1] + WR[3] * nx[2];
  S kL = 0.5 * (WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3]);
  S kR = 0.5 * (WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3]);
  S HL = g / (g - 1.0) * WL[4] / WL[0] + kL;
  S HR = g / (g - 1.0) * WR[4] / WR[0] + kR;
  // Roe averages
  S r = sqrt(WR[0] / WL[0]);
  S rt = r * WL[0];
  S ut[3];
  for (int a = 0; a < 3; ++a) ut[a] = (WL[1 + a] + r * WR[1 + a]) / (1.0 + r);
  S Ht = (HL + r * HR) / (1.0 + r);
  S kt = 0.5 * (ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
  S ct2 = (g - 1.0) * (Ht - kt);
  S ct = sqrt(ct2);
  S qt = ut[0] * nx[0] + ut[1] * nx[1] + ut[2] * nx[2];
  S qtr = qt - vgn;
  // wave speeds
  S l1 = qtr - ct, l2 = qtr, l3 = qtr + ct;
  if (mode == 0) {
    l1 = fabs(l1); l2 = fabs(l2); l3 = fabs(l3);
    if (C.entropy_fix) {
      S delta = C.ent_frac * ct;
      if (l1 < delta) l1 = (l1 * l1 + delta * delta) / (2.0 * delta);
      if (l3 < delta) l3 = (l3 * l3 + delta * delta) / (2.0 * delta);
    }
  } else if (mode == 2) {
    l1 = S(1.0); l2 = S(1.0); l3 = S(1.0);
  }
  // wave strengths
  S dp = WR[4] - WL[4], drho = WR[0] - WL[0], dq = qR - qL;
  S a1 = (dp - rt * ct * dq) / (2.0 * ct2);
  S a3 = (dp + rt * ct * dq) / (2.0 * ct2);
  S a2 = drho - dp / ct2;
  S dut[3];
  for (int a = 0; a < 3; ++a) dut[a] = (WR[1 + a] - WL[1 + a]) - dq * nx[a];
  S udut = ut[0] * dut[0] + ut[1] * dut[1] + ut[2] * dut[2];
  S Dm[5];
  Dm[0] = l1 * a1 + l2 * a2 + l3 * a3;
  for (int a = 0; a < 3; ++a)
    Dm[1 + a] = l1 * a1 * (ut[a] - ct * nx[a]) + l2 * (a2 * ut[a] + rt * dut[a]) +
                l3 * a3 * (ut[a] + ct * nx[a]);
  Dm[4] = l1 * a1 * (Ht - ct * qt) + l2 * (a2 * kt + rt * udut) + l3 * a3 * (Ht + ct * qt);
  if (mode != 0) {
    for (int v = 0; v < 5; ++v) F[v] = Dm[v];
    return;
  }
  // physical fluxes relative to the moving face
  S FL[5], FR[5];
  S qLr = qL - vgn, qRr = qR - vgn;
  S EL = WL[4] / (g - 1.0) + WL[0] * kL, ER = WR[4] / (g - 1.0) + WR[0] * kR;  // rho*E
  FL[0] = WL[0] * qLr; FR[0] = WR[0] * qRr;
  for (int a = 0; a < 3; ++a) {
    FL[1 + a] = WL[0] * WL[1 + a] * qLr + WL[4] * nx[a];
    FR[1 + a] = WR[0] * WR[1 + a] * qRr + WR[4] * nx[a];
  }
  FL[4] = EL * qLr + WL[4] * qL;
  FR[4] = ER * qRr + WR[4] * qR;
  for (int v = 0; v < 5; ++v) F[v] = (0.5 * (FL[v] + FR[v]) - 0.5 * Dm[v]) * A;
}

// ---------------------------------------------------------- gradients --
// Green-Gauss gradient of (u, v, w, T) at padded cell c, snapshot n, T = gamma p/rho
template <class S>
void gradient(const Case& C, const S* U, int b, int n, const Frame& f, int i, int j, int k,
              S G[4][3]) {
  const Block& B = C.B[b];
  auto phi = [&](int ii, int jj, int kk, S* out) {
    S W[5];
    load_prim(C, U, b, n, B.cell(ii, jj, kk), W);
    out[0] = W[1]; out[1] = W[2]; out[2] = W[3]; out[3] = C.gamma * W[4] / W[0];
  };
  S pc[4];
  phi(i, j, k, pc);
  for (int q = 0; q < 4; ++q) for (int a = 0; a < 3; ++a) G[q][a] = S(0.0);
  for (int d = 0; d < C.dim; ++d) {
    int e[3] = {d == 0, d == 1, d == 2};
    for (int side = 0; side < 2; ++side) {
      int ii = i + (side ? e[0] : -e[0]), jj = j + (side ? e[1] : -e[1]), kk = k + (side ? e[2] : -e[2]);
      int64_t fc = side ? B.cell(ii, jj, kk) : B.cell(i, j, k);   // owner of the low face
      double Sr[3];
      rotv(f, &B.S[d][3 * fc], Sr);
      double sg = side ? 1.0 : -1.0;
      S pn[4];
      phi(ii, jj, kk, pn);
      for (int q = 0; q < 4; ++q)
        for (int a = 0; a < 3; ++a) G[q][a] += 0.5 * (pc[q] + pn[q]) * (sg * Sr[a]);
    }
  }
  double V = B.vol[B.cell(i, j, k)];
  for (int q = 0; q < 4; ++q) for (int a = 0; a < 3; ++a) G[q][a] /= V;
}

// viscous flux through the face between cells L and R (S points L -> R)
template <class S>
void viscous_flux(const Case& C, const S* U, int b, int n, const Frame& f, const int* cL,
                  const int* cR, const double* Svec, S* Fv, S tau_out[3][3]) {
  const Block& B = C.B[b];
  S GL[4][3], GR[4][3];
  gradient(C, U, b, n, f, cL[0], cL[1], cL[2], GL);
  gradient(C, U, b, n, f, cR[0], cR[1], cR[2], GR);
  S WL[5], WR[5];
  load_prim(C, U, b, n, B.cell(cL[0], cL[1], cL[2]), WL);
  load_prim(C, U, b, n, B.cell(cR[0], cR[1], cR[2]), WR);
  S pL[4] = {WL[1], WL[2], WL[3], C.gamma * WL[4] / WL[0]};
  S pR[4] = {WR[1], WR[2], WR[3], C.gamma * WR[4] / WR[0]};
  // the rigid rotation is linear, so the rotated L->R centre difference is
  // the rotation of the static difference (no cancellation of |x| >> |t|)
  const double* xL = &B.xc[3 * B.cell(cL[0], cL[1], cL[2])];
  const double* xR = &B.xc[3 * B.cell(cR[0], cR[1], cR[2])];
  double d0[3] = {xR[0] - xL[0], xR[1] - xL[1], xR[2] - xL[2]}, t[3];
  rotv(f, d0, t);
  double len = std::sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  double th[3] = {t[0] / len, t[1] / len, t[2] / len};
  S Gf[4][3];
  for (int q = 0; q < 4; ++q) {
    S gb[3], proj = S(0.0);
    for (int a = 0; a < 3; ++a) { gb[a] = 0.5 * (GL[q][a] + GR[q][a]); proj += gb[a] * th[a]; }
    S corr = (pR[q] - pL[q]) / len - proj;
    for (int a = 0; a < 3; ++a) Gf[q][a] = gb[a] + corr * th[a];
  }
  // Stokes stress with constant mu; Fourier heat flux kappa grad T
  S div = Gf[0][0] + Gf[1][1] + Gf[2][2];
  S tau[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c)
      tau[a][c] = C.mu * (Gf[a][c] + Gf[c][a]) - (a == c ? (2.0 / 3.0) * C.mu * div : S(0.0));
  S uf[3];
  for (int a = 0; a < 3; ++a) uf[a] = 0.5 * (pL[a] + pR[a]);
  Fv[0] = S(0.0);
  S work = S(0.0);
  for (int a = 0; a < 3; ++a) {
    S ts = S(0.0);
    for (int c = 0; c < 3; ++c) ts += tau[a][c] * Svec[c];
    Fv[1 + a] = ts;
    work += uf[a] * ts;
  }
  S heat = S(0.0);
  for (int c = 0; c < 3; ++c) heat += Gf[3][c] * Svec[c];
  Fv[4] = work + C.kappa * heat;
  if (tau_out)
    for (int a = 0; a < 3; ++a) for (int c = 0; c < 3; ++c) tau_out[a][c] = tau[a][c];
}

// total flux (convective minus viscous) through the low face of cell cR along d
template <class S>
void face_flux(const Case& C, const S* U, int b, int n, const Frame& f, int d, const int* cR,
               S* F) {
  const Block& B = C.B[b];
  int e[3] = {d == 0, d == 1, d == 2};
  int cL[3] = {cR[0] - e[0], cR[1] - e[1], cR[2] - e[2]};
  int cLL[3] = {cL[0] - e[0], cL[1] - e[1], cL[2] - e[2]};
  int cRR[3] = {cR[0] + e[0], cR[1] + e[1], cR[2] + e[2]};
  S W0[5], W1[5], W2[5], W3[5];
  load_prim(C, U, b, n, B.cell(cLL[0], cLL[1], cLL[2]), W0);
  load_prim(C, U, b, n, B.cell(cL[0], cL[1], cL[2]), W1);
  load_prim(C, U, b, n, B.cell(cR[0], cR[1], cR[2]), W2);
  load_prim(C, U, b, n, B.cell(cRR[0], cRR[1], cRR[2]), W3);
  // MUSCL on primitives: W_L = W_{L} + s_L/2, W_R = W_{R} - s_R/2, s = va(backward, forward)
  S WL[5], WR[5];
  for (int q = 0; q < 5; ++q) {
    S sL = van_albada(W1[q] - W0[q], W2[q] - W1[q], C.lim_eps);
    S sR = van_albada(W2[q] - W1[q], W3[q] - W2[q], C.lim_eps);
    WL[q] = W1[q] + 0.5 * sL;
    WR[q] = W2[q] - 0.5 * sR;
  }
  int64_t fc = B.cell(cR[0], cR[1], cR[2]);
  double Sr[3], xf[3], vg[3];
  rotv(f, &B.S[d][3 * fc], Sr);
  rotp(f, &B.xf[d][3 * fc], xf);
  gridvel(f, xf, vg);
  roe(C, WL, WR, Sr, vg, 0, F);
  if (C.viscous) {
    S Fv[5];
    viscous_flux(C, U, b, n, f, cL, cR, Sr, Fv, (S(*)[3]) nullptr);
    for (int q = 0; q < 5; ++q) F[q] -= Fv[q];
  }
}

// HB residual of one interior cell at all snapshots: R[n][v]; optional scale[n][v]
// = sum of |face flux| + |HB source| (the magnitude the residual cancels)
// residual of cell (b, i, j, k) at snapshot n: R[v], scale[v] for v < nv
template <class S>
void snapshot_residual(const Case& C, const S* U, int b, int i, int j, int k, int n, S* R, double* scale) {
  const Block& B = C.B[b];
  int64_t c = B.cell(i, j, k);
  {
    Frame f = frame(C, n);
    S acc[5];
    for (int q = 0; q < 5; ++q) acc[q] = S(0.0);
    double sc[5] = {0, 0, 0, 0, 0};
    for (int d = 0; d < C.dim; ++d) {
      int lo[3] = {i, j, k};
      int hi[3] = {i + (d == 0), j + (d == 1), k + (d == 2)};
      S Fl[5], Fh[5];
      face_flux(C, U, b, n, f, d, lo, Fl);
      face_flux(C, U, b, n, f, d, hi, Fh);
      for (int q = 0; q < 5; ++q) {
        acc[q] += Fh[q] - Fl[q];
        sc[q] += std::fabs(val(Fh[q])) + std::fabs(val(Fl[q]));
      }
    }
    for (int v = 0; v < C.nv; ++v) {
      S hb = S(0.0);
      for (int m = 0; m < C.ns; ++m) hb += C.D[n * C.ns + m] * U[C.at(b, m, v, c)];
      hb = B.vol[c] * C.omega * hb;
      R[v] = acc[comp5(C, v)] + hb;
      if (scale) scale[v] = sc[comp5(C, v)] + std::fabs(val(hb));
    }
  }
}

// residual of cell (b, i, j, k) at every snapshot: R[n * nv + v]
template <class S>
void cell_residual(const Case& C, const S* U, int b, int i, int j, int k, S* R, double* scale) {
  for (int n = 0; n < C.ns; ++n)
    snapshot_residual(C, U, b, i, j, k, n, R + n * C.nv, scale ? scale + n * C.nv : nullptr);
}

// ------------------------------------------------------- ghost filling --
// boundary face of a BC at tangential cell t: the low face of cell (0 or n) along p
struct BFace { int64_t fc; double sgn; };
BFace bface(const Block& B, int p, int side, const int* t) {
  int c[3] = {t[0], t[1], t[2]};
  c[p] = side ? B.n[p] : 0;
  return {B.cell(c[0], c[1], c[2]), side ? 1.0 : -1.0};
}

template <class S>
void fill_pass(const Case& C, S* U, int pass);

template <class S>
void fill_ghosts(const Case& C, S* U) {
  for (int pass = 0; pass < C.dim; ++pass) fill_pass(C, U, pass);
}

// the cut copies, then the boundary ghosts, of one pass; a cut whose source
// block is -1 lies in another process's share of a block decomposition and
// is left for the exchange to fill
template <class S>
void fill_pass(const Case& C, S* U, int pass) {
  {
    for (const Cut& ct : C.cuts) {
      if (ct.pass != pass || ct.src < 0) continue;
      const Block& D = C.B[ct.dst];
      const Block& Sb = C.B[ct.src];
      for (int k = ct.lo[2]; k < ct.hi[2]; ++k)
        for (int j = ct.lo[1]; j < ct.hi[1]; ++j)
          for (int i = ct.lo[0]; i < ct.hi[0]; ++i) {
            int dd[3] = {i, j, k}, s[3];
            for (int a = 0; a < 3; ++a) s[a] = ct.off[a] + ct.sign[a] * dd[ct.perm[a]];
            int64_t cd = D.cell(i, j, k), cs = Sb.cell(s[0], s[1], s[2]);
            for (int n = 0; n < C.ns; ++n)
              for (int v = 0; v < C.nv; ++v) U[C.at(ct.dst, n, v, cd)] = U[C.at(ct.src, n, v, cs)];
          }
    }
    for (const Bc& bc : C.bcs) {
      int p = bc.face / 2, side = bc.face % 2;
      if (p != pass) continue;
      const Block& B = C.B[bc.blk];
      int lo[3] = {bc.lo[0], bc.lo[1], bc.lo[2]}, hi[3] = {bc.hi[0], bc.hi[1], bc.hi[2]};
      lo[p] = 0; hi[p] = 1;
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            int t[3] = {i, j, k};
            BFace bf = bface(B, p, side, t);
            for (int n = 0; n < C.ns; ++n) {
              Frame f = frame(C, n);
              double Sr[3], xf[3], vg[3], nrm[3];
              rotv(f, &B.S[p][3 * bf.fc], Sr);
              rotp(f, &B.xf[p][3 * bf.fc], xf);
              gridvel(f, xf, vg);
              double A = std::sqrt(Sr[0] * Sr[0] + Sr[1] * Sr[1] + Sr[2] * Sr[2]);
              for (int a = 0; a < 3; ++a) nrm[a] = bf.sgn * Sr[a] / A;   // outward
              for (int layer = 0; layer < 2; ++layer) {
                int gc[3] = {i, j, k}, mc[3] = {i, j, k};
                gc[p] = side ? B.n[p] + layer : -1 - layer;
                mc[p] = side ? B.n[p] - 1 - layer : layer;
                S Wm[5], Wg[5];
                if (bc.type == BC_FARFIELD) {
                  int ic[3] = {i, j, k};
                  ic[p] = side ? B.n[p] - 1 : 0;
                  S Wi[5];
                  load_prim(C, U, bc.blk, n, B.cell(ic[0], ic[1], ic[2]), Wi);
                  double Winf[5];
                  freestream(C, f, xf, Winf);
                  const double g = C.gamma;
                  S qi = (Wi[1] - vg[0]) * nrm[0] + (Wi[2] - vg[1]) * nrm[1] + (Wi[3] - vg[2]) * nrm[2];
                  double qinf = (Winf[1] - vg[0]) * nrm[0] + (Winf[2] - vg[1]) * nrm[1] +
                                (Winf[3] - vg[2]) * nrm[2];
                  S ci = sqrt(g * Wi[4] / Wi[0]);
                  double cinf = std::sqrt(g * Winf[4] / Winf[0]);
                  S Rp = qi + 2.0 * ci / (g - 1.0);
                  S Rm = S(qinf - 2.0 * cinf / (g - 1.0));
                  S qb = 0.5 * (Rp + Rm);
                  S cb = 0.25 * (g - 1.0) * (Rp - Rm);
                  S ent, ut[3];
                  if (val(qb) > 0.0) {   // outflow: entropy and tangential velocity from inside
                    ent = Wi[4] / pow(Wi[0], g);
                    for (int a = 0; a < 3; ++a) ut[a] = (Wi[1 + a] - vg[a]) - qi * nrm[a];
                  } else {               // inflow: from the freestream
                    ent = S(Winf[4] / std::pow(Winf[0], g));
                    for (int a = 0; a < 3; ++a) ut[a] = S((Winf[1 + a] - vg[a]) - qinf * nrm[a]);
                  }
                  S rb = pow(cb * cb / (g * ent), 1.0 / (g - 1.0));
                  Wg[0] = rb;
                  for (int a = 0; a < 3; ++a) Wg[1 + a] = vg[a] + ut[a] + qb * nrm[a];
                  Wg[4] = rb * cb * cb / g;
                } else {
                  load_prim(C, U, bc.blk, n, B.cell(mc[0], mc[1], mc[2]), Wm);
                  Wg[0] = Wm[0];
                  Wg[4] = Wm[4];
                  if (bc.type == BC_SLIP) {     // reflect the relative normal velocity
                    S qn = (Wm[1] - vg[0]) * nrm[0] + (Wm[2] - vg[1]) * nrm[1] + (Wm[3] - vg[2]) * nrm[2];
                    for (int a = 0; a < 3; ++a) Wg[1 + a] = Wm[1 + a] - 2.0 * qn * nrm[a];
                  } else {                      // no-slip adiabatic: u_g = 2 v_wall - u
                    for (int a = 0; a < 3; ++a) Wg[1 + a] = 2.0 * vg[a] - Wm[1 + a];
                  }
                }
                if (C.dim == 2) Wg[3] = S(0.0);
                S Ug[5];
                cons(C, Wg, Ug);
                int64_t cg = B.cell(gc[0], gc[1], gc[2]);
                for (int v = 0; v < C.nv; ++v) U[C.at(bc.blk, n, v, cg)] = Ug[v];
              }
            }
          }
    }
  }
}

// ------------------------------------------------------------- forces --
// cl, cd, cm per snapshot and body; pressure relative to p_inf plus viscous
// traction on wall faces, normalised by q_inf * c with c = 1.
template <class S>
void forces(const Case& C, const S* U, S* coef /*[ns][nb][3]*/, S* J) {
  for (int q = 0; q < C.ns * C.n_bodies * 3; ++q) coef[q] = S(0.0);
  double qinf = 0.5 * C.mach * C.mach;
  double eD[2] = {std::cos(C.alpha0), std::sin(C.alpha0)};
  double eL[2] = {-std::sin(C.alpha0), std::cos(C.alpha0)};
  for (const Bc& bc : C.bcs) {
    if (bc.type != BC_SLIP && bc.type != BC_NOSLIP) continue;
    if (bc.body < 0 || bc.body >= C.n_bodies) continue;
    int p = bc.face / 2, side = bc.face % 2;
    const Block& B = C.B[bc.blk];
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = std::max(bc.lo[a], 0); hi[a] = std::min(bc.hi[a], B.n[a]); }
    lo[p] = 0; hi[p] = 1;
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int t[3] = {i, j, k};
          BFace bf = bface(B, p, side, t);
          int ic[3] = {i, j, k}, gc[3] = {i, j, k};
          ic[p] = side ? B.n[p] - 1 : 0;
          gc[p] = side ? B.n[p] : -1;
          for (int n = 0; n < C.ns; ++n) {
            Frame f = frame(C, n);
            double Sr[3], xf[3], Sb[3];
            rotv(f, &B.S[p][3 * bf.fc], Sr);
            rotp(f, &B.xf[p][3 * bf.fc], xf);
            for (int a = 0; a < 3; ++a) Sb[a] = bf.sgn * Sr[a];   // into the body
            S W[5];
            load_prim(C, U, bc.blk, n, B.cell(ic[0], ic[1], ic[2]), W);
            S Fo[3];
            for (int a = 0; a < 3; ++a) Fo[a] = (W[4] - C.pinf) * Sb[a];
            if (C.viscous) {
              S Fv[5], tau[3][3];
              const int* cl = side ? ic : gc;
              const int* cr = side ? gc : ic;
              viscous_flux(C, U, bc.blk, n, f, cl, cr, Sr, Fv, tau);
              for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) Fo[a] -= tau[a][c] * Sb[c];
            }
            S* o = &coef[(n * C.n_bodies + bc.body) * 3];
            o[0] += (Fo[0] * eL[0] + Fo[1] * eL[1]) / qinf;
            o[1] += (Fo[0] * eD[0] + Fo[1] * eD[1]) / qinf;
            if (C.functag == 3)
              o[2] += ((xf[0] - C.pivot[0]) * Fo[1] - (xf[1] - C.pivot[1]) * Fo[0]) / qinf;
          }
        }
  }
  S j = S(0.0);
  for (int n = 0; n < C.ns; ++n)
    for (int bd = 0; bd < C.n_bodies; ++bd) j += coef[(n * C.n_bodies + bd) * 3];
  *J = j / (double)C.ns;
}

// ------------------------------------------------- local time step --
double local_dt(const Case& C, const double* U0, int b, int i, int j, int k, int n) {
  const Block& B = C.B[b];
  int64_t c = B.cell(i, j, k);
  Frame f = frame(C, n);
  double W[5];
  load_prim(C, U0, b, n, c, W);
  double cs = std::sqrt(C.gamma * W[4] / W[0]);
  double x[3], vg[3];
  rotp(f, &B.xc[3 * c], x);
  gridvel(f, x, vg);
  double ur[3] = {W[1] - vg[0], W[2] - vg[1], W[3] - vg[2]};
  double lam = 0.0, s2 = 0.0;
  for (int d = 0; d < C.dim; ++d) {
    int64_t ch = B.cell(i + (d == 0), j + (d == 1), k + (d == 2));
    double Sl[3], Sh[3], Sm[3];
    rotv(f, &B.S[d][3 * c], Sl);
    rotv(f, &B.S[d][3 * ch], Sh);
    for (int a = 0; a < 3; ++a) Sm[a] = 0.5 * (Sl[a] + Sh[a]);
    double mag2 = Sm[0] * Sm[0] + Sm[1] * Sm[1] + Sm[2] * Sm[2];
    lam += std::fabs(ur[0] * Sm[0] + ur[1] * Sm[1] + ur[2] * Sm[2]) + cs * std::sqrt(mag2);
    s2 += mag2;
  }
  double V = B.vol[c];
  if (C.viscous) lam += 4.0 * std::max(4.0 / 3.0, C.gamma / C.prandtl) * (C.mu / W[0]) * s2 / V;
  lam += C.omega * C.nh * V;
  lam += C.td_lam * V;
  return C.cfl * V / lam;
}

template <class F>
void for_interior(const Case& C, F fn) {
  for (int b = 0; b < (int)C.B.size(); ++b) {
    const Block& B = C.B[b];
    for (int k = 0; k < B.n[2]; ++k)
      for (int j = 0; j < B.n[1]; ++j)
        for (int i = 0; i < B.n[0]; ++i) fn(b, i, j, k);
  }
}

}  // namespace

// =================================================================== C API
extern "C" {

void orc_d_matrix(int ns, double* D) { d_matrix(ns, D); }

double orc_van_albada(double a, double b, double eps) { return van_albada(a, b, eps); }

// prm: gamma, entropy_fix, entropy_frac (the rest of the case is irrelevant here)
void orc_roe_flux(int dim, const double* prm, const double* WL, const double* WR,
                  const double* Svec, const double* vg, int mode, double* F) {
  Case C;
  C.dim = dim; C.nv = dim + 2;
  C.gamma = prm[0]; C.entropy_fix = (int)prm[1]; C.ent_frac = prm[2];
  roe(C, WL, WR, Svec, vg, mode, F);
}

// params (double[20]): gamma, prandtl, mach, reynolds, alpha0_deg, omega, cfl,
// lim_eps, entropy_frac, viscous, entropy_fix, motion, pitch_amp_deg, pivot_x,
// pivot_y, ubc, ubc_amp, n_bodies, functag, unused
void* orc_create(int dim, int n_harm, const double* prm, int n_blocks, const int* bdims,
                 const double* nodes, int n_cuts, const int* cuts, int n_bcs, const int* bcs) {
  Case* C = new Case();
  C->dim = dim; C->nv = dim + 2; C->nh = n_harm; C->ns = 2 * n_harm + 1;
  C->gamma = prm[0]; C->prandtl = prm[1]; C->mach = prm[2]; C->reynolds = prm[3];
  C->alpha0 = prm[4] * M_PI / 180.0; C->omega = prm[5]; C->cfl = prm[6]; C->lim_eps = prm[7];
  C->ent_frac = prm[8]; C->viscous = (int)prm[9]; C->entropy_fix = (int)prm[10];
  C->motion = (int)prm[11]; C->pitch_amp = prm[12] * M_PI / 180.0;
  C->pivot[0] = prm[13]; C->pivot[1] = prm[14]; C->ubc = (int)prm[15]; C->ubc_amp = prm[16];
  C->n_bodies = (int)prm[17]; C->functag = (int)prm[18];
  C->mu = C->mach / C->reynolds;
  C->kappa = C->mu / ((C->gamma - 1.0) * C->prandtl);
  C->pinf = 1.0 / C->gamma;
  C->D.assign(C->ns * C->ns, 0.0);
  d_matrix(C->ns, C->D.data());
  const double* np_ = nodes;
  int64_t off = 0;
  for (int b = 0; b < n_blocks; ++b) {
    Block B;
    for (int a = 0; a < 3; ++a) B.n[a] = bdims[3 * b + a];
    B.g[0] = 2; B.g[1] = 2; B.g[2] = (dim == 3) ? 2 : 0;
    if (dim == 2) B.n[2] = 1;
    for (int a = 0; a < 3; ++a) B.p[a] = B.n[a] + 2 * B.g[a];
    B.q[0] = B.p[0] + 1; B.q[1] = B.p[1] + 1; B.q[2] = (dim == 3) ? B.p[2] + 1 : 1;
    B.ncell = (int64_t)B.p[0] * B.p[1] * B.p[2];
    B.stride[0] = 1; B.stride[1] = B.p[0]; B.stride[2] = (int64_t)B.p[0] * B.p[1];
    int64_t nn = (int64_t)B.q[0] * B.q[1] * B.q[2];
    B.X.assign(3 * nn, 0.0);
    for (int64_t m = 0; m < nn; ++m)
      for (int a = 0; a < dim; ++a) B.X[3 * m + a] = np_[dim * m + a];
    np_ += dim * nn;
    C->B.push_back(B);
    C->boff.push_back(off);
    off += (int64_t)C->ns * C->nv * B.ncell;
  }
  C->total = off;
  for (auto& B : C->B) build_geometry(*C, B);
  for (int c = 0; c < n_cuts; ++c) {
    const int* r = cuts + 17 * c;
    Cut ct;
    ct.dst = r[0]; ct.src = r[1];
    for (int a = 0; a < 3; ++a) {
      ct.lo[a] = r[2 + a]; ct.hi[a] = r[5 + a]; ct.off[a] = r[8 + a];
      ct.perm[a] = r[11 + a]; ct.sign[a] = r[14 + a];
    }
    const Block& D = C->B[ct.dst];
    // the pass is the highest direction along which the box leaves the
    // interior; lower directions are only the corner extension
    ct.pass = -1;
    for (int a = 0; a < dim; ++a)
      if (ct.lo[a] < 0 || ct.hi[a] > D.n[a]) ct.pass = a;
    C->cuts.push_back(ct);
  }
  for (int c = 0; c < n_bcs; ++c) {
    const int* r = bcs + 10 * c;
    Bc bc;
    bc.blk = r[0]; bc.face = r[1];
    for (int a = 0; a < 3; ++a) { bc.lo[a] = r[2 + a]; bc.hi[a] = r[5 + a]; }
    bc.type = r[8]; bc.body = r[9];
    C->bcs.push_back(bc);
  }
  return C;
}

void orc_destroy(void* h) { delete (Case*)h; }

int64_t orc_state_size(void* h) { return ((Case*)h)->total; }

// offset of block b in the state, padded extents p[3], ghost layers g[3]
void orc_block_info(void* h, int b, int64_t* offset, int* p, int* g) {
  Case* C = (Case*)h;
  *offset = C->boff[b];
  for (int a = 0; a < 3; ++a) { p[a] = C->B[b].p[a]; g[a] = C->B[b].g[a]; }
}

// static geometry of block b over padded cells: vol[ncell], xc[ncell][3], S[d][ncell][3]
void orc_geometry(void* h, int b, double* vol, double* xc, double* S) {
  Case* C = (Case*)h;
  const Block& B = C->B[b];
  std::memcpy(vol, B.vol.data(), sizeof(double) * B.ncell);
  std::memcpy(xc, B.xc.data(), sizeof(double) * 3 * B.ncell);
  for (int d = 0; d < 3; ++d) std::memcpy(S + 3 * B.ncell * d, B.S[d].data(), sizeof(double) * 3 * B.ncell);
}

// initial state: freestream of each snapshot at the static cell centre times
// (1 + amp * noise); noise packed per block as [n][v][k][j][i]; ghosts zero
void orc_init_state(void* h, const double* noise, double amp, double* U) {
  Case* C = (Case*)h;
  std::fill(U, U + C->total, 0.0);
  const double* z = noise;
  for (int b = 0; b < (int)C->B.size(); ++b) {
    const Block& B = C->B[b];
    for (int n = 0; n < C->ns; ++n) {
      Frame f = frame(*C, n);
      for (int v = 0; v < C->nv; ++v)
        for (int k = 0; k < B.n[2]; ++k)
          for (int j = 0; j < B.n[1]; ++j)
            for (int i = 0; i < B.n[0]; ++i) {
              int64_t c = B.cell(i, j, k);
              double W[5], Ui[5];
              freestream(*C, f, &B.xc[3 * c], W);
              cons(*C, W, Ui);
              U[C->at(b, n, v, c)] = Ui[v] * (1.0 + amp * (*z++));
            }
    }
  }
}

void orc_fill_ghosts(void* h, double* U) { fill_ghosts(*(Case*)h, U); }

// residual of every interior cell (ghosts of a private copy of U are filled
// first); R and scale in the state layout, ghost entries zero
void orc_residual(void* h, const double* Uin, double* R, double* scale) {
  Case* C = (Case*)h;
  std::vector<double> U(Uin, Uin + C->total);
  fill_ghosts(*C, U.data());
  std::fill(R, R + C->total, 0.0);
  if (scale) std::fill(scale, scale + C->total, 0.0);
  std::vector<double> r(C->ns * C->nv), s(C->ns * C->nv);
  for_interior(*C, [&](int b, int i, int j, int k) {
    cell_residual(*C, U.data(), b, i, j, k, r.data(), s.data());
    int64_t c = C->B[b].cell(i, j, k);
    for (int n = 0; n < C->ns; ++n)
      for (int v = 0; v < C->nv; ++v) {
        R[C->at(b, n, v, c)] = r[n * C->nv + v];
        if (scale) scale[C->at(b, n, v, c)] = s[n * C->nv + v];
      }
  });
}

// residual at listed cells only (b,i,j,k quads); R, scale as [m][ns][nv]
void orc_residual_cells(void* h, const double* Uin, int m, const int* cells, double* R,
                        double* scale) {
  Case* C = (Case*)h;
  std::vector<double> U(Uin, Uin + C->total);
  fill_ghosts(*C, U.data());
  for (int q = 0; q < m; ++q) {
    const int* c = cells + 4 * q;
    cell_residual(*C, U.data(), c[0], c[1], c[2], c[3], R + (int64_t)q * C->ns * C->nv,
                  scale ? scale + (int64_t)q * C->ns * C->nv : nullptr);
  }
}

// local pseudo-time step of every interior cell and snapshot, state layout with nv = 1
// entries replaced by the same value for each variable
void orc_time_step(void* h, const double* U, double* dt) {
  Case* C = (Case*)h;
  std::fill(dt, dt + C->total, 0.0);
  for_interior(*C, [&](int b, int i, int j, int k) {
    int64_t c = C->B[b].cell(i, j, k);
    for (int n = 0; n < C->ns; ++n) {
      double t = local_dt(*C, U, b, i, j, k, n);
      for (int v = 0; v < C->nv; ++v) dt[C->at(b, n, v, c)] = t;
    }
  });
}

namespace {
// The residual sweep of a stage: every (block, snapshot) pair, split into
// rows of cells.  With threads > 1 (a library built with OpenMP) the items
// run on that many threads, the hybrid harmonic parallelisation the paper
// applies with OpenMP (Sec. 2): each item writes only its own entries of R,
// so the result is bit for bit the single-thread one.
void residual_sweep(const Case& C, const double* U, double* R, int threads) {
  struct Item { int b, n, j, k; };
  std::vector<Item> items;
  for (int b = 0; b < (int)C.B.size(); ++b)
    for (int n = 0; n < C.ns; ++n)
      for (int k = 0; k < C.B[b].n[2]; ++k)
        for (int j = 0; j < C.B[b].n[1]; ++j) items.push_back({b, n, j, k});
  const int64_t count = (int64_t)items.size();
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads > 0 ? threads : 1)
#endif
  for (int64_t q = 0; q < count; ++q) {
    const Item& it = items[q];
    const Block& B = C.B[it.b];
    double r[5];
    for (int i = 0; i < B.n[0]; ++i) {
      snapshot_residual(C, U, it.b, i, it.j, it.k, it.n, r, (double*)nullptr);
      int64_t c = B.cell(i, it.j, it.k);
      for (int v = 0; v < C.nv; ++v) R[C.at(it.b, it.n, v, c)] = r[v];
    }
  }
  (void)threads;
}

// n_iter iterations of the 4-stage Runge-Kutta smoother with local time steps
// (coefficients 1/4, 1/3, 1/2, 1); norms[it][v] = RMS of R/V over interior
// cells and snapshots at the first stage, or NULL
void rk_smooth(Case* C, double* U, int n_iter, double* norms, int threads) {
  const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  std::vector<double> U0(C->total), dt(C->total), R(C->total);
  int64_t ncells = 0;
  for (auto& B : C->B) ncells += (int64_t)B.n[0] * B.n[1] * B.n[2];
  for (int it = 0; it < n_iter; ++it) {
    std::copy(U, U + C->total, U0.begin());
    for_interior(*C, [&](int b, int i, int j, int k) {
      int64_t c = C->B[b].cell(i, j, k);
      for (int n = 0; n < C->ns; ++n) dt[C->at(b, n, 0, c)] = local_dt(*C, U0.data(), b, i, j, k, n);
    });
    for (int s = 0; s < 4; ++s) {
      fill_ghosts(*C, U);
      double acc[5] = {0, 0, 0, 0, 0};
      residual_sweep(*C, (const double*)U, R.data(), threads);
      for_interior(*C, [&](int b, int i, int j, int k) {
        int64_t c = C->B[b].cell(i, j, k);
        double V = C->B[b].vol[c];
        for (int n = 0; n < C->ns; ++n) {
          double t = dt[C->at(b, n, 0, c)];
          for (int v = 0; v < C->nv; ++v) {
            int64_t a = C->at(b, n, v, c);
            if (s == 0) acc[v] += (R[a] / V) * (R[a] / V);
            U[a] = U0[a] - alpha[s] * t / V * R[a];
          }
        }
      });
      if (s == 0 && norms)
        for (int v = 0; v < C->nv; ++v)
          norms[(int64_t)it * C->nv + v] = std::sqrt(acc[v] / (double)(ncells * C->ns));
    }
  }
}
}  // namespace

void orc_rk_smooth(void* h, double* U, int n_iter, double* norms) {
  rk_smooth((Case*)h, U, n_iter, norms, 1);
}

// one pass of the ghost fill in place (cuts with source block -1 skipped)
void orc_halo_pass(void* h, double* U, int pass) { fill_pass(*(Case*)h, U, pass); }

// one stage of the smoother above, out of place and without refilling the
// ghosts of Uin: Uout = U0 - alpha_stage dt(U0)/V R(Uin) on interior cells;
// at stage 0 sums[v] = sum over interior cells and snapshots of (R/V)^2
void orc_rk_stage(void* h, const double* Uin, const double* U0, double* Uout, int stage, double* sums) {
  Case* C = (Case*)h;
  const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  std::vector<double> R(C->total);
  residual_sweep(*C, Uin, R.data(), 1);
  double acc[5] = {0, 0, 0, 0, 0};
  for_interior(*C, [&](int b, int i, int j, int k) {
    int64_t c = C->B[b].cell(i, j, k);
    double V = C->B[b].vol[c];
    for (int n = 0; n < C->ns; ++n) {
      double t = local_dt(*C, U0, b, i, j, k, n);
      for (int v = 0; v < C->nv; ++v) {
        int64_t a = C->at(b, n, v, c);
        if (stage == 0) acc[v] += (R[a] / V) * (R[a] / V);
        Uout[a] = U0[a] - alpha[stage] * t / V * R[a];
      }
    }
  });
  if (stage == 0 && sums)
    for (int v = 0; v < C->nv; ++v) sums[v] = acc[v];
}

// the same iterations with the residual sweeps on `threads` threads (only in
// the OpenMP build of this file; otherwise one thread): the same result, bit
// for bit.  orc_openmp_threads reports the threads available (0 without OpenMP).
void orc_rk_smooth_threads(void* h, double* U, int n_iter, double* norms, int threads) {
  rk_smooth((Case*)h, U, n_iter, norms, threads);
}

int orc_openmp_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 0;
#endif
}

// ---- time-domain dual time stepping (a case with one snapshot).  Reading:
// the physical-time derivative by second-order backward differences (BDF2),
// each physical step solved by the same pseudo-time RK smoother with local
// time steps:  R*(U) = R(U; t) + V (a0 U + a1 U^n + a2 U^(n-1)) / dt,
// (a0, a1, a2) = (3/2, -2, 1/2), or (1, -1, 0) on the first step (U^(n-1)
// null); the pseudo time step adds a0 V / dt to its spectral radius.
namespace {
void td_coeffs(const double* Unm1, double* a) {
  if (Unm1) { a[0] = 1.5; a[1] = -2.0; a[2] = 0.5; }
  else { a[0] = 1.0; a[1] = -1.0; a[2] = 0.0; }
}

void td_residual(Case& C, const double* U, const double* Un, const double* Unm1, double dt, double* R) {
  double a[3];
  td_coeffs(Unm1, a);
  std::vector<double> W(U, U + C.total), r(C.nv);
  fill_ghosts(C, W.data());
  std::fill(R, R + C.total, 0.0);
  for_interior(C, [&](int b, int i, int j, int k) {
    cell_residual(C, (const double*)W.data(), b, i, j, k, r.data(), (double*)nullptr);
    const int64_t c = C.B[b].cell(i, j, k);
    const double V = C.B[b].vol[c];
    for (int v = 0; v < C.nv; ++v) {
      const int64_t e = C.at(b, 0, v, c);
      const double ut = a[0] * U[e] + a[1] * Un[e] + (Unm1 ? a[2] * Unm1[e] : 0.0);
      R[e] = r[v] + V * ut / dt;
    }
  });
}
}  // namespace

// R*(U) at physical time t (interior entries; the case has one snapshot)
void orc_td_residual(void* h, const double* U, const double* Un, const double* Unm1, double t, double dt,
                     double* R) {
  Case* C = (Case*)h;
  C->td = 1;
  C->td_t = t;
  td_residual(*C, U, Un, Unm1, dt, R);
  C->td = 0;
}

// n_inner pseudo-time RK iterations of R*(U) = 0 at physical time t, in
// place; norms[it][v] = RMS of R*/V at the first stage, or NULL
void orc_td_step(void* h, double* U, const double* Un, const double* Unm1, double t, double dt, int n_inner,
                 double* norms) {
  Case* C = (Case*)h;
  double a[3];
  td_coeffs(Unm1, a);
  C->td = 1;
  C->td_t = t;
  C->td_lam = a[0] / dt;
  const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  std::vector<double> U0(C->total), dtl(C->total), R(C->total);
  int64_t ncells = 0;
  for (auto& B : C->B) ncells += (int64_t)B.n[0] * B.n[1] * B.n[2];
  for (int it = 0; it < n_inner; ++it) {
    std::copy(U, U + C->total, U0.begin());
    for_interior(*C, [&](int b, int i, int j, int k) {
      dtl[C->at(b, 0, 0, C->B[b].cell(i, j, k))] = local_dt(*C, U0.data(), b, i, j, k, 0);
    });
    for (int s = 0; s < 4; ++s) {
      td_residual(*C, U, Un, Unm1, dt, R.data());
      double acc[5] = {0, 0, 0, 0, 0};
      for_interior(*C, [&](int b, int i, int j, int k) {
        const int64_t c = C->B[b].cell(i, j, k);
        const double V = C->B[b].vol[c];
        const double tl = dtl[C->at(b, 0, 0, c)];
        for (int v = 0; v < C->nv; ++v) {
          const int64_t e = C->at(b, 0, v, c);
          if (s == 0) acc[v] += (R[e] / V) * (R[e] / V);
          U[e] = U0[e] - alpha[s] * tl / V * R[e];
        }
      });
      if (s == 0 && norms)
        for (int v = 0; v < C->nv; ++v) norms[(int64_t)it * C->nv + v] = std::sqrt(acc[v] / (double)ncells);
    }
  }
  C->td = 0;
  C->td_lam = 0.0;
}

// forces at physical time t of a one-snapshot case
void orc_td_forces(void* h, const double* Uin, double t, double* coef, double* J) {
  Case* C = (Case*)h;
  C->td = 1;
  C->td_t = t;
  std::vector<double> U(Uin, Uin + C->total);
  fill_ghosts(*C, U.data());
  forces(*C, U.data(), coef, J);
  C->td = 0;
}

void orc_forces(void* h, const double* Uin, double* coef, double* J) {
  Case* C = (Case*)h;
  std::vector<double> U(Uin, Uin + C->total);
  fill_ghosts(*C, U.data());
  forces(*C, U.data(), coef, J);
}

// Columns of the gradient of L(U) = sum_rows psi . R(U) + J_seed * J(U) with
// respect to interior state entries cols[q] = (b, i, j, k, v, n).
// mode 0: forward-mode dual numbers (exact); mode 1: central differences with
// step h * max(1, |U|).  Only residual rows whose stencil (Chebyshev radius 2,
// ghosts included) meets a perturbed entry are evaluated: the others do not
// depend on the column, so their contribution is exactly zero.
void orc_adjoint_columns(void* h, const double* Uin, const double* psi, double J_seed, int ncols,
                         const int* cols, double* out, int mode, double hstep) {
  Case* C = (Case*)h;
  int nb = (int)C->B.size();
  std::vector<Dual> Ud(C->total);
  std::vector<double> Up(C->total), Um(C->total);
  std::vector<double> base(Uin, Uin + C->total);
  std::vector<double> r(C->ns * C->nv);
  std::vector<Dual> rd(C->ns * C->nv);
  std::vector<Dual> coefd(std::max(1, C->ns * C->n_bodies * 3));
  std::vector<double> coefp(std::max(1, C->ns * C->n_bodies * 3));
  std::vector<std::vector<char>> mark(nb);
  for (int b = 0; b < nb; ++b) mark[b].assign(C->B[b].ncell, 0);
  for (int64_t a = 0; a < C->total; ++a) Ud[a] = Dual(base[a], 0.0);
  std::copy(base.begin(), base.end(), Up.begin());
  fill_ghosts(*C, Ud.data());

  // cells that carry the column's perturbation: the seed itself plus the
  // ghost cells that the ghost fill derived from it; rows whose stencil
  // (Chebyshev radius 2) meets one of them are evaluated
  auto rows_from_tangent = [&](int sb, int64_t sc, auto tangent_at) {
    std::vector<std::array<int, 4>> rows;
    std::vector<std::vector<char>> seen(nb);
    for (int b = 0; b < nb; ++b) {
      const Block& B = C->B[b];
      std::vector<std::array<int, 3>> hot;
      for (int k = -B.g[2]; k < B.n[2] + B.g[2]; ++k)
        for (int j = -B.g[1]; j < B.n[1] + B.g[1]; ++j)
          for (int i = -B.g[0]; i < B.n[0] + B.g[0]; ++i) {
            const bool in = B.interior(i, j, k);
            const int64_t c = B.cell(i, j, k);
            if (in && !(b == sb && c == sc)) continue;
            bool t = false;
            for (int n = 0; n < C->ns && !t; ++n)
              for (int v = 0; v < C->nv && !t; ++v) t = tangent_at(C->at(b, n, v, c));
            if (t) hot.push_back({i, j, k});
          }
      if (hot.empty()) continue;
      seen[b].assign(B.ncell, 0);
      const int rk = (C->dim == 3) ? 2 : 0;
      for (auto& h : hot)
        for (int dk = -rk; dk <= rk; ++dk)
          for (int dj = -2; dj <= 2; ++dj)
            for (int di = -2; di <= 2; ++di) {
              int i = h[0] + di, j = h[1] + dj, k = h[2] + dk;
              if (!B.interior(i, j, k)) continue;
              int64_t c = B.cell(i, j, k);
              if (seen[b][c]) continue;
              seen[b][c] = 1;
              rows.push_back({b, i, j, k});
            }
    }
    std::sort(rows.begin(), rows.end());
    return rows;
  };

  for (int q = 0; q < ncols; ++q) {
    const int* cl = cols + 6 * q;
    int b = cl[0], v = cl[4], n = cl[5];
    int64_t a = C->at(b, n, v, C->B[b].cell(cl[1], cl[2], cl[3]));
    if (mode == 0) {
      Ud[a].d = 1.0;
      fill_ghosts(*C, Ud.data());
      auto rows = rows_from_tangent(b, C->B[b].cell(cl[1], cl[2], cl[3]),
                                    [&](int64_t x) { return Ud[x].d != 0.0; });
      double acc = 0.0;
      for (auto& rw : rows) {
        cell_residual(*C, (const Dual*)Ud.data(), rw[0], rw[1], rw[2], rw[3], rd.data(), (double*)nullptr);
        int64_t c = C->B[rw[0]].cell(rw[1], rw[2], rw[3]);
        for (int nn = 0; nn < C->ns; ++nn)
          for (int vv = 0; vv < C->nv; ++vv) acc += psi[C->at(rw[0], nn, vv, c)] * rd[nn * C->nv + vv].d;
      }
      if (J_seed != 0.0 && C->n_bodies > 0) {
        Dual Jd;
        forces(*C, (const Dual*)Ud.data(), coefd.data(), &Jd);
        acc += J_seed * Jd.d;
      }
      out[q] = acc;
      Ud[a].d = 0.0;
      // ghosts keep stale tangents; the next fill overwrites every ghost
    } else {
      // the rows come from the same structural dependence as the dual mode
      Ud[a].d = 1.0;
      fill_ghosts(*C, Ud.data());
      auto rows = rows_from_tangent(b, C->B[b].cell(cl[1], cl[2], cl[3]),
                                    [&](int64_t x) { return Ud[x].d != 0.0; });
      Ud[a].d = 0.0;
      double hh = hstep * std::max(1.0, std::fabs(base[a]));
      std::vector<double> rp((size_t)rows.size() * C->ns * C->nv), rm(rp.size());
      double Jp = 0.0, Jm = 0.0;
      for (int sgn = 0; sgn < 2; ++sgn) {
        Up[a] = base[a] + (sgn == 0 ? hh : -hh);
        fill_ghosts(*C, Up.data());
        std::vector<double>& dst = (sgn == 0) ? rp : rm;
        for (size_t w = 0; w < rows.size(); ++w)
          cell_residual(*C, (const double*)Up.data(), rows[w][0], rows[w][1], rows[w][2], rows[w][3],
                        dst.data() + w * C->ns * C->nv, (double*)nullptr);
        if (J_seed != 0.0 && C->n_bodies > 0)
          forces(*C, (const double*)Up.data(), coefp.data(), sgn == 0 ? &Jp : &Jm);
      }
      Up[a] = base[a];
      double acc = 0.0;
      for (size_t w = 0; w < rows.size(); ++w) {
        int64_t c = C->B[rows[w][0]].cell(rows[w][1], rows[w][2], rows[w][3]);
        for (int nn = 0; nn < C->ns; ++nn)
          for (int vv = 0; vv < C->nv; ++vv)
            acc += psi[C->at(rows[w][0], nn, vv, c)] *
                   (rp[w * C->ns * C->nv + nn * C->nv + vv] - rm[w * C->ns * C->nv + nn * C->nv + vv]);
      }
      acc += J_seed * (Jp - Jm);
      out[q] = acc / (2.0 * hh);
    }
  }
}

}  // extern "C"
