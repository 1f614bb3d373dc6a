// GR hydrodynamics of a perfect fluid on the evolving spacetime (Sec. 2.1.2,
// 2.2 of the SACRA-K paper), FP64.
//
//  - Variables: primitives (rho, eps, u_i) with u_i the spatial covariant
//    components of the four-velocity, w = alpha u^t = sqrt(1 + gamma^ij u_i
//    u_j); densitised conserved variables sqrt(gamma) (D, J_i, rho_H) with
//    D = rho w, J_i = rho h w u_i, rho_H = rho h w^2 - P, h = 1 + eps + P/rho.
//  - Hybrid EOS: P = P_cold(rho) + (Gamma_th - 1) rho (eps - eps_cold(rho)),
//    the cold part a piecewise polytrope.
//  - Fluxes along j with V^j = alpha gamma^jk u_k / w - beta^j:
//    D^ V^j, J^_i V^j + alpha sqrt(gamma) P delta^j_i, E^ V^j + sqrt(gamma)
//    P (V^j + beta^j); sources sqrt(gamma) (-rho_H d_i alpha + J_k d_i beta^k
//    + alpha/2 S^jk d_i gamma_jk) and sqrt(gamma) (alpha S^jk K_jk - J^j
//    d_j alpha), S^jk = rho h u^j u^k + P gamma^jk.
//  - Faces: PPM (Colella & Woodward) edge values with slopes limited by the
//    steep minmod of parameter b = 3, metric by the 4th-order Lagrange
//    interpolation (-1, 9, 9, -1)/16; the face flux is the HLLC flux of
//    special relativity (Mignone & Bodo 2005) in an orthonormal tetrad in
//    which the face is at rest, with the HLLE flux there where the
//    intermediate state is unphysical, or (MatterArgs::riemann = 1) the
//    HLLE flux in the coordinate frame with the relativistic characteristic
//    speeds; metric derivatives of the sources by the 4th-order centred
//    differences.
//  - Recovery: Newton-Raphson on w with the hybrid EOS solved for P(w) in
//    closed form, f(w) = w - (rho_H + P) / sqrt((rho_H + P)^2 - S^2), the
//    previous recovery's w as the guess and a bisection bracket; a negative
//    thermal part is repaired to the cold value; a cell below the floor or
//    without a root is reset to rest at the floor density (atmosphere).
//
// Kernels: one thread per active cell (recovery, update) or per face
// (fluxes, one launch per direction into a face-flux array), grid-striding.
#include <math.h>

#include "grhd.h"
#include "sacrak_dev.cuh"

namespace sacrak {
namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double PPM_B = 3.0;

struct Met {
  double al, be[3], g[6], gu[6], sg;
};

__device__ __forceinline__ double inv_sym(const double g[6], double gu[6]) {
  const double c0 = g[3] * g[5] - g[4] * g[4];
  const double c1 = g[2] * g[4] - g[1] * g[5];
  const double c2 = g[1] * g[4] - g[2] * g[3];
  const double det = g[0] * c0 + g[1] * c1 + g[2] * c2;
  const double id = 1.0 / det;
  gu[0] = c0 * id;
  gu[1] = c1 * id;
  gu[2] = c2 * id;
  gu[3] = (g[0] * g[5] - g[2] * g[2]) * id;
  gu[4] = (g[1] * g[2] - g[0] * g[4]) * id;
  gu[5] = (g[0] * g[3] - g[1] * g[1]) * id;
  return det;
}

// alpha, beta^i, gamma_ij at cell q (what the face interpolation needs)
__device__ __forceinline__ void metric_ll_at(const double* __restrict__ u, long long q, long long fs, double v[10]) {
  const double W = __ldg(u + F_W * fs + q);
  const double iW2 = 1.0 / (W * W);
  v[0] = __ldg(u + F_ALP * fs + q);
#pragma unroll
  for (int d = 0; d < 3; ++d) v[1 + d] = __ldg(u + (F_BETX + d) * fs + q);
#pragma unroll
  for (int a = 0; a < 6; ++a) v[4 + a] = __ldg(u + (F_GXX + a) * fs + q) * iW2;
}

// 3+1 metric at cell q of the Z4c state u (optionally K_ij)
__device__ __forceinline__ void metric_at(const double* __restrict__ u, long long q, long long fs, Met& m,
                                          double* K_ll) {
  const double W = __ldg(u + F_W * fs + q);
  double gt[6], gtu[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) gt[a] = __ldg(u + (F_GXX + a) * fs + q);
  const double det = inv_sym(gt, gtu);
  const double iW2 = 1.0 / (W * W);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    m.g[a] = gt[a] * iW2;
    m.gu[a] = gtu[a] * (W * W);
  }
  m.sg = sqrt(det) / (W * W * W);
  m.al = __ldg(u + F_ALP * fs + q);
#pragma unroll
  for (int d = 0; d < 3; ++d) m.be[d] = __ldg(u + (F_BETX + d) * fs + q);
  if (K_ll) {
    const double K = __ldg(u + F_KH * fs + q) + 2.0 * __ldg(u + F_TH * fs + q);
#pragma unroll
    for (int a = 0; a < 6; ++a) K_ll[a] = (__ldg(u + (F_AXX + a) * fs + q) + gt[a] * K / 3.0) * iW2;
  }
}

__device__ __forceinline__ void raise3(const double gu[6], const double v[3], double r[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) r[i] = gu[S2(i, 0)] * v[0] + gu[S2(i, 1)] * v[1] + gu[S2(i, 2)] * v[2];
}

// ------------------------------------------------------------------ EOS

// rho^x for the polytrope exponent x = Gamma - 1: the exponents 1, 1/2, 3/2
// and 2 without pow (the same values to rounding)
__device__ __forceinline__ double pow_gm1(double rho, double x) {
  if (x == 1.0) return rho;
  if (x == 0.5) return sqrt(rho);
  if (x == 1.5) return rho * sqrt(rho);
  if (x == 2.0) return rho * rho;
  return pow(rho, x);
}

__device__ __forceinline__ void eos_cold(const DevEOS& e, double rho, double& P, double& eps, double& dP) {
  int i = 0;
  for (int b = 0; b < e.n - 1; ++b) i += rho >= e.rb[b] ? 1 : 0;
  const double K = e.K[i], G = e.G[i];
  const double rg = pow_gm1(rho, G - 1.0);
  P = K * rg * rho;
  eps = e.a[i] + K * rg / (G - 1.0);
  dP = G * K * rg;
}

__device__ __forceinline__ double eos_pressure(const DevEOS& e, double rho, double eps) {
  double Pc, ec, dP;
  eos_cold(e, rho, Pc, ec, dP);
  return Pc + (e.gth - 1.0) * rho * (eps - ec);
}

// ------------------------------------------------------------------ prim <-> con

__device__ __forceinline__ void prim2con(const DevEOS& e, const Met& m, const double pr[NM], double c[NM],
                                         double& w, double& h, double& P) {
  const double ul[3] = {pr[2], pr[3], pr[4]};
  double uu[3];
  raise3(m.gu, ul, uu);
  w = sqrt(1.0 + ul[0] * uu[0] + ul[1] * uu[1] + ul[2] * uu[2]);
  P = eos_pressure(e, pr[0], pr[1]);
  h = 1.0 + pr[1] + P / pr[0];
  c[0] = m.sg * pr[0] * w;
#pragma unroll
  for (int i = 0; i < 3; ++i) c[1 + i] = m.sg * pr[0] * h * w * ul[i];
  c[4] = m.sg * (pr[0] * h * w * w - P);
}

// P(w) of the hybrid EOS at fixed D, rho_H (closed form) and dP/dw
__device__ __forceinline__ void pressure_of_w(const DevEOS& e, double w, double D, double E, double& P,
                                              double& dPdw) {
  const double rho = D / w;
  double Pc, ec, dPc;
  eos_cold(e, rho, Pc, ec, dPc);
  const double g = e.gth - 1.0;
  const double iw = 1.0 / w, iw2 = iw * iw;
  const double N = Pc + g * (E * iw2 - D * iw * (1.0 + ec));
  const double Q = 1.0 + g * (1.0 - iw2);
  // d eps_cold / d rho = P_cold / rho^2, d rho / d w = -D / w^2
  const double dN = -D * iw2 * dPc + g * (-2.0 * E * iw2 * iw + D * iw2 * (1.0 + ec) + Pc * iw);
  const double dQ = 2.0 * g * iw2 * iw;
  const double iQ = 1.0 / Q;
  P = N * iQ;
  dPdw = (dN - P * dQ) * iQ;
}

// Newton-Raphson on w within the bracket [lo, hi] (bisection where a step
// leaves it); returns true for a physical root
__device__ bool con2prim(const DevEOS& e, const Met& m, const double c[NM], double wg, double pr[NM],
                         double& wout) {
  const double D = c[0] / m.sg, E = c[4] / m.sg;
  const double J[3] = {c[1] / m.sg, c[2] / m.sg, c[3] / m.sg};
  double Ju[3];
  raise3(m.gu, J, Ju);
  const double S2 = J[0] * Ju[0] + J[1] * Ju[1] + J[2] * Ju[2];
  if (!(D > 0.0) || !(E > 0.0) || !isfinite(D) || !isfinite(E)) return false;
  double w = fmin(fmax(wg, 1.0), 1e4), lo = 1.0, hi = 1e4;
  double P = 0.0, dP = 0.0;
#pragma unroll 1
  for (int it = 0; it < 60; ++it) {
    pressure_of_w(e, w, D, E, P, dP);
    const double X = E + P;
    const double q = X * X - S2;
    const double iR = 1.0 / sqrt(fmax(q, 1e-300));
    const double f = w - X * iR;
    if (f < 0.0) lo = fmax(lo, w);
    if (f > 0.0) hi = fmin(hi, w);
    const double fp = 1.0 + dP * S2 * (iR * iR * iR);
    double wn = w - f / (fp != 0.0 ? fp : 1.0);
    const bool newton = wn >= lo && wn <= hi;  // closed: w = 1 (at rest) is a root
    if (!newton) wn = 0.5 * (lo + hi);
    // quadratic convergence: a Newton step below 1e-10 w leaves an iterate
    // accurate to rounding (a bisection step never ends the iteration)
    const bool done = newton && fabs(wn - w) <= 1e-10 * wn;
    w = wn;
    if (done) break;
  }
  pressure_of_w(e, w, D, E, P, dP);
  const double X = E + P;
  const double q = X * X - S2;
  const double f = w - X / sqrt(fmax(q, 1e-300));
  const double rho = D / w;
  const double h = X / (D * w);
  pr[0] = rho;
  pr[1] = h - 1.0 - P / rho;
#pragma unroll
  for (int i = 0; i < 3; ++i) pr[2 + i] = J[i] / (rho * h * w);
  wout = w;
  return isfinite(w) && q > 0.0 && rho > 0.0 && fabs(f) <= 1e-10 * w;
}

__device__ __forceinline__ double floor_at(const MatterArgs& A, int i, int j, int k) {
  const double x = A.origin[0] + (i + 0.5) * A.dx, y = A.origin[1] + (j + 0.5) * A.dx,
               z = A.origin[2] + (k + 0.5) * A.dx;
  const double r = sqrt(x * x + y * y + z * z);
  if (r <= A.r_atm) return A.rho_atm;
  const double s = A.r_atm / fmax(r, 1e-300);
  return A.rho_atm * s * s * s;
}

__device__ __forceinline__ const double* z4c_stage_state(const MatterArgs& A, int ring) {
  const int s = A.stage;
  return A.P->buf[s == 0 ? ring : (s == 5 ? stage_out_slot(4, ring) : stage_in_slot(s, ring))];
}
__device__ __forceinline__ double* matter_stage_state(const MatterArgs& A, int ring) {
  const int s = A.stage;
  return A.P->mcons[s == 0 ? ring : (s == 5 ? stage_out_slot(4, ring) : stage_in_slot(s, ring))];
}

// ------------------------------------------------------------------ kernels

__global__ void __launch_bounds__(128) matter_prep_kernel(MatterArgs A) {
  const long long nact = (long long)A.n[0] * A.n[1] * A.n[2];
  const int ring = A.lev->ring;
  const double* __restrict__ u = z4c_stage_state(A, ring);
  double* __restrict__ cons = matter_stage_state(A, ring);
  double* __restrict__ prim = A.P->mprim;
  double* __restrict__ zs = A.P->mzsrc;
  const long long fs = A.fs;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < nact;
       id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % A.n[0]);
    const int j = (int)((id / A.n[0]) % A.n[1]);
    const int k = (int)(id / ((long long)A.n[0] * A.n[1]));
    const long long q = (i + GH) + (j + GH) * A.sy + (k + GH) * A.sz;
    Met m;
    metric_at(u, q, fs, m, nullptr);
    double c[NM], pr[NM], w;
#pragma unroll
    for (int f = 0; f < NM; ++f) c[f] = cons[f * fs + q];
    bool ok = con2prim(A.eos, m, c, prim[NM * fs + q], pr, w);
    double Pc, ec, dP;
    eos_cold(A.eos, ok ? pr[0] : 1.0, Pc, ec, dP);
    bool fix = false;
    if (ok && pr[1] < ec) {
      pr[1] = ec;
      fix = true;
    }
    const double fl = floor_at(A, i, j, k);
    if (!ok || pr[0] < fl) {
      double Pf, ef, dPf;
      eos_cold(A.eos, fl, Pf, ef, dPf);
      pr[0] = fl;
      pr[1] = ef;
      pr[2] = pr[3] = pr[4] = 0.0;
      fix = true;
    }
    double h, P;
    if (fix) {
      prim2con(A.eos, m, pr, c, w, h, P);
#pragma unroll
      for (int f = 0; f < NM; ++f) cons[f * fs + q] = c[f];
    } else {
      P = eos_pressure(A.eos, pr[0], pr[1]);
      h = 1.0 + pr[1] + P / pr[0];
    }
#pragma unroll
    for (int f = 0; f < NM; ++f) prim[f * fs + q] = pr[f];
    prim[NM * fs + q] = w;
    if (A.coupled) {
      // rho_ADM = rho_H, S_i = J_i, S_ij = rho h u_i u_j + P gamma_ij and the
      // Z4c matter terms (Khat, Theta, At_ij, Gamt^i)
      const double rho = pr[0];
      const double ul[3] = {pr[2], pr[3], pr[4]};
      const double E = rho * h * w * w - P;
      double Sl[3], Sll[6], Str = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) Sl[a] = rho * h * w * ul[a];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) Sll[S2(a, b)] = rho * h * ul[a] * ul[b] + P * m.g[S2(a, b)];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Str += m.gu[S2(a, b)] * Sll[S2(a, b)];
      const double W = u[F_W * fs + q];
      const double al = m.al;
      zs[0 * fs + q] = 4.0 * PI * al * (Str + E);
      zs[1 * fs + q] = -8.0 * PI * al * E;
#pragma unroll
      for (int a = 0; a < 6; ++a) zs[(2 + a) * fs + q] = -8.0 * PI * al * W * W * (Sll[a] - m.g[a] * Str / 3.0);
      // gt^ij = gamma^ij / W^2
#pragma unroll
      for (int a = 0; a < 3; ++a)
        zs[(8 + a) * fs + q] = -16.0 * PI * al *
                               (m.gu[S2(a, 0)] * Sl[0] + m.gu[S2(a, 1)] * Sl[1] + m.gu[S2(a, 2)] * Sl[2]) / (W * W);
    }
  }
}

// ghost cells of the NMP primitive arrays: nearest active cell (outflow) or
// the periodic image
__global__ void __launch_bounds__(128) matter_ghost_kernel(MatterArgs A) {
  const long long ntot = (long long)A.NX * A.NY * A.NZ;
  double* __restrict__ prim = A.P->mprim;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < ntot;
       id += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(id % A.NX), J = (int)((id / A.NX) % A.NY), K = (int)(id / ((long long)A.NX * A.NY));
    const int c[3] = {I, J, K}, N[3] = {A.n[0], A.n[1], A.n[2]};
    bool ghost = false;
    int s[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int a = c[d] - GH;  // active index
      ghost |= (a < 0 || a >= N[d]);
      s[d] = A.periodic ? ((a % N[d]) + N[d]) % N[d] : (a < 0 ? 0 : (a >= N[d] ? N[d] - 1 : a));
    }
    if (!ghost) continue;
    const long long q = I + J * A.sy + K * A.sz;
    const long long qs = (s[0] + GH) + (s[1] + GH) * A.sy + (s[2] + GH) * A.sz;
#pragma unroll
    for (int f = 0; f < NMP; ++f) prim[f * A.fs + q] = prim[f * A.fs + qs];
  }
}

// equatorial symmetry (Sec. 2.2.2): the z < 0 ghost layers of a patch on
// z = 0 mirror the layers above (layer k < GH takes layer 2 GH - 1 - k), the
// primitives and the stage's conserved variables; u_z and J^_z are odd in z,
// the rest even
__global__ void __launch_bounds__(128) matter_zreflect_kernel(MatterArgs A) {
  if (!A.P->zrefl) return;
  const long long nlay = (long long)A.NX * A.NY;
  double* __restrict__ prim = A.P->mprim;
  double* __restrict__ cons = matter_stage_state(A, A.lev->ring);
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < GH * nlay;
       id += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(id / nlay);
    const long long r = id - k * nlay;
    const int I = (int)(r % A.NX), J = (int)(r / A.NX);
    const long long q = I + J * A.sy + k * A.sz;
    const long long qm = I + J * A.sy + (2 * GH - 1 - k) * A.sz;
#pragma unroll
    for (int f = 0; f < NMP; ++f) prim[f * A.fs + q] = (f == 4 ? -1.0 : 1.0) * prim[f * A.fs + qm];
#pragma unroll
    for (int f = 0; f < NM; ++f) cons[f * A.fs + q] = (f == 3 ? -1.0 : 1.0) * cons[f * A.fs + qm];
  }
}

__device__ __forceinline__ double minmod3(double a, double b, double c) {
  const bool pos = a > 0.0 && b > 0.0 && c > 0.0, neg = a < 0.0 && b < 0.0 && c < 0.0;
  if (!(pos || neg)) return 0.0;
  const double m = fmin(fmin(fabs(a), fabs(b)), fabs(c));
  return pos ? m : -m;
}

// PPM states at the face between cells 2 and 3 of v[0..5] (cells m-2 .. m+3)
__device__ __forceinline__ void ppm_face(const double v[6], double& left, double& right) {
  double sl[4];  // limited slopes at cells 1..4
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double a0 = v[i], a1 = v[i + 1], a2 = v[i + 2];
    sl[i] = minmod3(0.5 * (a2 - a0), PPM_B * (a2 - a1), PPM_B * (a1 - a0));
  }
  // face values between cells (1,2), (2,3), (3,4)
  double af[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) af[i] = 0.5 * (v[i + 1] + v[i + 2]) - (sl[i + 1] - sl[i]) * (1.0 / 6.0);
  // cell 2 (aL = af[0], aR = af[1]) and cell 3 (aL = af[1], aR = af[2]), monotonised
#pragma unroll
  for (int cidx = 0; cidx < 2; ++cidx) {
    const double c = v[2 + cidx];
    double aL = af[cidx], aR = af[cidx + 1];
    if ((aR - c) * (c - aL) <= 0.0) {
      aL = c;
      aR = c;
    }
    const double d = aR - aL, mid = c - 0.5 * (aL + aR);
    const double d6 = d * d * (1.0 / 6.0);
    const bool ol = d * mid > d6;
    if (ol) aL = 3.0 * c - 2.0 * aR;
    if (!ol && -d6 > d * mid) aR = 3.0 * c - 2.0 * aL;
    if (cidx == 0)
      left = aR;
    else
      right = aL;
  }
}

// conserved variables, flux along d and characteristic speeds of a state
template <int d>
__device__ __forceinline__ void phys_flux(const DevEOS& e, const Met& m, const double pr[NM], double U[NM],
                                          double F[NM], double& lp, double& lm) {
  // one cold-EOS evaluation for the pressure and the sound speed
  double Pc, ec, dPc;
  eos_cold(e, pr[0], Pc, ec, dPc);
  const double P = Pc + (e.gth - 1.0) * pr[0] * (pr[1] - ec);
  const double irho = 1.0 / pr[0];
  const double h = 1.0 + pr[1] + P * irho;
  double w;
  {
    const double ul[3] = {pr[2], pr[3], pr[4]};
    double uu[3];
    raise3(m.gu, ul, uu);
    w = sqrt(1.0 + ul[0] * uu[0] + ul[1] * uu[1] + ul[2] * uu[2]);
    U[0] = m.sg * pr[0] * w;
#pragma unroll
    for (int i = 0; i < 3; ++i) U[1 + i] = m.sg * pr[0] * h * w * ul[i];
    U[4] = m.sg * (pr[0] * h * w * w - P);
  }
  const double ul[3] = {pr[2], pr[3], pr[4]};
  double uu[3];
  raise3(m.gu, ul, uu);
  const double V = m.al * uu[d] / w - m.be[d];
#pragma unroll
  for (int f = 0; f < NM; ++f) F[f] = U[f] * V;
  F[1 + d] += m.al * m.sg * P;
  F[4] += m.sg * P * (V + m.be[d]);
  const double vd = uu[d] / w;
  const double v2 = 1.0 - 1.0 / (w * w);
  // sound speed: (dP/drho|_eps + P/rho^2 dP/deps|_rho) / h
  const double g1 = e.gth - 1.0;
  const double cs2 = (dPc + g1 * (pr[1] - ec) - g1 * Pc * irho + P * irho * g1) / h;
  const double gdd = m.gu[S2(d, d)];
  const double root = sqrt(fmax(cs2 * (1.0 - v2) * (gdd * (1.0 - v2 * cs2) - vd * vd * (1.0 - cs2)), 0.0));
  const double pre = m.al / (1.0 - v2 * cs2);
  lp = pre * (vd * (1.0 - cs2) + root) - m.be[d];
  lm = pre * (vd * (1.0 - cs2) - root) - m.be[d];
}

// ------------------------------------------------------------------ HLLC in the face tetrad

// Orthonormal tetrad at a face normal to x^d: e1 along the spacetime gradient
// of x^d (g^{mu d} / sqrt(g^dd)), e0 the Eulerian observer n projected onto
// the face's world-sheet x^d = const and normalised, e2 and e3 the two
// coordinate directions along the face made orthonormal to e0 (and e2).
// e0, e2, e3 are tangent to the world-sheet: the face is at rest in the frame.
struct Tetrad {
  double e[4][4];  // e[a][mu], contravariant
  double lo[4][3]; // (e_a)_i, the spatial components lowered with the 4-metric
  double s1;       // sqrt(g^dd)
};

// The Gram-Schmidt steps in closed form: with p0 = (e0)_a and q0 = (e0)_b
// (a, b the face's directions), e2 = (d_a + p0 e0) / N2 with N2^2 = g_aa +
// p0^2 (e0 . e0 = -1), e3 = (d_b + q0 e0 - p2 e2) / N3 with p2 = (g_ab + p0
// q0) / N2 and N3^2 = g_bb + q0^2 - p2^2.  Lowered: (e1)_i = delta^d_i / s1
// and (e0)_i = -c / (s1 sqrt(1 + c^2)) delta^d_i (n_i = 0), so p0 = q0 = 0.
template <int d>
__device__ __forceinline__ void face_tetrad(const Met& m, Tetrad& T) {
  constexpr int a = (d + 1) % 3, b = (d + 2) % 3;
  const double ia2 = 1.0 / (m.al * m.al);
  T.s1 = sqrt(m.gu[S2(d, d)] - m.be[d] * m.be[d] * ia2);
  const double is1 = 1.0 / T.s1;
  double* e0 = T.e[0];
  double* e1 = T.e[1];
  e1[0] = m.be[d] * ia2 * is1;
#pragma unroll
  for (int i = 0; i < 3; ++i) e1[1 + i] = (m.gu[S2(i, d)] - m.be[i] * m.be[d] * ia2) * is1;
  const double c = -m.be[d] / m.al * is1;  // n . e1
  const double ic = 1.0 / sqrt(1.0 + c * c);
  e0[0] = (1.0 / m.al - c * e1[0]) * ic;
#pragma unroll
  for (int i = 0; i < 3; ++i) e0[1 + i] = (-m.be[i] / m.al - c * e1[1 + i]) * ic;
  const double e0d = -c * is1 * ic;  // (e0)_d, the only spatial lowered component
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T.lo[0][i] = (i == d) ? e0d : 0.0;
    T.lo[1][i] = (i == d) ? is1 : 0.0;
  }
  const double iN2 = 1.0 / sqrt(m.g[S2(a, a)]);
  const double p2 = m.g[S2(a, b)] * iN2;
  const double iN3 = 1.0 / sqrt(m.g[S2(b, b)] - p2 * p2);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const double e2 = (mu == 1 + a ? 1.0 : 0.0) * iN2;
    T.e[2][mu] = e2;
    T.e[3][mu] = ((mu == 1 + b ? 1.0 : 0.0) - p2 * e2) * iN3;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double l2 = m.g[S2(a, i)] * iN2;
    T.lo[2][i] = l2;
    T.lo[3][i] = (m.g[S2(b, i)] - p2 * l2) * iN3;
  }
}

// special-relativistic state in the tetrad frame: conserved (D, S_1, S_2,
// S_3, E = rho h W^2 - P), flux along 1, speeds along 1, v_1 and P
__device__ __forceinline__ void sr_state(const DevEOS& e, const Met& m, const Tetrad& T, const double pr[NM],
                                         double U[5], double F[5], double& lp, double& lm, double& v1,
                                         double& P) {
  double Pc, ec, dPc;
  eos_cold(e, pr[0], Pc, ec, dPc);
  P = Pc + (e.gth - 1.0) * pr[0] * (pr[1] - ec);
  const double irho = 1.0 / pr[0];
  const double h = 1.0 + pr[1] + P * irho;
  const double ul[3] = {pr[2], pr[3], pr[4]};
  double uu[3];
  raise3(m.gu, ul, uu);
  const double w = sqrt(1.0 + ul[0] * uu[0] + ul[1] * uu[1] + ul[2] * uu[2]);
  const double u0 = -m.al * w + m.be[0] * ul[0] + m.be[1] * ul[1] + m.be[2] * ul[2];  // u_t
  double comp[4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
    comp[a] = T.e[a][0] * u0 + T.e[a][1] * ul[0] + T.e[a][2] * ul[1] + T.e[a][3] * ul[2];
  const double Wt = -comp[0], iW = 1.0 / Wt;
  const double v[3] = {comp[1] * iW, comp[2] * iW, comp[3] * iW};
  const double rhw2 = pr[0] * h * Wt * Wt;
  U[0] = pr[0] * Wt;
  U[1] = rhw2 * v[0];
  U[2] = rhw2 * v[1];
  U[3] = rhw2 * v[2];
  U[4] = rhw2 - P;
#pragma unroll
  for (int f = 0; f < 5; ++f) F[f] = U[f] * v[0];
  F[1] += P;
  F[4] = U[1];
  const double g1 = e.gth - 1.0;
  const double cs2 = (dPc + g1 * (pr[1] - ec) - g1 * Pc * irho + P * irho * g1) / h;
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double root = sqrt(fmax(cs2 * (1.0 - v2) * (1.0 - v2 * cs2 - v[0] * v[0] * (1.0 - cs2)), 0.0));
  const double id = 1.0 / (1.0 - v2 * cs2);
  lp = (v[0] * (1.0 - cs2) + root) * id;
  lm = (v[0] * (1.0 - cs2) - root) * id;
  v1 = v[0];
}

// HLLC flux across an interface at rest (Mignone & Bodo 2005), the HLLE flux
// where the intermediate state is unphysical: no real contact speed, a
// contact speed outside the outer waves or not below light speed, or a
// non-positive intermediate pressure
__device__ __forceinline__ void sr_hllc(const double UL[5], const double FL[5], double lpl, double lml, double vL,
                                        double PL, const double UR[5], const double FR[5], double lpr, double lmr,
                                        double vR, double PR, double out[5]) {
  const double lL = fmin(lml, lmr), lR = fmax(lpl, lpr);
  if (lL >= 0.0) {
#pragma unroll
    for (int f = 0; f < 5; ++f) out[f] = FL[f];
    return;
  }
  if (lR <= 0.0) {
#pragma unroll
    for (int f = 0; f < 5; ++f) out[f] = FR[f];
    return;
  }
  const double iden = 1.0 / (lR - lL);
  double Uh[5], Fh[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    Uh[f] = (lR * UR[f] - lL * UL[f] + FL[f] - FR[f]) * iden;
    Fh[f] = (lR * FL[f] - lL * FR[f] + lL * lR * (UR[f] - UL[f])) * iden;
  }
  const double b = Uh[4] + Fh[1];
  const double disc = b * b - 4.0 * Fh[4] * Uh[1];
  const double ls = 2.0 * Uh[1] / (b + sqrt(fmax(disc, 0.0)));
  const double ps = Fh[1] - ls * Fh[4];
  if (!(disc >= 0.0 && ps > 0.0 && fabs(ls) < 1.0 && ls > lL && ls < lR)) {
#pragma unroll
    for (int f = 0; f < 5; ++f) out[f] = Fh[f];
    return;
  }
  const bool left = ls >= 0.0;
  const double* U = left ? UL : UR;
  const double* F = left ? FL : FR;
  const double lK = left ? lL : lR, vK = left ? vL : vR, PK = left ? PL : PR;
  const double r = 1.0 / (lK - ls), a = lK - vK;
  const double Us[5] = {U[0] * a * r, (U[1] * a + ps - PK) * r, U[2] * a * r, U[3] * a * r,
                        (U[4] * a + ps * ls - PK * vK) * r};
#pragma unroll
  for (int f = 0; f < 5; ++f) out[f] = F[f] + lK * (Us[f] - U[f]);
}

// Coordinate-frame flux of the densitised conserved variables from the
// tetrad-frame flux row Ft = (F_D, F_S1, F_S2, F_S3, F_E): with xi = dx^d and
// xi . e_a = 0 for a != 1, rho u^d = sqrt(g^dd) F_D and T^d_nu = sqrt(g^dd)
// [F_E (e0)_nu + sum_j F_Sj (e_j)_nu], so (sqrt(-g) = alpha sqrt(gamma))
// D^: alpha sqrt(gamma) sqrt(g^dd) F_D; J^_i: alpha sqrt(gamma) sqrt(g^dd)
// [F_E (e0)_i + sum_j F_Sj (e_j)_i]; E^ (alpha sqrt(gamma) times -T^d_nu n^nu):
// alpha^2 sqrt(gamma) sqrt(g^dd) [F_E e0^t + sum_j F_Sj e_j^t].
__device__ __forceinline__ void tetrad_to_coordinate(const Met& m, const Tetrad& T, const double Ft[5],
                                                     double out[NM]) {
  const double pre = m.al * m.sg * T.s1;
  const double rows[4] = {Ft[4], Ft[1], Ft[2], Ft[3]};
  out[0] = pre * Ft[0];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    out[1 + i] = pre * (rows[0] * T.lo[0][i] + rows[1] * T.lo[1][i] + rows[2] * T.lo[2][i] + rows[3] * T.lo[3][i]);
  out[4] = pre * m.al * (rows[0] * T.e[0][0] + rows[1] * T.e[1][0] + rows[2] * T.e[2][0] + rows[3] * T.e[3][0]);
}

// RK4-weighted sum of a face's fluxes over the step's stages (the reflux of
// Sec. 2.2.1): mfs = sum_s b_s F_s; on levels > 0 after stage 4 also mfa, the
// sum of the level's first step, then the mean of its two steps
__device__ __forceinline__ void accumulate_flux(const MatterArgs& A, int dir, long long q, const double F[NM]) {
  if (A.stage < 1 || A.stage > 4 || !A.P->mfs) return;
  const double bw = (A.stage == 1 || A.stage == 4) ? 1.0 / 6.0 : 1.0 / 3.0;
  double* __restrict__ fsum = A.P->mfs + (long long)dir * NM * A.fs;
  double* __restrict__ favg = A.P->mfa + (long long)dir * NM * A.fs;
#pragma unroll
  for (int f = 0; f < NM; ++f) {
    const long long o = f * A.fs + q;
    const double v = (A.stage == 1 ? 0.0 : fsum[o]) + bw * F[f];
    fsum[o] = v;
    if (A.stage == 4 && A.plev) favg[o] = A.first_substep ? v : 0.5 * (favg[o] + v);
  }
}

// one thread per face: faces m+1/2 along dir for m = 2 .. n+2 (array index),
// the other axes over active cells; flux stored at cell m
template <int dir>
__global__ void __launch_bounds__(128) matter_flux_kernel(MatterArgs A) {
  constexpr int a1 = (dir + 1) % 3, a2 = (dir + 2) % 3;
  const long long nf = (long long)(A.n[dir] + 1) * A.n[a1] * A.n[a2];
  const int ring = A.lev->ring;
  const double* __restrict__ u = z4c_stage_state(A, ring);
  const double* __restrict__ prim = A.P->mprim;
  double* __restrict__ flux = A.P->mflux + (long long)dir * NM * A.fs;
  const long long sd = dir == 0 ? 1 : (dir == 1 ? A.sy : A.sz);
  // faces m+1/2 along dir for array index m = 2 .. n+2, active cells along
  // the other axes; x varies fastest over the threads (coalesced rows)
  const int ex = A.n[0] + (dir == 0 ? 1 : 0), ey = A.n[1] + (dir == 1 ? 1 : 0);
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < nf;
       id += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(id % ex);
    const int iy = (int)((id / ex) % ey);
    const int iz = (int)(id / ((long long)ex * ey));
    const int cx = ix + (dir == 0 ? 2 : GH), cy = iy + (dir == 1 ? 2 : GH), cz = iz + (dir == 2 ? 2 : GH);
    const long long q = cx + cy * A.sy + cz * A.sz;
    // face metric: (-1, 9, 9, -1)/16 of alpha, beta, gamma_ij from cells m-1 .. m+2
    Met mf;
    {
      double vals[10];
      for (int t = 0; t < 10; ++t) vals[t] = 0.0;
      const double wts[4] = {-1.0 / 16.0, 9.0 / 16.0, 9.0 / 16.0, -1.0 / 16.0};
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        double vc[10];
        metric_ll_at(u, q + (o - 1) * sd, A.fs, vc);
#pragma unroll
        for (int b = 0; b < 10; ++b) vals[b] += wts[o] * vc[b];
      }
      mf.al = vals[0];
#pragma unroll
      for (int b = 0; b < 3; ++b) mf.be[b] = vals[1 + b];
#pragma unroll
      for (int b = 0; b < 6; ++b) mf.g[b] = vals[4 + b];
      mf.sg = sqrt(inv_sym(mf.g, mf.gu));
    }
    double pl[NM], pr[NM];
#pragma unroll
    for (int f = 0; f < NM; ++f) {
      double v[6];
#pragma unroll
      for (int o = 0; o < 6; ++o) v[o] = prim[f * A.fs + q + (o - 2) * sd];
      ppm_face(v, pl[f], pr[f]);
    }
    double UL[NM], FL[NM], UR[NM], FR[NM], lpl, lml, lpr, lmr;
    if (A.riemann == 0) {
      Tetrad T;
      face_tetrad<dir>(mf, T);
      double vL, PL, vR, PR, Ft[5], out[NM];
      sr_state(A.eos, mf, T, pl, UL, FL, lpl, lml, vL, PL);
      sr_state(A.eos, mf, T, pr, UR, FR, lpr, lmr, vR, PR);
      sr_hllc(UL, FL, lpl, lml, vL, PL, UR, FR, lpr, lmr, vR, PR, Ft);
      tetrad_to_coordinate(mf, T, Ft, out);
#pragma unroll
      for (int f = 0; f < NM; ++f) flux[f * A.fs + q] = out[f];
      accumulate_flux(A, dir, q, out);
      continue;
    }
    phys_flux<dir>(A.eos, mf, pl, UL, FL, lpl, lml);
    phys_flux<dir>(A.eos, mf, pr, UR, FR, lpr, lmr);
    const double ap = fmax(0.0, fmax(lpl, lpr)), am = fmin(0.0, fmin(lml, lmr));
    const double den = (ap - am > 0.0) ? ap - am : 1.0;
    double out[NM];
#pragma unroll
    for (int f = 0; f < NM; ++f) {
      out[f] = (ap * FL[f] - am * FR[f] + ap * am * (UR[f] - UL[f])) / den;
      flux[f * A.fs + q] = out[f];
    }
    accumulate_flux(A, dir, q, out);
  }
}

// 4th-order centred first derivative of a metric quantity computed by `get`
// at the cells q + k st (k = -2..2)
template <class G>
__device__ __forceinline__ double d1c(const G& get, long long q, long long st, double ih12) {
  return (8.0 * (get(q + st) - get(q - st)) - (get(q + 2 * st) - get(q - 2 * st))) * ih12;
}

__global__ void __launch_bounds__(128) matter_update_kernel(MatterArgs A) {
  const long long nact = (long long)A.n[0] * A.n[1] * A.n[2];
  const int ring = A.lev->ring;
  const int s = A.stage;
  const double* __restrict__ u = z4c_stage_state(A, ring);
  const double* __restrict__ prim = A.P->mprim;
  const double* __restrict__ flux = A.P->mflux;
  const long long fs = A.fs;
  const long long st[3] = {1, A.sy, A.sz};
  const double ih = 1.0 / A.dx, ih12 = 1.0 / (12.0 * A.dx);
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < nact;
       id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % A.n[0]);
    const int j = (int)((id / A.n[0]) % A.n[1]);
    const int k = (int)(id / ((long long)A.n[0] * A.n[1]));
    const long long q = (i + GH) + (j + GH) * A.sy + (k + GH) * A.sz;
    double rhs[NM];
#pragma unroll
    for (int f = 0; f < NM; ++f) rhs[f] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double* Fd = flux + (long long)d * NM * fs;
#pragma unroll
      for (int f = 0; f < NM; ++f) rhs[f] -= (Fd[f * fs + q] - Fd[f * fs + q - st[d]]) * ih;
    }
    // sources at the cell
    Met m;
    double K_ll[6];
    metric_at(u, q, fs, m, K_ll);
    double pr[NM];
#pragma unroll
    for (int f = 0; f < NM; ++f) pr[f] = prim[f * fs + q];
    double U[NM], w, h, P;
    prim2con(A.eos, m, pr, U, w, h, P);
    const double rho = pr[0];
    const double ul[3] = {pr[2], pr[3], pr[4]};
    double uu[3];
    raise3(m.gu, ul, uu);
    const double E = rho * h * w * w - P;
    double J[3], Ju[3], Suu[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) J[a] = rho * h * w * ul[a];
    raise3(m.gu, J, Ju);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) Suu[S2(a, b)] = rho * h * uu[a] * uu[b] + P * m.gu[S2(a, b)];
    double dal[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dal[d] = d1c([&](long long p) { return __ldg(u + F_ALP * fs + p); }, q, st[d], ih12);
      // gamma_jk = gt_jk / W^2 at the four neighbours (one reciprocal each)
      double iw2[4];
      const int off[4] = {1, -1, 2, -2};
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const double Wp = __ldg(u + F_W * fs + q + off[o] * st[d]);
        iw2[o] = 1.0 / (Wp * Wp);
      }
      double sgd = 0.0;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const double* ga = u + (F_GXX + a) * fs + q;
        const double gp1 = __ldg(ga + st[d]) * iw2[0], gm1 = __ldg(ga - st[d]) * iw2[1];
        const double gp2 = __ldg(ga + 2 * st[d]) * iw2[2], gm2 = __ldg(ga - 2 * st[d]) * iw2[3];
        const double dg = (8.0 * (gp1 - gm1) - (gp2 - gm2)) * ih12;
        sgd += ((a == 0 || a == 3 || a == 5) ? 1.0 : 2.0) * Suu[a] * dg;
      }
      double jdb = 0.0;
#pragma unroll
      for (int b = 0; b < 3; ++b)
        jdb += J[b] * d1c([&](long long p) { return __ldg(u + (F_BETX + b) * fs + p); }, q, st[d], ih12);
      rhs[1 + d] += m.sg * (-E * dal[d] + jdb + 0.5 * m.al * sgd);
    }
    double SK = 0.0;
#pragma unroll
    for (int a = 0; a < 6; ++a) SK += ((a == 0 || a == 3 || a == 5) ? 1.0 : 2.0) * Suu[a] * K_ll[a];
    rhs[4] += m.sg * (m.al * SK - (Ju[0] * dal[0] + Ju[1] * dal[1] + Ju[2] * dal[2]));
    if (s == 0) {
#pragma unroll
      for (int f = 0; f < NM; ++f) A.out[f * fs + q] = rhs[f];
      continue;
    }
    // RK4 stage update (the spacetime's weights)
    double* __restrict__ un = A.P->mcons[ring];
    double* __restrict__ y = A.P->mcons[B_Y];
    double* __restrict__ out = A.P->mcons[stage_out_slot(s, ring)];
    const double bw = (s == 1 || s == 4) ? (1.0 / 6.0) : (1.0 / 3.0);
    const double cw = (s == 3) ? 1.0 : 0.5;
    bool bad = false;
#pragma unroll
    for (int f = 0; f < NM; ++f) {
      const long long o = f * fs + q;
      double v;
      if (s == 4) {
        v = y[o] + bw * A.dt * rhs[f];
      } else {
        const double a = un[o];
        y[o] = (s == 1 ? a : y[o]) + bw * A.dt * rhs[f];
        v = a + cw * A.dt * rhs[f];
      }
      out[o] = v;
      bad |= !isfinite(v);
    }
    if (bad) atomicOr(A.err, (unsigned)ERR_NONFINITE);
  }
}

__global__ void __launch_bounds__(128) matter_prim2con_kernel(MatterArgs A) {
  const long long ntot = (long long)A.NX * A.NY * A.NZ;
  const int ring = A.lev->ring;
  const double* __restrict__ u = A.P->buf[ring];
  double* __restrict__ cons = A.P->mcons[ring];
  double* __restrict__ prim = A.P->mprim;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < ntot;
       id += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(id % A.NX), J = (int)((id / A.NX) % A.NY), K = (int)(id / ((long long)A.NX * A.NY));
    const long long q = I + J * A.sy + K * A.sz;
    Met m;
    metric_at(u, q, A.fs, m, nullptr);
    double pr[NM], c[NM], w, h, P;
#pragma unroll
    for (int f = 0; f < NM; ++f) pr[f] = prim[f * A.fs + q];
    prim2con(A.eos, m, pr, c, w, h, P);
#pragma unroll
    for (int f = 0; f < NM; ++f) cons[f * A.fs + q] = c[f];
    prim[NM * A.fs + q] = w;
  }
}

// ------------------------------------------------------------------ refinement boundary (Sec. 2.2.1)

__device__ __forceinline__ int fdiv2(int i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

__device__ __forceinline__ long long shell_count(const DevPatch* P) {
  return (long long)P->NX * P->NY * P->NZ - (long long)(P->NX - 2 * GH) * (P->NY - 2 * GH) * (P->NZ - 2 * GH);
}

// Average over the left (right: the right) half of cell c from the cell
// averages a..e of cells -2..2: the left-half averages of the three
// quadratic interpolants, (-a + 4b + 5c)/8, (b + 8c - d)/8, (11c - 4d + e)/8,
// weighted gamma_k / (eps + beta_k)^2 (gamma = 3/16, 5/8, 3/16, the 5-cell
// quartic; beta_k the Jiang-Shu indicators; eps = 1e-6 times the mean square
// of a..e), normalised; the right half is 2c - left (conservative).
__device__ __forceinline__ double weno_half(double a, double b, double c, double d, double e, bool right) {
  const double L0 = (-a + 4.0 * b + 5.0 * c) / 8.0, L1 = (b + 8.0 * c - d) / 8.0, L2 = (11.0 * c - 4.0 * d + e) / 8.0;
  const double t0 = a - 2.0 * b + c, t1 = b - 2.0 * c + d, t2 = c - 2.0 * d + e;
  const double v0 = a - 4.0 * b + 3.0 * c, v1 = b - d, v2 = 3.0 * c - 4.0 * d + e;
  const double B0 = 13.0 / 12.0 * t0 * t0 + 0.25 * v0 * v0;
  const double B1 = 13.0 / 12.0 * t1 * t1 + 0.25 * v1 * v1;
  const double B2 = 13.0 / 12.0 * t2 * t2 + 0.25 * v2 * v2;
  const double eps = 1e-6 * (a * a + b * b + c * c + d * d + e * e) / 5.0 + 1e-300;
  const double r0 = eps + B0, r1 = eps + B1, r2 = eps + B2;
  const double a0 = (3.0 / 16.0) / (r0 * r0), a1 = (5.0 / 8.0) / (r1 * r1), a2 = (3.0 / 16.0) / (r2 * r2);
  const double left = (a0 * L0 + a1 * L1 + a2 * L2) / (a0 + a1 + a2);
  return right ? 2.0 * c - left : left;
}

// 6-point Lagrange weights at +1/4 (nodes -2..3) and -1/4 (nodes -3..2)
__constant__ double c_lp[6] = {77.0 / 8192, -693.0 / 8192, 6930.0 / 8192, 2310.0 / 8192, -495.0 / 8192, 63.0 / 8192};
__constant__ double c_lm[6] = {63.0 / 8192, -495.0 / 8192, 2310.0 / 8192, 6930.0 / 8192, -693.0 / 8192, 77.0 / 8192};

// The parent's fluid at cell ci (active index, ghosts negative) of child C,
// from the parent's ring slot pr: D^ by the conservative WENO5 (x, y, z),
// eps and u_i by the tensor-product 6th-order Lagrange interpolation, the
// parent cell's D^ where the WENO value is not positive, trilinear eps where
// that or the Lagrange eps is not positive.  v = (D^, eps, u_x, u_y, u_z).
__device__ __forceinline__ void prolong_fluid_cell(const DevPatch* C, const DevPatch* P, int pr, const int ci[3],
                                                   double v[NM]) {
  const long long sy = P->px, sz = P->plane, fs = P->fstride;
  const double* __restrict__ D = P->mcons[pr];
  const double* __restrict__ prim = P->mprim;
  int pc[3];
  bool odd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    pc[d] = C->off[d] + fdiv2(ci[d]) + GH;
    odd[d] = (ci[d] & 1) != 0;
  }
  auto at = [&](const double* f, int x, int y, int z) { return f[x + y * sy + (long long)z * sz]; };
  // D^: WENO along x (5 x 5 rows), then y (5 rows), then z
  double vz[5];
  for (int c = 0; c < 5; ++c) {
    double vy[5];
    const int z = pc[2] - 2 + c;
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      const int y = pc[1] - 2 + b;
      vy[b] = weno_half(at(D, pc[0] - 2, y, z), at(D, pc[0] - 1, y, z), at(D, pc[0], y, z), at(D, pc[0] + 1, y, z),
                        at(D, pc[0] + 2, y, z), odd[0]);
    }
    vz[c] = weno_half(vy[0], vy[1], vy[2], vy[3], vy[4], odd[1]);
  }
  double Dv = weno_half(vz[0], vz[1], vz[2], vz[3], vz[4], odd[2]);
  const bool bad = !(Dv > 0.0);
  if (bad) Dv = at(D, pc[0], pc[1], pc[2]);
  // eps, u_i: 6th-order Lagrange (nodes -3..2 for even child indices, -2..3 for odd)
  double lag[4] = {0.0, 0.0, 0.0, 0.0};
  const int n0[3] = {odd[0] ? -2 : -3, odd[1] ? -2 : -3, odd[2] ? -2 : -3};
  for (int c = 0; c < 6; ++c)
    for (int b = 0; b < 6; ++b)
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const double w = (odd[0] ? c_lp[a] : c_lm[a]) * (odd[1] ? c_lp[b] : c_lm[b]) * (odd[2] ? c_lp[c] : c_lm[c]);
        const long long q = (pc[0] + n0[0] + a) + (pc[1] + n0[1] + b) * sy + (long long)(pc[2] + n0[2] + c) * sz;
#pragma unroll
        for (int f = 0; f < 4; ++f) lag[f] += w * prim[(1 + f) * fs + q];
      }
  double eps = lag[0];
  if (bad || !(eps > 0.0)) {  // trilinear: 3/4 of the cell, 1/4 of the neighbour on the child's side
    const int o[3] = {odd[0] ? 1 : -1, odd[1] ? 1 : -1, odd[2] ? 1 : -1};
    double vzl[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      double vyl[2];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int y = pc[1] + b * o[1], z = pc[2] + c * o[2];
        vyl[b] = 0.75 * at(prim + fs, pc[0], y, z) + 0.25 * at(prim + fs, pc[0] + o[0], y, z);
      }
      vzl[c] = 0.75 * vyl[0] + 0.25 * vyl[1];
    }
    eps = 0.75 * vzl[0] + 0.25 * vzl[1];
  }
  v[0] = Dv;
  v[1] = eps;
  v[2] = lag[1];
  v[3] = lag[2];
  v[4] = lag[3];
}

// one thread per ghost-shell cell of a child: the parent's current fluid
// prolonged, cached in the child's slot of the parent's current ring slot
__global__ void __launch_bounds__(128) matter_prolong_kernel(MatterAmrArgs A) {
  const DevPatch* C = A.patches + A.child_ids[blockIdx.y];
  const DevPatch* P = A.patches + C->parent;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= shell_count(C)) return;
  int i, j, k;
  shell_ijk(id, C->NX, C->NY, C->NZ, i, j, k);
  // a child on z = 0 (equatorial symmetry): its z < 0 ghosts are reflected,
  // and their stencils would reach below the parent's array
  if (C->zrefl && k < GH) return;
  const int pr = A.plev->ring;
  const int ci[3] = {i - GH, j - GH, k - GH};
  double v[NM];
  prolong_fluid_cell(C, P, pr, ci, v);
  double* __restrict__ cache = C->mgsh[pr];
  const long long fc = C->fstride;
  const long long qc = i + (long long)j * C->px + (long long)k * C->plane;
#pragma unroll
  for (int f = 0; f < NM; ++f) cache[f * fc + qc] = v[f];
}

// The fluid of a patch shifted by sh child cells (its geometry already the
// new one, the spacetime already moved): every cell of its array that was
// active before and is active now keeps (conserved, primitives, w); every
// other cell takes the parent's prolongation (prolong_fluid_cell) with
// rho = D^ / (sqrt(gamma) w) on the new metric and its conserved variables.
// Output to the patch's face-flux arrays (dead between steps): fields 0..4
// the conserved variables, 5..10 the primitives and w.
__global__ void __launch_bounds__(128) matter_move_kernel(MatterMoveArgs A) {
  const DevPatch* C = A.patches + A.patch;
  const DevPatch* P = A.patches + C->parent;
  const long long ntot = (long long)C->NX * C->NY * C->NZ;
  const long long sy = C->px, sz = C->plane, fs = C->fstride;
  const double* __restrict__ cons = C->mcons[A.ring];
  const double* __restrict__ prim = C->mprim;
  const double* __restrict__ u = C->buf[A.ring];
  double* __restrict__ out = C->mflux;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < ntot;
       id += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(id % C->NX), J = (int)((id / C->NX) % C->NY), K = (int)(id / ((long long)C->NX * C->NY));
    const long long q = I + J * sy + K * sz;
    const int ci[3] = {I - GH, J - GH, K - GH};
    bool copy = true;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      copy = copy && ci[d] >= 0 && ci[d] < C->n[d] && ci[d] + A.sh[d] >= 0 && ci[d] + A.sh[d] < C->n[d];
    if (copy) {
      const long long qo = q + A.sh[0] + A.sh[1] * sy + A.sh[2] * sz;
#pragma unroll
      for (int f = 0; f < NM; ++f) out[f * fs + q] = cons[f * fs + qo];
#pragma unroll
      for (int f = 0; f < NMP; ++f) out[(NM + f) * fs + q] = prim[f * fs + qo];
      continue;
    }
    if (C->zrefl && K < GH) {  // reflected afterwards
#pragma unroll
      for (int f = 0; f < NM + NMP; ++f) out[f * fs + q] = 0.0;
      continue;
    }
    double v[NM];
    prolong_fluid_cell(C, P, A.pring, ci, v);
    Met m;
    metric_at(u, q, fs, m, nullptr);
    const double ul[3] = {v[2], v[3], v[4]};
    double uu[3];
    raise3(m.gu, ul, uu);
    const double w = sqrt(1.0 + ul[0] * uu[0] + ul[1] * uu[1] + ul[2] * uu[2]);
    double pr[NM] = {v[0] / (m.sg * w), v[1], v[2], v[3], v[4]}, c[NM], w2, h, Pp;
    prim2con(A.eos, m, pr, c, w2, h, Pp);
    bool finite = true;
#pragma unroll
    for (int f = 0; f < NM; ++f) {
      out[f * fs + q] = c[f];
      out[(NM + f) * fs + q] = pr[f];
      finite = finite && isfinite(c[f]);
    }
    out[(NM + NM) * fs + q] = w2;
    if (!finite) atomicOr(A.err, (unsigned)ERR_NONFINITE);
  }
}

// Density maximum (a neutron star is located there, Sec. 2.2.1): per block
// the largest rest-mass density over the patch's active cells and the first
// active index (z, y, x order) that holds it; NaN cells never win.
__device__ __forceinline__ void argmax_merge(double& v, long long& i, double v2, long long i2) {
  if (i2 >= 0 && (i < 0 || v2 > v || (v2 == v && i2 < i))) {
    v = v2;
    i = i2;
  }
}

__global__ void __launch_bounds__(256) density_max_kernel(const DevPatch* patches, int patch, double* part) {
  const DevPatch* P = patches + patch;
  const long long nact = (long long)P->n[0] * P->n[1] * P->n[2];
  double best = 0.0;
  long long bi = -1;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < nact;
       id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % P->n[0]), j = (int)((id / P->n[0]) % P->n[1]);
    const int k = (int)(id / ((long long)P->n[0] * P->n[1]));
    const double r = P->mprim[(i + GH) + (long long)(j + GH) * P->px + (long long)(k + GH) * P->plane];
    if (r == r) argmax_merge(best, bi, r, id);
  }
  __shared__ double sv[256];
  __shared__ long long si[256];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      double v = sv[threadIdx.x];
      long long ix = si[threadIdx.x];
      argmax_merge(v, ix, sv[threadIdx.x + h], si[threadIdx.x + h]);
      sv[threadIdx.x] = v;
      si[threadIdx.x] = ix;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sv[0];
    part[2 * blockIdx.x + 1] = (double)si[0];
  }
}

// the blocks' pairs reduced the same way; the result in part[0], part[1]
__global__ void __launch_bounds__(256) density_max_final_kernel(double* part, int nblocks) {
  double best = 0.0;
  long long bi = -1;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) argmax_merge(best, bi, part[2 * b], (long long)part[2 * b + 1]);
  __shared__ double sv[256];
  __shared__ long long si[256];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      double v = sv[threadIdx.x];
      long long ix = si[threadIdx.x];
      argmax_merge(v, ix, sv[threadIdx.x + h], si[threadIdx.x + h]);
      sv[threadIdx.x] = v;
      si[threadIdx.x] = ix;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[0] = sv[0];
    part[1] = (double)si[0];
  }
}

// ghost cells of a level > 0 fluid: the time interpolant of the cached
// prolongations, rho = D^ / (sqrt(gamma) w) with this patch's stage metric
__global__ void __launch_bounds__(128) matter_child_ghost_kernel(MatterArgs A) {
  const DevPatch* C = A.P;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= shell_count(C)) return;
  int i, j, k;
  shell_ijk(id, C->NX, C->NY, C->NZ, i, j, k);
  if (C->zrefl && k < GH) return;  // reflected afterwards (not prolonged)
  const int pr = A.plev->ring;
  const bool q3 = A.plev->nvalid >= 3;
  const double w0 = q3 ? A.wq[0] : 0.0, w1 = q3 ? A.wq[1] : A.wl[1], w2 = q3 ? A.wq[2] : A.wl[2];
  const double* __restrict__ g0 = C->mgsh[(pr + 1) % 3];
  const double* __restrict__ g1 = C->mgsh[(pr + 2) % 3];
  const double* __restrict__ g2 = C->mgsh[pr];
  const long long fs = A.fs;
  const long long q = i + (long long)j * A.sy + (long long)k * A.sz;
  double v[NM];
#pragma unroll
  for (int f = 0; f < NM; ++f) {
    const long long o = f * fs + q;
    // (slots of zero weight are not read: they may hold no data yet)
    double t = (w1 != 0.0 ? w1 * g1[o] : 0.0);
    if (q3 && w0 != 0.0) t = w0 * g0[o] + t;
    v[f] = t + (w2 != 0.0 ? w2 * g2[o] : 0.0);
  }
  Met m;
  metric_at(z4c_stage_state(A, A.lev->ring), q, fs, m, nullptr);
  const double ul[3] = {v[2], v[3], v[4]};
  double uu[3];
  raise3(m.gu, ul, uu);
  const double w = sqrt(1.0 + ul[0] * uu[0] + ul[1] * uu[1] + ul[2] * uu[2]);
  double* __restrict__ prim = C->mprim;
  prim[q] = v[0] / (m.sg * w);
  prim[fs + q] = v[1];
  prim[2 * fs + q] = v[2];
  prim[3 * fs + q] = v[3];
  prim[4 * fs + q] = v[4];
  prim[NM * fs + q] = w;
}

// parent cells under a child's active cells <- mean of their 8 children
__global__ void __launch_bounds__(128) matter_restrict_kernel(MatterAmrArgs A) {
  const DevPatch* C = A.patches + A.child_ids[blockIdx.y];
  const DevPatch* P = A.patches + C->parent;
  const int mx = C->n[0] / 2, my = C->n[1] / 2, mz = C->n[2] / 2;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)mx * my * mz) return;
  const int I = (int)(id % mx), J = (int)((id / mx) % my), K = (int)(id / ((long long)mx * my));
  const double* __restrict__ cc = C->mcons[A.clev->ring];
  double* __restrict__ cp = P->mcons[A.plev->ring];
  const long long sy = C->px, sz = C->plane, fc = C->fstride;
  const long long q0 = (2 * I + GH) + (2 * J + GH) * sy + (long long)(2 * K + GH) * sz;
  const long long qp = (I + C->off[0] + GH) + (J + C->off[1] + GH) * P->px + (long long)(K + C->off[2] + GH) * P->plane;
#pragma unroll
  for (int f = 0; f < NM; ++f) {
    const double* x = cc + f * fc + q0;
    const double s = x[0] + x[1] + x[sy] + x[sy + 1] + x[sz] + x[sz + 1] + x[sz + sy] + x[sz + sy + 1];
    cp[f * P->fstride + qp] = 0.125 * s;
  }
}

// parent cells outside a child next to its boundary: the parent step's
// boundary-face flux replaced by the child's (4 fine faces, 2 steps averaged)
__global__ void __launch_bounds__(128) matter_reflux_kernel(MatterAmrArgs A) {
  const DevPatch* C = A.patches + A.child_ids[blockIdx.y];
  const DevPatch* P = A.patches + C->parent;
  const int m[3] = {C->n[0] / 2, C->n[1] / 2, C->n[2] / 2};
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int d = 0, side = 0;
  for (; d < 3; ++d) {
    const long long nfd = 2LL * m[(d + 1) % 3] * m[(d + 2) % 3];
    if (id < nfd) break;
    id -= nfd;
  }
  if (d == 3) return;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;  // tangential directions, t1 < t2
  const long long per = (long long)m[t1] * m[t2];
  side = (int)(id / per);
  id -= side * per;
  const int T1 = (int)(id % m[t1]), T2 = (int)(id / m[t1]);
  const long long sp[3] = {1, P->px, P->plane}, sc[3] = {1, C->px, C->plane};
  // parent face (array index along d), the parent cell outside, the child face
  const int mp = side ? C->off[d] + m[d] - 1 + GH : C->off[d] - 1 + GH;
  const int cell = side ? C->off[d] + m[d] + GH : C->off[d] - 1 + GH;
  const int mc = side ? C->n[d] - 1 + GH : GH - 1;
  const long long pt = (C->off[t1] + T1 + GH) * sp[t1] + (long long)(C->off[t2] + T2 + GH) * sp[t2];
  const long long qf = mp * sp[d] + pt, qcell = cell * sp[d] + pt;
  const long long qc = mc * sc[d] + (2 * T1 + GH) * sc[t1] + (long long)(2 * T2 + GH) * sc[t2];
  const double* __restrict__ fp = P->mfs + (long long)d * NM * P->fstride;
  const double* __restrict__ fcs = C->mfa + (long long)d * NM * C->fstride;
  double* __restrict__ cp = P->mcons[A.plev->ring];
  const double h = P->dx, sgn = side ? 1.0 : -1.0;
#pragma unroll
  for (int f = 0; f < NM; ++f) {
    const double* x = fcs + f * C->fstride + qc;
    // the fine faces in array order: (t2, t1) = (0,0), (0,1), (1,0), (1,1)
    const double fine = 0.25 * (x[0] + x[sc[t1]] + x[sc[t2]] + x[sc[t2] + sc[t1]]);
    cp[f * P->fstride + qcell] += (A.dt_parent / h) * (fine - fp[f * P->fstride + qf]) * sgn;
  }
}

int blocks_for(long long n) {
  long long b = (n + 127) / 128;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

void launch_matter_prep(const MatterArgs& a, cudaStream_t st) {
  matter_prep_kernel<<<blocks_for((long long)a.n[0] * a.n[1] * a.n[2]), 128, 0, st>>>(a);
}
void launch_matter_ghosts(const MatterArgs& a, cudaStream_t st) {
  matter_ghost_kernel<<<blocks_for((long long)a.NX * a.NY * a.NZ), 128, 0, st>>>(a);
}
void launch_matter_flux(const MatterArgs& a, int dir, cudaStream_t st) {
  const int a1 = (dir + 1) % 3, a2 = (dir + 2) % 3;
  const int nb = blocks_for((long long)(a.n[dir] + 1) * a.n[a1] * a.n[a2]);
  if (dir == 0)
    matter_flux_kernel<0><<<nb, 128, 0, st>>>(a);
  else if (dir == 1)
    matter_flux_kernel<1><<<nb, 128, 0, st>>>(a);
  else
    matter_flux_kernel<2><<<nb, 128, 0, st>>>(a);
}
void launch_matter_update(const MatterArgs& a, cudaStream_t st) {
  matter_update_kernel<<<blocks_for((long long)a.n[0] * a.n[1] * a.n[2]), 128, 0, st>>>(a);
}
void launch_matter_zreflect(const MatterArgs& a, cudaStream_t st) {
  matter_zreflect_kernel<<<blocks_for((long long)GH * a.NX * a.NY), 128, 0, st>>>(a);
}
void launch_matter_prim2con(const MatterArgs& a, cudaStream_t st) {
  matter_prim2con_kernel<<<blocks_for((long long)a.NX * a.NY * a.NZ), 128, 0, st>>>(a);
}
void launch_matter_child_ghosts(const MatterArgs& a, cudaStream_t st) {
  const long long sh = (long long)a.NX * a.NY * a.NZ - (long long)a.n[0] * a.n[1] * a.n[2];
  matter_child_ghost_kernel<<<(unsigned)((sh + 127) / 128), 128, 0, st>>>(a);
}
void launch_matter_prolong(const MatterAmrArgs& a, int nchildren, long long max_shell, cudaStream_t st) {
  if (nchildren == 0 || max_shell == 0) return;
  matter_prolong_kernel<<<dim3((unsigned)((max_shell + 127) / 128), nchildren), 128, 0, st>>>(a);
}
void launch_matter_move(const MatterMoveArgs& a, long long ncells, cudaStream_t st) {
  matter_move_kernel<<<blocks_for(ncells), 128, 0, st>>>(a);
}
void launch_density_max(const DevPatch* patches, int patch, long long nact, double* part, int max_blocks,
                        cudaStream_t st) {
  long long b = (nact + 255) / 256;
  if (b > max_blocks) b = max_blocks;
  if (b < 1) b = 1;
  density_max_kernel<<<(unsigned)b, 256, 0, st>>>(patches, patch, part);
  density_max_final_kernel<<<1, 256, 0, st>>>(part, (int)b);
}
void launch_matter_restrict(const MatterAmrArgs& a, int nchildren, long long max_cells, cudaStream_t st) {
  if (nchildren == 0 || max_cells == 0) return;
  matter_restrict_kernel<<<dim3((unsigned)((max_cells + 127) / 128), nchildren), 128, 0, st>>>(a);
}
void launch_matter_reflux(const MatterAmrArgs& a, int nchildren, long long max_faces, cudaStream_t st) {
  if (nchildren == 0 || max_faces == 0) return;
  matter_reflux_kernel<<<dim3((unsigned)((max_faces + 127) / 128), nchildren), 128, 0, st>>>(a);
}

}  // namespace sacrak
