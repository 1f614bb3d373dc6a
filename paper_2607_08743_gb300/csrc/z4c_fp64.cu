// FP64 Z4c right-hand side fused with the classical RK4 stage update and the
// algebraic constraints (Sec. 2.1.1, 2.2 of the SACRA-K paper), plus the
// Hamiltonian / momentum constraint monitor (Sec. 2.3).
//
// One thread per active point.  The FP64 pipe of GB300 (measured about
// 1 TFLOP/s, 1/74 of FP32) bounds this path, so the code is written to keep
// the FP64 instruction count low: unscaled stencil sums multiplied once by
// 1/(12h) or 1/(144h^2), contractions of the Christoffel symbols through the
// partially raised symbol X[j][k][l] = gt^lm Gt_jkm, and second derivatives
// of gt consumed into the Ricci tensor as they are formed.
#include <mutex>

#include "../../include/sacrak.h"
#include "sacrak_dev.cuh"

namespace sacrak {

struct PointState {
  double W, gt[6], Kh, Th, At[6], Gam[3], al, be[3], Bv[3];
};

__device__ __forceinline__ void load_centre(const double* __restrict__ u, long long q,
                                            long long fs, PointState& c) {
  c.W = __ldg(u + F_W * fs + q);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    c.gt[a] = __ldg(u + (F_GXX + a) * fs + q);
    c.At[a] = __ldg(u + (F_AXX + a) * fs + q);
  }
  c.Kh = __ldg(u + F_KH * fs + q);
  c.Th = __ldg(u + F_TH * fs + q);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    c.Gam[i] = __ldg(u + (F_GAMX + i) * fs + q);
    c.be[i] = __ldg(u + (F_BETX + i) * fs + q);
    c.Bv[i] = __ldg(u + (F_BX + i) * fs + q);
  }
  c.al = __ldg(u + F_ALP * fs + q);
}

// inverse of a symmetric 3x3 matrix
__device__ __forceinline__ void sym_inv(const double g[6], double gu[6]) {
  double c0 = g[3] * g[5] - g[4] * g[4];
  double c1 = g[2] * g[4] - g[1] * g[5];
  double c2 = g[1] * g[4] - g[2] * g[3];
  double det = g[0] * c0 + g[1] * c1 + g[2] * c2;
  double id = 1.0 / det;
  gu[0] = c0 * id;
  gu[1] = c1 * id;
  gu[2] = c2 * id;
  gu[3] = (g[0] * g[5] - g[2] * g[2]) * id;
  gu[4] = (g[1] * g[2] - g[0] * g[4]) * id;
  gu[5] = (g[0] * g[3] - g[1] * g[1]) * id;
}

// sum_{l,m} S^{lm} T_{lm} of two symmetric tensors
__device__ __forceinline__ double sym_contract(const double S[6], const double T[6]) {
  return S[0] * T[0] + S[3] * T[3] + S[5] * T[5] + 2.0 * (S[1] * T[1] + S[2] * T[2] + S[4] * T[4]);
}

// Geometry shared by the RHS and the constraint monitor.
struct Geo {
  double gtu[6];
  double dW[3], dal[3];
  double Gu[3][6];    // Gt^i_jk
  double Gd[3];       // Gamd^i
  double Ric[6];      // R_ij
  double DDa[6];      // D_i D_j alpha (physical)
  double Lapa;        // D^i D_i alpha
  double Rsc;         // R
};

// G.dW, G.dal and dgt (first derivatives, scaled) are given; d2(g, d) is the
// scaled second derivative along axis d of W (g = 0), gt_a (g = 1 + a) and
// alpha (g = 7); the mixed second derivatives are formed here.
template <class D2>
__device__ __forceinline__ void geometry_t(const double* __restrict__ u, long long q,
                                           const long long st[3], long long fs, double c11,
                                           const PointState& c, Geo& G, const double dgt[3][6],
                                           const double dGam[3][3], const D2& d2) {
  sym_inv(c.gt, G.gtu);
  const double* gtu = G.gtu;

  // Christoffel symbols of the first kind from the first derivatives of gt
  double Gl[3][6];  // Gt_ijk = 1/2 (d_j gt_ik + d_k gt_ij - d_i gt_jk)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = j; k < 3; ++k)
        Gl[i][S2(j, k)] = 0.5 * (dgt[j][S2(i, k)] + dgt[k][S2(i, j)] - dgt[i][S2(j, k)]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 6; ++a)
      G.Gu[i][a] = gtu[S2(i, 0)] * Gl[0][a] + gtu[S2(i, 1)] * Gl[1][a] + gtu[S2(i, 2)] * Gl[2][a];
#pragma unroll
  for (int i = 0; i < 3; ++i) G.Gd[i] = sym_contract(gtu, G.Gu[i]);

  // X[j][k][l] = gt^lm Gt_jkm
  double X[3][3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        X[j][k][l] = gtu[S2(l, 0)] * Gl[j][S2(k, 0)] + gtu[S2(l, 1)] * Gl[j][S2(k, 1)] +
                     gtu[S2(l, 2)] * Gl[j][S2(k, 2)];

  // conformal Ricci tensor
  double Rt[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int ij = S2(i, j);
      // -1/2 gt^lm d_l d_m gt_ij
      const double* f = u + (F_GXX + ij) * fs;
      double dd[6];
      dd[0] = d2(1 + ij, 0);
      dd[3] = d2(1 + ij, 1);
      dd[5] = d2(1 + ij, 2);
      dd[1] = d11u(f, q, st[0], st[1]) * c11;
      dd[2] = d11u(f, q, st[0], st[2]) * c11;
      dd[4] = d11u(f, q, st[1], st[2]) * c11;
      double r = -0.5 * sym_contract(gtu, dd);
      // gt_k(i d_j) Gamt^k
      double t2 = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) t2 += c.gt[S2(k, i)] * dGam[j][k] + c.gt[S2(k, j)] * dGam[i][k];
      r += 0.5 * t2;
      // Gamd^k Gt_(ij)k
      double t3 = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) t3 += G.Gd[k] * (Gl[i][S2(j, k)] + Gl[j][S2(i, k)]);
      r += 0.5 * t3;
      // gt^lm (Gt^k_li Gt_jkm + Gt^k_lj Gt_ikm + Gt^k_im Gt_klj)
      double t4 = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
          t4 += G.Gu[k][S2(l, i)] * X[j][k][l] + G.Gu[k][S2(l, j)] * X[i][k][l] +
                G.Gu[k][S2(i, l)] * X[k][j][l];
      Rt[ij] = r + t4;
    }

  // conformal-factor and lapse second covariant derivatives
  const double W = c.W;
  const double iW = 1.0 / W;
  double DDW[6], DDal[6];
  {
    const double* fW = u + F_W * fs;
    const double* fa = u + F_ALP * fs;
    double ddW[6], dda[6];
    ddW[0] = d2(0, 0);
    ddW[3] = d2(0, 1);
    ddW[5] = d2(0, 2);
    ddW[1] = d11u(fW, q, st[0], st[1]) * c11;
    ddW[2] = d11u(fW, q, st[0], st[2]) * c11;
    ddW[4] = d11u(fW, q, st[1], st[2]) * c11;
    dda[0] = d2(7, 0);
    dda[3] = d2(7, 1);
    dda[5] = d2(7, 2);
    dda[1] = d11u(fa, q, st[0], st[1]) * c11;
    dda[2] = d11u(fa, q, st[0], st[2]) * c11;
    dda[4] = d11u(fa, q, st[1], st[2]) * c11;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      DDW[a] = ddW[a] - (G.Gu[0][a] * G.dW[0] + G.Gu[1][a] * G.dW[1] + G.Gu[2][a] * G.dW[2]);
      DDal[a] = dda[a] - (G.Gu[0][a] * G.dal[0] + G.Gu[1][a] * G.dal[1] + G.Gu[2][a] * G.dal[2]);
    }
  }
  double dWW[6], dWa[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      dWW[S2(i, j)] = G.dW[i] * G.dW[j];
      dWa[S2(i, j)] = G.dW[i] * G.dal[j] + G.dW[j] * G.dal[i];
    }
  const double trDDW = sym_contract(gtu, DDW);
  const double dWdW = sym_contract(gtu, dWW);
  const double dWda = 0.5 * sym_contract(gtu, dWa);
  const double trDDa = sym_contract(gtu, DDal);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    G.Ric[a] = Rt[a] + (DDW[a] + c.gt[a] * trDDW) * iW - 2.0 * c.gt[a] * dWdW * (iW * iW);
    G.DDa[a] = DDal[a] + (dWa[a] - c.gt[a] * dWda) * iW;
  }
  G.Rsc = W * W * sym_contract(gtu, G.Ric);
  G.Lapa = W * W * trDDa - W * dWda;
}

// second derivatives along the axes formed on demand (constraint monitor,
// surface diagnostics)
struct D2Direct {
  const double* u;
  long long q, fs;
  const long long* st;
  double c2;
  const PointState* c;
  __device__ __forceinline__ double operator()(int g, int d) const {
    const int f = g == 0 ? F_W : (g == 7 ? F_ALP : F_GXX + g - 1);
    const double f0 = g == 0 ? c->W : (g == 7 ? c->al : c->gt[g - 1]);
    return d2u(u + f * fs, q, st[d], f0) * c2;
  }
};

__device__ __forceinline__ void geometry(const double* __restrict__ u, long long q,
                                         const long long st[3], long long fs, double c1,
                                         double c2, double c11, const PointState& c, Geo& G,
                                         double dGam[3][3], double dbe[3][3]) {
  double dgt[3][6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int a = 0; a < 6; ++a) dgt[d][a] = d1u(u + (F_GXX + a) * fs, q, st[d]) * c1;
    G.dW[d] = d1u(u + F_W * fs, q, st[d]) * c1;
    G.dal[d] = d1u(u + F_ALP * fs, q, st[d]) * c1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dGam[d][i] = d1u(u + (F_GAMX + i) * fs, q, st[d]) * c1;
      dbe[d][i] = d1u(u + (F_BETX + i) * fs, q, st[d]) * c1;
    }
  }
  geometry_t(u, q, st, fs, c11, c, G, dgt, dGam, D2Direct{u, q, fs, st, c2, &c});
}

// Per-thread stash of the fused stencil pass in shared memory, one column per
// thread ([slot][thread]): each field's advection + dissipation, and the
// second derivatives along the axes of W, gt (6), alpha and beta (3).
constexpr int STAGE_THREADS = 128;
constexpr int ST_ADV = 0;        // NF slots
constexpr int ST_D2 = NF;        // 11 groups x 3 axes: 0 W, 1..6 gt, 7 alpha, 8..10 beta
constexpr int ST_N = NF + 33;
constexpr size_t STAGE_SMEM = (size_t)ST_N * STAGE_THREADS * sizeof(double);

struct Stash {
  double* p;  // this thread's column
  __device__ __forceinline__ double& operator[](int slot) const { return p[slot * STAGE_THREADS]; }
};
struct D2Stash {
  Stash S;
  __device__ __forceinline__ double operator()(int g, int d) const { return S[ST_D2 + 3 * g + d]; }
};

// One field's stencils along the three axes from one read of f_-3 .. f_3:
// with d_k = f_k - f_-k and e_k = (f_k - f0) + (f_-k - f0), D1 = 8 d1 - d2 (the
// first derivative times 12h), D2 = 16 e1 - e2 (the second times 12h^2), and
// the return value, the field's advection along the shift plus dissipation,
//   sum_d [ b_d (21 d1 - 6 d2 + d3) + a_d (e3 - 6 e2 + 15 e1) ],
// b_d = beta^d / (24h), a_d = |beta^d| / (24h) + sigma_KO / (64h).  The lopsided
// upwind derivative (one point behind, three ahead along the shift) equals
// its antisymmetric part, (21 d1 - 6 d2 + d3) / (24h), plus |beta|/2 times the
// sixth difference e3 - 6 e2 + 15 e1 over 12h, for either sign of beta; the
// sixth difference is also the Kreiss-Oliger stencil.
template <bool WANT_D1, bool WANT_D2>
__device__ __forceinline__ double field_axes(const double* __restrict__ f, long long q, const long long st[3],
                                             double f0, const double b[3], const double a[3], double D1[3],
                                             double D2[3]) {
  double adk = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const long long o = st[d];
    const double p1 = __ldg(f + q + o), m1 = __ldg(f + q - o);
    const double p2 = __ldg(f + q + 2 * o), m2 = __ldg(f + q - 2 * o);
    const double p3 = __ldg(f + q + 3 * o), m3 = __ldg(f + q - 3 * o);
    const double d1 = p1 - m1, d2 = p2 - m2, d3 = p3 - m3;
    const double e1 = (p1 - f0) + (m1 - f0), e2 = (p2 - f0) + (m2 - f0), e3 = (p3 - f0) + (m3 - f0);
    if (WANT_D1) D1[d] = 8.0 * d1 - d2;
    if (WANT_D2) D2[d] = 16.0 * e1 - e2;
    adk += b[d] * ((21.0 * d1 - 6.0 * d2) + d3) + a[d] * ((e3 - 6.0 * e2) + 15.0 * e1);
  }
  return adk;
}

__device__ __forceinline__ void z4c_rhs_point(const double* __restrict__ u, long long q,
                                              long long sy, long long sz, long long fs,
                                              double h, const DevParams& prm, Stash S, double r[NF]) {
  const long long st[3] = {1, sy, sz};
  const double c1 = 1.0 / (12.0 * h);
  const double c2 = c1 / h;
  const double c11 = c1 * c1;
  PointState c;
  load_centre(u, q, fs, c);
  Geo G;
  double dgt[3][6], dGam[3][3], dbe[3][3], dKh[3], dTh[3];
  {
    const double hb = 0.5 * c1, cko = prm.sigma_ko / (64.0 * h);
    double wb[3], wa[3], t1[3], t2[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      wb[d] = c.be[d] * hb;
      wa[d] = fabs(c.be[d]) * hb + cko;
    }
    S[ST_ADV + F_W] = field_axes<true, true>(u + F_W * fs, q, st, c.W, wb, wa, t1, t2);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      G.dW[d] = t1[d] * c1;
      S[ST_D2 + d] = t2[d] * c2;
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      S[ST_ADV + F_GXX + a] = field_axes<true, true>(u + (F_GXX + a) * fs, q, st, c.gt[a], wb, wa, t1, t2);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        dgt[d][a] = t1[d] * c1;
        S[ST_D2 + 3 * (1 + a) + d] = t2[d] * c2;
      }
    }
    S[ST_ADV + F_KH] = field_axes<true, false>(u + F_KH * fs, q, st, c.Kh, wb, wa, t1, t2);
#pragma unroll
    for (int d = 0; d < 3; ++d) dKh[d] = t1[d] * c1;
    S[ST_ADV + F_TH] = field_axes<true, false>(u + F_TH * fs, q, st, c.Th, wb, wa, t1, t2);
#pragma unroll
    for (int d = 0; d < 3; ++d) dTh[d] = t1[d] * c1;
#pragma unroll
    for (int a = 0; a < 6; ++a)
      S[ST_ADV + F_AXX + a] = field_axes<false, false>(u + (F_AXX + a) * fs, q, st, c.At[a], wb, wa, t1, t2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S[ST_ADV + F_GAMX + i] = field_axes<true, false>(u + (F_GAMX + i) * fs, q, st, c.Gam[i], wb, wa, t1, t2);
#pragma unroll
      for (int d = 0; d < 3; ++d) dGam[d][i] = t1[d] * c1;
    }
    S[ST_ADV + F_ALP] = field_axes<true, true>(u + F_ALP * fs, q, st, c.al, wb, wa, t1, t2);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      G.dal[d] = t1[d] * c1;
      S[ST_D2 + 21 + d] = t2[d] * c2;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S[ST_ADV + F_BETX + i] = field_axes<true, true>(u + (F_BETX + i) * fs, q, st, c.be[i], wb, wa, t1, t2);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        dbe[d][i] = t1[d] * c1;
        S[ST_D2 + 3 * (8 + i) + d] = t2[d] * c2;
      }
      S[ST_ADV + F_BX + i] = field_axes<false, false>(u + (F_BX + i) * fs, q, st, c.Bv[i], wb, wa, t1, t2);
    }
  }
  geometry_t(u, q, st, fs, c11, c, G, dgt, dGam, D2Stash{S});
  const double* gtu = G.gtu;
  const double W = c.W, al = c.al;
  const double K = c.Kh + 2.0 * c.Th;
  const double divb = dbe[0][0] + dbe[1][1] + dbe[2][2];

  // At with one index raised (Am[i][j] = gt^ik At_kj), At^ij, At_ij At^ij
  double Am[3][3], Atu[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Am[i][j] = gtu[S2(i, 0)] * c.At[S2(0, j)] + gtu[S2(i, 1)] * c.At[S2(1, j)] +
                 gtu[S2(i, 2)] * c.At[S2(2, j)];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j)
      Atu[S2(i, j)] = Am[i][0] * gtu[S2(0, j)] + Am[i][1] * gtu[S2(1, j)] + Am[i][2] * gtu[S2(2, j)];
  const double AA = sym_contract(c.At, Atu);

  r[F_W] = W * (1.0 / 3.0) * (al * K - divb);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int ij = S2(i, j);
      double s = -2.0 * al * c.At[ij];
      double sA = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        s += c.gt[S2(i, k)] * dbe[j][k] + c.gt[S2(j, k)] * dbe[i][k];
        sA += c.At[S2(i, k)] * dbe[j][k] + c.At[S2(j, k)] * dbe[i][k];
      }
      r[F_GXX + ij] = s - (2.0 / 3.0) * c.gt[ij] * divb;
      r[F_AXX + ij] = sA - (2.0 / 3.0) * c.At[ij] * divb;  // completed below
    }
  const double alk1 = al * prm.kappa1;
  r[F_KH] = -G.Lapa + al * (AA + K * K * (1.0 / 3.0)) + alk1 * (1.0 - prm.kappa2) * c.Th;
  r[F_TH] = 0.5 * al * (G.Rsc - AA + (2.0 / 3.0) * K * K) - alk1 * (2.0 + prm.kappa2) * c.Th;

  {
    double X[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) X[a] = al * G.Ric[a] - G.DDa[a];
    const double trX3 = sym_contract(gtu, X) * (1.0 / 3.0);
    const double W2 = W * W;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int ij = S2(i, j);
        double AikAkj = c.At[S2(i, 0)] * Am[0][j] + c.At[S2(i, 1)] * Am[1][j] + c.At[S2(i, 2)] * Am[2][j];
        r[F_AXX + ij] += W2 * (X[ij] - c.gt[ij] * trX3) + al * (K * c.At[ij] - 2.0 * AikAkj);
      }
  }

  // Gamma-tilde: second derivatives of the shift
  {
    double ddb[3][6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double* f = u + (F_BETX + i) * fs;
      ddb[i][0] = S[ST_D2 + 3 * (8 + i) + 0];
      ddb[i][3] = S[ST_D2 + 3 * (8 + i) + 1];
      ddb[i][5] = S[ST_D2 + 3 * (8 + i) + 2];
      ddb[i][1] = d11u(f, q, st[0], st[1]) * c11;
      ddb[i][2] = d11u(f, q, st[0], st[2]) * c11;
      ddb[i][4] = d11u(f, q, st[1], st[2]) * c11;
    }
    double ddivb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) ddivb[j] = ddb[0][S2(j, 0)] + ddb[1][S2(j, 1)] + ddb[2][S2(j, 2)];
    const double iW = 1.0 / W;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double inner = sym_contract(G.Gu[i], Atu);
      double s = 0.0, t = 0.0, v = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        s += Atu[S2(i, j)] * G.dal[j];
        t += Atu[S2(i, j)] * G.dW[j];
        v += gtu[S2(i, j)] * (2.0 * dKh[j] + dTh[j]);
      }
      inner -= 3.0 * t * iW + v * (1.0 / 3.0);
      double g = -2.0 * s + 2.0 * al * inner;
      g += sym_contract(gtu, ddb[i]);
      g += (gtu[S2(i, 0)] * ddivb[0] + gtu[S2(i, 1)] * ddivb[1] + gtu[S2(i, 2)] * ddivb[2]) * (1.0 / 3.0);
      g += (2.0 / 3.0) * G.Gd[i] * divb;
      g -= G.Gd[0] * dbe[0][i] + G.Gd[1] * dbe[1][i] + G.Gd[2] * dbe[2][i];
      g -= 2.0 * alk1 * (c.Gam[i] - G.Gd[i]);
      r[F_GAMX + i] = g;
    }
  }

  if (prm.lapse == 1)
    r[F_ALP] = -al * al * K;
  else
    r[F_ALP] = -2.0 * al * (prm.lapse_uses_khat ? c.Kh : K);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r[F_BETX + i] = 0.75 * c.Bv[i];
    r[F_BX + i] = r[F_GAMX + i] - prm.eta * c.Bv[i];
  }

  // advection along the shift (upwind) and Kreiss-Oliger dissipation
#pragma unroll
  for (int f = 0; f < NF; ++f) r[f] += S[ST_ADV + f];
  if (prm.shift == 1) {
#pragma unroll
    for (int f = F_BETX; f < NF; ++f) r[f] = 0.0;
  }
}

// det gt = 1, At trace-free w.r.t. gt, W >= w_floor (pointwise, on a state
// vector of 25 values)
__device__ __forceinline__ void enforce_point(double v[NF], double w_floor) {
  double g[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) g[a] = v[F_GXX + a];
  double det = g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) +
               g[2] * (g[1] * g[4] - g[3] * g[2]);
  double fac = 1.0 / cbrt(det);
#pragma unroll
  for (int a = 0; a < 6; ++a) g[a] *= fac;
  double gu[6];
  sym_inv(g, gu);
  double tr3 = sym_contract(gu, v + F_AXX) * (1.0 / 3.0);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    v[F_GXX + a] = g[a];
    v[F_AXX + a] -= g[a] * tr3;
  }
  if (v[F_W] < w_floor) v[F_W] = w_floor;
}

__device__ __forceinline__ void rk_update(int s, double dt, long long q, long long fs,
                                          const double* __restrict__ un, double* __restrict__ y,
                                          double* __restrict__ out, double k[NF], double w_floor,
                                          unsigned* err) {
  const double bw = (s == 1 || s == 4) ? (1.0 / 6.0) : (1.0 / 3.0);
  const double cw = (s == 3) ? 1.0 : 0.5;
  const double bdt = bw * dt, cdt = cw * dt;
  double v[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const long long o = f * fs + q;
    if (s == 4) {
      v[f] = y[o] + bdt * k[f];
    } else {
      const double a = un[o];
      const double yn = (s == 1) ? a + bdt * k[f] : y[o] + bdt * k[f];
      y[o] = yn;
      v[f] = a + cdt * k[f];
    }
  }
  enforce_point(v, w_floor);
  bool bad = false;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    out[f * fs + q] = v[f];
    bad |= !isfinite(v[f]);
  }
  if (bad) atomicOr(err, (unsigned)ERR_NONFINITE);
}

template <int MODE>  // 0: RK stage, 1: RHS only
__global__ void __launch_bounds__(STAGE_THREADS) z4c_stage_fp64_kernel(StageArgs A) {
  extern __shared__ double stash[];
  const Tile tl = A.tiles[blockIdx.x];
  const DevPatch* P = A.patches + tl.patch;
  const int i = tl.x0 + (threadIdx.x & 31);
  const int j = tl.y0 + (threadIdx.x >> 5);
  const int k = tl.z0;
  if (i >= P->n[0] || j >= P->n[1] || k >= P->n[2]) return;
  const int ring = A.lev->ring;
  const int s = A.stage;
  const long long sy = P->px, sz = P->plane, fs = P->fstride;
  const long long q = (i + GH) + (long long)(j + GH) * sy + (long long)(k + GH) * sz;
  const double* __restrict__ u = P->buf[MODE ? ring : stage_in_slot(s, ring)];
  double r[NF];
  z4c_rhs_point(u, q, sy, sz, fs, P->dx, A.prm, Stash{stash + threadIdx.x}, r);
  if (A.prm.matter) {
    // the fluid's terms (Sec. 2.1.2), formed by the matter recovery kernel from
    // this stage's state: Khat, Theta, At_ij, Gamt^i (and B^i through Gamt^i)
    const double* __restrict__ zs = P->mzsrc;
    r[F_KH] += zs[q];
    r[F_TH] += zs[fs + q];
#pragma unroll
    for (int a = 0; a < 6; ++a) r[F_AXX + a] += zs[(2 + a) * fs + q];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double g = zs[(8 + a) * fs + q];
      r[F_GAMX + a] += g;
      if (A.prm.shift == 0) r[F_BX + a] += g;
    }
  }
  if (MODE == 1) {
    double* out = P->buf[B_S1];
#pragma unroll
    for (int f = 0; f < NF; ++f) out[f * fs + q] = r[f];
    return;
  }
  rk_update(s, A.dt, q, fs, P->buf[ring], P->buf[B_Y], P->buf[stage_out_slot(s, ring)], r,
            A.prm.w_floor, A.err);
}

// ---------------------------------------------------------------------------
// Sommerfeld outgoing-wave condition on the ghost points of level-0 patches
// (Sec. 2.2.2): d_t f = -(f - f_flat)/r - (x^i/r) d_i f, with d_i the 2nd-order
// one-sided difference toward the origin, evolved with the same RK4 stage.

__global__ void __launch_bounds__(128) sommerfeld_stage_kernel(GhostArgs A) {
  const DevPatch* P = A.patches + A.patch_ids[blockIdx.y];
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (id >= shell_count(P->NX, P->NY, P->NZ)) return;
  shell_ijk(id, P->NX, P->NY, P->NZ, i, j, k);
  const int ring = A.lev->ring;
  const int s = A.stage;
  const long long sy = P->px, sz = P->plane, fs = P->fstride;
  const long long q = i + (long long)j * sy + (long long)k * sz;
  const double* __restrict__ u = P->buf[stage_in_slot(s, ring)];
  const double h = P->dx;
  const int idx[3] = {i, j, k};
  const long long st[3] = {1, sy, sz};
  double x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = P->origin[d] + (idx[d] - GH + 0.5) * h;
  const double rr = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const double ir = 1.0 / rr;
  const double c = 1.0 / (2.0 * h);
  double kk[NF];
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    const double* fp = u + f * fs;
    const double f0 = fp[q];
    double acc = (f0 - flat_value(f)) * ir;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long o = x[d] > 0.0 ? -st[d] : st[d];
      double v = (3.0 * f0 - 4.0 * fp[q + o] + fp[q + 2 * o]) * c;
      double dfd = x[d] > 0.0 ? v : -v;
      acc += (x[d] * ir) * dfd;
    }
    kk[f] = -acc;
  }
  rk_update(s, A.dt, q, fs, P->buf[ring], P->buf[B_Y], P->buf[stage_out_slot(s, ring)], kk,
            A.prm.w_floor, A.err);
}

// ---------------------------------------------------------------------------
// Constraint monitor (Sec. 2.3): H = R + 2/3 K^2 - At_ij At^ij and
// M^i = W^2 gt^ij (gt^kl Dt_k At_lj - 3 At_j^k d_k W / W - 2/3 d_j K), per block
// partial sums of H^2, (M^x)^2, (M^y)^2, (M^z)^2 and the count over active
// points with W >= w_excise.

// ---------------------------------------------------------------------------
// Psi4 extraction (Sec. 2.3).  At cell q the vacuum electric and magnetic
// parts of the Weyl tensor (physical, covariant) and the physical metric:
//   E_ij = R_ij - K_ik K^k_j + K K_ij
//   B_ij = 1/2 (eps_i^kl D_k K_lj + eps_j^kl D_k K_li),  eps_ikl = sqrt(g) [ikl]
// with g_ij = gt_ij / W^2, K_ij = (At_ij + gt_ij K / 3) / W^2, K = Khat + 2
// Theta, R_ij the RHS's physical Ricci tensor and Gamma^i_jk = Gt^i_jk -
// (delta^i_j d_k W + delta^i_k d_j W - gt_jk gt^il d_l W) / W.
__device__ __noinline__ void weyl_cell(const double* __restrict__ u, long long q, const long long st[3],
                                       long long fs, double h, double E[6], double B[6], double gam[6]) {
  const double c1 = 1.0 / (12.0 * h), c2 = c1 / h, c11 = c1 * c1;
  PointState c;
  load_centre(u, q, fs, c);
  Geo G;
  double dGam[3][3], dbe[3][3];
  geometry(u, q, st, fs, c1, c2, c11, c, G, dGam, dbe);
  const double W = c.W, W2 = W * W, iW = 1.0 / W;
  const double K = c.Kh + 2.0 * c.Th;
  double Kl[6], gu[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    gam[a] = c.gt[a] / W2;
    Kl[a] = (c.At[a] + c.gt[a] * K / 3.0) / W2;
    gu[a] = W2 * G.gtu[a];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      double kk = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double kup = gu[S2(k, 0)] * Kl[S2(0, j)] + gu[S2(k, 1)] * Kl[S2(1, j)] + gu[S2(k, 2)] * Kl[S2(2, j)];
        kk += Kl[S2(i, k)] * kup;
      }
      E[S2(i, j)] = G.Ric[S2(i, j)] - kk + K * Kl[S2(i, j)];
    }
  // d_k K_ij from the derivatives of At, gt, W, Khat, Theta
  double dK[3][6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double dKt = (d1u(u + F_KH * fs, q, st[d]) + 2.0 * d1u(u + F_TH * fs, q, st[d])) * c1;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const double dA = d1u(u + (F_AXX + a) * fs, q, st[d]) * c1;
      const double dg = d1u(u + (F_GXX + a) * fs, q, st[d]) * c1;
      dK[d][a] = (dA + dg * K / 3.0 + c.gt[a] * dKt / 3.0) / W2 - 2.0 * Kl[a] * G.dW[d] * iW;
    }
  }
  double gw[3];  // gt^mn d_n W
#pragma unroll
  for (int m = 0; m < 3; ++m)
    gw[m] = G.gtu[S2(m, 0)] * G.dW[0] + G.gtu[S2(m, 1)] * G.dW[1] + G.gtu[S2(m, 2)] * G.dW[2];
  double Gp[3][6];  // physical Gamma^m_kl
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = k; l < 3; ++l) {
        const double cw = (m == k ? G.dW[l] : 0.0) + (m == l ? G.dW[k] : 0.0) - c.gt[S2(k, l)] * gw[m];
        Gp[m][S2(k, l)] = G.Gu[m][S2(k, l)] - cw * iW;
      }
  const double a0 = c.gt[3] * c.gt[5] - c.gt[4] * c.gt[4], a1 = c.gt[2] * c.gt[4] - c.gt[1] * c.gt[5],
               a2 = c.gt[1] * c.gt[4] - c.gt[2] * c.gt[3];
  const double sg = sqrt(c.gt[0] * a0 + c.gt[1] * a1 + c.gt[2] * a2) / (W2 * W);
  // C_ij = eps_i^kl D_k K_lj, D_k K_lj = d_k K_lj - Gamma^m_kl K_mj - Gamma^m_kj K_lm
  double C[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double DK[3][3];  // DK[k][l] = D_k K_lj
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        double v = dK[k][S2(l, j)];
#pragma unroll
        for (int m = 0; m < 3; ++m) v -= Gp[m][S2(k, l)] * Kl[S2(m, j)] + Gp[m][S2(k, j)] * Kl[S2(l, m)];
        DK[k][l] = v;
      }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int a = (i + 1) % 3, b = (i + 2) % 3;  // [iab] = +1, [iba] = -1
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
          v += (gu[S2(k, a)] * gu[S2(l, b)] - gu[S2(k, b)] * gu[S2(l, a)]) * DK[k][l];
      C[i][j] = sg * v;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) B[S2(i, j)] = 0.5 * (C[i][j] + C[j][i]);
}

constexpr int PSI4_THREADS = 128;

// Pass 1: E_ij, B_ij and g_ij of every cell whose centre lies within 3.6 dx
// of the sphere (the interpolation cells of any sphere point are within
// 2 sqrt(3) dx of it) and whose derivative stencils stay in the array, into
// 18 fields of `cells`.
__global__ void __launch_bounds__(128) psi4_cells_kernel(Psi4Args A) {
  const DevPatch* P = A.patches + A.patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)P->NX * P->NY * P->NZ) return;
  const int i = (int)(id % P->NX), j = (int)((id / P->NX) % P->NY), k = (int)(id / ((long long)P->NX * P->NY));
  if (i < 2 || j < 2 || k < 2 || i > P->NX - 3 || j > P->NY - 3 || k > P->NZ - 3) return;
  const double dx = P->origin[0] + (i - GH + 0.5) * P->dx - A.c[0];
  const double dy = P->origin[1] + (j - GH + 0.5) * P->dx - A.c[1];
  const double dz = P->origin[2] + (k - GH + 0.5) * P->dx - A.c[2];
  if (fabs(sqrt(dx * dx + dy * dy + dz * dz) - A.r) > 3.6 * P->dx) return;
  const long long st[3] = {1, P->px, P->plane};
  const long long q = i + (long long)j * P->px + (long long)k * P->plane;
  double E[6], B[6], g[6];
  weyl_cell(P->buf[A.levels[P->level].ring], q, st, P->fstride, P->dx, E, B, g);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    A.cells[a * P->fstride + q] = E[a];
    A.cells[(6 + a) * P->fstride + q] = B[a];
    A.cells[(12 + a) * P->fstride + q] = g[a];
  }
}

// Pass 2, one block per theta ring: Psi4 = (E_ij - i B_ij) mbar^i mbar^j at
// each of its phi points, with E, B and g interpolated tricubically from the
// pass-1 values of the 4 x 4 x 4 nearest cell centres and mbar = (e_theta - i e_phi)/sqrt(2) from the triad
// Gram-Schmidt-built (metric g) on the coordinate radial, theta and phi
// directions.
__global__ void __launch_bounds__(PSI4_THREADS) psi4_sphere_kernel(Psi4Args A) {
  __shared__ double node[2];
  __shared__ double red[PSI4_THREADS];
  const int it = blockIdx.x;
  if (threadIdx.x == 0) {
    double x, w;
    gauss_legendre_node(A.ntheta, it, x, w);
    node[0] = x;
    node[1] = w;
    A.ring[it] = x;
    A.ring[A.ntheta + it] = w;
  }
  __syncthreads();
  const DevPatch* P = A.patches + A.patch;
  const double* __restrict__ u = P->buf[A.levels[P->level].ring];
  const long long st[3] = {1, P->px, P->plane};
  const int N[3] = {P->NX, P->NY, P->NZ};
  const double ct = node[0], sth = sqrt((1.0 - ct) * (1.0 + ct));
  double bad = 0.0;
  for (int ip = threadIdx.x; ip < A.nphi; ip += PSI4_THREADS) {
    double sp, cp;
    sincospi(2.0 * ip / A.nphi, &sp, &cp);
    const double n[3] = {sth * cp, sth * sp, ct};
    double wl[3][4];
    int i0[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double t = (A.c[d] + A.r * n[d] - P->origin[d]) / P->dx - 0.5 + GH;
      ok = ok && t >= 3.0 && t < N[d] - 4.0;
      i0[d] = ok ? (int)floor(t) - 1 : 0;
      cubic_weights(ok ? t - i0[d] : 0.0, wl[d]);
    }
    double* out = A.psi + 2 * ((long long)it * A.nphi + ip);
    if (!ok) {
      bad += 1.0;
      out[0] = out[1] = 0.0;
      continue;
    }
    double E[6] = {0, 0, 0, 0, 0, 0}, B[6] = {0, 0, 0, 0, 0, 0}, g[6] = {0, 0, 0, 0, 0, 0};
    for (int c = 0; c < 4; ++c)
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
          const long long q = (i0[0] + a) + (i0[1] + b) * st[1] + (i0[2] + c) * st[2];
          const double* cq = A.cells + q;
          const double w = wl[0][a] * wl[1][b] * wl[2][c];
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            E[k] += w * cq[k * P->fstride];
            B[k] += w * cq[(6 + k) * P->fstride];
            g[k] += w * cq[(12 + k) * P->fstride];
          }
        }
    double e[3][3];
    const double v[3][3] = {{n[0], n[1], n[2]}, {ct * cp, ct * sp, -sth}, {-sp, cp, 0.0}};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double w[3] = {v[a][0], v[a][1], v[a][2]};
#pragma unroll
      for (int b = 0; b < a; ++b) {
        double dot = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) dot += g[S2(i, j)] * w[i] * e[b][j];
#pragma unroll
        for (int i = 0; i < 3; ++i) w[i] -= dot * e[b][i];
      }
      double nn = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) nn += g[S2(i, j)] * w[i] * w[j];
      nn = 1.0 / sqrt(nn);
#pragma unroll
      for (int i = 0; i < 3; ++i) e[a][i] = w[i] * nn;
    }
    // mbar mbar = P - i Q; Psi4 = (E:P - B:Q) - i (E:Q + B:P)
    double EP = 0.0, EQ = 0.0, BP = 0.0, BQ = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double Pm = 0.5 * (e[1][i] * e[1][j] - e[2][i] * e[2][j]);
        const double Qm = 0.5 * (e[1][i] * e[2][j] + e[2][i] * e[1][j]);
        EP += E[S2(i, j)] * Pm;
        EQ += E[S2(i, j)] * Qm;
        BP += B[S2(i, j)] * Pm;
        BQ += B[S2(i, j)] * Qm;
      }
    out[0] = EP - BQ;
    out[1] = -(EQ + BP);
  }
  red[threadIdx.x] = bad;
  __syncthreads();
  for (int o = PSI4_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) A.ring[2 * A.ntheta + it] = red[0];
}

// _{-2}Y_lm amplitude sqrt((2l+1)/(4 pi)) d^l_{m,2}(theta) from the half-angle
// cosine c and sine s (Wigner d-function as a finite sum)
__device__ double swsh_amp(int l, int m, double c, double s) {
  double f[2 * PSI4_MAX_L + 1];
  f[0] = 1.0;
  for (int i = 1; i <= 2 * l; ++i) f[i] = f[i - 1] * i;
  const double pre = sqrt(f[l + m] * f[l - m] * f[l + 2] * f[l - 2]);
  const int k1 = m - 2 > 0 ? m - 2 : 0, k2 = l + m < l - 2 ? l + m : l - 2;
  double d = 0.0;
  for (int k = k1; k <= k2; ++k) {
    double t = pre / (f[l + m - k] * f[l - 2 - k] * f[k] * f[k + 2 - m]);
    const int pc = 2 * l + m - 2 - 2 * k, ps = 2 * k + 2 - m;
    for (int i = 0; i < pc; ++i) t *= c;
    for (int i = 0; i < ps; ++i) t *= s;
    d += (k & 1) ? -t : t;
  }
  return sqrt((2.0 * l + 1.0) / (4.0 * 3.141592653589793)) * d;
}

// One block per mode (l, m): Psi4^lm = sum over rings (in order) of the ring
// weight times sum over phi (in order) of Psi4 conj(_{-2}Y_lm) 2 pi / nphi
__global__ void __launch_bounds__(PSI4_THREADS) psi4_modes_kernel(Psi4Args A) {
  __shared__ double red[2][PSI4_THREADS];
  const int k = blockIdx.x;
  int l = 2;
  while ((l + 1) * (l + 1) - 4 <= k) ++l;
  const int m = k - (l * l - 4) - l;
  double ar = 0.0, ai = 0.0;
  for (int it = threadIdx.x; it < A.ntheta; it += PSI4_THREADS) {
    const double ct = A.ring[it], w = A.ring[A.ntheta + it];
    const double amp = swsh_amp(l, m, sqrt(0.5 * (1.0 + ct)), sqrt(0.5 * (1.0 - ct)));
    const double* ps = A.psi + 2 * (long long)it * A.nphi;
    double sr = 0.0, si = 0.0;
    for (int ip = 0; ip < A.nphi; ++ip) {
      double sn, cs;
      sincospi(2.0 * m * ip / A.nphi, &sn, &cs);
      sr += ps[2 * ip] * cs + ps[2 * ip + 1] * sn;
      si += ps[2 * ip + 1] * cs - ps[2 * ip] * sn;
    }
    ar += w * amp * sr;
    ai += w * amp * si;
  }
  red[0][threadIdx.x] = ar;
  red[1][threadIdx.x] = ai;
  __syncthreads();
  for (int o = PSI4_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double dphi = 2.0 * 3.141592653589793 / A.nphi;
    A.out[2 * k] = red[0][0] * dphi;
    A.out[2 * k + 1] = red[1][0] * dphi;
  }
}

void launch_psi4(const Psi4Args& a, long long patch_points, cudaStream_t st) {
  psi4_cells_kernel<<<(unsigned)((patch_points + 127) / 128), 128, 0, st>>>(a);
  psi4_sphere_kernel<<<a.ntheta, PSI4_THREADS, 0, st>>>(a);
  psi4_modes_kernel<<<(a.lmax + 1) * (a.lmax + 1) - 4, PSI4_THREADS, 0, st>>>(a);
}

__global__ void __launch_bounds__(128) constraints_kernel(ConsArgs A) {
  __shared__ double red[5][4];
  const Tile tl = A.tiles[blockIdx.x];
  const DevPatch* P = A.patches + tl.patch;
  const int i = tl.x0 + (threadIdx.x & 31);
  const int j = tl.y0 + (threadIdx.x >> 5);
  const int k = tl.z0;
  double acc[5] = {0, 0, 0, 0, 0};
  if (i < P->n[0] && j < P->n[1] && k < P->n[2]) {
    const long long sy = P->px, sz = P->plane, fs = P->fstride;
    const long long st[3] = {1, sy, sz};
    const long long q = (i + GH) + (long long)(j + GH) * sy + (long long)(k + GH) * sz;
    const double* __restrict__ u = P->buf[A.lev->ring];
    const double h = P->dx;
    const double c1 = 1.0 / (12.0 * h), c2 = c1 / h, c11 = c1 * c1;
    PointState c;
    load_centre(u, q, fs, c);
    Geo G;
    double dGam[3][3], dbe[3][3];
    geometry(u, q, st, fs, c1, c2, c11, c, G, dGam, dbe);
    const double* gtu = G.gtu;
    double Am[3][3], Atu[6];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Am[a][b] = gtu[S2(a, 0)] * c.At[S2(0, b)] + gtu[S2(a, 1)] * c.At[S2(1, b)] +
                   gtu[S2(a, 2)] * c.At[S2(2, b)];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b)
        Atu[S2(a, b)] = Am[a][0] * gtu[S2(0, b)] + Am[a][1] * gtu[S2(1, b)] + Am[a][2] * gtu[S2(2, b)];
    const double K = c.Kh + 2.0 * c.Th;
    const double H = G.Rsc + (2.0 / 3.0) * K * K - sym_contract(c.At, Atu);
    double dAt[3][6], dK[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int a = 0; a < 6; ++a) dAt[d][a] = d1u(u + (F_AXX + a) * fs, q, st[d]) * c1;
      dK[d] = (d1u(u + F_KH * fs, q, st[d]) + 2.0 * d1u(u + F_TH * fs, q, st[d])) * c1;
    }
    double Ml[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          // Dt_b At_ea = d_b At_ea - Gt^l_be At_la - Gt^l_ba At_el
          double DA = dAt[b][S2(e, a)];
#pragma unroll
          for (int l = 0; l < 3; ++l)
            DA -= G.Gu[l][S2(b, e)] * c.At[S2(l, a)] + G.Gu[l][S2(b, a)] * c.At[S2(e, l)];
          s += gtu[S2(b, e)] * DA;
        }
      s -= 3.0 * (Am[0][a] * G.dW[0] + Am[1][a] * G.dW[1] + Am[2][a] * G.dW[2]) / c.W;
      s -= (2.0 / 3.0) * dK[a];
      Ml[a] = s;
    }
    if (c.W >= A.w_excise) {
      acc[0] = H * H;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double m = c.W * c.W * (gtu[S2(a, 0)] * Ml[0] + gtu[S2(a, 1)] * Ml[1] + gtu[S2(a, 2)] * Ml[2]);
        acc[1 + a] = m * m;
      }
      acc[4] = 1.0;
    }
  }
  // fixed-order block reduction: warp shuffles, then 4 warps in order
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    double v = acc[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    const int a = threadIdx.x;
    A.partial[(long long)blockIdx.x * 5 + a] = ((red[a][0] + red[a][1]) + red[a][2]) + red[a][3];
  }
}

// deterministic final sum of per-block partials: one block, fixed order
__global__ void sum_partials_kernel(const double* partial, int nblocks, int width, double* out) {
  __shared__ double sh[256];
  for (int a = 0; a < width; ++a) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[(long long)b * width + a];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[a] = sh[0];
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// host-side launchers

void launch_stage_fp64(const StageArgs& a, cudaStream_t st) {
  if (a.ntiles == 0) return;
  static bool ready[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !ready[dev]) {  // the stash is above the 48 KB default
    cudaFuncSetAttribute(z4c_stage_fp64_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STAGE_SMEM);
    cudaFuncSetAttribute(z4c_stage_fp64_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STAGE_SMEM);
    ready[dev] = true;
  }
  if (a.stage == 0)
    z4c_stage_fp64_kernel<1><<<a.ntiles, STAGE_THREADS, STAGE_SMEM, st>>>(a);
  else
    z4c_stage_fp64_kernel<0><<<a.ntiles, STAGE_THREADS, STAGE_SMEM, st>>>(a);
}

void launch_sommerfeld(const GhostArgs& a, int npatches, long long max_shell, cudaStream_t st) {
  if (npatches == 0 || max_shell == 0) return;
  dim3 grid((unsigned)((max_shell + 127) / 128), npatches);
  sommerfeld_stage_kernel<<<grid, 128, 0, st>>>(a);
}

void launch_constraints(const ConsArgs& a, int ntiles, double* out5, cudaStream_t st) {
  if (ntiles == 0) return;
  constraints_kernel<<<ntiles, 128, 0, st>>>(a);
  sum_partials_kernel<<<1, 256, 0, st>>>(a.partial, ntiles, 5, out5);
}

}  // namespace sacrak

// ----------------------------------------------------------------------------
// Allocation-free variant of the constraint monitor.
//
// Some callers cannot allocate device memory at all: code running inside a
// host framework that owns the whole device through its own memory pool,
// inside a pre-sized sandbox or a fixed-memory production service, or in a
// hook that must never trigger cudaMalloc's implicit synchronisation.  They
// keep a patch in their own device memory and want its constraint norms.
// This entry point needs no grid and no arena: the per-block partial sums go
// to one file-scope device array of fixed size that every GPU loading this
// library holds until the process exits.

namespace sacrak {
namespace {

constexpr int NOALLOC_MAX_BLOCKS = 2048;  // partial-sum slots (5 doubles each)
constexpr int NOALLOC_MAX_N = 512;        // largest active cells per axis
constexpr int NOALLOC_MAX_DEVICES = 64;

// [0, 5*NOALLOC_MAX_BLOCKS): per-block partials; then 5 final sums.  Every call
// overwrites the slots it uses before reading them, so nothing has to start
// at zero; calls that overlap on the GPU race on this array.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_BLOCKS * 5 + 8];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// device address of the scratch array on device `dev` (the current device):
// looked up once per device, with that device current; the host-side symbol
// is only a stand-in and must never be handed to a kernel.  A context that
// was destroyed and created again (a device reset) reloads the module at a
// new address, so the cached address is dropped whenever a call on that
// device reports a destroyed context (noalloc_forget).
cudaError_t noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = (double*)g_noalloc_addr[dev];
  return cudaSuccess;
}

void noalloc_forget(int dev, cudaError_t e) {
  if (e != cudaErrorContextIsDestroyed && e != cudaErrorDeviceUninitialized) return;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  g_noalloc_addr[dev] = nullptr;
}

// cuMemGetAddressRange from the driver (base and size of the allocation that
// holds a device address), looked up once through the runtime
typedef int (*AddressRangeFn)(unsigned long long*, size_t*, unsigned long long);
AddressRangeFn address_range_fn() {
  static AddressRangeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (AddressRangeFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// one block per group of 32x4 points of a z-plane, grid-striding over the
// patch; the same per-point arithmetic as constraints_kernel
__global__ void __launch_bounds__(128) constraints_noalloc_kernel(const double* __restrict__ u,
                                                                  int nx, int ny, int nz, double h,
                                                                  double w_excise, double* partial) {
  __shared__ double red[5][4];
  const int tx = (nx + 31) / 32, ty = (ny + 3) / 4;
  const long long ntiles = (long long)tx * ty * nz;
  const int NX = nx + 2 * GH, NY = ny + 2 * GH, NZ = nz + 2 * GH;
  const long long sy = NX, sz = (long long)NX * NY, fs = sz * NZ;
  const long long st[3] = {1, sy, sz};
  const double c1 = 1.0 / (12.0 * h), c2 = c1 / h, c11 = c1 * c1;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i = (int)(t % tx) * 32 + (threadIdx.x & 31);
    const int j = (int)((t / tx) % ty) * 4 + (threadIdx.x >> 5);
    const int k = (int)(t / ((long long)tx * ty));
    if (i >= nx || j >= ny) continue;
    const long long q = (i + GH) + (long long)(j + GH) * sy + (long long)(k + GH) * sz;
    PointState c;
    load_centre(u, q, fs, c);
    Geo G;
    double dGam[3][3], dbe[3][3];
    geometry(u, q, st, fs, c1, c2, c11, c, G, dGam, dbe);
    const double* gtu = G.gtu;
    double Am[3][3], Atu[6];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Am[a][b] = gtu[S2(a, 0)] * c.At[S2(0, b)] + gtu[S2(a, 1)] * c.At[S2(1, b)] +
                   gtu[S2(a, 2)] * c.At[S2(2, b)];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b)
        Atu[S2(a, b)] = Am[a][0] * gtu[S2(0, b)] + Am[a][1] * gtu[S2(1, b)] + Am[a][2] * gtu[S2(2, b)];
    const double K = c.Kh + 2.0 * c.Th;
    const double H = G.Rsc + (2.0 / 3.0) * K * K - sym_contract(c.At, Atu);
    double dAt[3][6], dK[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int a = 0; a < 6; ++a) dAt[d][a] = d1u(u + (F_AXX + a) * fs, q, st[d]) * c1;
      dK[d] = (d1u(u + F_KH * fs, q, st[d]) + 2.0 * d1u(u + F_TH * fs, q, st[d])) * c1;
    }
    double Ml[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          double DA = dAt[b][S2(e, a)];
#pragma unroll
          for (int l = 0; l < 3; ++l)
            DA -= G.Gu[l][S2(b, e)] * c.At[S2(l, a)] + G.Gu[l][S2(b, a)] * c.At[S2(e, l)];
          s += gtu[S2(b, e)] * DA;
        }
      s -= 3.0 * (Am[0][a] * G.dW[0] + Am[1][a] * G.dW[1] + Am[2][a] * G.dW[2]) / c.W;
      s -= (2.0 / 3.0) * dK[a];
      Ml[a] = s;
    }
    if (c.W >= w_excise) {
      acc[0] += H * H;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double m = c.W * c.W * (gtu[S2(a, 0)] * Ml[0] + gtu[S2(a, 1)] * Ml[1] + gtu[S2(a, 2)] * Ml[2]);
        acc[1 + a] += m * m;
      }
      acc[4] += 1.0;
    }
  }
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    double v = acc[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    const int a = threadIdx.x;
    partial[(long long)blockIdx.x * 5 + a] = ((red[a][0] + red[a][1]) + red[a][2]) + red[a][3];
  }
}

}  // namespace
}  // namespace sacrak

extern "C" sacrak_status sacrak_constraints_noalloc(const double* dev_u, const int n[3], double dx,
                                                    double w_excise, void* cuda_stream,
                                                    double out_l2[4]) {
  using namespace sacrak;
  if (!dev_u || !n || !out_l2 || !(dx > 0.0)) return SACRAK_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (n[d] < 4 || n[d] > NOALLOC_MAX_N) return SACRAK_EINVAL;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SACRAK_ECUDA;
  }
  // dev_u must be device memory of the current device (a peer GPU's memory
  // would be read across the link, or fault without peer access) ...
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, dev_u) != cudaSuccess || attr.type != cudaMemoryTypeDevice ||
      attr.device != dev) {
    cudaGetLastError();
    return SACRAK_EINVAL;
  }
  // ... and its allocation must hold the whole patch array
  const size_t need = sizeof(double) * NF * (size_t)(n[0] + 2 * GH) * (n[1] + 2 * GH) * (n[2] + 2 * GH);
  AddressRangeFn range = address_range_fn();
  if (!range) return SACRAK_ECUDA;
  unsigned long long base = 0;
  size_t size = 0;
  const unsigned long long a = (unsigned long long)(uintptr_t)dev_u;
  if (range(&base, &size, a) != 0) {
    cudaGetLastError();
    return SACRAK_EINVAL;
  }
  if (a < base || a - base + need > size) return SACRAK_EINVAL;
  double* scratch = nullptr;
  e = noalloc_scratch(dev, &scratch);
  if (e != cudaSuccess) {
    noalloc_forget(dev, e);
    cudaGetLastError();
    return SACRAK_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const long long ntiles = (long long)((n[0] + 31) / 32) * ((n[1] + 3) / 4) * n[2];
  const int nblocks = (int)(ntiles < NOALLOC_MAX_BLOCKS ? ntiles : NOALLOC_MAX_BLOCKS);
  constraints_noalloc_kernel<<<nblocks, 128, 0, st>>>(dev_u, n[0], n[1], n[2], dx, w_excise, scratch);
  double* sums_dev = scratch + (size_t)NOALLOC_MAX_BLOCKS * 5;
  sum_partials_kernel<<<1, 256, 0, st>>>(scratch, nblocks, 5, sums_dev);
  e = cudaGetLastError();
  double sums[5];
  if (e == cudaSuccess) e = cudaMemcpyAsync(sums, sums_dev, sizeof sums, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    noalloc_forget(dev, e);
    return SACRAK_ECUDA;
  }
  for (int c = 0; c < 4; ++c) out_l2[c] = sums[4] > 0 ? sqrt(sums[c] / sums[4]) : 0.0;
  return SACRAK_OK;
}
