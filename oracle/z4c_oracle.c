/*
 * Z4c oracle: plain FP64 CPU implementation of the Z4c right-hand side, the
 * classical RK4 update, the outer boundary, the algebraic constraints, the
 * constraint monitor, the pi-symmetry monitor and the Berger-Oliger inter-level
 * operators (Sec. 2.1.1, 2.2, 2.2.1, 2.2.2, 2.3, 3.2 of the SACRA-K paper).
 *
 * TEST INFRASTRUCTURE ONLY.  Written point by point from the definitions, for
 * a reader to check against the equations by eye; no blocking, no fusion.
 * Build with -O2 -ffp-contract=off -fno-fast-math (the paper's
 * reproducibility flags, Sec. 2.4 and Sec. 3.2) so that every point evaluates
 * the same operations in the same order and pi symmetry holds bit for bit.
 *
 * Continuum equations (vacuum, W-variable Z4c with K = Khat + 2 Theta, and
 * d0 = d_t - beta^k d_k; the paper cites Z4c without printing it):
 *   d0 W      = W/3 (alpha K - d_k beta^k)
 *   d0 gt_ij  = -2 alpha At_ij + gt_ik d_j beta^k + gt_jk d_i beta^k
 *               - 2/3 gt_ij d_k beta^k
 *   d0 Khat   = -D^i D_i alpha + alpha (At_ij At^ij + K^2/3)
 *               + alpha kappa1 (1 - kappa2) Theta
 *   d0 Theta  = alpha/2 (R - At_ij At^ij + 2/3 K^2) - alpha kappa1 (2 + kappa2) Theta
 *   d0 At_ij  = W^2 [-D_i D_j alpha + alpha R_ij]^TF
 *               + alpha (K At_ij - 2 At_ik gt^kl At_lj)
 *               + At_ik d_j beta^k + At_jk d_i beta^k - 2/3 At_ij d_k beta^k
 *   d0 Gamt^i = -2 At^ij d_j alpha
 *               + 2 alpha (Gamt^i_jk At^jk - 3 At^ij d_j W / W
 *                          - 1/3 gt^ij (2 d_j Khat + d_j Theta))
 *               + gt^jk d_j d_k beta^i + 1/3 gt^ij d_j d_k beta^k
 *               + 2/3 Gamd^i d_k beta^k - Gamd^k d_k beta^i
 *               - 2 alpha kappa1 (Gamt^i - Gamd^i)
 *   d0 alpha  = -2 alpha K (1+log, Sec. 2.1.1) or -alpha^2 K (harmonic)
 *   d0 beta^i = 3/4 B^i ;  d0 B^i = d0 Gamt^i - eta B^i   (Sec. 2.1.1)
 * with R_ij = Rt_ij + RW_ij,
 *   Rt_ij = -1/2 gt^lm d_l d_m gt_ij + gt_k(i d_j) Gamt^k + Gamd^k Gt_(ij)k
 *           + gt^lm (2 Gt^k_l(i Gt_j)km + Gt^k_im Gt_klj)
 *   RW_ij = (Dt_i Dt_j W + gt_ij gt^kl Dt_k Dt_l W) / W - 2 gt_ij gt^kl d_k W d_l W / W^2
 *   D_i D_j alpha = Dt_i Dt_j alpha + (d_i W d_j alpha + d_j W d_i alpha
 *                   - gt_ij gt^kl d_k W d_l alpha) / W
 *   R = W^2 gt^ij R_ij.
 * Discretisation (Sec. 2.2): 4th-order centred first and second derivatives,
 * mixed derivatives nested (D_a applied to D_b f), 4th-order lopsided upwind
 * advection biased by the sign of the shift, 6th-order Kreiss-Oliger
 * dissipation sigma/(64 h) sum_dirs Delta^6 f added to every field.
 */
#include "z4c_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
  F_W = 0, F_GXX, F_GXY, F_GXZ, F_GYY, F_GYZ, F_GZZ, F_KH, F_TH,
  F_AXX, F_AXY, F_AXZ, F_AYY, F_AYZ, F_AZZ, F_GAMX, F_GAMY, F_GAMZ,
  F_ALP, F_BETX, F_BETY, F_BETZ, F_BX, F_BY, F_BZ
};
#define NF ORC_NF

/* symmetric-index map (i,j) -> 0..5 in the order xx,xy,xz,yy,yz,zz */
static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

/* pi-rotation parity of every field: x,y change sign, z does not */
static const int PARITY[NF] = {
    +1,                 /* W */
    +1, +1, -1, +1, -1, +1, /* gt: xx xy xz yy yz zz */
    +1, +1,             /* Khat Theta */
    +1, +1, -1, +1, -1, +1, /* At */
    -1, -1, +1,         /* Gamt */
    +1,                 /* alpha */
    -1, -1, +1,         /* beta */
    -1, -1, +1};        /* B */

/* flat-space value of every field, used by the Sommerfeld condition */
static double flat_value(int f) {
  return (f == F_W || f == F_GXX || f == F_GYY || f == F_GZZ || f == F_ALP) ? 1.0 : 0.0;
}

typedef struct {
  int NX, NY, NZ;       /* array extents incl. ghosts */
  ptrdiff_t s[3];       /* strides of x, y, z */
  ptrdiff_t sf;         /* stride between fields */
} layout;

static layout make_layout(const orc_patch* p) {
  layout L;
  L.NX = p->n[0] + 2 * p->g;
  L.NY = p->n[1] + 2 * p->g;
  L.NZ = p->n[2] + 2 * p->g;
  L.s[0] = 1;
  L.s[1] = L.NX;
  L.s[2] = (ptrdiff_t)L.NX * L.NY;
  L.sf = (ptrdiff_t)L.NX * L.NY * L.NZ;
  return L;
}

size_t orc_patch_points(const orc_patch* p) {
  layout L = make_layout(p);
  return (size_t)L.sf;
}

/* threads of the OpenMP loops (timing of the oracle on a given core count) */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------- finite-difference operators (Sec. 2.2) ---------------- */

/* 4th-order centred first derivative along stride s */
static double D1(const double* f, ptrdiff_t q, ptrdiff_t s, double h) {
  return (8.0 * (f[q + s] - f[q - s]) - (f[q + 2 * s] - f[q - 2 * s])) / (12.0 * h);
}

/* Every stencil below is a linear combination whose coefficients sum to
 * zero, so it is evaluated on differences from the centre value f_k - f_0:
 * the same combination, rounded relative to the result instead of to the
 * field value (this matters where the RHS is many orders of magnitude below
 * the field, e.g. dissipation of 1e-10 noise on gt_xx = 1). */

/* 4th-order centred second derivative along stride s:
 * (16 (f1 + f-1) - (f2 + f-2) - 30 f0) / (12 h^2) */
static double D2(const double* f, ptrdiff_t q, ptrdiff_t s, double h) {
  double f0 = f[q];
  return (16.0 * ((f[q + s] - f0) + (f[q - s] - f0)) - ((f[q + 2 * s] - f0) + (f[q - 2 * s] - f0))) /
         (12.0 * h * h);
}

/* mixed derivative: D along sa applied to (D along sb) */
static double D11(const double* f, ptrdiff_t q, ptrdiff_t sa, ptrdiff_t sb, double h) {
  double p1 = D1(f, q + sa, sb, h), m1 = D1(f, q - sa, sb, h);
  double p2 = D1(f, q + 2 * sa, sb, h), m2 = D1(f, q - 2 * sa, sb, h);
  return (8.0 * (p1 - m1) - (p2 - m2)) / (12.0 * h);
}

/* lopsided stencil with one point behind and three ahead:
 * (-3 f_{-1} - 10 f_0 + 18 f_{+1} - 6 f_{+2} + f_{+3}) / 12  (times 1/h) */
static double lop(double am1, double a0, double ap1, double ap2, double ap3) {
  return (-3.0 * (am1 - a0) + 18.0 * (ap1 - a0) - 6.0 * (ap2 - a0) + (ap3 - a0)) / 12.0;
}

/* 4th-order upwind derivative along stride s, biased toward the side the
 * shift component b points to; for b <= 0 the mirrored stencil is the same
 * expression on mirrored points, negated (this keeps pi symmetry bitwise). */
static double Dup(const double* f, ptrdiff_t q, ptrdiff_t s, double h, double b) {
  if (b > 0.0)
    return lop(f[q - s], f[q], f[q + s], f[q + 2 * s], f[q + 3 * s]) / h;
  return -lop(f[q + s], f[q], f[q - s], f[q - 2 * s], f[q - 3 * s]) / h;
}

/* 6th difference along stride s (the Kreiss-Oliger operator's stencil) */
static double Delta6(const double* f, ptrdiff_t q, ptrdiff_t s) {
  double f0 = f[q];
  return ((f[q - 3 * s] - f0) + (f[q + 3 * s] - f0)) - 6.0 * ((f[q - 2 * s] - f0) + (f[q + 2 * s] - f0)) +
         15.0 * ((f[q - s] - f0) + (f[q + s] - f0));
}

void orc_stencils(const orc_patch* p, const double* u, int field, int i, int j, int k,
                  const double b[3], double out[15]) {
  layout L = make_layout(p);
  const double h = p->dx;
  const double* f = u + field * L.sf;
  ptrdiff_t q = i + j * L.s[1] + k * L.s[2];
  for (int d = 0; d < 3; ++d) {
    out[d] = D1(f, q, L.s[d], h);
    out[3 + d] = D2(f, q, L.s[d], h);
    out[9 + d] = Dup(f, q, L.s[d], h, b[d]);
    out[12 + d] = Delta6(f, q, L.s[d]);
  }
  out[6] = D11(f, q, L.s[0], L.s[1], h);
  out[7] = D11(f, q, L.s[0], L.s[2], h);
  out[8] = D11(f, q, L.s[1], L.s[2], h);
}

/* ---------------- geometry helpers ---------------- */

/* symmetric 3x3 inverse from the 6 components; returns the determinant */
static double sym_inverse(const double g[6], double gu[6]) {
  double xx = g[0], xy = g[1], xz = g[2], yy = g[3], yz = g[4], zz = g[5];
  double det = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
  gu[0] = (yy * zz - yz * yz) / det;
  gu[1] = (xz * yz - xy * zz) / det;
  gu[2] = (xy * yz - xz * yy) / det;
  gu[3] = (xx * zz - xz * xz) / det;
  gu[4] = (xy * xz - xx * yz) / det;
  gu[5] = (xx * yy - xy * xy) / det;
  return det;
}

/* per-point geometric quantities shared by the RHS and the constraints */
typedef struct {
  double W, gt[6], Kh, Th, At[6], Gam[3], alp, bet[3], B[3];
  double gtu[6];                 /* gt^ij */
  double dW[3], dgt[3][6];       /* d_k W, d_k gt_ij */
  double dKh[3], dTh[3], dalp[3];
  double dGam[3][3];             /* dGam[k][i] = d_k Gamt^i */
  double dbet[3][3];             /* dbet[k][i] = d_k beta^i */
  double ddW[6], ddgt[6][6];     /* ddgt[ij][kl] = d_k d_l gt_ij */
  double ddalp[6], ddbet[3][6];  /* ddbet[i][kl] = d_k d_l beta^i */
  double Gl[3][6];               /* Gt_ijk, first index lowered: Gl[i][jk] */
  double Gu[3][6];               /* Gt^i_jk */
  double Gd[3];                  /* Gamd^i = gt^jk Gt^i_jk */
  double Ric[6];                 /* R_ij = Rt_ij + RW_ij */
  double Rsc;                    /* R = W^2 gt^ij R_ij */
  double DDa[6];                 /* D_i D_j alpha (physical) */
  double Lapa;                   /* D^i D_i alpha */
  double Atu[6];                 /* At^ij */
  double AA;                     /* At_ij At^ij */
  double K;                      /* K = Khat + 2 Theta */
} pointgeo;

static void load_point(const double* u, const layout* L, ptrdiff_t q, pointgeo* G) {
  const double* F[NF];
  for (int f = 0; f < NF; ++f) F[f] = u + f * L->sf;
  G->W = F[F_W][q];
  for (int a = 0; a < 6; ++a) {
    G->gt[a] = F[F_GXX + a][q];
    G->At[a] = F[F_AXX + a][q];
  }
  G->Kh = F[F_KH][q];
  G->Th = F[F_TH][q];
  for (int i = 0; i < 3; ++i) {
    G->Gam[i] = F[F_GAMX + i][q];
    G->bet[i] = F[F_BETX + i][q];
    G->B[i] = F[F_BX + i][q];
  }
  G->alp = F[F_ALP][q];
}

/* derivatives and the curvature quantities at active point q */
static void point_geometry(const double* u, const layout* L, double h, ptrdiff_t q,
                           pointgeo* G) {
  const double* F[NF];
  for (int f = 0; f < NF; ++f) F[f] = u + f * L->sf;
  load_point(u, L, q, G);

  /* first derivatives */
  for (int k = 0; k < 3; ++k) {
    ptrdiff_t s = L->s[k];
    G->dW[k] = D1(F[F_W], q, s, h);
    for (int a = 0; a < 6; ++a) G->dgt[k][a] = D1(F[F_GXX + a], q, s, h);
    G->dKh[k] = D1(F[F_KH], q, s, h);
    G->dTh[k] = D1(F[F_TH], q, s, h);
    G->dalp[k] = D1(F[F_ALP], q, s, h);
    for (int i = 0; i < 3; ++i) {
      G->dGam[k][i] = D1(F[F_GAMX + i], q, s, h);
      G->dbet[k][i] = D1(F[F_BETX + i], q, s, h);
    }
  }
  /* second derivatives: pure ones by D2, mixed ones nested D_k (D_l f), k < l */
  for (int k = 0; k < 3; ++k) {
    for (int l = k; l < 3; ++l) {
      int kl = SYM[k][l];
      if (k == l) {
        ptrdiff_t s = L->s[k];
        G->ddW[kl] = D2(F[F_W], q, s, h);
        for (int a = 0; a < 6; ++a) G->ddgt[a][kl] = D2(F[F_GXX + a], q, s, h);
        G->ddalp[kl] = D2(F[F_ALP], q, s, h);
        for (int i = 0; i < 3; ++i) G->ddbet[i][kl] = D2(F[F_BETX + i], q, s, h);
      } else {
        ptrdiff_t sa = L->s[k], sb = L->s[l];
        G->ddW[kl] = D11(F[F_W], q, sa, sb, h);
        for (int a = 0; a < 6; ++a) G->ddgt[a][kl] = D11(F[F_GXX + a], q, sa, sb, h);
        G->ddalp[kl] = D11(F[F_ALP], q, sa, sb, h);
        for (int i = 0; i < 3; ++i) G->ddbet[i][kl] = D11(F[F_BETX + i], q, sa, sb, h);
      }
    }
  }

  /* inverse conformal metric */
  sym_inverse(G->gt, G->gtu);
  const double* gt = G->gt;
  const double* gtu = G->gtu;

  /* Christoffel symbols: Gt_ijk = 1/2 (d_j gt_ik + d_k gt_ij - d_i gt_jk) */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = j; k < 3; ++k)
        G->Gl[i][SYM[j][k]] =
            0.5 * (G->dgt[j][SYM[i][k]] + G->dgt[k][SYM[i][j]] - G->dgt[i][SYM[j][k]]);
  for (int i = 0; i < 3; ++i)
    for (int jk = 0; jk < 6; ++jk) {
      double s = 0.0;
      for (int l = 0; l < 3; ++l) s += gtu[SYM[i][l]] * G->Gl[l][jk];
      G->Gu[i][jk] = s;
    }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += gtu[SYM[j][k]] * G->Gu[i][SYM[j][k]];
    G->Gd[i] = s;
  }

  /* conformal Ricci tensor Rt_ij */
  double Rt[6];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      int ij = SYM[i][j];
      double t1 = 0.0; /* -1/2 gt^lm d_l d_m gt_ij */
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) t1 += gtu[SYM[l][m]] * G->ddgt[ij][SYM[l][m]];
      t1 *= -0.5;
      double t2 = 0.0; /* gt_k(i d_j) Gamt^k */
      for (int k = 0; k < 3; ++k)
        t2 += 0.5 * (gt[SYM[k][i]] * G->dGam[j][k] + gt[SYM[k][j]] * G->dGam[i][k]);
      double t3 = 0.0; /* Gamd^k Gt_(ij)k */
      for (int k = 0; k < 3; ++k)
        t3 += G->Gd[k] * 0.5 * (G->Gl[i][SYM[j][k]] + G->Gl[j][SYM[i][k]]);
      double t4 = 0.0; /* gt^lm (Gt^k_li Gt_jkm + Gt^k_lj Gt_ikm + Gt^k_im Gt_klj) */
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          double s = 0.0;
          for (int k = 0; k < 3; ++k)
            s += G->Gu[k][SYM[l][i]] * G->Gl[j][SYM[k][m]] +
                 G->Gu[k][SYM[l][j]] * G->Gl[i][SYM[k][m]] +
                 G->Gu[k][SYM[i][m]] * G->Gl[k][SYM[l][j]];
          t4 += gtu[SYM[l][m]] * s;
        }
      Rt[ij] = t1 + t2 + t3 + t4;
    }

  /* conformal-factor part RW_ij and second covariant derivatives */
  double W = G->W;
  double DDW[6], DDalpt[6];
  for (int ij = 0; ij < 6; ++ij) {
    double cw = 0.0, ca = 0.0;
    for (int k = 0; k < 3; ++k) {
      cw += G->Gu[k][ij] * G->dW[k];
      ca += G->Gu[k][ij] * G->dalp[k];
    }
    DDW[ij] = G->ddW[ij] - cw;
    DDalpt[ij] = G->ddalp[ij] - ca;
  }
  double trDDW = 0.0, dWdW = 0.0, dWda = 0.0, trDDa = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      trDDW += gtu[SYM[k][l]] * DDW[SYM[k][l]];
      dWdW += gtu[SYM[k][l]] * G->dW[k] * G->dW[l];
      dWda += gtu[SYM[k][l]] * G->dW[k] * G->dalp[l];
      trDDa += gtu[SYM[k][l]] * DDalpt[SYM[k][l]];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      int ij = SYM[i][j];
      double RW = (DDW[ij] + gt[ij] * trDDW) / W - 2.0 * gt[ij] * dWdW / (W * W);
      G->Ric[ij] = Rt[ij] + RW;
      G->DDa[ij] = DDalpt[ij] +
                   (G->dW[i] * G->dalp[j] + G->dW[j] * G->dalp[i] - gt[ij] * dWda) / W;
    }
  double trR = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) trR += gtu[SYM[k][l]] * G->Ric[SYM[k][l]];
  G->Rsc = W * W * trR;
  G->Lapa = W * W * trDDa - W * dWda;

  /* At^ij and At_ij At^ij */
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += gtu[SYM[i][k]] * gtu[SYM[j][l]] * G->At[SYM[k][l]];
      G->Atu[SYM[i][j]] = s;
    }
  double AA = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) AA += G->At[SYM[i][j]] * G->Atu[SYM[i][j]];
  G->AA = AA;
  G->K = G->Kh + 2.0 * G->Th;
}

/* Z4c sources (everything but advection and dissipation) at active point q */
static void z4c_sources(const pointgeo* G, const orc_params* prm, double src[NF]) {
  const double* gt = G->gt;
  const double* gtu = G->gtu;
  const double* At = G->At;
  double W = G->W, alp = G->alp, K = G->K, Th = G->Th;
  double k1 = prm->kappa1, k2 = prm->kappa2;

  double divb = G->dbet[0][0] + G->dbet[1][1] + G->dbet[2][2];

  src[F_W] = W / 3.0 * (alp * K - divb);

  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      int ij = SYM[i][j];
      double s = -2.0 * alp * At[ij];
      for (int k = 0; k < 3; ++k)
        s += gt[SYM[i][k]] * G->dbet[j][k] + gt[SYM[j][k]] * G->dbet[i][k];
      s -= 2.0 / 3.0 * gt[ij] * divb;
      src[F_GXX + ij] = s;
    }

  src[F_KH] = -G->Lapa + alp * (G->AA + K * K / 3.0) + alp * k1 * (1.0 - k2) * Th;
  src[F_TH] = 0.5 * alp * (G->Rsc - G->AA + 2.0 / 3.0 * K * K) - alp * k1 * (2.0 + k2) * Th;

  /* X_ij = -D_i D_j alpha + alpha R_ij, trace-free part w.r.t. gt */
  double X[6], trX = 0.0;
  for (int ij = 0; ij < 6; ++ij) X[ij] = -G->DDa[ij] + alp * G->Ric[ij];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) trX += gtu[SYM[k][l]] * X[SYM[k][l]];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      int ij = SYM[i][j];
      double AikAkj = 0.0; /* At_ik gt^kl At_lj */
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) AikAkj += At[SYM[i][k]] * gtu[SYM[k][l]] * At[SYM[l][j]];
      double s = W * W * (X[ij] - gt[ij] * trX / 3.0);
      s += alp * (K * At[ij] - 2.0 * AikAkj);
      for (int k = 0; k < 3; ++k)
        s += At[SYM[i][k]] * G->dbet[j][k] + At[SYM[j][k]] * G->dbet[i][k];
      s -= 2.0 / 3.0 * At[ij] * divb;
      src[F_AXX + ij] = s;
    }

  /* d_j d_k beta^k (gradient of the divergence) */
  double ddivb[3];
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += G->ddbet[k][SYM[j][k]];
    ddivb[j] = s;
  }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += -2.0 * G->Atu[SYM[i][j]] * G->dalp[j];
    double inner = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) inner += G->Gu[i][SYM[j][k]] * G->Atu[SYM[j][k]];
    for (int j = 0; j < 3; ++j) inner -= 3.0 * G->Atu[SYM[i][j]] * G->dW[j] / W;
    for (int j = 0; j < 3; ++j)
      inner -= gtu[SYM[i][j]] * (2.0 * G->dKh[j] + G->dTh[j]) / 3.0;
    s += 2.0 * alp * inner;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += gtu[SYM[j][k]] * G->ddbet[i][SYM[j][k]];
    for (int j = 0; j < 3; ++j) s += gtu[SYM[i][j]] * ddivb[j] / 3.0;
    s += 2.0 / 3.0 * G->Gd[i] * divb;
    for (int k = 0; k < 3; ++k) s -= G->Gd[k] * G->dbet[k][i];
    s -= 2.0 * alp * k1 * (G->Gam[i] - G->Gd[i]);
    src[F_GAMX + i] = s;
  }

  if (prm->lapse == 1)
    src[F_ALP] = -alp * alp * K;
  else
    src[F_ALP] = -2.0 * alp * (prm->lapse_uses_khat ? G->Kh : K);

  for (int i = 0; i < 3; ++i) {
    if (prm->shift == 1) {
      src[F_BETX + i] = 0.0;
      src[F_BX + i] = 0.0;
    } else {
      src[F_BETX + i] = 0.75 * G->B[i];
      src[F_BX + i] = src[F_GAMX + i] - prm->eta * G->B[i];
    }
  }
}

void orc_z4c_rhs_terms(const orc_patch* p, const orc_params* prm, const double* u,
                       double* rhs, int mask) {
  layout L = make_layout(p);
  const int g = p->g;
  const double h = p->dx;
  memset(rhs, 0, sizeof(double) * (size_t)L.sf * NF);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int k = g; k < g + p->n[2]; ++k)
    for (int j = g; j < g + p->n[1]; ++j)
      for (int i = g; i < g + p->n[0]; ++i) {
        ptrdiff_t q = i + j * L.s[1] + k * L.s[2];
        pointgeo G;
        double src[NF];
        if (mask & 1) {
          point_geometry(u, &L, h, q, &G);
          z4c_sources(&G, prm, src);
        } else {
          load_point(u, &L, q, &G);
          for (int f = 0; f < NF; ++f) src[f] = 0.0;
        }
        for (int f = 0; f < NF; ++f) {
          const double* fp = u + f * L.sf;
          double adv = 0.0, ko = 0.0;
          if (mask & 2)
            for (int d = 0; d < 3; ++d) adv += G.bet[d] * Dup(fp, q, L.s[d], h, G.bet[d]);
          if (mask & 4) {
            for (int d = 0; d < 3; ++d) ko += Delta6(fp, q, L.s[d]);
            ko *= prm->sigma_ko / (64.0 * h);
          }
          double r = src[f] + adv + ko;
          if (prm->shift == 1 && f >= F_BETX) r = 0.0; /* frozen gauge fields */
          rhs[f * L.sf + q] = r;
        }
      }
}

void orc_z4c_rhs(const orc_patch* p, const orc_params* prm, const double* u, double* rhs) {
  orc_z4c_rhs_terms(p, prm, u, rhs, 7);
}

/* ---------------- outer boundary (Sec. 2.2.2) ---------------- */

static int is_ghost(const orc_patch* p, int i, int j, int k) {
  int g = p->g;
  return i < g || i >= g + p->n[0] || j < g || j >= g + p->n[1] || k < g || k >= g + p->n[2];
}

/* d_t f = -(f - f_flat)/r - (x^i/r) d_i f, with d_i the 2nd-order one-sided
 * difference pointing toward the origin along each axis. */
void orc_sommerfeld_rhs(const orc_patch* p, const double* u, double* rhs) {
  layout L = make_layout(p);
  const double h = p->dx;
  const int g = p->g;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int k = 0; k < L.NZ; ++k)
    for (int j = 0; j < L.NY; ++j)
      for (int i = 0; i < L.NX; ++i) {
        if (!is_ghost(p, i, j, k)) continue;
        ptrdiff_t q = i + j * L.s[1] + k * L.s[2];
        int idx[3] = {i, j, k};
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = p->origin[d] + (idx[d] - g + 0.5) * h;
        double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (int f = 0; f < NF; ++f) {
          const double* fp = u + f * L.sf;
          double s = -(fp[q] - flat_value(f)) / r;
          for (int d = 0; d < 3; ++d) {
            ptrdiff_t st = L.s[d];
            double df;
            if (x[d] > 0.0)
              df = (3.0 * fp[q] - 4.0 * fp[q - st] + fp[q - 2 * st]) / (2.0 * h);
            else
              df = -(3.0 * fp[q] - 4.0 * fp[q + st] + fp[q + 2 * st]) / (2.0 * h);
            s -= x[d] / r * df;
          }
          rhs[f * L.sf + q] = s;
        }
      }
}

void orc_fill_periodic(const orc_patch* p, double* u) {
  layout L = make_layout(p);
  const int g = p->g;
  for (int f = 0; f < NF; ++f)
    for (int k = 0; k < L.NZ; ++k)
      for (int j = 0; j < L.NY; ++j)
        for (int i = 0; i < L.NX; ++i) {
          if (!is_ghost(p, i, j, k)) continue;
          int si = g + (((i - g) % p->n[0]) + p->n[0]) % p->n[0];
          int sj = g + (((j - g) % p->n[1]) + p->n[1]) % p->n[1];
          int sk = g + (((k - g) % p->n[2]) + p->n[2]) % p->n[2];
          u[f * L.sf + i + j * L.s[1] + k * L.s[2]] =
              u[f * L.sf + si + sj * L.s[1] + sk * L.s[2]];
        }
}

/* Equatorial reflection symmetry (Sec. 2.2.2): only z >= 0 is evolved; a
 * field with an odd number of z indices changes sign under z -> -z. */
static int zparity(int f) {
  return (f == F_GXZ || f == F_GYZ || f == F_AXZ || f == F_AYZ || f == F_GAMZ || f == F_BETZ || f == F_BZ)
             ? -1
             : 1;
}

int orc_fill_zreflect(const orc_patch* p, double* u) {
  if (fabs(p->origin[2]) > 1e-12 * p->dx) return -1;
  layout L = make_layout(p);
  const int g = p->g;
  for (int f = 0; f < NF; ++f)
    for (int k = 0; k < g; ++k) /* ghost layer z-index k - g < 0 mirrors 2g - 1 - k */
      for (int j = 0; j < L.NY; ++j)
        for (int i = 0; i < L.NX; ++i)
          u[f * L.sf + i + j * L.s[1] + k * L.s[2]] =
              zparity(f) * u[f * L.sf + i + j * L.s[1] + (2 * g - 1 - k) * L.s[2]];
  return 0;
}

/* ---------------- ADM surface integrals (Sec. 2.3) ---------------- */

#define ORC_PI 3.14159265358979323846

/* Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on the
 * Legendre polynomial P_n (three-term recurrence), Chebyshev-like starting
 * points. */
void orc_gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (n == 1) {
        p1 = z;
        p0 = 1.0;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0); /* P_n'(z) */
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* At cell q: the mass integrand vector sqrt(gamma) gamma^ik gamma^jl
 * (d_j gamma_kl - d_k gamma_jl) (out m[3]), the mixed extrinsic curvature
 * times sqrt(gamma), kk[i][j] = sqrt(gamma) K_i^j, and sqrt(gamma) K (out
 * sk), from gamma_ij = gt_ij / W^2, K_ij = (At_ij + gt_ij K / 3) / W^2,
 * K = Khat + 2 Theta; derivatives by the 4th-order centred D1.  The proper
 * surface element of the coordinate sphere is dS_i = sqrt(gamma) n_i r^2
 * dOmega (n_i = x_i / r), so these are the integrands per coordinate area. */
static void adm_cell(const double* u, const layout* L, double h, ptrdiff_t q, double m[3], double kk[3][3],
                     double* sk) {
  const double W = u[F_W * L->sf + q];
  double gt[6], gtu[6], At[6];
  for (int a = 0; a < 6; ++a) {
    gt[a] = u[(F_GXX + a) * L->sf + q];
    At[a] = u[(F_AXX + a) * L->sf + q];
  }
  const double det = sym_inverse(gt, gtu);
  double gamu[6], dgam[3][6];
  for (int a = 0; a < 6; ++a) gamu[a] = gtu[a] * W * W;
  for (int d = 0; d < 3; ++d) {
    const double dW = D1(u + F_W * L->sf, q, L->s[d], h);
    for (int a = 0; a < 6; ++a) {
      const double dgt = D1(u + (F_GXX + a) * L->sf, q, L->s[d], h);
      dgam[d][a] = dgt / (W * W) - 2.0 * gt[a] * dW / (W * W * W);
    }
  }
  const double sg = sqrt(det) / (W * W * W);
  for (int i = 0; i < 3; ++i) {
    double v = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l)
          v += gamu[SYM[i][k]] * gamu[SYM[j][l]] * (dgam[j][SYM[k][l]] - dgam[k][SYM[j][l]]);
    m[i] = sg * v;
  }
  const double K = u[F_KH * L->sf + q] + 2.0 * u[F_TH * L->sf + q];
  /* K_i^j = gamma^jk K_ik = gt^jk (At_ik + gt_ik K / 3) */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += gtu[SYM[j][k]] * (At[SYM[i][k]] + gt[SYM[i][k]] * K / 3.0);
      kk[i][j] = sg * a;
    }
  *sk = sg * K;
}

int orc_adm_integrals(const orc_patch* p, const double* u, const double c[3], double r, int ntheta, int nphi,
                      double out[5]) {
  layout L = make_layout(p);
  const double h = p->dx;
  const int g = p->g;
  const int N[3] = {L.NX, L.NY, L.NZ};
  double* xg = (double*)malloc(sizeof(double) * ntheta);
  double* wg = (double*)malloc(sizeof(double) * ntheta);
  orc_gauss_legendre(ntheta, xg, wg);
  static const int nodes[4] = {0, 1, 2, 3};
  double M = 0.0, J = 0.0, P[3] = {0.0, 0.0, 0.0};
  int bad = 0;
  for (int it = 0; it < ntheta && !bad; ++it) {
    const double ct = xg[it], st = sqrt(1.0 - ct * ct);
    for (int ip = 0; ip < nphi && !bad; ++ip) {
      const double ph = 2.0 * ORC_PI * ip / nphi;
      const double n[3] = {st * cos(ph), st * sin(ph), ct};
      const double x[3] = {c[0] + r * n[0], c[1] + r * n[1], c[2] + r * n[2]};
      /* 4 nearest cell centres per axis: array index of cell i is i + g,
       * its centre origin + (i + 1/2) h */
      int i0[3];
      double wl[3][4];
      for (int d = 0; d < 3; ++d) {
        const double t = (x[d] - p->origin[d]) / h - 0.5 + g; /* array coordinate */
        i0[d] = (int)floor(t) - 1;
        if (i0[d] < 2 || i0[d] + 3 > N[d] - 3) bad = 1;
        orc_lagrange_weights(4, nodes, t - i0[d], wl[d]);
      }
      if (bad) break;
      double m[3] = {0, 0, 0}, kk[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, sk = 0.0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          for (int e = 0; e < 4; ++e) {
            const ptrdiff_t q = (i0[0] + a) + (ptrdiff_t)(i0[1] + b) * L.s[1] + (ptrdiff_t)(i0[2] + e) * L.s[2];
            double mc[3], kc[3][3], skc;
            adm_cell(u, &L, h, q, mc, kc, &skc);
            const double w = wl[0][a] * wl[1][b] * wl[2][e];
            for (int d = 0; d < 3; ++d) {
              m[d] += w * mc[d];
              for (int f = 0; f < 3; ++f) kk[d][f] += w * kc[d][f];
            }
            sk += w * skc;
          }
      const double dA = wg[it] * (2.0 * ORC_PI / nphi) * r * r; /* coordinate area of the node */
      double mn = 0.0, jn = 0.0;
      for (int d = 0; d < 3; ++d) {
        mn += m[d] * n[d];
        jn += ((x[0] - c[0]) * kk[1][d] - (x[1] - c[1]) * kk[0][d]) * n[d];
      }
      M += dA * mn;
      J += dA * jn;
      /* (K_i^j - delta_i^j K) n_j */
      for (int i = 0; i < 3; ++i) {
        double pn = -sk * n[i];
        for (int d = 0; d < 3; ++d) pn += kk[i][d] * n[d];
        P[i] += dA * pn;
      }
    }
  }
  free(xg);
  free(wg);
  if (bad) return -1;
  out[0] = M / (16.0 * ORC_PI);
  out[1] = J / (8.0 * ORC_PI);
  for (int i = 0; i < 3; ++i) out[2 + i] = P[i] / (8.0 * ORC_PI);
  return 0;
}

/* ---------------- Psi4 extraction (Sec. 2.3) ---------------- */

/* Electric and magnetic parts of the Weyl tensor (vacuum, physical,
 * covariant) and the physical metric at cell q:
 *   E_ij = R_ij - K_ik K^k_j + K K_ij
 *   B_ij = 1/2 (eps_i^kl D_k K_lj + eps_j^kl D_k K_li),  eps_ikl = sqrt(g) [ikl]
 * with g_ij = gt_ij / W^2, K_ij = (At_ij + gt_ij K / 3) / W^2, K = Khat + 2
 * Theta, R_ij the physical Ricci tensor of the RHS (conformal part plus W
 * part), Gamma^i_jk = Gt^i_jk - (delta^i_j d_k W + delta^i_k d_j W - gt_jk
 * gt^il d_l W) / W. */
static void weyl_cell(const double* u, const layout* L, double h, ptrdiff_t q, double E[6], double B[6],
                      double gam[6]) {
  pointgeo G;
  point_geometry(u, L, h, q, &G);
  const double W = G.W, W2 = W * W;
  double Kl[6], gu[6], Kud[3][3]; /* K_ij, g^ij, K^i_j */
  for (int a = 0; a < 6; ++a) {
    gam[a] = G.gt[a] / W2;
    Kl[a] = (G.At[a] + G.gt[a] * G.K / 3.0) / W2;
    gu[a] = W2 * G.gtu[a];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += gu[SYM[i][k]] * Kl[SYM[k][j]];
      Kud[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double kk = 0.0;
      for (int k = 0; k < 3; ++k) kk += Kl[SYM[i][k]] * Kud[k][j];
      E[SYM[i][j]] = G.Ric[SYM[i][j]] - kk + G.K * Kl[SYM[i][j]];
    }
  /* d_k K_ij from the derivatives of At, gt, W, Khat, Theta */
  double dK[3][6];
  for (int k = 0; k < 3; ++k) {
    const double dKt = G.dKh[k] + 2.0 * G.dTh[k];
    for (int a = 0; a < 6; ++a) {
      const double dA = D1(u + (F_AXX + a) * L->sf, q, L->s[k], h);
      dK[k][a] = (dA + G.dgt[k][a] * G.K / 3.0 + G.gt[a] * dKt / 3.0) / W2 - 2.0 * Kl[a] * G.dW[k] / W;
    }
  }
  /* physical Christoffels Gamma^m_kl */
  double Gp[3][6];
  for (int m = 0; m < 3; ++m)
    for (int k = 0; k < 3; ++k)
      for (int l = k; l < 3; ++l) {
        double gw = 0.0; /* gt^mn d_n W */
        for (int n = 0; n < 3; ++n) gw += G.gtu[SYM[m][n]] * G.dW[n];
        const double c = ((m == k) ? G.dW[l] : 0.0) + ((m == l) ? G.dW[k] : 0.0) - G.gt[SYM[k][l]] * gw;
        Gp[m][SYM[k][l]] = G.Gu[m][SYM[k][l]] - c / W;
      }
  /* DK[k][l][j] = D_k K_lj */
  double DK[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l)
      for (int j = 0; j < 3; ++j) {
        double v = dK[k][SYM[l][j]];
        for (int m = 0; m < 3; ++m)
          v -= Gp[m][SYM[k][l]] * Kl[SYM[m][j]] + Gp[m][SYM[k][j]] * Kl[SYM[l][m]];
        DK[k][l][j] = v;
      }
  /* eps_i^kl = g^ka g^lb sqrt(g) [iab]; sqrt(g) = sqrt(det gt) / W^3 */
  const double gtdet = G.gt[0] * (G.gt[3] * G.gt[5] - G.gt[4] * G.gt[4]) -
                       G.gt[1] * (G.gt[1] * G.gt[5] - G.gt[4] * G.gt[2]) +
                       G.gt[2] * (G.gt[1] * G.gt[4] - G.gt[3] * G.gt[2]);
  const double sg = sqrt(gtdet) / (W2 * W);
  double C[3][3]; /* C_ij = eps_i^kl D_k K_lj */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          const int lc = (a == (i + 1) % 3 && b == (i + 2) % 3) ? 1 : ((b == (i + 1) % 3 && a == (i + 2) % 3) ? -1 : 0);
          if (!lc) continue;
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) v += lc * gu[SYM[k][a]] * gu[SYM[l][b]] * DK[k][l][j];
        }
      C[i][j] = sg * v;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) B[SYM[i][j]] = 0.5 * (C[i][j] + C[j][i]);
}

/* spin-weight -2 spherical harmonic: sqrt((2l+1)/(4 pi)) d^l_{m,2}(theta)
 * e^{i m phi}, with the Wigner d-function
 * d^l_{m,2} = sum_k (-1)^k sqrt((l+m)!(l-m)!(l+2)!(l-2)!) / ((l+m-k)! (l-2-k)!
 *             k! (k+2-m)!) cos(theta/2)^(2l+m-2-2k) sin(theta/2)^(2k+2-m),
 * k from max(0, m-2) to min(l+m, l-2) */
static double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

void orc_swsh(int l, int m, double theta, double phi, double out[2]) {
  const double c = cos(0.5 * theta), s = sin(0.5 * theta);
  const double pre = sqrt(fact(l + m) * fact(l - m) * fact(l + 2) * fact(l - 2));
  double d = 0.0;
  const int k1 = m - 2 > 0 ? m - 2 : 0, k2 = (l + m < l - 2) ? l + m : l - 2;
  for (int k = k1; k <= k2; ++k) {
    const double t = pre / (fact(l + m - k) * fact(l - 2 - k) * fact(k) * fact(k + 2 - m));
    d += ((k & 1) ? -t : t) * pow(c, 2 * l + m - 2 - 2 * k) * pow(s, 2 * k + 2 - m);
  }
  const double a = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI)) * d;
  out[0] = a * cos(m * phi);
  out[1] = a * sin(m * phi);
}

/* Psi4 at the sphere point with angles (theta, phi) about c at radius r:
 * E, B, g interpolated tricubically from the 4 nearest cell centres per axis;
 * orthonormal triad (Gram-Schmidt with g) from the coordinate radial, theta
 * and phi directions; mbar = (e_theta - i e_phi)/sqrt(2);
 * Psi4 = (E_ij - i B_ij) mbar^i mbar^j.  -1 if the stencils leave the array. */
static int psi4_at(const orc_patch* p, const double* u, const double c[3], double r, double ct, double st,
                   double cp, double sp, double out[2]) {
  layout L = make_layout(p);
  const int g = p->g;
  const int N[3] = {L.NX, L.NY, L.NZ};
  static const int nodes[4] = {0, 1, 2, 3};
  const double n[3] = {st * cp, st * sp, ct};
  int i0[3];
  double wl[3][4];
  for (int d = 0; d < 3; ++d) {
    const double x = c[d] + r * n[d];
    const double t = (x - p->origin[d]) / p->dx - 0.5 + g;
    i0[d] = (int)floor(t) - 1;
    if (!(t >= 3.0 && t < N[d] - 4.0)) return -1;
    orc_lagrange_weights(4, nodes, t - i0[d], wl[d]);
  }
  double E[6] = {0}, B[6] = {0}, gam[6] = {0};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int e = 0; e < 4; ++e) {
        const ptrdiff_t q = (i0[0] + a) + (ptrdiff_t)(i0[1] + b) * L.s[1] + (ptrdiff_t)(i0[2] + e) * L.s[2];
        double Ec[6], Bc[6], gc[6];
        weyl_cell(u, &L, p->dx, q, Ec, Bc, gc);
        const double w = wl[0][a] * wl[1][b] * wl[2][e];
        for (int k = 0; k < 6; ++k) {
          E[k] += w * Ec[k];
          B[k] += w * Bc[k];
          gam[k] += w * gc[k];
        }
      }
  /* Gram-Schmidt: e_r, e_theta, e_phi orthonormal in g */
  double v[3][3] = {{n[0], n[1], n[2]}, {ct * cp, ct * sp, -st}, {-sp, cp, 0.0}};
  double e[3][3];
  for (int a = 0; a < 3; ++a) {
    double w[3] = {v[a][0], v[a][1], v[a][2]};
    for (int b = 0; b < a; ++b) {
      double dot = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) dot += gam[SYM[i][j]] * w[i] * e[b][j];
      for (int i = 0; i < 3; ++i) w[i] -= dot * e[b][i];
    }
    double nn = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) nn += gam[SYM[i][j]] * w[i] * w[j];
    nn = sqrt(nn);
    for (int i = 0; i < 3; ++i) e[a][i] = w[i] / nn;
  }
  /* mbar mbar = P - i Q, P = (e_th e_th - e_ph e_ph)/2, Q = (e_th e_ph + e_ph e_th)/2 */
  double EP = 0.0, EQ = 0.0, BP = 0.0, BQ = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double P = 0.5 * (e[1][i] * e[1][j] - e[2][i] * e[2][j]);
      const double Q = 0.5 * (e[1][i] * e[2][j] + e[2][i] * e[1][j]);
      EP += E[SYM[i][j]] * P;
      EQ += E[SYM[i][j]] * Q;
      BP += B[SYM[i][j]] * P;
      BQ += B[SYM[i][j]] * Q;
    }
  out[0] = EP - BQ;
  out[1] = -(EQ + BP);
  return 0;
}

int orc_psi4_point(const orc_patch* p, const double* u, const double c[3], double r, double theta, double phi,
                   double out[2]) {
  return psi4_at(p, u, c, r, cos(theta), sin(theta), cos(phi), sin(phi), out);
}

int orc_psi4_modes(const orc_patch* p, const double* u, const double c[3], double r, int ntheta, int nphi,
                   int lmax, double* out) {
  const int nm = (lmax + 1) * (lmax + 1) - 4;
  double* xg = (double*)malloc(sizeof(double) * ntheta);
  double* wg = (double*)malloc(sizeof(double) * ntheta);
  orc_gauss_legendre(ntheta, xg, wg);
  for (int k = 0; k < 2 * nm; ++k) out[k] = 0.0;
  int bad = 0;
  for (int it = 0; it < ntheta && !bad; ++it) {
    const double ct = xg[it], st = sqrt(1.0 - ct * ct), th = acos(ct);
    for (int ip = 0; ip < nphi && !bad; ++ip) {
      const double ph = 2.0 * ORC_PI * ip / nphi;
      double psi[2];
      if (psi4_at(p, u, c, r, ct, st, cos(ph), sin(ph), psi)) {
        bad = 1;
        break;
      }
      const double w = wg[it] * 2.0 * ORC_PI / nphi;
      int k = 0;
      for (int l = 2; l <= lmax; ++l)
        for (int m = -l; m <= l; ++m, ++k) {
          double y[2];
          orc_swsh(l, m, th, ph, y);
          /* Psi4 conj(Y) */
          out[2 * k] += w * (psi[0] * y[0] + psi[1] * y[1]);
          out[2 * k + 1] += w * (psi[1] * y[0] - psi[0] * y[1]);
        }
    }
  }
  free(xg);
  free(wg);
  return bad ? -1 : 0;
}

/* ---------------- algebraic constraints ---------------- */

static void enforce_point(double* u, ptrdiff_t sf, ptrdiff_t q, double w_floor) {
  double gt[6], gtu[6];
  for (int a = 0; a < 6; ++a) gt[a] = u[(F_GXX + a) * sf + q];
  double xx = gt[0], xy = gt[1], xz = gt[2], yy = gt[3], yz = gt[4], zz = gt[5];
  double det = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
  double fac = 1.0 / cbrt(det); /* det gt = 1 */
  for (int a = 0; a < 6; ++a) gt[a] *= fac;
  sym_inverse(gt, gtu);
  double tr = 0.0; /* gt^kl At_kl */
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) tr += gtu[SYM[k][l]] * u[(F_AXX + SYM[k][l]) * sf + q];
  for (int a = 0; a < 6; ++a) {
    u[(F_GXX + a) * sf + q] = gt[a];
    u[(F_AXX + a) * sf + q] -= gt[a] * tr / 3.0;
  }
  double W = u[F_W * sf + q];
  if (W < w_floor) u[F_W * sf + q] = w_floor;
}

void orc_enforce(const orc_patch* p, double w_floor, int all_points, double* u) {
  layout L = make_layout(p);
  for (int k = 0; k < L.NZ; ++k)
    for (int j = 0; j < L.NY; ++j)
      for (int i = 0; i < L.NX; ++i) {
        if (!all_points && is_ghost(p, i, j, k)) continue;
        enforce_point(u, L.sf, i + j * L.s[1] + k * L.s[2], w_floor);
      }
}

/* ---------------- classical RK4 (Sec. 2.2) ---------------- */

/* src (may be NULL): a term added to the right-hand side at the active
 * points, e.g. the matter terms of the Z4c equations (Sec. 2.1.2) */
void orc_rk4_stage_src(const orc_patch* p, const orc_params* prm, int s, double dt,
                       int evolve_ghosts, const double* us, const double* un, double* y,
                       double* out, const double* src) {
  layout L = make_layout(p);
  size_t np = (size_t)L.sf * NF;
  double* k = (double*)malloc(sizeof(double) * np);
  orc_z4c_rhs(p, prm, us, k);
  if (src)
    for (int kk = 0; kk < L.NZ; ++kk)
      for (int j = 0; j < L.NY; ++j)
        for (int i = 0; i < L.NX; ++i)
          if (!is_ghost(p, i, j, kk))
            for (int f = 0; f < NF; ++f) {
              ptrdiff_t q = f * L.sf + i + j * L.s[1] + kk * L.s[2];
              k[q] += src[q];
            }
  if (evolve_ghosts) {
    double* kg = (double*)malloc(sizeof(double) * np);
    orc_sommerfeld_rhs(p, us, kg);
    for (int kk = 0; kk < L.NZ; ++kk)
      for (int j = 0; j < L.NY; ++j)
        for (int i = 0; i < L.NX; ++i)
          if (is_ghost(p, i, j, kk))
            for (int f = 0; f < NF; ++f) {
              ptrdiff_t q = f * L.sf + i + j * L.s[1] + kk * L.s[2];
              k[q] = kg[q];
            }
    free(kg);
  }
  static const double c[4] = {0.5, 0.5, 1.0, 0.0};
  static const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  double bdt = b[s - 1] * dt, cdt = c[s - 1] * dt;
  memcpy(out, un, sizeof(double) * np);
  for (int kk = 0; kk < L.NZ; ++kk)
    for (int j = 0; j < L.NY; ++j)
      for (int i = 0; i < L.NX; ++i) {
        if (!evolve_ghosts && is_ghost(p, i, j, kk)) continue;
        ptrdiff_t q0 = i + j * L.s[1] + kk * L.s[2];
        for (int f = 0; f < NF; ++f) {
          ptrdiff_t q = f * L.sf + q0;
          if (s == 1) {
            y[q] = un[q] + bdt * k[q];
            out[q] = un[q] + cdt * k[q];
          } else if (s < 4) {
            y[q] = y[q] + bdt * k[q];
            out[q] = un[q] + cdt * k[q];
          } else {
            out[q] = y[q] + bdt * k[q];
          }
        }
        enforce_point(out, L.sf, q0, prm->w_floor);
      }
  free(k);
}

void orc_rk4_stage(const orc_patch* p, const orc_params* prm, int s, double dt,
                   int evolve_ghosts, const double* us, const double* un, double* y,
                   double* out) {
  orc_rk4_stage_src(p, prm, s, dt, evolve_ghosts, us, un, y, out, NULL);
}

void orc_rk4_step(const orc_patch* p, const orc_params* prm, int bc, double dt, double* u) {
  layout L = make_layout(p);
  size_t np = (size_t)L.sf * NF;
  double* un = (double*)malloc(sizeof(double) * np);
  double* y = (double*)malloc(sizeof(double) * np);
  double* a = (double*)malloc(sizeof(double) * np);
  double* b = (double*)malloc(sizeof(double) * np);
  const int zsym = (bc & ORC_BC_ZREFLECT) != 0;
  bc &= ~ORC_BC_ZREFLECT;
  if (zsym) orc_fill_zreflect(p, u);
  memcpy(un, u, sizeof(double) * np);
  int eg = (bc == ORC_BC_SOMMERFELD);
  const double* cur = un;
  double* bufs[2] = {a, b};
  for (int s = 1; s <= 4; ++s) {
    double* out = (s == 4) ? u : bufs[(s - 1) % 2];
    if (bc == ORC_BC_PERIODIC) orc_fill_periodic(p, (double*)cur);
    if (zsym) orc_fill_zreflect(p, (double*)cur);
    orc_rk4_stage(p, prm, s, dt, eg, cur, un, y, out);
    cur = out;
  }
  if (bc == ORC_BC_PERIODIC) orc_fill_periodic(p, u);
  if (zsym) orc_fill_zreflect(p, u);
  free(un);
  free(y);
  free(a);
  free(b);
}

/* ---------------- constraint monitor (Sec. 2.3) ---------------- */

void orc_constraints(const orc_patch* p, const double* u, double w_excise, double* c,
                     double norms[4]) {
  layout L = make_layout(p);
  const int g = p->g;
  const double h = p->dx;
  memset(c, 0, sizeof(double) * (size_t)L.sf * 4);
  double sums[4] = {0, 0, 0, 0};
  long cnt = 0;
  for (int k = g; k < g + p->n[2]; ++k)
    for (int j = g; j < g + p->n[1]; ++j)
      for (int i = g; i < g + p->n[0]; ++i) {
        ptrdiff_t q = i + j * L.s[1] + k * L.s[2];
        pointgeo G;
        point_geometry(u, &L, h, q, &G);
        /* H = R + 2/3 K^2 - At_ij At^ij */
        double H = G.Rsc + 2.0 / 3.0 * G.K * G.K - G.AA;
        /* M_i = gt^jk Dt_j At_ki - 3 At_i^j d_j W / W - 2/3 d_i K */
        double dAt[3][6];
        for (int d = 0; d < 3; ++d)
          for (int a = 0; a < 6; ++a) dAt[d][a] = D1(u + (F_AXX + a) * L.sf, q, L.s[d], h);
        double Ml[3];
        for (int i2 = 0; i2 < 3; ++i2) {
          double s = 0.0;
          for (int j2 = 0; j2 < 3; ++j2)
            for (int k2 = 0; k2 < 3; ++k2) {
              /* Dt_j At_ki = d_j At_ki - Gt^l_jk At_li - Gt^l_ji At_kl */
              double DA = dAt[j2][SYM[k2][i2]];
              for (int l = 0; l < 3; ++l)
                DA -= G.Gu[l][SYM[j2][k2]] * G.At[SYM[l][i2]] +
                      G.Gu[l][SYM[j2][i2]] * G.At[SYM[k2][l]];
              s += G.gtu[SYM[j2][k2]] * DA;
            }
          for (int j2 = 0; j2 < 3; ++j2) {
            double Aij = 0.0; /* At_i^j = gt^jk At_ik */
            for (int k2 = 0; k2 < 3; ++k2) Aij += G.gtu[SYM[j2][k2]] * G.At[SYM[i2][k2]];
            s -= 3.0 * Aij * G.dW[j2] / G.W;
          }
          s -= 2.0 / 3.0 * (G.dKh[i2] + 2.0 * G.dTh[i2]);
          Ml[i2] = s;
        }
        double Mu[3];
        for (int i2 = 0; i2 < 3; ++i2) {
          double s = 0.0;
          for (int j2 = 0; j2 < 3; ++j2) s += G.gtu[SYM[i2][j2]] * Ml[j2];
          Mu[i2] = G.W * G.W * s;
        }
        c[q] = H;
        for (int d = 0; d < 3; ++d) c[(1 + d) * L.sf + q] = Mu[d];
        if (G.W >= w_excise) {
          sums[0] += H * H;
          for (int d = 0; d < 3; ++d) sums[1 + d] += Mu[d] * Mu[d];
          cnt++;
        }
      }
  for (int a = 0; a < 4; ++a) norms[a] = cnt > 0 ? sqrt(sums[a] / (double)cnt) : 0.0;
}

/* ---------------- pi-symmetry monitor (Sec. 3.2) ---------------- */

double orc_pi_symmetry(const orc_patch* p, const double* u, int include_ghosts) {
  layout L = make_layout(p);
  double mx = 0.0;
  for (int f = 0; f < NF; ++f)
    for (int k = 0; k < L.NZ; ++k)
      for (int j = 0; j < L.NY; ++j)
        for (int i = 0; i < L.NX; ++i) {
          if (!include_ghosts && is_ghost(p, i, j, k)) continue;
          int im = L.NX - 1 - i, jm = L.NY - 1 - j;
          double a = u[f * L.sf + i + j * L.s[1] + k * L.s[2]];
          double b = u[f * L.sf + im + jm * L.s[1] + k * L.s[2]];
          double d = fabs(a - PARITY[f] * b);
          if (d > mx || d != d) mx = (d != d) ? INFINITY : d;
        }
  return mx;
}

/* ---------------- Berger-Oliger inter-level operators (Sec. 2.2.1) ---------------- */

void orc_lagrange_weights(int nnodes, const int* nodes, double x, double* w) {
  for (int j = 0; j < nnodes; ++j) {
    double num = 1.0, den = 1.0;
    for (int m = 0; m < nnodes; ++m) {
      if (m == j) continue;
      num *= x - nodes[m];
      den *= (double)(nodes[j] - nodes[m]);
    }
    w[j] = num / den;
  }
}

/* offset of the child's origin in parent cells; -1 if not an integer */
static int child_offset(const orc_patch* parent, const orc_patch* child, int off[3]) {
  if (fabs(parent->dx - 2.0 * child->dx) > 1e-14 * parent->dx) return -1;
  for (int d = 0; d < 3; ++d) {
    double t = (child->origin[d] - parent->origin[d]) / parent->dx;
    double r = floor(t + 0.5);
    if (fabs(t - r) > 1e-9) return -1;
    off[d] = (int)r;
  }
  return 0;
}

static int floor_div2(int i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

int orc_prolong_ghosts(const orc_patch* parent, const double* up, const orc_patch* child,
                       double* uc) {
  return orc_prolong_ghosts_ex(parent, up, child, uc, 0);
}

/* 6th-order prolongation of the parent's data onto the child's ghost cells
 * (all_cells = 0) or onto every cell of the child's array (all_cells = 1). */
static int prolong_cells(const orc_patch* parent, const double* up, const orc_patch* child, double* uc,
                         int skip_zlower, int all_cells);

int orc_prolong_ghosts_ex(const orc_patch* parent, const double* up, const orc_patch* child,
                          double* uc, int skip_zlower) {
  return prolong_cells(parent, up, child, uc, skip_zlower, 0);
}

int orc_move_patch(const orc_patch* parent, const double* up, const orc_patch* oldc, const double* uo,
                   const orc_patch* newc, double* un, int skip_zlower) {
  int sh[3];
  if (oldc->g != newc->g || fabs(oldc->dx - newc->dx) > 1e-14 * oldc->dx) return -1;
  for (int d = 0; d < 3; ++d) {
    if (oldc->n[d] != newc->n[d]) return -1;
    const double t = (newc->origin[d] - oldc->origin[d]) / newc->dx;
    const double r = floor(t + 0.5);
    if (fabs(t - r) > 1e-9) return -1;
    sh[d] = (int)r; /* new array index + sh = old array index */
  }
  if (prolong_cells(parent, up, newc, un, skip_zlower, 1)) return -1;
  layout L = make_layout(newc);
  const int g = newc->g;
  for (int k = 0; k < L.NZ; ++k)
    for (int j = 0; j < L.NY; ++j)
      for (int i = 0; i < L.NX; ++i) {
        const int io = i + sh[0], jo = j + sh[1], ko = k + sh[2];
        if (io < g || io >= g + oldc->n[0] || jo < g || jo >= g + oldc->n[1] || ko < g ||
            ko >= g + oldc->n[2])
          continue; /* not an active cell of the old patch: keep the prolonged value */
        const ptrdiff_t qn = i + j * L.s[1] + (ptrdiff_t)k * L.s[2];
        const ptrdiff_t qo = io + jo * L.s[1] + (ptrdiff_t)ko * L.s[2];
        for (int f = 0; f < NF; ++f) un[f * L.sf + qn] = uo[f * L.sf + qo];
      }
  return 0;
}

int orc_interp_point(const orc_patch* p, const double* u, int f, const double x[3], double* out) {
  layout L = make_layout(p);
  const int g = p->g;
  static const int nodes[4] = {0, 1, 2, 3};
  int i0[3];
  double w[3][4];
  for (int d = 0; d < 3; ++d) {
    const double t = (x[d] - p->origin[d]) / p->dx - 0.5 + g; /* array coordinate */
    if (!(t >= g + 1.0 && t < g + p->n[d] - 2.0)) return -1; /* 4 active cells */
    i0[d] = (int)floor(t) - 1;
    orc_lagrange_weights(4, nodes, t - i0[d], w[d]);
  }
  double v = 0.0;
  for (int c = 0; c < 4; ++c)
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a)
        v += w[0][a] * w[1][b] * w[2][c] *
             u[f * L.sf + (i0[0] + a) + (i0[1] + b) * L.s[1] + (ptrdiff_t)(i0[2] + c) * L.s[2]];
  *out = v;
  return 0;
}

static int prolong_cells(const orc_patch* parent, const double* up, const orc_patch* child, double* uc,
                         int skip_zlower, int all_cells) {
  int off[3];
  if (child_offset(parent, child, off)) return -1;
  layout Lp = make_layout(parent), Lc = make_layout(child);
  const int gc = child->g, gp = parent->g;
  /* 6-point Lagrange weights for the two offsets +1/4 and -1/4 */
  static const int nodes_p[6] = {-2, -1, 0, 1, 2, 3};
  static const int nodes_m[6] = {-3, -2, -1, 0, 1, 2};
  double wp[6], wm[6];
  orc_lagrange_weights(6, nodes_p, 0.25, wp);
  orc_lagrange_weights(6, nodes_m, -0.25, wm);
  int pdim[3] = {Lp.NX, Lp.NY, Lp.NZ};
  int cdim[3] = {Lc.NX, Lc.NY, Lc.NZ};
  /* check that every stencil stays inside the parent array */
  for (int d = 0; d < 3; ++d)
    for (int ic = (d == 2 && skip_zlower) ? 0 : -gc; ic < child->n[d] + gc; ++ic) {
      int P = off[d] + floor_div2(ic);
      int lo = (ic & 1) ? P - 2 : P - 3, hi = (ic & 1) ? P + 3 : P + 2;
      if (lo + gp < 0 || hi + gp >= pdim[d]) return -1;
    }
  for (int kc = 0; kc < cdim[2]; ++kc)
    for (int jc = 0; jc < cdim[1]; ++jc)
      for (int ic = 0; ic < cdim[0]; ++ic) {
        if (!all_cells && !is_ghost(child, ic, jc, kc)) continue;
        if (skip_zlower && kc < gc) continue; /* left to the reflection */
        int ci[3] = {ic - gc, jc - gc, kc - gc};
        int base[3];
        const double* w[3];
        const int* nd[3];
        for (int d = 0; d < 3; ++d) {
          base[d] = off[d] + floor_div2(ci[d]) + gp;
          int odd = ci[d] & 1; /* odd child index: offset +1/4 */
          w[d] = odd ? wp : wm;
          nd[d] = odd ? nodes_p : nodes_m;
        }
        for (int f = 0; f < NF; ++f) {
          const double* fp = up + f * Lp.sf;
          double v = 0.0;
          for (int c = 0; c < 6; ++c)
            for (int b = 0; b < 6; ++b)
              for (int a = 0; a < 6; ++a) {
                ptrdiff_t q = (base[0] + nd[0][a]) + (base[1] + nd[1][b]) * Lp.s[1] +
                              (ptrdiff_t)(base[2] + nd[2][c]) * Lp.s[2];
                v += w[0][a] * w[1][b] * w[2][c] * fp[q];
              }
          uc[f * Lc.sf + ic + jc * Lc.s[1] + kc * Lc.s[2]] = v;
        }
      }
  return 0;
}

int orc_restrict(const orc_patch* parent, double* up, const orc_patch* child,
                 const double* uc) {
  int off[3];
  if (child_offset(parent, child, off)) return -1;
  for (int d = 0; d < 3; ++d)
    if (child->n[d] % 2) return -1;
  layout Lp = make_layout(parent), Lc = make_layout(child);
  const int gc = child->g, gp = parent->g;
  static const int nodes[4] = {-1, 0, 1, 2};
  double w[4];
  orc_lagrange_weights(4, nodes, 0.5, w);
  for (int d = 0; d < 3; ++d)
    if (off[d] < 0 || off[d] + child->n[d] / 2 > parent->n[d]) return -1;
  for (int K = 0; K < child->n[2] / 2; ++K)
    for (int J = 0; J < child->n[1] / 2; ++J)
      for (int I = 0; I < child->n[0] / 2; ++I) {
        ptrdiff_t qp = (I + off[0] + gp) + (J + off[1] + gp) * Lp.s[1] +
                       (ptrdiff_t)(K + off[2] + gp) * Lp.s[2];
        for (int f = 0; f < NF; ++f) {
          const double* fc = uc + f * Lc.sf;
          double v = 0.0;
          for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
              for (int a = 0; a < 4; ++a) {
                ptrdiff_t q = (2 * I + nodes[a] + gc) + (2 * J + nodes[b] + gc) * Lc.s[1] +
                              (ptrdiff_t)(2 * K + nodes[c] + gc) * Lc.s[2];
                v += w[a] * w[b] * w[c] * fc[q];
              }
          up[f * Lp.sf + qp] = v;
        }
      }
  return 0;
}

long orc_exchange(const orc_patch* a, double* ua, const orc_patch* b, double* ub) {
  if (fabs(a->dx - b->dx) > 1e-14 * a->dx || a->g != b->g) return -1;
  int off[3]; /* b's cell index of a's cell 0 */
  for (int d = 0; d < 3; ++d) {
    double t = (a->origin[d] - b->origin[d]) / a->dx;
    double r = floor(t + 0.5);
    if (fabs(t - r) > 1e-9) return -1;
    off[d] = (int)r;
  }
  layout La = make_layout(a), Lb = make_layout(b);
  const int g = a->g;
  long touched = 0;
  for (int k = -g; k < a->n[2] + g; ++k)
    for (int j = -g; j < a->n[1] + g; ++j)
      for (int i = -g; i < a->n[0] + g; ++i) {
        int ib = i + off[0], jb = j + off[1], kb = k + off[2];
        int a_act = i >= 0 && i < a->n[0] && j >= 0 && j < a->n[1] && k >= 0 && k < a->n[2];
        int b_in = ib >= -g && ib < b->n[0] + g && jb >= -g && jb < b->n[1] + g &&
                   kb >= -g && kb < b->n[2] + g;
        if (!b_in) continue;
        int b_act = ib >= 0 && ib < b->n[0] && jb >= 0 && jb < b->n[1] && kb >= 0 && kb < b->n[2];
        ptrdiff_t qa = (i + g) + (j + g) * La.s[1] + (ptrdiff_t)(k + g) * La.s[2];
        ptrdiff_t qb = (ib + g) + (jb + g) * Lb.s[1] + (ptrdiff_t)(kb + g) * Lb.s[2];
        if (a_act && b_act) {
          for (int f = 0; f < NF; ++f) {
            double m = 0.5 * (ua[f * La.sf + qa] + ub[f * Lb.sf + qb]);
            ua[f * La.sf + qa] = m;
            ub[f * Lb.sf + qb] = m;
          }
          touched++;
        } else if (b_act && !a_act) {
          for (int f = 0; f < NF; ++f) ua[f * La.sf + qa] = ub[f * Lb.sf + qb];
          touched++;
        } else if (a_act && !b_act) {
          for (int f = 0; f < NF; ++f) ub[f * Lb.sf + qb] = ua[f * La.sf + qa];
          touched++;
        }
      }
  return touched;
}
