/*
 * Z4c oracle: a plain, slow, FP64 CPU statement of the hot path (test
 * infrastructure only -- only the tests, the smoke check and the benchmark's
 * CPU-baseline arm may load it; the product library never does).
 *
 * What pins each function (tests/test_oracle_*.py), i.e. checks it against
 * something other than itself:
 *   orc_stencils        exact on polynomials to each stencil's order; upwind
 *                       bias closed form on x^6; 6th difference = 720 h^6 x^6
 *   orc_z4c_rhs(_terms) every field converges at 4th order to the continuum
 *                       ADM time derivative on generic smooth data (physical
 *                       Christoffels/Ricci by definition, autograd
 *                       derivatives); Minkowski exactly 0; Brill-Lindquist
 *                       closed forms (W, alpha, gt, Gamt RHS exactly 0;
 *                       d_t Khat -> -2 psi^-8 |grad psi|^2); gauge-wave RHS ->
 *                       d/dt of the closed form; KO and advection closed forms
 *   orc_constraints     H, M^i converge at 4th order to the ADM constraints
 *   orc_sommerfeld_rhs  2nd-order convergence on an exact outgoing wave
 *   orc_rk4_step/stage  gauge wave (closed form in time) at 4th order
 *   orc_fill_periodic   brute force
 *   orc_fill_zreflect   brute force; a z-symmetric full-domain evolution
 *                       equals the half-domain one with reflection
 *   orc_enforce         det gt = 1 and gt^ij At_ij = 0 to rounding
 *   orc_pi_symmetry     symmetrised data 0, noisy data > 0; RHS and RK4 keep 0
 *   orc_prolong_ghosts  exact on degree <= 5, not on degree 6
 *   orc_restrict        exact on degree <= 3, not on degree 4
 *   orc_exchange        brute force of the three overlap rules
 *   orc_lagrange_weights exact fractions (Fraction arithmetic)
 *   orc_move_patch      copies equal the old cells, prolonged cells exact
 *                       on degree-5 polynomials; shift and back restores
 *   orc_interp_point    exact on tricubic polynomials
 *   orc_swsh            closed forms of l = 2, orthonormality to l = 8
 *   orc_psi4_point      linearised plane waves along several directions:
 *                       -d_t^2 (h_+ - i h_x) at 4th order; Schwarzschild:
 *                       0 at 4th order
 *   orc_psi4_modes      modes of a plane wave against a fine quadrature of
 *                       its closed-form Psi4 on the sphere
 *   orc_adm_integrals   Schwarzschild in isotropic coordinates: M psi(r)
 *                       (closed form) at 4th order in dx; Bowen-York spin:
 *                       J_z = J and boost: P = P for any conformal factor;
 *                       a pure-gauge perturbation of flat space gives a
 *                       mass of second order; nodes integrate polynomials
 *                       exactly (orc_gauss_legendre)
 *   Berger-Oliger driver (oracle/__init__.py) gauge wave on 3 nested levels,
 *                       2nd-order convergence with quadratic time interpolation
 * No function is left "parity unpinned".
 *
 * Field order (25 evolved fields of the Z4c/BSSN puncture system, Sec. 2.1.1):
 *   0 W; 1-6 gt_xx,xy,xz,yy,yz,zz; 7 Khat; 8 Theta; 9-14 At_xx..zz;
 *   15-17 Gamt^x,y,z; 18 alpha; 19-21 beta^x,y,z; 22-24 B^x,y,z.
 * Storage of one patch: double u[25][n2+2g][n1+2g][n0+2g], x fastest, no
 * padding.  Active cell i (0 <= i < n) has its centre at
 * origin + (i + 1/2) dx; ghost cells are i = -g..-1 and n..n+g-1.
 */
#ifndef Z4C_ORACLE_H
#define Z4C_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NF 25

typedef struct {
  int n[3];          /* active cells per axis */
  int g;             /* ghost width (3) */
  double dx;         /* grid spacing, same on all axes */
  double origin[3];  /* lower face of active cell 0 */
} orc_patch;

typedef struct {
  double kappa1, kappa2;  /* Z4c damping (Sec. 3: 0.005/M, 0) */
  double eta;             /* Gamma-driver damping (Sec. 3: 0.36/M) */
  double sigma_ko;        /* Kreiss-Oliger coefficient (Sec. 2.2: 0.5) */
  double w_floor;         /* floor applied to W after each stage write */
  int lapse;              /* 0: 1+log slicing, 1: harmonic slicing */
  int shift;              /* 0: hyperbolic Gamma driver, 1: frozen (beta=B=0) */
  int lapse_uses_khat;    /* 0: lapse source uses K = Khat + 2 Theta; 1: Khat */
} orc_params;

/* ghost treatment of a uniform patch; ORC_BC_ZREFLECT may be or-ed in:
 * equatorial reflection symmetry at z = 0 (Sec. 2.2.2) for a patch whose
 * lower z face is z = 0 -- its z < 0 ghosts mirror z > 0 before every stage */
enum { ORC_BC_SOMMERFELD = 0, ORC_BC_PERIODIC = 1, ORC_BC_FROZEN = 2, ORC_BC_NONE = 3, ORC_BC_ZREFLECT = 8 };

size_t orc_patch_points(const orc_patch* p);

/* Z4c right-hand side at every active point (ghost entries of rhs set to 0). */
void orc_z4c_rhs(const orc_patch* p, const orc_params* prm, const double* u, double* rhs);

/* Same, with only the selected terms: bit0 = sources, bit1 = advection,
 * bit2 = Kreiss-Oliger.  orc_z4c_rhs == mask 7. */
void orc_z4c_rhs_terms(const orc_patch* p, const orc_params* prm, const double* u,
                       double* rhs, int mask);

/* Sommerfeld outgoing-wave right-hand side at every ghost point. */
void orc_sommerfeld_rhs(const orc_patch* p, const double* u, double* rhs);

/* periodic ghost fill */
void orc_fill_periodic(const orc_patch* p, double* u);

/* equatorial reflection: the z < 0 ghost layers (all x, y) take the mirror
 * value f(x, y, -z) = s_z f(x, y, z), s_z = -1 for fields with an odd number
 * of z indices (gt_xz, gt_yz, At_xz, At_yz, Gamt^z, beta^z, B^z).  The patch's
 * lower z face must be z = 0 (else -1). */
int orc_fill_zreflect(const orc_patch* p, double* u);

/* algebraic constraints: det gt = 1, At trace-free, W >= w_floor; at active
 * points (all points when all_points != 0) */
void orc_enforce(const orc_patch* p, double w_floor, int all_points, double* u);

/* one classical RK4 step of a uniform patch in place.  For ORC_BC_NONE the
 * caller must fill ghosts itself, so this variant is not offered here; the
 * AMR driver uses orc_rk4_stage. */
void orc_rk4_step(const orc_patch* p, const orc_params* prm, int bc, double dt, double* u);

/* one RK4 stage s (1..4), as used by the Berger-Oliger driver:
 *   k = F(us) at active points (+ Sommerfeld at ghost points if evolve_ghosts)
 *   s==1: y = un + dt/6 k ; s==2,3: y += dt/3 k ; s==4: out = y + dt/6 k
 *   s<4: out = un + c_s dt k (c = 1/2, 1/2, 1)
 * then enforcement on the written points.  Points that are not updated keep
 * the values of un in out. */
/* orc_rk4_stage with src (NULL or a patch array) added to the right-hand
 * side at the active points (the matter terms of the Z4c equations). */
void orc_rk4_stage_src(const orc_patch* p, const orc_params* prm, int s, double dt,
                       int evolve_ghosts, const double* us, const double* un, double* y,
                       double* out, const double* src);
void orc_rk4_stage(const orc_patch* p, const orc_params* prm, int s, double dt,
                   int evolve_ghosts, const double* us, const double* un, double* y,
                   double* out);

/* Hamiltonian and momentum constraints (index up) at active points:
 * c[4][points] (ghost entries 0) and volume-normalised L2 norms over active
 * points with W >= w_excise. */
void orc_constraints(const orc_patch* p, const double* u, double w_excise, double* c,
                     double norms[4]);

/* Rotation-by-pi (x,y -> -x,-y) symmetry monitor: max over points and fields
 * of |f(x,y,z) - s_f f(-x,-y,z)|.  Patch must be centred on x=y=0. */
double orc_pi_symmetry(const orc_patch* p, const double* u, int include_ghosts);

/* 6th-order Lagrange prolongation from a parent state into every ghost point
 * of a child patch (2:1, cell centred). Returns 0, or -1 if the stencil leaves
 * the parent array or the patches are not aligned. */
int orc_prolong_ghosts(const orc_patch* parent, const double* up, const orc_patch* child,
                       double* uc);
/* Same; with skip_zlower the child's z < 0 ghost layers are left alone (they
 * come from the equatorial reflection) and the parent is only read at z >= -3
 * cells. */
int orc_prolong_ghosts_ex(const orc_patch* parent, const double* up, const orc_patch* child,
                          double* uc, int skip_zlower);

/* 4th-order Lagrange restriction of the child onto every parent cell covered
 * by the child's active region (child ghosts must be valid). */
int orc_restrict(const orc_patch* parent, double* up, const orc_patch* child,
                 const double* uc);

/* Same-level exchange between two aligned patches: ghosts of each that lie in
 * the other's active region are overwritten; active points present in both are
 * replaced by the average. Returns the number of points touched. */
long orc_exchange(const orc_patch* a, double* ua, const orc_patch* b, double* ub);

/* The finite-difference operators of the RHS at one point (i,j,k are array
 * indices incl. ghosts) of one field: out[0..2] = D_x, D_y, D_z (centred);
 * out[3..5] = D_xx, D_yy, D_zz; out[6..8] = D_x(D_y), D_x(D_z), D_y(D_z);
 * out[9..11] = upwind D_x, D_y, D_z for shift components b[0..2];
 * out[12..14] = 6th differences along x, y, z. */
void orc_stencils(const orc_patch* p, const double* u, int field, int i, int j, int k,
                  const double b[3], double out[15]);

/* ADM mass, angular momentum (Sec. 2.3) and linear momentum (Sec. 3.2) on
 * the coordinate sphere of radius r around c, with the proper surface
 * element dS_i = sqrt(g) n_i r^2 dOmega:
 *   M   = 1/(16 pi) int g^ik g^jl (d_j g_kl - d_k g_jl) dS_i
 *   J_z = 1/(8 pi)  int (x K_y^j - y K_x^j) dS_j      (x, y relative to c)
 *   P_i = 1/(8 pi)  int (K_i^j - delta_i^j K) dS_j
 * the integrands formed at cell centres (4th-order derivatives), interpolated
 * to the sphere with the 4 nearest cell centres per axis (cubic Lagrange),
 * Gauss-Legendre in cos(theta) (ntheta nodes) times the trapezoid rule in phi
 * (nphi points).  out = {M, J_z, P_x, P_y, P_z}; -1 if an interpolation
 * stencil comes within 2 cells of the array edge. */
int orc_adm_integrals(const orc_patch* p, const double* u, const double c[3], double r, int ntheta, int nphi,
                      double out[5]);
void orc_gauss_legendre(int n, double* x, double* w);

/* Psi4 extraction (Sec. 2.3).  Psi4 = (E_ij - i B_ij) mbar^i mbar^j with the
 * vacuum electric and magnetic Weyl parts E_ij = R_ij - K_ik K^k_j + K K_ij,
 * B_ij = sym(eps_i^kl D_k K_lj), interpolated (tricubic, cell centres) to the
 * point, and mbar = (e_theta - i e_phi)/sqrt(2) from the orthonormal triad
 * Gram-Schmidt-built (metric g) on the coordinate radial, theta and phi
 * directions about c; for an outgoing wave h = h_+ - i h_x this gives
 * Psi4 = -d_t^2 h.  orc_psi4_point: at angles (theta, phi), radius r.
 * orc_psi4_modes: Psi4^lm = int Psi4 conj(_{-2}Y_lm) dOmega for l = 2..lmax,
 * m = -l..l (out: Re, Im pairs in that order), Gauss-Legendre in cos(theta)
 * times the trapezoid rule in phi.  -1 if a stencil leaves the array. */
int orc_psi4_point(const orc_patch* p, const double* u, const double c[3], double r, double theta, double phi,
                   double out[2]);
int orc_psi4_modes(const orc_patch* p, const double* u, const double c[3], double r, int ntheta, int nphi,
                   int lmax, double* out);
/* spin-weight -2 spherical harmonic _{-2}Y_lm(theta, phi) (Re, Im) */
void orc_swsh(int l, int m, double theta, double phi, double out[2]);

/* Moving boxes (Sec. 2.2.1): the data of a patch shifted from geometry oldc
 * to newc (same level and size, origins a whole number of cells apart):
 * every cell of newc's array that is an active cell of oldc takes the old
 * value, every other cell (ghosts included) the 6th-order prolongation of the
 * parent data (as for ghosts; with skip_zlower the z < 0 ghost layers are
 * left to the reflection).  -1 if misaligned or a stencil leaves the parent. */
int orc_move_patch(const orc_patch* parent, const double* up, const orc_patch* oldc, const double* uo,
                   const orc_patch* newc, double* un, int skip_zlower);
/* Field f at point x: tricubic Lagrange interpolation from the 4 nearest
 * cell centres per axis, all of them active cells; -1 otherwise. */
int orc_interp_point(const orc_patch* p, const double* u, int f, const double x[3], double* out);

/* Lagrange basis weights of a set of integer nodes at position x. */
void orc_lagrange_weights(int nnodes, const int* nodes, double x, double* w);

/* number of threads the OpenMP loops use (1 without OpenMP) */
void orc_set_num_threads(int n);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
