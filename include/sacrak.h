/*
 * sacrak.h -- C ABI of the GB300 (sm_103a) Z4c hot path.
 *
 * The library evolves the 25 Z4c/BSSN puncture fields (Sec. 2.1.1 of the
 * SACRA-K paper) with 4th-order finite differences, lopsided upwind advection
 * along the shift, 6th-order Kreiss-Oliger dissipation and classical RK4
 * (Sec. 2.2), on static box-in-box Berger-Oliger patches with subcycling,
 * 6th-order Lagrange prolongation, time interpolation between parent time
 * levels and 4th-order Lagrange restriction (Sec. 2.2.1), with the Sommerfeld
 * outgoing-wave condition on the coarsest level and optional equatorial
 * reflection symmetry (Sec. 2.2.2), puncture tracking with moving patches
 * (Sec. 2.2.1), and the diagnostics of Sec. 2.3 and 3.2: constraint norms,
 * pi symmetry, ADM mass / angular / linear momentum, Psi4 modes and the
 * waveform post-processing (Nakano extrapolation, fixed frequency
 * integration).
 *
 * Conventions shared by every call
 *  - Field order: 0 W; 1-6 gt_xx,xy,xz,yy,yz,zz; 7 Khat; 8 Theta;
 *    9-14 At_xx..zz; 15-17 Gamt^x,y,z; 18 alpha; 19-21 beta^x,y,z;
 *    22-24 B^x,y,z.
 *  - A "patch array" exchanged with the caller is double[25][NZ][NY][NX] with
 *    NX = n[0]+6, NY = n[1]+6, NZ = n[2]+6 (ghost width 3 on every side), x
 *    fastest, no padding.  Active cell i has its centre at
 *    origin + (i + 1/2) dx_level; ghost cells are i = -3..-1 and n..n+2.
 *  - Pointers named host_or_dev may be host memory (pageable or pinned) or
 *    device memory; the library asks CUDA which it is.
 *  - Ownership: the caller owns every buffer it passes, including the device
 *    arena given to sacrak_grid_create, which the library never frees and
 *    never reallocates.  The library allocates no device memory on any call
 *    (except the tables cuFFT keeps for the duration of sacrak_ffi_strain).
 *  - Ordering: all device work is ordered on the grid's CUDA stream, in call
 *    order.  (Refined levels' ghost work may run on a second stream owned by
 *    the grid, forked from and joined back into the grid's stream within the
 *    same call: sacrak_set_overlap.)  Calls that return values computed on
 *    the device (constraints, pi symmetry, surface integrals, puncture
 *    positions, downloads to host memory) and the regrid calls synchronise
 *    that stream.
 *  - Errors: no call aborts or throws across the ABI.  Invalid arguments
 *    return SACRAK_EINVAL before any device work is issued; a CUDA error
 *    returns SACRAK_ECUDA; a non-finite value detected by a stage returns
 *    SACRAK_ENONFINITE at the next call that synchronises; a bounded device
 *    wait that runs out returns SACRAK_ETIMEOUT (reported ahead of a
 *    non-finite value seen in the same interval: the stage that gave up left
 *    its outputs unwritten).  After ECUDA, ENONFINITE or ETIMEOUT the grid
 *    is marked invalid and every stepping call returns SACRAK_ESTATE until
 *    new data is uploaded or set.  sacrak_last_error gives a one-line
 *    description.
 *  - Thread safety: one grid per host thread.
 */
#ifndef SACRAK_H
#define SACRAK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SACRAK_OK = 0,
  SACRAK_EINVAL = 1,
  SACRAK_ENOMEM = 2,
  SACRAK_ECUDA = 3,
  SACRAK_ENONFINITE = 4,
  SACRAK_ETIMEOUT = 5,
  SACRAK_ESTATE = 6
} sacrak_status;

typedef struct sacrak_grid sacrak_grid; /* opaque, host memory */

/* Run parameters (Sec. 2.2, Sec. 3: kappa1 = 0.005/M, kappa2 = 0,
 * eta = 0.36/M, sigma_KO = 0.5, Courant factor 0.5). */
typedef struct {
  double kappa1, kappa2; /* Z4c constraint damping */
  double eta;            /* Gamma-driver damping */
  double sigma_ko;       /* Kreiss-Oliger coefficient */
  double courant;        /* dt_level = courant * dx_level */
  double w_floor;        /* W >= w_floor after every stage write */
  int lapse;             /* 0: 1+log (d0 alpha = -2 alpha K), 1: harmonic (-alpha^2 K) */
  int shift;             /* 0: hyperbolic Gamma driver, 1: frozen (beta = B = 0) */
  int bc;                /* coarsest level ghosts: 0 Sommerfeld, 1 periodic, 2 frozen */
  int precision;         /* 0: FP64, 1: mixed (FP32 stencils/sources, FP64 state) */
  int lapse_uses_khat;   /* 0: 1+log source uses K = Khat + 2 Theta, 1: Khat */
  int zsym;              /* 1: equatorial reflection symmetry (Sec. 2.2.2): only z >= 0 is
                            evolved; patches whose lower z face is z = 0 get their z < 0
                            ghosts by reflection (f(-z) = s_z f(z), s_z = -1 for fields with
                            an odd number of z indices) after every other ghost treatment;
                            not with bc = 1 */
  int matter;            /* 1: a perfect fluid evolved with the spacetime (Sec. 2.1.2, 2.2):
                            FP64, no overlapping patches on a level; with zsym the
                            fluid's z < 0 ghosts are reflected too (u_z and J_z odd,
                            the rest even); see the matter calls below */
} sacrak_params;

/* One patch: refinement level, active cells per axis, lower face of active
 * cell 0.  Level l has spacing dx0 / 2^l.  A patch of level l > 0 must lie
 * inside one patch of level l-1 with its faces on that parent's cell faces
 * and at least 4 parent cells between its active region and the parent's
 * active edge (the 6-point prolongation stencils of its ghosts then read
 * parent active cells only); n must be even on levels > 0.  With zsym, a
 * patch and its parent may both start at z = 0 (the margin below is then the
 * parent's reflected ghosts). */
typedef struct {
  int level;
  int n[3];
  double origin[3];
} sacrak_patch_desc;

/* Bytes of device memory a grid of this shape needs.  Sec. 2.4 keeps every
 * evolved field in device memory for the whole evolution; this is that
 * resident state, held in one caller-owned arena: per patch 6 FP64 state
 * copies (3 time levels, the RK accumulator, 2 stage buffers), 3 more on
 * levels > 0 (the parent's time levels prolonged onto the ghost shell), and
 * with params->precision == 1 five copies of FP32 hi/lo pairs (the split of
 * the 3 time levels, 2 stage states) and 103 FP32 derivative planes over the
 * 32 x 4 x 1 tiles of the level with the most tiles (stage kernel 7); plus
 * tables and reduction scratch.  params may be NULL (FP64).  Returns 0 for
 * an invalid description. */
size_t sacrak_arena_bytes(int nlevels, int npatches, const sacrak_patch_desc* patches,
                          const sacrak_params* params);

/* Create a grid on the current CUDA device: the box-in-box refinement levels
 * of Sec. 2.2.1 (factor-2 spacing per level, dx_level = dx0 / 2^level) over
 * the caller's arena.  device_arena must point to at
 * least sacrak_arena_bytes(...) bytes of device memory, 256-byte aligned.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream). Fields start
 * as Minkowski.  With the Sommerfeld boundary (bc = 0) every level-0 patch must
 * contain the coordinate origin (with zsym: on its lower z face). */
sacrak_status sacrak_grid_create(int nlevels, double dx0, int npatches,
                                 const sacrak_patch_desc* patches, const sacrak_params* params,
                                 void* cuda_stream, void* device_arena, size_t arena_bytes,
                                 sacrak_grid** out);

sacrak_status sacrak_grid_destroy(sacrak_grid* grid);

/* Analytic initial data on every patch (ghosts included), generated on the
 * device.  kind: 0 Minkowski, 1 Brill-Lindquist punctures (m[a], pos[3a..]),
 * 2 gauge wave (H = 1 - gw_amp sin(2 pi x / gw_len), harmonic slicing, zero
 * shift).  noise_amp > 0 adds uniform noise in [-noise_amp, noise_amp) from
 * the counter hash h = sm(sm(sm(sm(seed + f) ^ i) ^ j) ^ k), SplitMix64's
 * output function sm, level-global cell indices (i,j,k) counted from the
 * level-0 patch's origin.  symmetrise_pi replaces every point with x < 0 by
 * its pi partner (-x,-y,z) times the field parity (Sec. 3.2); it needs patches
 * centred on x = y = 0.  Resets the time levels (the next step interpolates
 * linearly in time, Sec. 2.2.1). */
sacrak_status sacrak_set_initial_data(sacrak_grid* grid, int kind, int npunct, const double* m,
                                      const double* pos, double gw_amp, double gw_len,
                                      double noise_amp, uint64_t seed, int symmetrise_pi);

/* Copy a whole patch array (ghosts included) into / out of the current time
 * level: the transfers of Sec. 2.4 (initial data copied to the device at the
 * start; fields copied back only for diagnostics and snapshots).  Host
 * memory goes through one contiguous copy and a repacking kernel; device
 * memory through a device copy.  Upload resets the time levels like
 * sacrak_set_initial_data.  SACRAK_EINVAL for a bad patch or a null pointer. */
sacrak_status sacrak_upload_fields(sacrak_grid* grid, int patch, const double* host_or_dev);
sacrak_status sacrak_download_fields(sacrak_grid* grid, int patch, double* host_or_dev);

/* Z4c right-hand side (sources + upwind advection + Kreiss-Oliger) of the
 * current state of one patch at its active points, ghosts used as they are:
 * the Z4c equations with the 1+log / harmonic slicing and the Gamma-driver
 * shift of Sec. 2.1.1, discretised as Sec. 2.2 states (4th-order centred
 * derivatives, 4th-order lopsided upwind advection following the sign of the
 * shift, 6th-order Kreiss-Oliger dissipation with sigma_ko), evaluated by
 * the level's stage kernel (FP64, or with precision = 1 in FP32 on
 * centre-referenced hi/lo differences).  Output is a patch array whose ghost entries are
 * 0; the call returns when it is written.  SACRAK_EINVAL for a bad patch or
 * a null pointer. */
sacrak_status sacrak_rhs(sacrak_grid* grid, int patch, double* host_or_dev_rhs);

/* One classical RK4 step (Sec. 2.2: method of lines, classical fourth-order
 * Runge-Kutta, dt = Courant factor x spacing) of every patch of one level
 * with dt (dt <= 0: use courant * dx_level), each stage fused with the
 * right-hand side and the algebraic constraints (det gt = 1, trace-free At,
 * W floor).  Level 0's ghosts follow params.bc; ghosts of finer
 * levels are prolonged from the parent at every stage time.  Does not recurse
 * into finer levels and does not restrict. */
sacrak_status sacrak_rk4_step(sacrak_grid* grid, int level, double dt);

/* Berger-Oliger step of `level` and everything finer (Sec. 2.2.1): RK4 step of
 * the level, two recursive steps of level+1, restriction of level+1 onto it.
 * sacrak_level_step(grid, 0) is one coarse step.  The first call records the
 * launch sequence into a CUDA graph; later calls replay it. */
sacrak_status sacrak_level_step(sacrak_grid* grid, int level);

/* Volume-normalised L2 norms of H, M^x, M^y, M^z over the active cells of a
 * level with W >= w_excise (Sec. 2.3). */
sacrak_status sacrak_constraints(sacrak_grid* grid, int level, double w_excise,
                                 double out_l2[4]);

/* ---- Moving boxes (Sec. 2.2.1) ----
 * Punctures are tracked by integrating dx/dt = -beta^i(x); the patches that
 * follow them are shifted in steps of two of their cells (one parent cell),
 * which keeps parent and child cell faces aligned, and the region a shifted
 * patch newly covers is prolonged from its parent. */

/* Up to 8 punctures at pos[3 p .. 3 p + 2] (host array); follow[patch] (host
 * array of npatches entries) is the puncture that patch follows, -1 for
 * none (level-0 patches cannot follow).  Each puncture must be followed by
 * some patch; it is tracked on the finest of them (the first of equal
 * level): after every step of that patch's level, inside the captured
 * coarse step, x <- x - dt/2 (beta_n(x) + beta_{n+1}(x - dt beta_n(x)))
 * (Heun's method), beta interpolated tricubically from the 4 x 4 x 4 nearest
 * active cell centres of the old and new time levels.  A puncture whose
 * stencil would leave the active cells keeps its position and the next
 * synchronising call returns SACRAK_EINVAL once.  npunct = 0 stops tracking.
 * Synchronises the stream. */
sacrak_status sacrak_track_punctures(sacrak_grid* grid, int npunct, const double* pos, const int* follow);

/* Current puncture positions into pos[3 * npunct] (host); synchronises. */
sacrak_status sacrak_get_punctures(sacrak_grid* grid, double* pos);

/* Shift patch (level > 0) by shift[d] cells of its parent (2 shift[d] of its
 * own) while all levels are at the same time (between coarse steps): cells
 * that were active keep their values, every other cell of the patch's
 * current time level (ghosts included) is the 6th-order prolongation of the
 * parent's current time level; the parent offsets of its children follow.
 * The time-level history of the patch's level restarts (the ghosts of its
 * children are interpolated linearly in time during its next step, as at
 * the start of a run) and the captured coarse step is rebuilt at the next
 * sacrak_level_step.  SACRAK_EINVAL unless the patch and its children stay
 * nested (4 parent cells of margin; under equatorial symmetry no shift along
 * z).  With a fluid (Sec. 2.2.1) the same holds for its conserved variables
 * and primitives: cells active before and after keep them, every other
 * cell takes the parent's fluid prolongation (D^ by the conservative WENO5,
 * eps and u_i by the 6th-order Lagrange interpolation, with the fallbacks of
 * the refinement-boundary ghosts) with rho = D^ / (sqrt(gamma) w) on the
 * moved metric; the parent level's time-level history restarts too (the
 * fluid's primitives exist for the current time level only); SACRAK_ESTATE
 * before sacrak_upload_matter.  Synchronises. */
sacrak_status sacrak_move_patch(sacrak_grid* grid, int patch, const int shift[3]);

/* Lower face of active cell 0 of a patch (host array of 3), as moved. */
sacrak_status sacrak_patch_origin(sacrak_grid* grid, int patch, double origin[3]);

/* Regrid between coarse steps: coarse to fine, every patch that follows a
 * puncture or a star is shifted by trunc((x_p - centre) / dx_parent) parent
 * cells per axis (the object then lies within one parent cell of the patch
 * centre), clamped so that it nests in its parent's new position and keeps
 * its children that follow nothing nested; the whole plan is checked before
 * any data moves (SACRAK_EINVAL and nothing moved if the result would not
 * nest).  A star's position is the density maximum (sacrak_density_maximum)
 * of the finest patch that follows it, taken before any patch moves.
 * *moved = patches shifted.  Synchronises. */
sacrak_status sacrak_regrid(sacrak_grid* grid, int* moved);

/* Fluid grids: the largest rest-mass density rho over the active cells of a
 * patch's current time level, out[0], and the centre of that cell,
 * out[1..3] (the first in z, y, x order where several are equal).  A
 * neutron star is located there (Sec. 2.2.1).  SACRAK_ENONFINITE when no
 * cell holds a finite density.  Synchronises. */
sacrak_status sacrak_density_maximum(sacrak_grid* grid, int patch, double out[4]);

/* Fluid grids: follow[q] (host array of npatches entries) is the star patch
 * q follows, -1 for none (level-0 patches cannot follow, nor can a patch
 * that follows a puncture); every star 0..nstars-1 must be followed by some
 * patch.  sacrak_regrid moves the followers; nstars = 0 stops following.
 * Host only. */
sacrak_status sacrak_track_stars(sacrak_grid* grid, int nstars, const int* follow);

/* ADM mass, angular momentum about z (Sec. 2.3) and linear momentum
 * (Sec. 3.2) on the coordinate sphere |x - centre| = radius of one patch's
 * current time level (FP64 in both precisions), with the proper surface
 * element dS_i = sqrt(g) n_i r^2 dOmega:
 *   out[0]   = M   = 1/(16 pi) int g^ik g^jl (d_j g_kl - d_k g_jl) dS_i
 *   out[1]   = J_z = 1/(8 pi)  int (x K_y^j - y K_x^j) dS_j
 *   out[2+i] = P_i = 1/(8 pi)  int (K_i^j - delta_i^j K) dS_j
 * (x, y relative to centre; g_ij = gt_ij / W^2, K_ij = (At_ij + gt_ij K/3) / W^2,
 * K = Khat + 2 Theta).  The integrands are formed at cell centres with the
 * 4th-order centred first derivative, interpolated to the sphere from the
 * 4 x 4 x 4 nearest cell centres (tricubic Lagrange) and integrated with
 * ntheta Gauss-Legendre nodes in cos(theta) (1..1024) times nphi equally
 * spaced phi points (1..2^20).  centre and out are host pointers; the call
 * returns when out is written.  Ghost cells are read, so a sphere closer than
 * 5 cells to the active region's edge needs current ghosts.  SACRAK_EINVAL
 * for bad arguments or when a sphere point's stencil would leave the array
 * (some cell within 2 cells of its edge); out is then not written. */
sacrak_status sacrak_adm_integrals(sacrak_grid* grid, int patch, const double centre[3],
                                   double radius, int ntheta, int nphi, double out[5]);

/* Psi4 modes (Sec. 2.3) on the coordinate sphere |x - centre| = radius of
 * one patch's current FP64 time level.  Psi4 = (E_ij - i B_ij) mbar^i mbar^j
 * with the vacuum electric and magnetic Weyl parts E_ij = R_ij - K_ik K^k_j
 * + K K_ij and B_ij = sym(eps_i^kl D_k K_lj) (R_ij the physical Ricci tensor
 * of the right-hand side, D the physical covariant derivative), formed at
 * cell centres and interpolated tricubically to the sphere points, and
 * mbar = (e_theta - i e_phi)/sqrt(2) from the triad orthonormalised
 * (Gram-Schmidt with g_ij) from the coordinate radial, theta and phi
 * directions about centre; an outgoing wave h = h_+ - i h_x gives
 * Psi4 = -d_t^2 h.  out[2k], out[2k+1] = Re, Im of
 * Psi4^lm = int Psi4 conj(_{-2}Y_lm) dOmega for l = 2..lmax (lmax 2..8),
 * m = -l..l, k counting in that order ((lmax+1)^2 - 4 modes), with ntheta
 * Gauss-Legendre nodes in cos(theta) (1..1024) and nphi equally spaced phi
 * points; 2 ntheta nphi must not exceed the doubles of one state copy of the
 * patch, whose first RK stage buffer (dead between steps) holds the sphere
 * values (its second holds E, B and g of the cells near the sphere, formed
 * once each).  Host pointers; returns when out is written.  SACRAK_EINVAL for
 * bad arguments or a sphere point within 2 cells of the array's edge. */
sacrak_status sacrak_psi4_modes(sacrak_grid* grid, int patch, const double centre[3], double radius,
                                int ntheta, int nphi, int lmax, double* out);

/* ---- Waveform post-processing (Sec. 2.3) ----
 * Stream-ordered on cuda_stream (a cudaStream_t, NULL = legacy default), on
 * device arrays owned by the caller; no grid needed. */

/* Nakano extrapolation of one Psi4 mode's time series: n samples at times
 * t[n], psi[2n] (Re, Im interleaved), mode index l >= 2, extraction radius
 * r0 > 0 and total mass m0 > 0 with D0 / (2 m0) > 1, D0 = r0 (1 + m0/(2 r0))^2.
 * Writes t_ret[n] = t - [D0 + 2 m0 ln(D0/(2 m0) - 1)] and out[2n] =
 * D0 Psi4^{l,m,inf} = C [D0 psi - (l-1)(l+2)/2 int_{t_0}^t psi dt'] with
 * C = 1 - 2 m0 / D0, the integral by the trapezoid rule from the first
 * sample (a fixed-order chunked scan).  out must not alias psi.
 * SACRAK_EINVAL for bad arguments. */
sacrak_status sacrak_nakano(const double* t, const double* psi, int n, int l, double r0, double m0,
                            double* t_ret, double* out, void* cuda_stream);

/* Device work-area bytes sacrak_ffi_strain needs for n samples (0 if cuFFT
 * cannot be loaded or n < 1). */
size_t sacrak_ffi_work_bytes(int n);

/* Fixed frequency integration of a uniformly sampled Psi4 mode psi[2n]
 * (spacing dt) to the strain h[2n] (Re, Im; h = h_+ - i h_x):
 * h = IFFT[ FFT(psi) / (2 pi max(|f|, f_cut))^2 ] over the DFT frequencies.
 * cuFFT (libcufft.so, loaded at the first call) runs the transforms on the
 * caller's work area (>= sacrak_ffi_work_bytes(n) bytes); its plan keeps its
 * own small tables for the duration of the call.  Synchronises the stream.
 * SACRAK_EINVAL for bad arguments or a short work area, SACRAK_ECUDA if
 * cuFFT is missing or fails. */
sacrak_status sacrak_ffi_strain(const double* psi, int n, double dt, double f_cut, double* h, void* work,
                                size_t work_bytes, void* cuda_stream);

/* max over all points (ghosts included) and fields of |f(x,y,z) - s_f f(-x,-y,z)|
 * for one patch centred on x = y = 0 (Sec. 3.2). */
sacrak_status sacrak_pi_symmetry(sacrak_grid* grid, int patch, double* max_abs_diff);

/* Kernel timing for roofline reports.  While enabled, level steps launch
 * eagerly (no graph) and every launch of the fused RHS + RK4 stage kernel is
 * bracketed by CUDA events on the grid's stream.  sacrak_profile_read
 * synchronises the stream and returns the summed duration of those launches
 * (ms), their number and the zones they updated; enabling again clears the
 * totals. */
sacrak_status sacrak_profile_enable(sacrak_grid* grid, int enable);
sacrak_status sacrak_profile_read(sacrak_grid* grid, double* stage_ms, long long* stage_launches,
                                  long long* stage_zones);

/* Allocation-free constraint monitor for callers that cannot allocate device
 * memory (a process whose device memory belongs to another framework's pool,
 * a fixed-size sandbox or service, a hook that must not call cudaMalloc).  No
 * counterpart in the paper: it computes what sacrak_constraints computes for
 * one level (the L2 norms of H, M^x, M^y, M^z over active cells with
 * W >= w_excise), for one patch array that the caller keeps in its own device
 * memory (dev_u, the unpadded patch-array layout above, n[3] active cells,
 * 4 <= n <= 512 per axis, spacing dx), without a grid.  Its partial sums live
 * in one static device array of 2048 x 5 + 8 doubles (about 80 KB) that every
 * GPU which loads the library keeps until the process exits; nothing is
 * allocated or freed.  The first call on a device looks that array up (with
 * the device current) and should come before any stream capture.  Calls that
 * overlap on the GPU share the array and race; serialise them (one stream,
 * or one call at a time).  Runs on cuda_stream (a cudaStream_t, NULL = legacy
 * default) and synchronises it to return out_l2 (host memory).  Sizes beyond
 * the limits return SACRAK_EINVAL, and so does a dev_u that is not device
 * memory of the current device or whose allocation (as the driver reports
 * it) does not hold the whole patch array; all before any launch.  The
 * cached address of the array is dropped when a call finds the device's
 * context destroyed (after a device reset), and looked up again. */
sacrak_status sacrak_constraints_noalloc(const double* dev_u, const int n[3], double dx,
                                         double w_excise, void* cuda_stream, double out_l2[4]);

/* Stage kernel of a level.  kernel 0: the direct kernel (every stencil value
 * read through the L1 cache, second derivatives kept in full).  Mixed
 * precision only: kernels 1..4, the TMA-staged kernel with tiles of
 * 32 x 4 x 1, 32 x 2 x 2, 32 x 4 x 2 and 32 x 8 x 1 points, which copies each
 * field's tile plus its 3-cell halo into shared memory with
 * tensor-memory-accelerator loads and walks all tiles of the level in one
 * persistent launch; kernels 5 and 6, the same arithmetic as 1..4 (hi/lo
 * pairs in packed FP32x2 instructions, branch-free upwinding, second
 * derivatives contracted as they are formed) reading through the L1 cache,
 * 3 CTAs per SM; kernel 6 also prefetches the next field's stencil rows
 * into L1 and the RK update's streaming reads into L2; kernel 7 splits the
 * stage into two launches, the derivatives (five fields per thread) into FP32
 * planes in the arena and then the algebra and RK4 update; kernel 8 is
 * kernel 6 with 4 CTAs per SM (128 registers), kernels 9, 10 and 11 are
 * kernel 6 prefetching only the star rows, only the z-arm rows, and only the
 * RK update's streaming reads; kernel 12 is kernel 10 with the inner
 * differences of D_x D_y f and D_x D_z f at the x neighbours taken from the
 * neighbouring lanes of the warp by shuffles (loads where a tile does not
 * fill its 32 x), kernel 13 is kernel 12 with 4 CTAs per SM, kernel 14 is
 * kernel 10 with 4 CTAs per SM (128 registers); kernels 15..17 take two
 * x-adjacent points per thread with 128-bit loads of the hi/lo pairs (15
 * plain, 16 prefetching the z-arm rows, 17 as 16 with 3 CTAs per SM; they
 * need 25 x the field stride < 2^31); kernel 18 is kernel 10 as a persistent
 * grid of resident CTAs walking the level's tiles; kernel 19 is kernel 10
 * with the row and plane pitches fixed at compile time where every patch of
 * the level has n[0] = n[1] = n for n in {32, 48, 64, 96, 128, 160, 192}
 * (the stencil offsets become constants of the loads), and kernel 10 itself
 * elsewhere and for the RHS alone (sacrak_rhs); kernel 19 gives kernel 10's
 * results bit for bit; kernel 20 is kernel 19 with 4 CTAs per SM (128
 * registers) where an instance fits, and kernel 10 elsewhere.  All kernels
 * compute the same RHS up to FP32 rounding order.  A TMA kernel needs at most 8 patches on the level and at
 * least 32 x TY x TZ active cells per patch, else SACRAK_EINVAL.  New grids
 * use kernel 20 in mixed precision and 0 in FP64.  Changing the kernel of a
 * level drops the recorded CUDA graph of the coarse step (it is recorded
 * again at the next sacrak_level_step). */
sacrak_status sacrak_set_stage_kernel(sacrak_grid* grid, int level, int kernel);
sacrak_status sacrak_get_stage_kernel(sacrak_grid* grid, int level, int* kernel);

/* Autotuner of the stage kernel: for every level, times RK4 stage 1 (which
 * reads the current time level and writes only the RK accumulator and the
 * first stage buffer, so the state is unchanged) with every kernel usable on
 * that level, `reps` launches each after one warm-up launch (CUDA events on
 * the grid's stream), and selects the fastest; the level's current kernel
 * stays unless the fastest beats it by more than 2% (stage 1 stands in for
 * all four stages).  Results are cached for the
 * process, keyed by device, precision and the level's patch shapes (levels
 * of identical shapes share one timing and one choice); with use_cache != 0
 * a cached level is not timed again.  us_per_launch, if not
 * NULL, receives nlevels x 21 timings in microseconds (kernel 0..20 of each
 * level; -1 where not timed).  Synchronises the stream; must not be called
 * while the stream is being captured (SACRAK_ESTATE). */
sacrak_status sacrak_autotune(sacrak_grid* grid, int reps, int use_cache, double* us_per_launch);

/* Bound of the TMA stage kernels' (kernels 1..4) wait for each field's copy,
 * in SM clock cycles: 0 restores the default (4e9, about 2 s); cycles < 0
 * makes every such wait count as run out at once, a test hook for the
 * time-out path (no paper counterpart).  A wait that runs out sets the
 * device error flag (SACRAK_ETIMEOUT at the next synchronising call, the
 * grid then invalid until new data); the CTA issues no further copy, waits
 * with the default bound for the copies it has in flight, and returns
 * without writing results.  Drops the recorded coarse-step graph. */
sacrak_status sacrak_set_wait_limit(sacrak_grid* grid, long long cycles);

/* Schedule of the refined levels' ghost work (Sec. 2.2.1).  on = 1 (the
 * default): within each RK4 step of a level > 0, the time fill of the
 * stage-2 and stage-3 inputs runs on a second stream of the library's
 * concurrently with the stage-1 kernel, the fill of the stage-4 input with
 * the stage-3 kernel, the spatial prolongation of a parent's new time level
 * with the children's first stage, and (without zsym) that of its restricted
 * level with the parent's next step; every call that launches them
 * makes the caller's stream wait for that stream before it returns (under
 * capture these are graph edges).  on = 0: every launch on the caller's
 * stream, one after another.  Results are the same bit for bit.  Drops the
 * recorded coarse-step graph; SACRAK_EINVAL for other values. */
sacrak_status sacrak_set_overlap(sacrak_grid* grid, int on);

/* ---- Matter: a perfect fluid on the evolving spacetime (Sec. 2.1.2, 2.2) ----
 * Grids created with params.matter = 1 (FP64) carry a perfect
 * fluid: primitives (rho, eps, u_x, u_y, u_z) -- rest-mass density, specific
 * internal energy, spatial covariant components of the four-velocity -- and
 * the densitised conserved variables sqrt(gamma) (D, J_i, rho_H), D = rho w,
 * J_i = rho h w u_i, rho_H = rho h w^2 - P, w = sqrt(1 + gamma^ij u_i u_j),
 * h = 1 + eps + P/rho.  Every RK4 stage recovers the primitives from the
 * stage's conserved variables (Newton-Raphson on w, the previous w as the
 * guess; a negative thermal part is repaired to the cold value; a cell below
 * the floor or without a root is reset to rest at the floor density on the
 * cold curve), adds the fluid's terms to the Z4c right-hand side (Khat
 * 4 pi alpha (S + rho_H), Theta -8 pi alpha rho_H, At_ij -8 pi alpha W^2
 * [S_ij]^TF, Gamt^i and B^i -16 pi alpha gt^ij J_j), and advances the
 * conserved variables with PPM face states (steep minmod b = 3), face fluxes
 * (sacrak_set_riemann: HLLC in the face tetrad by default, or HLLE), the
 * metric at faces by 4th-order interpolation and the geometric sources
 * (4th-order metric derivatives).  Ghost cells of the fluid: on level 0 zero
 * gradient (outflow), periodic with bc = 1; on finer levels from the parent
 * (Sec. 2.2.1): every parent time level is prolonged onto the child's ghost
 * shell -- D^ by a conservative fifth-order WENO interpolation (applied along
 * x, y, z; the parent cell's value where it is not positive), eps and u_i by
 * the 6th-order Lagrange interpolation of the spacetime (eps trilinear where
 * D^ fell back or eps is not positive) -- and interpolated in time like the
 * spacetime's ghosts, rho = D^ / (sqrt(gamma) w) with the child's metric.
 * After a level's two child steps the parent cells under a child take the
 * mean of their 8 children's conserved variables, and the parent cells next
 * to a child have their boundary-face fluxes of the parent's step (RK4-
 * weighted) replaced by the children's (averaged over the 4 fine faces and
 * the 2 child steps): the reflux, which conserves the total rest mass.  A
 * "matter array" exchanged with the caller is
 * double[5][NZ][NY][NX] in the patch-array layout above.  The stepping calls
 * return SACRAK_ESTATE until sacrak_upload_matter has run. */

/* Hybrid EOS (Sec. 2.1.2): P = P_cold(rho) + (gamma_th - 1) rho (eps -
 * eps_cold(rho)), cold part a piecewise polytrope P = K_i rho^gammas[i] on
 * [rho_bounds[i-1], rho_bounds[i]) (npieces 1..4, npieces - 1 increasing
 * boundaries, K_0 = K0 >= 0, the other K_i and the eps offsets fixed by
 * continuity of P and eps).  K0 = 0 gives the ideal gas P = (gamma_th - 1)
 * rho eps.  SACRAK_EINVAL for bad values or a grid without a fluid. */
sacrak_status sacrak_set_eos(sacrak_grid* grid, int npieces, double K0, const double* gammas,
                             const double* rho_bounds, double gamma_th);

/* Density floor of the atmosphere (Sec. 2.2): rho_atm within the coordinate
 * radius r_atm, falling as r^-3 outside (the paper: 1e-12 of the maximum
 * density within eight times the finest domain). */
sacrak_status sacrak_set_atmosphere(sacrak_grid* grid, double rho_atm, double r_atm);

/* Face flux of the fluid (Sec. 2.2).  solver = 0 (the default): the HLLC
 * flux of special relativity (Mignone & Bodo 2005) solved in an orthonormal
 * tetrad in which the face is at rest (e1 along the gradient of the face
 * coordinate, e0 the Eulerian observer projected onto the face), with the
 * HLLE flux there where the intermediate state is unphysical (no real
 * contact speed, a contact speed outside the outer waves or not below light
 * speed, a non-positive intermediate pressure), transformed back to the
 * coordinate frame.  solver = 1: the HLLE flux in the coordinate frame with
 * the relativistic characteristic speeds.  SACRAK_EINVAL for other values or
 * a grid without a fluid.  Drops the recorded coarse-step graph. */
sacrak_status sacrak_set_riemann(sacrak_grid* grid, int solver);

/* Primitives of one patch (a matter array, ghosts included, host or device
 * memory) into the current time level; the conserved variables are formed
 * with the patch's current metric, so upload the spacetime first.  Needs the
 * EOS and the atmosphere (SACRAK_ESTATE otherwise).  Synchronises. */
sacrak_status sacrak_upload_matter(sacrak_grid* grid, int patch, const double* host_or_dev_prim);

/* The primitives of the last recovery (after a step: of the new time level)
 * into a matter array (host or device memory).  Synchronises. */
sacrak_status sacrak_download_matter(sacrak_grid* grid, int patch, double* host_or_dev_prim);

/* d_t of the conserved variables of the current state of one patch (flux
 * divergence + sources, active cells; ghost entries 0) after recovering its
 * primitives (which may repair cells as a stage does).  Synchronises. */
sacrak_status sacrak_matter_rhs(sacrak_grid* grid, int patch, double* host_or_dev_rhs);

/* Current time of a level. */
sacrak_status sacrak_level_time(sacrak_grid* grid, int level, double* t);

/* One-line description of the last error on this grid ("" if none). */
const char* sacrak_last_error(const sacrak_grid* grid);

#ifdef __cplusplus
}
#endif
#endif /* SACRAK_H */
