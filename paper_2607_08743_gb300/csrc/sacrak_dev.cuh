// Device-side data structures and finite-difference helpers shared by the
// kernels of the GB300 Z4c hot path.
//
// Memory layout (HBM): every patch owns six state copies (three time levels,
// the RK4 accumulator y and two stage buffers).  A state copy is
// double[25][NZ][NY][px]: x fastest, the row pitch px = NX + 1 rounded up to
// 8 doubles (64 B), every copy starting one element past a 256-byte
// boundary, so that active cell i of a row sits at element i + 4 of its
// 64-byte aligned row and the cells (2m, 2m+1) form one 16-byte vector.
// Ghost width is 3 on every side.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sacrak {

constexpr int NF = 25;
constexpr int GH = 3;
constexpr int NBUF = 6;

enum Field {
  F_W = 0, F_GXX, F_GXY, F_GXZ, F_GYY, F_GYZ, F_GZZ, F_KH, F_TH,
  F_AXX, F_AXY, F_AXZ, F_AYY, F_AYZ, F_AZZ, F_GAMX, F_GAMY, F_GAMZ,
  F_ALP, F_BETX, F_BETY, F_BETZ, F_BX, F_BY, F_BZ
};

// buffer slots of a patch
enum { B_TL0 = 0, B_TL1 = 1, B_TL2 = 2, B_Y = 3, B_S0 = 4, B_S1 = 5 };

struct DevPatch {
  int n[3];          // active cells
  int NX, NY, NZ;    // extents incl. ghosts
  int px;            // row pitch in doubles
  int level;
  int parent;        // parent patch index, -1 on level 0
  int off[3];        // this patch's origin in parent cell units
  int zrefl;         // equatorial symmetry: lower z face at z = 0, ghosts below by reflection
  long long plane;   // px * NY
  long long fstride; // doubles between consecutive fields
  double dx;
  double origin[3];
  double* buf[NBUF];
  // levels > 0: the parent's time level in each ring slot, prolonged in space
  // onto this patch (full patch layout; only the ghost shell is written; in
  // mixed precision each 8-byte entry holds the hi/lo float2 split instead)
  double* gsh[3];
  // mixed precision only (null otherwise): each time level split into FP32
  // hi + lo, interleaved (hl, same ring slots as buf), and the stage states
  // u_s = hi_n + lo_s stored the same way (sa, sb): stage s reads hl[ring],
  // sa, sb, sa; stages 1-3 write sa, sb, sa; stage 4 writes hl[ring + 1]
  float2* hl[3];
  float2* sa;
  float2* sb;
  // matter (FP64 grids with a fluid): the densitised conserved
  // variables in the same slots as buf (5 fields each), the primitives and
  // the Lorentz factor (6 fields), the face fluxes along x, y, z (15) and the
  // matter terms of the Z4c right-hand side (11); null without a fluid
  double* mcons[NBUF];
  double* mprim;
  double* mflux;
  double* mzsrc;
  // levels > 0 of a fluid grid: the parent's fluid in each ring slot prolonged
  // onto this patch's ghost shell (D^, eps, u_i; 5 fields per slot), and the
  // RK4-weighted face fluxes of the patch's last step (mfs) and of its last
  // two steps averaged (mfa), 3 directions x 5 fields each, for the reflux
  double* mgsh[3];
  double* mfs;
  double* mfa;
};

struct DevLevel {
  int ring;    // slot of the current time level
  int nvalid;  // valid time levels (1..3)
  int steps;
  int pad_;
  double t;    // time of the current time level
};

struct Tile {
  int patch;
  int x0, y0, z0;
};

struct DevParams {
  double kappa1, kappa2, eta, sigma_ko, w_floor;
  int lapse, shift, lapse_uses_khat;
  int matter;  // 1: add the fluid's terms (DevPatch::mzsrc) to the Z4c right-hand side
};

// error flags written by kernels (bitmask), read by the host after a sync
enum { ERR_NONFINITE = 1, ERR_BOUNDS = 2, ERR_TIMEOUT = 4, ERR_TRACK = 8 };

// pi-rotation parity of each field (x,y -> -x,-y)
__host__ __device__ inline int pi_parity(int f) {
  // W gt(xx xy xz yy yz zz) Khat Theta At(..) Gamt(x y z) alpha beta(x y z) B(x y z)
  const unsigned odd_mask = (1u << F_GXZ) | (1u << F_GYZ) | (1u << F_AXZ) | (1u << F_AYZ) |
                            (1u << F_GAMX) | (1u << F_GAMY) | (1u << F_BETX) |
                            (1u << F_BETY) | (1u << F_BX) | (1u << F_BY);
  return (odd_mask >> f) & 1u ? -1 : 1;
}

__host__ __device__ inline double flat_value(int f) {
  return (f == F_W || f == F_GXX || f == F_GYY || f == F_GZZ || f == F_ALP) ? 1.0 : 0.0;
}

// symmetric index (i,j) -> 0..5 (xx,xy,xz,yy,yz,zz)
__host__ __device__ constexpr int S2(int i, int j) {
  return (i == j) ? (i == 0 ? 0 : (i == 1 ? 3 : 5))
                  : ((i + j) == 1 ? 1 : ((i + j) == 2 ? 2 : 4));
}

// mixed precision: split stage state read (in) / written (out) by stage s
__host__ __device__ inline float2* mixed_in(const DevPatch* P, int s, int ring) {
  return s == 1 ? P->hl[ring] : (s == 3 ? P->sb : P->sa);
}
__host__ __device__ inline float2* mixed_out(const DevPatch* P, int s) {
  return s == 2 ? P->sb : P->sa;  // stage 4 writes the split of the new level instead
}

// slot of the stage input / output buffer for RK4 stage s (1..4)
__host__ __device__ inline int stage_in_slot(int s, int ring) {
  return s == 1 ? ring : (s == 3 ? B_S1 : B_S0);
}
__host__ __device__ inline int stage_out_slot(int s, int ring) {
  return s == 4 ? (ring + 1) % 3 : (s == 2 ? B_S1 : B_S0);
}

// ---------------------------------------------------------------------------
// Finite-difference operators on a field pointer f at linear offset q with
// stride st.  The pair forms (f+ - f-) and (f+ + f-) make every operator
// exactly antisymmetric/symmetric under mirroring, which keeps pi symmetry
// bitwise for any contraction pattern the compiler picks.

// 4th-order centred first derivative, unscaled: 8 (f1 - f-1) - (f2 - f-2);
// multiply by 1/(12 h).
__device__ __forceinline__ double d1u(const double* __restrict__ f, long long q, long long st) {
  double a = __ldg(f + q + st) - __ldg(f + q - st);
  double b = __ldg(f + q + 2 * st) - __ldg(f + q - 2 * st);
  return 8.0 * a - b;
}

// The stencils whose coefficients sum to zero are evaluated on differences
// from the centre value, f_k - f_0, so that they round relative to the result
// rather than to the field value.

// 4th-order centred second derivative, unscaled:
// 16 (f1 + f-1) - (f2 + f-2) - 30 f0; multiply by 1/(12 h^2).
__device__ __forceinline__ double d2u(const double* __restrict__ f, long long q, long long st,
                                      double f0) {
  double a = (__ldg(f + q + st) - f0) + (__ldg(f + q - st) - f0);
  double b = (__ldg(f + q + 2 * st) - f0) + (__ldg(f + q - 2 * st) - f0);
  return 16.0 * a - b;
}

// nested mixed derivative D_a(D_b f), unscaled; multiply by 1/(144 h^2).
__device__ __forceinline__ double d11u(const double* __restrict__ f, long long q, long long sa,
                                       long long sb) {
  double p1 = d1u(f, q + sa, sb), m1 = d1u(f, q - sa, sb);
  double p2 = d1u(f, q + 2 * sa, sb), m2 = d1u(f, q - 2 * sa, sb);
  return 8.0 * (p1 - m1) - (p2 - m2);
}

// lopsided upwind derivative (one point behind, three ahead along the side
// the shift points to), unscaled: (-3 f-s - 10 f0 + 18 fs - 6 f2s + f3s) * s;
// multiply by 1/(12 h).  The mirrored case is the same expression on mirrored
// points, negated.
__device__ __forceinline__ double dupu(const double* __restrict__ f, long long q, long long st,
                                       double b, double f0) {
  long long s = b > 0.0 ? st : -st;
  double v = -3.0 * (__ldg(f + q - s) - f0) + 18.0 * (__ldg(f + q + s) - f0) -
             6.0 * (__ldg(f + q + 2 * s) - f0) + (__ldg(f + q + 3 * s) - f0);
  return b > 0.0 ? v : -v;
}

// 6th difference along st (Kreiss-Oliger stencil)
__device__ __forceinline__ double delta6(const double* __restrict__ f, long long q, long long st,
                                         double f0) {
  double a = (__ldg(f + q + 3 * st) - f0) + (__ldg(f + q - 3 * st) - f0);
  double b = (__ldg(f + q + 2 * st) - f0) + (__ldg(f + q - 2 * st) - f0);
  double c = (__ldg(f + q + st) - f0) + (__ldg(f + q - st) - f0);
  return (a - 6.0 * b) + 15.0 * c;
}

// Sphere quadrature and interpolation shared by the surface diagnostics

// Node i (descending in x) and weight of the n-point Gauss-Legendre rule on
// [-1, 1]: Newton's method on P_n, evaluated with the three-term recurrence
// (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, from cos(pi (4i+3)/(4n+2)).
__device__ inline void gauss_legendre_node(int n, int i, double& x, double& w) {
  double z = cospi((4.0 * i + 3.0) / (4.0 * n + 2.0)), dpn = 1.0;
  for (int it = 0; it < 64; ++it) {
    double pkm1 = 1.0, pk = z;
    for (int k = 1; k < n; ++k) {
      const double pk1 = ((2.0 * k + 1.0) * z * pk - k * pkm1) / (k + 1.0);
      pkm1 = pk;
      pk = pk1;
    }
    dpn = n * (z * pk - pkm1) / (z * z - 1.0);  // P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1)
    const double step = pk / dpn;
    z -= step;
    if (fabs(step) < 1e-16) break;
  }
  x = z;
  w = 2.0 / ((1.0 - z * z) * dpn * dpn);
}

// cubic Lagrange basis on the nodes 0, 1, 2, 3 at position s
__device__ __forceinline__ void cubic_weights(double s, double w[4]) {
  const double s1 = s - 1.0, s2 = s - 2.0, s3 = s - 3.0;
  w[0] = -s1 * s2 * s3 / 6.0;
  w[1] = s * s2 * s3 / 2.0;
  w[2] = -s * s1 * s3 / 2.0;
  w[3] = s * s1 * s2 / 6.0;
}

// Kernel argument bundles ----------------------------------------------------

// linear ghost-shell index -> (i,j,k) array indices (ghosts included): two z
// slabs, then two y slabs over the middle z range, then two x slabs.  32-bit
// arithmetic: a shell has fewer than 2^31 points for patches of up to 4096
// cells per axis, and 64-bit division would dominate the cost of the fills.
__device__ __forceinline__ void shell_ijk(long long id64, int NX, int NY, int NZ, int& i, int& j, int& k) {
  int id = (int)id64;
  const int zslab = GH * NY * NX;
  const int nz = NZ - 2 * GH, ny = NY - 2 * GH;
  const int yslab = GH * NX * nz;
  if (id < 2 * zslab) {
    const int side = id >= zslab;
    int r = id - side * zslab;
    const int rr = r / NX;
    i = r - rr * NX;
    k = rr / NY;
    j = rr - k * NY;
    k += side ? NZ - GH : 0;
    return;
  }
  id -= 2 * zslab;
  if (id < 2 * yslab) {
    const int side = id >= yslab;
    const int r = id - side * yslab;
    const int rr = r / NX;
    i = r - rr * NX;
    k = rr / GH;
    j = rr - k * GH + (side ? NY - GH : 0);
    k += GH;
    return;
  }
  id -= 2 * yslab;
  const int xslab = GH * ny * nz;
  const int side = id >= xslab;
  const int r = id - side * xslab;
  const int rr = r / GH;
  i = r - rr * GH + (side ? NX - GH : 0);
  k = rr / ny;
  j = rr - k * ny + GH;
  k += GH;
}

__host__ __device__ inline long long shell_count(int NX, int NY, int NZ) {
  return (long long)NX * NY * NZ - (long long)(NX - 2 * GH) * (NY - 2 * GH) * (NZ - 2 * GH);
}

struct StageArgs {
  const Tile* tiles;
  int ntiles;
  const DevPatch* patches;
  const DevLevel* lev;  // the level being stepped
  int stage;            // 1..4; 0 = write the RHS into S1 (no RK update)
  double dt;
  DevParams prm;
  unsigned* err;
};

struct GhostArgs {
  const DevPatch* patches;
  const int* patch_ids;  // patches of the level
  const DevLevel* lev;
  int stage;
  double dt;
  DevParams prm;
  unsigned* err;
};

struct ConsArgs {
  const Tile* tiles;
  const DevPatch* patches;
  const DevLevel* lev;
  double w_excise;
  double* partial;  // [ntiles][5]
};

// ghost fills: mode 0 = stage input of stage s, 1 = current time level,
// 2 = next time level
struct FillArgs {
  const DevPatch* patches;
  const int* patch_ids;
  const DevLevel* lev;   // level of the patches being filled
  const DevLevel* plev;  // parent level (prolongation / restriction)
  int mode, stage;
  // prolongation: weights of the parent's (oldest, middle, newest) time levels,
  // for three valid levels (wq) and for two (wl, oldest weight 0)
  double wq[3], wl[3];
  int mixed;  // also maintain the FP32 split buffers
  int dual;   // time fill of stage 2: also fill the stage-3 input (same stage time)
};

struct ExchArgs {
  const DevPatch* patches;
  const DevLevel* lev;
  int a, b;
  int off[3];  // b's cell index of a's cell 0
  int mode, stage;
  int mixed;
};

struct InitArgs {
  const DevPatch* patches;
  const DevLevel* levels;
  int kind;  // 0 Minkowski, 1 punctures, 2 gauge wave
  int npunct;
  double m[8];
  double pos[24];
  double gw_amp, gw_len;
  double noise_amp;
  uint64_t seed;
  double lo[3];  // level-0 origin (origin of level-global cell indices)
};

// ADM surface integrals on the sphere |x - c| = r of one patch's current time
// level: ring holds 6 * ntheta doubles (per-ring M, J_z, P_x, P_y, P_z and
// points whose stencil leaves the array)
constexpr int ADM_MAX_THETA = 1024;
struct AdmArgs {
  const DevPatch* patches;
  const DevLevel* levels;
  int patch, ntheta, nphi;
  double c[3], r;
  double* ring;
};

// Moving boxes (Sec. 2.2.1).  A tracked puncture: position, the patch it is
// tracked on (the finest patch that follows it) and that patch's level.
constexpr int MAX_PUNCT = 8;
struct DevPunct {
  double x[3];
  int patch, level;
};
// the punctures tracked on `level`, after the stage 4 of its step (old time
// level in the ring slot, new one in the next slot): Heun's method for
// dx/dt = -beta(x) over dt
struct TrackArgs {
  const DevPatch* patches;
  const DevLevel* levels;
  DevPunct* punct;
  int np, level;
  double dt;
  unsigned* err;
};
// data of patch `patch` shifted by sh own cells (new array index + sh = old
// array index) with its new offset noff in parent cells, written to dst (a
// full patch buffer): old active cells copied from the current slot, the
// rest prolonged from the parent's current slot; with skip_zlower the z < 0
// ghost layers are left to the reflection.  The device table still holds the
// old geometry.
struct MoveArgs {
  const DevPatch* patches;
  const DevLevel* levels;
  int patch;
  int sh[3], noff[3];
  int skip_zlower;
  double* dst;
  unsigned* err;
};

// Psi4 extraction (Sec. 2.3) on the sphere |x - c| = r of one patch's current
// time level: Psi4 at the ntheta x nphi sphere points into psi (2 doubles
// each), per ring the node, its weight and the points whose stencil leaves
// the array into ring (3 * ntheta); then the modes l = 2..lmax, m = -l..l
// into out (2 doubles each)
constexpr int PSI4_MAX_L = 8;
struct Psi4Args {
  const DevPatch* patches;
  const DevLevel* levels;
  int patch, ntheta, nphi, lmax;
  double c[3], r;
  double* psi;
  double* ring;
  double* out;
  double* cells;  // E_ij, B_ij, g_ij (18 fields, patch layout) of the cells near the sphere
};

// launchers (host)
void launch_stage_fp64(const StageArgs& a, cudaStream_t st);
void launch_stage_mixed(const StageArgs& a, cudaStream_t st);
void launch_sommerfeld(const GhostArgs& a, int npatches, long long max_shell, cudaStream_t st);
void launch_constraints(const ConsArgs& a, int ntiles, double* out5, cudaStream_t st);
void launch_fill(int kind, const FillArgs& a, int npatches, long long maxpts, cudaStream_t st);
void launch_exchange(const ExchArgs& e, long long tot, cudaStream_t st);
// equatorial reflection of the z < 0 ghost layers of the level's zrefl
// patches, in the buffer selected by (mode, stage) as for the other fills
void launch_zreflect(const FillArgs& a, int npatches, long long maxpts, cudaStream_t st);
// bricks of the spatial prolongation of one child patch (n active cells)
int prolong_bricks(int n0, int n1, int n2);
// back = 0: the parent's current slot; 1, 2: the one and two time levels
// before it (after a patch moved, every cached slot is recomputed)
void launch_prolong_space(const DevPatch* patches, const int* ids, const DevLevel* plev, int nchildren,
                          long long max_bricks, int mixed, cudaStream_t st, int back = 0);
void launch_track(const TrackArgs& a, cudaStream_t st);
void launch_move(const MoveArgs& a, long long tot, cudaStream_t st);
void launch_set_nvalid(DevLevel* L, int nvalid, cudaStream_t st);
void launch_sommerfeld_mixed(const GhostArgs& a, int npatches, long long max_shell, cudaStream_t st);
void launch_split(const DevPatch* patches, const DevLevel* levels, int patch, long long tot,
                  cudaStream_t st);
void launch_level_advance(DevLevel* L, double dt, cudaStream_t st);
// pitched patch buffer <-> contiguous patch array (rows of NX doubles)
void launch_repack(double* dst, const double* src, long long rows, int NX, int px, int to_pitched,
                   cudaStream_t st);
void launch_init(const InitArgs& a, int patch, long long tot, cudaStream_t st);
void launch_psi4(const Psi4Args& a, long long patch_points, cudaStream_t st);
// out6 = {M, J_z, P_x, P_y, P_z, points outside}
void launch_adm(const AdmArgs& a, double* out6, cudaStream_t st);
void launch_symmetrise(const DevPatch* p, const DevLevel* l, int patch, long long half_tot,
                       cudaStream_t st);
int launch_pi_symmetry(const DevPatch* p, const DevLevel* l, int patch, long long tot,
                       double* partial, double* out, cudaStream_t st);

}  // namespace sacrak
