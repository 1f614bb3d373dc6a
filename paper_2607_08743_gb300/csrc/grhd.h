// Launch interface of the GR hydrodynamics (matter) kernels (grhd.cu).
//
// The fluid of Sec. 2.1.2 of the SACRA-K paper: primitives (rho, eps, u_i)
// and the densitised conserved variables sqrt(gamma) (D, J_i, rho_H), with
// the hybrid EOS (piecewise polytrope + thermal part), evolved with the
// spacetime by the same RK4 stages (Sec. 2.2): PPM (steep minmod b = 3) +
// HLLE face fluxes, geometric sources, Newton-Raphson recovery on the
// Lorentz factor w, atmosphere floor.  FP64 throughout.  (Face fluxes:
// HLLC of special relativity in an orthonormal tetrad in which the face is
// at rest, HLLE there where the intermediate state is unphysical; or HLLE
// in the coordinate frame.)
#pragma once
#include "sacrak_dev.cuh"

namespace sacrak {

constexpr int NM = 5;        // rho, eps, u_x, u_y, u_z  /  D^, J^_x, J^_y, J^_z, E^
constexpr int NMP = 6;       // primitive arrays: the five plus the Lorentz factor w
constexpr int NZSRC = 11;    // matter terms of the Z4c RHS: Khat, Theta, At (6), Gamt (3)
constexpr int MAX_PIECES = 4;

struct DevEOS {
  int n;                      // pieces of the cold polytrope
  double K[MAX_PIECES], G[MAX_PIECES], a[MAX_PIECES];
  double rb[MAX_PIECES - 1];  // density boundaries between pieces
  double gth;                 // Gamma_th
};

struct MatterArgs {
  const DevPatch* P;          // device pointer to the patch
  const DevLevel* lev;        // its level (ring slot on the device)
  int n[3], NX, NY, NZ;
  long long sy, sz, fs;
  double dx, origin[3];
  DevEOS eos;
  double rho_atm, r_atm;      // floor f_atm rho_max inside r_atm, r^-3 outside
  int periodic;               // ghost cells: 0 outflow (zero gradient), 1 periodic
  int stage;                  // 1..4 RK stage; 5: the new level after stage 4; 0: current level
  int coupled;                // write the Z4c matter terms (spacetime evolved with the fluid)
  int riemann;                // face flux: 0 HLLC in the face tetrad (HLLE fallback), 1 HLLE in the coordinate frame
  double dt;
  double* out;                // update kernel with stage 0: d_t of the conserved variables
  unsigned* err;
  // levels > 0: ghost cells from the parent (Sec. 2.2.1) -- the parent level,
  // the time weights of its (oldest, middle, newest) time levels at this
  // call's time (three valid levels / two), and whether the flux sums of the
  // two-step average start with this step
  const DevLevel* plev;
  double wq[3], wl[3];
  int first_substep;
};

// The fluid of one patch just shifted (Sec. 2.2.1): its level's ring slot,
// its parent's, the shift in its own cells
struct MatterMoveArgs {
  const DevPatch* patches;
  int patch;
  int ring, pring;
  int sh[3];
  DevEOS eos;
  unsigned* err;
};

// One child level's fluid operators at the refinement boundary (Sec. 2.2.1)
struct MatterAmrArgs {
  const DevPatch* patches;
  const int* child_ids;       // the children (one level)
  const DevLevel* plev;       // their parent level
  const DevLevel* clev;       // their level
  double dt_parent;           // reflux: the parent's step
};

// Primitive recovery of the stage's conserved state (active cells) with the
// atmosphere, the Lorentz factor of the previous recovery as the Newton
// guess, and (coupled) the Z4c matter terms of the recovered fluid.
void launch_matter_prep(const MatterArgs& a, cudaStream_t st);
// ghost cells of the primitive arrays
void launch_matter_ghosts(const MatterArgs& a, cudaStream_t st);
// the fluid of a shifted patch into its face-flux arrays (copy where active
// before and after, the parent's prolongation elsewhere; see grhd.cu)
void launch_matter_move(const MatterMoveArgs& a, long long ncells, cudaStream_t st);
// the largest rest-mass density over a patch's active cells and its first
// active index: part[0], part[1] (index -1: no finite density); part holds
// 2 x max_blocks doubles
void launch_density_max(const DevPatch* patches, int patch, long long nact, double* part, int max_blocks,
                        cudaStream_t st);
// equatorial symmetry: the z < 0 ghost layers of the primitives and of the
// stage's conserved variables mirror those above z = 0 (patches on z = 0)
void launch_matter_zreflect(const MatterArgs& a, cudaStream_t st);
// face fluxes along dir (0, 1, 2) from the PPM states (MatterArgs::riemann)
void launch_matter_flux(const MatterArgs& a, int dir, cudaStream_t st);
// flux divergence + sources: RK4 stage update (stage 1..4) or d_t (stage 0)
void launch_matter_update(const MatterArgs& a, cudaStream_t st);
// conserved variables of the primitives (after an upload of primitives)
void launch_matter_prim2con(const MatterArgs& a, cudaStream_t st);
// ghost cells of a level > 0 fluid from the cached prolongations of the
// parent's time levels (instead of launch_matter_ghosts)
void launch_matter_child_ghosts(const MatterArgs& a, cudaStream_t st);
// prolongation of the parent's current fluid onto every child's ghost shell,
// cached in the child's slot of the parent's current ring slot: conservative
// WENO5 of D^ (x, y, z), 6th-order Lagrange of eps and u_i, fallbacks
void launch_matter_prolong(const MatterAmrArgs& a, int nchildren, long long max_shell, cudaStream_t st);
// parent cells under the children's active cells <- the mean of the 8 children
void launch_matter_restrict(const MatterAmrArgs& a, int nchildren, long long max_cells, cudaStream_t st);
// parent cells next to the children: the parent's boundary-face fluxes of its
// last step replaced by the children's (averaged over 4 faces and 2 steps)
void launch_matter_reflux(const MatterAmrArgs& a, int nchildren, long long max_faces, cudaStream_t st);

}  // namespace sacrak
