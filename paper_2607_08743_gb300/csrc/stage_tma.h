// Launch interface of the TMA-staged mixed-precision stage kernels
// (z4c_mixed_tma.cu).  Host code builds one CUtensorMap per patch and split
// buffer (hl[0..2], sa, sb) for the tile shape of the chosen variant and
// passes them by value (__grid_constant__), so that the kernel can pick the
// stage input from the ring slot it reads on the device.
#pragma once
#include <cuda.h>

#include "sacrak_dev.cuh"

namespace sacrak {

constexpr int TMA_MAXP = 8;       // patches of one level in one launch
// bound of a TMA stage kernel's wait for one copy: about 2 s of SM clock
constexpr long long TMA_WAIT_CYCLES = 4000000000LL;
constexpr int TMA_NVARIANTS = 4;  // tile shapes 32x4x1, 32x2x2, 32x4x2, 32x8x1

struct TmaStageArgs {
  CUtensorMap map[TMA_MAXP][5];  // per patch slot: hl[0], hl[1], hl[2], sa, sb
  StageArgs st;                  // tiles / ntiles of st are not used
  int np;                        // patches in this launch
  int ntiles;                    // tiles over all of them
  int pid[TMA_MAXP];             // patch index of each slot
  int tstart[TMA_MAXP + 1];      // first tile of each slot
  int ntx[TMA_MAXP], nty[TMA_MAXP];  // tiles along x and y of each slot
  int nz[TMA_MAXP];              // NZ (z extent incl. ghosts) of each slot
  long long wait_cycles;         // bound of the wait for a field's copy (SM clock cycles);
                                 // < 0: every such wait counts as run out at once (tests)
};

// tile shape (TY, TZ) of variant v; tiles are 32 x TY x TZ points
void tma_variant_shape(int v, int* ty, int* tz);
// bytes of one field box (40 x (TY+6) x (TZ+6) hi/lo pairs)
int tma_box_bytes(int v);
// opt the kernels of variant v in to their shared memory; returns the
// resident CTAs per SM (0 on failure)
int tma_setup_variant(int v);
void launch_stage_tma(int v, const TmaStageArgs& a, int grid, cudaStream_t st);

// The same arithmetic reading every stencil value through the L1 cache, over
// the 32 x 4 x 1 tile list of StageArgs.  Variant v: 0 3 CTAs per SM; 1 also
// prefetches the next field's stencil rows into L1 and the epilogue's
// streaming reads into L2; 2 as 1 with 4 CTAs per SM (128 registers); 3 as 1
// with only the star rows prefetched; 4 only the z-arm rows; 5 only the
// epilogue's reads; 6 as 4 with the x-neighbour inner differences of the
// mixed derivatives D_x D_y, D_x D_z exchanged by warp shuffles; 7 as 6 with
// 4 CTAs per SM; 8 as 4 with 4 CTAs per SM.  ldg_setup opts the kernels in to their shared memory
// (false on failure).
int ldg_setup(int v);
void launch_stage_ldg(int v, const StageArgs& a, cudaStream_t st);

// Variant 4 with the row and plane pitches of the level's patches fixed at
// compile time (z4c_mixed_fixed.cu), 3 or 4 CTAs per SM: instances for
// patches n[0] = n[1] = n, n in {32, 48, 64, 96, 128, 160, 192} (row pitch
// align8(n + 7) pairs, plane pitch that times n + 6).  launch_stage_fixed
// launches the instance of pitches (sy, sz) for a stage 1..4 and returns
// true; it returns false, and launches nothing, for other pitches or for
// stage 0 (the RHS alone).
bool fixed_setup(int ctas_per_sm);
bool launch_stage_fixed(const StageArgs& a, long long sy, long long sz, int ctas_per_sm, cudaStream_t st);

// The stage split in two launches: derivatives of five fields per thread into
// FP32 slot planes in global memory (dslot, split_slot_floats(ntiles) floats
// for a launch over ntiles tiles), then the algebra and the RK4 update.
long long split_slot_floats(long long ntiles);
void launch_stage_split(const StageArgs& a, float* dslot, cudaStream_t st);

// Two x-adjacent points per thread with 128-bit loads of the hi/lo pairs
// (z4c_mixed_pair.cu), one 64-thread CTA per 32 x 4 x 1 tile of StageArgs;
// element offsets are 32-bit, so every patch needs 25 * fstride < 2^31.
// Variant v: 0 prefetches the epilogue's streaming reads into L2; 1 also the
// next field's z-arm rows into L1; 2 as 1 with 3 CTAs per SM.  pair_setup opts the kernels in to their
// shared memory (false on failure).
int pair_setup(int v);
void launch_stage_pair(int v, const StageArgs& a, cudaStream_t st);

}  // namespace sacrak
