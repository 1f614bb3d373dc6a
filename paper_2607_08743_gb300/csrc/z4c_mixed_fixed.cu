// The L1-path mixed-precision stage (variant 4 of launch_stage_ldg: the next
// field's z-arm rows prefetched into L1) instantiated for the row and plane
// pitches of patches of common widths, with 3 or 4 CTAs per SM.  With the pitches
// known at compile time every stencil offset of a field is a constant of its
// load instruction, so the 64-bit address arithmetic per stencil value of the
// runtime-pitch kernel goes away; the arithmetic is the same, value for value.
#include "ldg_stage.cuh"
#include "sacrak_dev.cuh"
#include "stage_tma.h"

namespace sacrak {
namespace {

using namespace mixed;

// row pitch (pairs) of a patch n cells wide with its ghosts: n + 6 cells and
// one spare element, rounded up to 8; plane pitch: rows of n + 6 cells
template <int N>
struct Pitch {
  static constexpr int SY = (N + 7 + 7) / 8 * 8;
  static constexpr int SZ = SY * (N + 6);
};

template <int MINB, int SY, int SZ>
__global__ void __launch_bounds__(128, MINB) z4c_stage_fixed_kernel(StageArgs S) {
  extern __shared__ float sd[];
  ldg_tile<MINB, 0, 3, false, SY, SZ>(S, blockIdx.x, sd);
}

template <int MINB, int N>
bool setup_one() {
  return cudaFuncSetAttribute(z4c_stage_fixed_kernel<MINB, Pitch<N>::SY, Pitch<N>::SZ>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, NSLOT * 128 * 4) == cudaSuccess;
}

template <int MINB, int N>
bool launch_one(const StageArgs& a, long long sy, long long sz, cudaStream_t st) {
  if (sy != Pitch<N>::SY || sz != Pitch<N>::SZ) return false;
  z4c_stage_fixed_kernel<MINB, Pitch<N>::SY, Pitch<N>::SZ><<<a.ntiles, 128, NSLOT * 128 * 4, st>>>(a);
  return true;
}

template <int MINB>
bool setup_all() {
  return setup_one<MINB, 32>() && setup_one<MINB, 48>() && setup_one<MINB, 64>() && setup_one<MINB, 96>() &&
         setup_one<MINB, 128>() && setup_one<MINB, 160>() && setup_one<MINB, 192>();
}

template <int MINB>
bool launch_all(const StageArgs& a, long long sy, long long sz, cudaStream_t st) {
  return launch_one<MINB, 32>(a, sy, sz, st) || launch_one<MINB, 48>(a, sy, sz, st) ||
         launch_one<MINB, 64>(a, sy, sz, st) || launch_one<MINB, 96>(a, sy, sz, st) ||
         launch_one<MINB, 128>(a, sy, sz, st) || launch_one<MINB, 160>(a, sy, sz, st) ||
         launch_one<MINB, 192>(a, sy, sz, st);
}

}  // namespace

bool fixed_setup(int ctas_per_sm) { return ctas_per_sm == 4 ? setup_all<4>() : setup_all<3>(); }

bool launch_stage_fixed(const StageArgs& a, long long sy, long long sz, int ctas_per_sm, cudaStream_t st) {
  if (a.stage < 1 || a.stage > 4) return false;
  if (a.ntiles == 0) return true;
  return ctas_per_sm == 4 ? launch_all<4>(a, sy, sz, st) : launch_all<3>(a, sy, sz, st);
}

}  // namespace sacrak
