// The fused mixed-precision stage on the L1 path: one thread per point of a
// 32 x 4 x 1 tile, every stencil value of the hi/lo pairs read from global
// memory through L1 (the RHS of Sec. 2.1.1 with the stencils of Sec. 2.2,
// and the RK4 stage update).  Shared by the runtime-pitch kernels and the
// instances with the pitches of common patch widths fixed at compile time.
#pragma once

#include "mixed_common.cuh"
#include "mixed_stage.cuh"
#include "sacrak_dev.cuh"

namespace sacrak {
namespace mixed {

// Prefetch into L1 the centre row and the z arms of the next field (rows of
// other planes, which the other warps of the CTA do not load)
__device__ __forceinline__ void prefetch_zarms(const float2* F, long long sz) {
  prefetch_l1(F);
#pragma unroll
  for (int k = 1; k <= 3; ++k) {
    prefetch_l1(F + k * sz);
    prefetch_l1(F - k * sz);
  }
}

// Prefetch into L1 the rows of the next field that its stencils read: the
// centre row, the y and z arms of the star, and (for fields with second
// derivatives) the 16 rows of the y-z mixed stencil.  x neighbours share the
// rows.  A warp's 32 points cover two 128-byte lines per row.
__device__ __forceinline__ void prefetch_field(const float2* F, long long sy, long long sz, bool mixed) {
  prefetch_l1(F);
#pragma unroll
  for (int k = 1; k <= 3; ++k) {
    prefetch_l1(F + k * sy);
    prefetch_l1(F - k * sy);
    prefetch_l1(F + k * sz);
    prefetch_l1(F - k * sz);
  }
  if (mixed) {
#pragma unroll
    for (int a = -2; a <= 2; ++a)
#pragma unroll
      for (int b = -2; b <= 2; ++b)
        if (a != 0 && b != 0) prefetch_l1(F + a * sy + b * sz);
  }
}

// The same arithmetic with every stencil value read from global memory
// through the L1 cache (no staging and no barriers, so threads beyond the
// patch leave at once): one thread per point of the level's 32 x 4 x 1 tile
// list, MINB CTAs per SM (NSLOT x 128 shared-memory slots each).
// SY, SZ > 0: every patch of the level has row pitch SY and plane pitch SZ
// (pairs), so each stencil offset is a constant of the load instruction.
// PF: 0 no prefetching, 1 the next field's star and mixed-derivative rows,
// 2 its star rows only, 3 its z-arm rows only, 4 none of its rows (only the
// epilogue's streaming reads into L2)
template <int MINB, int MODE, int PF, bool SHF = false, int SY = 0, int SZ = 0>
__device__ __forceinline__ void ldg_tile(const StageArgs& S, int tile, float* sd) {
  const Tile tl = S.tiles[tile];
  const DevPatch* P = S.patches + tl.patch;
  const int t = threadIdx.x;
  const int i = tl.x0 + (t & 31), j = tl.y0 + (t >> 5), k = tl.z0;
  if (i >= P->n[0] || j >= P->n[1] || k >= P->n[2]) return;
  // every lane of the warp is alive (its row is inside the patch, and so are
  // all 32 x of the tile): the x-neighbour exchange by shuffles is allowed
  const bool full = tl.x0 + 32 <= P->n[0];
  const int ring = S.lev->ring, s = S.stage;
  const long long sy = SY > 0 ? SY : P->px, sz = SY > 0 ? SZ : P->plane, fs = P->fstride;
  const long long q = (i + GH) + (long long)(j + GH) * sy + (long long)(k + GH) * sz;
  const float2* __restrict__ U = (MODE == 1) ? P->hl[ring] : mixed_in(P, s, ring);
  if (PF && MODE == 0) {
    // the epilogue's streaming reads (RK accumulator or time level, and the
    // split of the time level) start their way from HBM into L2 now
    const double* ya = (s == 1) ? P->buf[ring] : P->buf[B_Y];
    const float2* hn = P->hl[ring];
#pragma unroll 5
    for (int f = 0; f < NF; ++f) {
      prefetch_l2(ya + f * fs + q);
      if (s < 4) prefetch_l2(hn + f * fs + q);
    }
  }
  float gt[6], be[3], gtu[6], wko[3], wup[3], c1, c2, c11;
  point_setup(U, q, fs, true, P->dx, S.prm.sigma_ko, gt, be, gtu, wko, wup, c1, c2, c11);
  // one field at a time (a loop, not unrolled: the register budget of 3 or 4
  // CTAs per SM has no room for hoisting loads across fields); with PF the
  // next field's rows are prefetched into L1 while this one is formed
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    if (PF >= 1 && PF <= 2 && f + 1 < NF)
      prefetch_field(U + (long long)(f + 1) * fs + q, sy, sz, PF == 1 && plan(f + 1).d2 != 0);
    if (PF == 3 && f + 1 < NF) prefetch_zarms(U + (long long)(f + 1) * fs + q, sz);
    if constexpr (SY > 0) {
      const FixedAcc<SY, SZ> at{U + (long long)f * fs + q};
      field_pass_p<false, FixedAcc<SY, SZ>, SmemSlots<128>, SHF>(at, plan(f), f, SmemSlots<128>{sd, t}, wko, wup,
                                                                 c1, c2, c11, gtu, full);
    } else {
      const GlobalAcc at{U + (long long)f * fs + q, sy, sz};
      field_pass_p<false, GlobalAcc, SmemSlots<128>, SHF>(at, plan(f), f, SmemSlots<128>{sd, t}, wko, wup, c1,
                                                           c2, c11, gtu, full);
    }
  }
  float cen[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const float2 v = __ldg(U + (long long)f * fs + q);
    cen[f] = v.x + v.y;
  }
  float r[NF];
  sources<false>(SmemSlots<128>{sd, t}, cen, gt, gtu, S.prm, r);
  if (MODE == 1) {
    double* out = P->buf[B_S1];
#pragma unroll
    for (int f = 0; f < NF; ++f) out[f * fs + q] = (double)r[f];
  } else {
    rk_update_mixed(P, s, ring, S.dt, q, r, S.prm.w_floor, S.err);
  }
}

}  // namespace mixed
}  // namespace sacrak
