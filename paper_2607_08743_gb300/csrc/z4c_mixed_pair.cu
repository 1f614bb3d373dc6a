// Mixed-precision Z4c RHS + RK4 stage kernel with two points per thread.
//
// Same equations, stencils and precision split as the other mixed stage
// kernels (Sec. 2.1.1, 2.2 of the SACRA-K paper; mixed_stage.cuh), with the
// memory access organised around 128-bit loads:
//
//  - A thread owns the two x-adjacent cells (x, x+1), x even.  The state
//    buffers start one element past a 16-byte boundary and the row pitch is
//    even, so the hi/lo pairs of cells (x, x+1) of any row form one aligned
//    16-byte vector: every stencil row the two points need is one 128-bit
//    load instead of two 64-bit loads.
//  - The x arms of the two points (cells x-3 .. x+4) are three 128-bit and
//    two 64-bit loads.  The nested mixed derivatives D_x D_y f and D_x D_z f
//    of the two points need the inner y (z) differences at the six columns
//    x-2 .. x+3; they are formed once per column and shared (the centre
//    columns come with the y (z) arm loads).  D_y D_z f: 16 loads serve both.
//    A field with second derivatives costs 49 loads for the two points
//    (134 with one point per thread and 64-bit loads), one with first
//    derivatives only 17 (38).
//  - Addresses are 32-bit element offsets from the field's base pointer of
//    the thread's pair.
//  - A CTA of 64 threads covers one 32 x 4 x 1 tile of the level's tile list
//    (16 pair columns x 4 rows); its 97 derivative slots per point live in
//    shared memory, one plane per slot and point.  The curvature algebra
//    and the RK4 update then run for one point after the other.
//
// Bitwise pi symmetry: each point's derivatives are the same expressions of
// its own neighbours whichever slot of the pair it occupies (the shared
// inner differences depend only on their column), so a point and its
// mirror partner (x -> -x, the other slot of another pair) round alike.
#include <math.h>

#include "mixed_common.cuh"
#include "mixed_stage.cuh"
#include "sacrak_dev.cuh"
#include "stage_tma.h"

namespace sacrak {
namespace {

using namespace mixed;

constexpr int PNT = 64;  // threads per CTA: 16 pair columns x 4 rows

// the hi/lo pairs of the cells (x, x+1) at p (16-byte aligned)
struct Two {
  float2 a, b;
};
__device__ __forceinline__ Two ld2(const float2* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return Two{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ float2 ld1(const float2* p) { return __ldg(p); }

// Star terms of one point along one axis from its seven values: adds the
// advection + dissipation to acc, sets the scaled second derivative d2 and
// returns the unscaled first difference 8 (f1 - f-1) - (f2 - f-2).  The same
// expressions as the one-point field pass.
__device__ __forceinline__ float star_axis(float2 m3, float2 m2, float2 m1, float2 c0, float2 p1, float2 p2,
                                           float2 p3, float wko, float wup, float c2, float2& acc, float& d2) {
  const float2 a = add2(sub2(m3, c0), sub2(p3, c0));
  const float2 b = add2(sub2(m2, c0), sub2(p2, c0));
  const float2 cc = add2(sub2(m1, c0), sub2(p1, c0));
  const float2 ko = fma2s(cc, 15.0f, fma2s(b, -6.0f, a));  // Delta^6
  const float2 e1 = sub2(p1, m1), e2n = sub2(m2, p2), e3 = sub2(p3, m3);
  const float2 as = fma2s(e1, 21.0f, fma2s(e2n, 6.0f, e3));
  acc = fma2s(ko, wko, acc);
  acc = fma2s(as, wup, acc);
  d2 = hsum(fma2s(cc, 16.0f, neg2(b))) * c2;
  return hsum(fma2s(e1, 8.0f, e2n));
}

// unscaled first difference of (hi, lo) pairs from the values at +1, -1, +2, -2
__device__ __forceinline__ float2 inner2(float2 p1, float2 m1, float2 p2, float2 m2) {
  return fma2s(sub2(p1, m1), 8.0f, sub2(m2, p2));
}
// D_A (D_B f) from the inner differences at A-offsets +1, -1, +2, -2
__device__ __forceinline__ float outer2(float2 ip1, float2 im1, float2 ip2, float2 im2, float c11) {
  return hsum(fma2s(sub2(ip1, im1), 8.0f, sub2(im2, ip2))) * c11;
}

// D_x D_B f of the two points: st is the pitch along B, cp1 .. cm2 the arm
// rows of the pair at B-offsets +1, -1, +2, -2.  The inner B differences at
// the six columns x-2 .. x+3 are formed once and shared.
__device__ __forceinline__ void mixed_x(const float2* __restrict__ F, int st, const Two cp1, const Two cm1,
                                        const Two cp2, const Two cm2, float c11, float& d0, float& d1) {
  const Two lp1 = ld2(F + st - 2), lm1 = ld2(F - st - 2), lp2 = ld2(F + 2 * st - 2), lm2 = ld2(F - 2 * st - 2);
  const Two rp1 = ld2(F + st + 2), rm1 = ld2(F - st + 2), rp2 = ld2(F + 2 * st + 2), rm2 = ld2(F - 2 * st + 2);
  const float2 im2 = inner2(lp1.a, lm1.a, lp2.a, lm2.a);  // column x-2
  const float2 im1 = inner2(lp1.b, lm1.b, lp2.b, lm2.b);  // x-1
  const float2 i0 = inner2(cp1.a, cm1.a, cp2.a, cm2.a);   // x
  const float2 i1 = inner2(cp1.b, cm1.b, cp2.b, cm2.b);   // x+1
  const float2 i2 = inner2(rp1.a, rm1.a, rp2.a, rm2.a);   // x+2
  const float2 i3 = inner2(rp1.b, rm1.b, rp2.b, rm2.b);   // x+3
  d0 = outer2(i1, im1, i2, im2, c11);
  d1 = outer2(i2, i0, i3, im1, c11);
}

// derivative slots: one plane of PNT floats per slot and point
struct PairSlots {
  float* sd;
  int t;
  __device__ __forceinline__ void put(int k, float v0, float v1) const {
    sd[k * PNT + t] = v0;
    sd[(NSLOT + k) * PNT + t] = v1;
  }
  __device__ __forceinline__ void add(int k, float v0, float v1) const {
    sd[k * PNT + t] += v0;
    sd[(NSLOT + k) * PNT + t] += v1;
  }
};
// the slots of one point, as the curvature algebra reads them
struct PointSlots {
  const float* sd;
  __device__ __forceinline__ float operator()(int k) const { return sd[k * PNT]; }
};

// One field for the two points: F is the field at cell x of the thread's
// row; sy, sz the row and plane pitch in elements.
__device__ __forceinline__ void pair_field(const float2* __restrict__ F, int sy, int sz, const FieldPlan P,
                                           const int f, const PairSlots& SD, const float (&wko)[2][3],
                                           const float (&wup)[2][3], float c1, float c2, float c11,
                                           const float (&gtu0)[6], const float (&gtu1)[6]) {
  float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
  float dd0[6], dd1[6], g0[3], g1[3];
  // x arms: cells x-3 .. x+4
  const float2 xm3 = ld1(F - 3);
  const Two xa = ld2(F - 2), xc = ld2(F), xb = ld2(F + 2);
  const float2 x4 = ld1(F + 4);
  g0[0] = star_axis(xm3, xa.a, xa.b, xc.a, xc.b, xb.a, xb.b, wko[0][0], wup[0][0], c2, acc0, dd0[0]);
  g1[0] = star_axis(xa.a, xa.b, xc.a, xc.b, xb.a, xb.b, x4, wko[1][0], wup[1][0], c2, acc1, dd1[0]);
  // y and z arms: one 128-bit load per row serves both points
  Two ya[6], za[6];  // offsets -3, -2, -1, +1, +2, +3
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ya[2 - k] = ld2(F - (k + 1) * sy);
    ya[3 + k] = ld2(F + (k + 1) * sy);
    za[2 - k] = ld2(F - (k + 1) * sz);
    za[3 + k] = ld2(F + (k + 1) * sz);
  }
  g0[1] = star_axis(ya[0].a, ya[1].a, ya[2].a, xc.a, ya[3].a, ya[4].a, ya[5].a, wko[0][1], wup[0][1], c2, acc0,
                    dd0[3]);
  g1[1] = star_axis(ya[0].b, ya[1].b, ya[2].b, xc.b, ya[3].b, ya[4].b, ya[5].b, wko[1][1], wup[1][1], c2, acc1,
                    dd1[3]);
  g0[2] = star_axis(za[0].a, za[1].a, za[2].a, xc.a, za[3].a, za[4].a, za[5].a, wko[0][2], wup[0][2], c2, acc0,
                    dd0[5]);
  g1[2] = star_axis(za[0].b, za[1].b, za[2].b, xc.b, za[3].b, za[4].b, za[5].b, wko[1][2], wup[1][2], c2, acc1,
                    dd1[5]);
  if (P.d1 >= 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) SD.put(P.d1 + P.d1s * d, g0[d] * c1, g1[d] * c1);
  }
  if (P.d2 != 0) {
    // D_x D_y and D_x D_z: the inner y (z) differences at the columns
    // x-2 .. x+3, from the rows at +-1, +-2 (the centre columns are the arms)
    mixed_x(F, sy, ya[3], ya[2], ya[4], ya[1], c11, dd0[1], dd1[1]);
    mixed_x(F, sz, za[3], za[2], za[4], za[1], c11, dd0[2], dd1[2]);
    // D_y D_z: the inner z difference at the rows y-2 .. y+2 (not y)
    float2 iz0[4], iz1[4];  // rows +1, -1, +2, -2
    constexpr int KY[4] = {1, -1, 2, -2};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2* R = F + KY[u] * sy;
      const Two p1 = ld2(R + sz), m1 = ld2(R - sz), p2 = ld2(R + 2 * sz), m2 = ld2(R - 2 * sz);
      iz0[u] = inner2(p1.a, m1.a, p2.a, m2.a);
      iz1[u] = inner2(p1.b, m1.b, p2.b, m2.b);
    }
    dd0[4] = outer2(iz0[0], iz0[1], iz0[2], iz0[3], c11);
    dd1[4] = outer2(iz1[0], iz1[1], iz1[2], iz1[3], c11);
    if (P.d2 == 1) {
#pragma unroll
      for (int q = 0; q < 6; ++q) SD.put(P.d2slot + q, dd0[q], dd1[q]);
    } else {
      SD.put(P.d2slot, symc(gtu0, dd0), symc(gtu1, dd1));
      if (P.d2 == 3) {
        // d_j d_I beta^I (compile-time indices: a runtime index would put
        // dd in local memory)
        const int I = f - F_BETX;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float v0 = I == 0 ? dd0[S2(j, 0)] : (I == 1 ? dd0[S2(j, 1)] : dd0[S2(j, 2)]);
          const float v1 = I == 0 ? dd1[S2(j, 0)] : (I == 1 ? dd1[S2(j, 1)] : dd1[S2(j, 2)]);
          if (I == 0)
            SD.put(S_DVB + j, v0, v1);
          else
            SD.add(S_DVB + j, v0, v1);
        }
      }
    }
  }
  SD.put(S_AK + f, hsum(acc0), hsum(acc1));
}

__device__ __forceinline__ void prefetch_l1p(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
__device__ __forceinline__ void prefetch_l2p(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// PF: 1 the epilogue's streaming reads prefetched into L2 at the start;
// 3 also the next field's centre row and z arms into L1 while a field is
// formed.  MODE 1: right-hand side only (into the second stage buffer).
template <int MODE, int PF, int MINB>
__global__ void __launch_bounds__(PNT, MINB) z4c_stage_pair_kernel(StageArgs S) {
  extern __shared__ float sdp[];
  const Tile tl = S.tiles[blockIdx.x];
  const DevPatch* P = S.patches + tl.patch;
  const int t = threadIdx.x;
  const int i = tl.x0 + 2 * (t & 15), j = tl.y0 + (t >> 4), k = tl.z0;
  if (i >= P->n[0] || j >= P->n[1] || k >= P->n[2]) return;
  const bool valid1 = i + 1 < P->n[0];  // odd n: the pair's second cell is a ghost
  const int ring = S.lev->ring, s = S.stage;
  const int sy = P->px, sz = (int)P->plane, fs = (int)P->fstride;
  const int q = (i + GH) + (j + GH) * sy + (k + GH) * sz;
  const float2* __restrict__ U = (MODE == 1) ? P->hl[ring] : mixed_in(P, s, ring);
  if (PF && MODE == 0) {
    const double* ya = (s == 1) ? P->buf[ring] : P->buf[B_Y];
    const float2* hn = P->hl[ring];
#pragma unroll 5
    for (int f = 0; f < NF; ++f) {
      prefetch_l2p(ya + f * fs + q);
      if (s < 4) prefetch_l2p(hn + f * fs + q);
    }
  }
  // centre values of gt and beta of both points, inverse metric, weights
  float gt0[6], gt1[6], gtu0[6], gtu1[6], wko[2][3], wup[2][3];
  {
    float be[2][3];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const Two v = ld2(U + (F_GXX + a) * fs + q);
      gt0[a] = v.a.x + v.a.y;
      gt1[a] = valid1 ? v.b.x + v.b.y : gt0[a];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const Two v = ld2(U + (F_BETX + d) * fs + q);
      be[0][d] = v.a.x + v.a.y;
      be[1][d] = valid1 ? v.b.x + v.b.y : be[0][d];
    }
    sym_inv_f(gt0, gtu0);
    sym_inv_f(gt1, gtu1);
    const float h = (float)P->dx;
    const float c1 = 1.0f / (12.0f * h);
    const float cko = (float)(S.prm.sigma_ko / (64.0 * P->dx));
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        wko[p][d] = 0.5f * fabsf(be[p][d]) * c1 + cko;
        wup[p][d] = 0.5f * be[p][d] * c1;
      }
  }
  const float h = (float)P->dx;
  const float c1 = 1.0f / (12.0f * h), c2 = c1 / h, c11 = c1 * c1;
  const PairSlots SD{sdp, t};
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    const float2* F = U + f * fs + q;
    if (PF == 3 && f + 1 < NF) {
      const float2* Fn = F + fs;
      prefetch_l1p(Fn);
#pragma unroll
      for (int kk = 1; kk <= 3; ++kk) {
        prefetch_l1p(Fn + kk * sz);
        prefetch_l1p(Fn - kk * sz);
      }
    }
    pair_field(F, sy, sz, plan(f), f, SD, wko, wup, c1, c2, c11, gtu0, gtu1);
  }
  // curvature algebra and RK4 update, one point after the other
#pragma unroll 1
  for (int pp = 0; pp < 2; ++pp) {
    if (pp == 1 && !valid1) break;
    const int qp = q + pp;
    float cen[NF], gt[6], gtu[6], r[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float2 v = __ldg(U + f * fs + qp);
      cen[f] = v.x + v.y;
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      gt[a] = pp ? gt1[a] : gt0[a];
      gtu[a] = pp ? gtu1[a] : gtu0[a];
    }
    sources<false>(PointSlots{sdp + pp * NSLOT * PNT + t}, cen, gt, gtu, S.prm, r);
    if (MODE == 1) {
      double* out = P->buf[B_S1];
#pragma unroll
      for (int f = 0; f < NF; ++f) out[f * fs + qp] = (double)r[f];
    } else {
      rk_update_mixed(P, s, ring, S.dt, qp, r, S.prm.w_floor, S.err);
    }
  }
}

constexpr int PAIR_SMEM = 2 * NSLOT * PNT * 4;

// MINB CTAs per SM; with MINB = 3 the shared-memory carveout is held to
// 164 KB (3 CTAs of slots), which leaves the rest of the SM's 256 KB to L1
template <int PF, int MINB>
bool setup_pair() {
  bool ok = cudaFuncSetAttribute(z4c_stage_pair_kernel<0, PF, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 PAIR_SMEM) == cudaSuccess &&
            cudaFuncSetAttribute(z4c_stage_pair_kernel<1, PF, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 PAIR_SMEM) == cudaSuccess;
  if (ok && MINB == 3)
    ok = cudaFuncSetAttribute(z4c_stage_pair_kernel<0, PF, MINB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              72) == cudaSuccess &&
         cudaFuncSetAttribute(z4c_stage_pair_kernel<1, PF, MINB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              72) == cudaSuccess;
  return ok;
}

template <int PF, int MINB>
void launch_pair(const StageArgs& a, cudaStream_t st) {
  if (a.stage == 0)
    z4c_stage_pair_kernel<1, PF, MINB><<<a.ntiles, PNT, PAIR_SMEM, st>>>(a);
  else
    z4c_stage_pair_kernel<0, PF, MINB><<<a.ntiles, PNT, PAIR_SMEM, st>>>(a);
}

}  // namespace

// variant v: 0 L2 prefetch of the epilogue's reads, 4 CTAs per SM; 1 also
// the next field's z-arm rows into L1; 2 as 1 with 3 CTAs per SM
int pair_setup(int v) {
  switch (v) {
    case 0: return setup_pair<1, 4>();
    case 1: return setup_pair<3, 4>();
    case 2: return setup_pair<3, 3>();
  }
  return 0;
}

void launch_stage_pair(int v, const StageArgs& a, cudaStream_t st) {
  if (a.ntiles == 0) return;
  switch (v) {
    case 0: launch_pair<1, 4>(a, st); break;
    case 1: launch_pair<3, 4>(a, st); break;
    case 2: launch_pair<3, 3>(a, st); break;
  }
}

}  // namespace sacrak
