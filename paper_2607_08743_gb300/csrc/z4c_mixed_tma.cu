// Mixed-precision Z4c RHS + RK4 stage kernel with TMA-staged field tiles.
//
// Same equations and precision split as z4c_mixed.cu (Sec. 2.1.1, 2.2 of the
// SACRA-K paper: 4th-order centred derivatives, lopsided upwind advection,
// 6th-order Kreiss-Oliger dissipation, classical RK4), organised for the
// memory system of sm_103a:
//
//  - A CTA owns a tile of 32 x TY x TZ points (one thread per point, x along
//    the lanes).  For every field it needs the tile plus a 3-cell halo, a box
//    of 38 x (TY+6) x (TZ+6) hi/lo pairs, which one elected thread copies into
//    shared memory with a TMA tensor load (cp.async.bulk.tensor, completion on
//    an mbarrier).  Two buffers alternate: the copy of the next field (or of
//    the next tile's first field) runs while the current field is processed.
//  - Every stencil value is then a shared-memory load at a compile-time
//    offset.  The hi and lo parts are processed together with packed FP32x2
//    arithmetic (one instruction per pair).
//  - The lopsided upwind stencil is split into its symmetric part, which is
//    the Kreiss-Oliger sixth difference, and its antisymmetric part
//    21 (f1 - f-1) - 6 (f2 - f-2) + (f3 - f-3): for either sign of the shift,
//    beta * upwind = |beta|/2 * Delta6 + beta/2 * antisymmetric part, so no
//    branch or select depends on the sign of the shift.
//  - Second derivatives of gt and beta are contracted with gt^lm as they are
//    formed (the Ricci tensor and the Gamma-driver only need those
//    contractions), so 97 derivative values per point are kept in shared
//    memory for the curvature algebra instead of 139.
//  - The kernel is persistent: the grid is sized to the resident CTAs and
//    every CTA walks the tiles of all patches of a level with a static stride.
//
// Waits on the mbarriers are bounded: a wait that runs out sets ERR_TIMEOUT,
// the CTA stops issuing copies, waits (bounded) for the copy it has in
// flight and returns without writing results.
#include <cuda.h>  // CUtensorMap (the type only)
#include <math.h>

#include "mixed_common.cuh"
#include "sacrak_dev.cuh"
#include "stage_tma.h"

namespace sacrak {
namespace {

using namespace mixed;

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 3D tensor tile -> shared memory, completion counted on `bar` in bytes
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// bounded wait: about 2 s of SM clock at most
constexpr long long WAIT_CYCLES = 4000000000LL;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > WAIT_CYCLES) return false;
  return true;
}

// ------------------------------------------------------------------ FP32x2

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 ra, rb, rr;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rr, ra, rb;\n\tmov.b64 {%0, %1}, rr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// a * s + c with a scalar s for both halves
__device__ __forceinline__ float2 fma2s(float2 a, float s, float2 c) {
  return __ffma2_rn(a, make_float2(s, s), c);
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float hsum(float2 a) { return a.x + a.y; }

// ------------------------------------------------------------------ layout

// derivative slots kept per point (one column per thread)
enum {
  S_DGT = 0,    // d_d gt_a at 6 d + a
  S_DW = 18,    // d_d W
  S_DAL = 21,   // d_d alpha
  S_DGAM = 24,  // d_d Gamt^i at 3 d + i
  S_DBE = 33,   // d_d beta^i at 3 d + i
  S_DKH = 42,
  S_DTH = 45,
  S_LGT = 48,   // gt^lm d_l d_m gt_a
  S_DDW = 54,   // d_a d_b W (symmetric index)
  S_DDAL = 60,  // d_a d_b alpha
  S_LBE = 66,   // gt^lm d_l d_m beta^i
  S_DVB = 69,   // d_j d_k beta^k
  S_AK = 72,    // advection + dissipation of field f
  NSLOT = 97
};
// The split kernels (derivatives to global memory, then the algebra) keep
// the three contributions d_j d_i beta^i of the three beta fields apart
// (they are formed by different threads): S_DVB + 3 i + j, then S_AK.
enum { S_AK_SPLIT = 78, NSLOT_SPLIT = 103 };

// slot storage: one column per thread in shared memory, or one plane per
// slot in global memory (point index p of n points)
template <int NT>
struct SmemSlots {
  float* sd;
  int t;
  __device__ __forceinline__ float& operator()(int k) const { return sd[k * NT + t]; }
};
struct GlobalSlots {
  float* d;
  long long n, p;
  __device__ __forceinline__ float& operator()(int k) const { return d[k * n + p]; }
};
struct GlobalSlotsIn {
  const float* __restrict__ d;
  long long n, p;
  __device__ __forceinline__ float operator()(int k) const { return __ldg(d + k * n + p); }
};

// what phase 1 forms for each field
struct FieldPlan {
  int d1;    // slot of d_x f (-1: none); d_y, d_z follow at +d1s, +2 d1s
  int d1s;
  int d2;    // 0 none, 1 all six into slots at d2slot, 2 contract with gt^lm into d2slot,
             // 3 contract (beta^i: d2slot = S_LBE + i) and add d_j d_i beta^i into S_DVB + j
  int d2slot;
  int cen;   // keep the centre value for phase 2
};

__host__ __device__ constexpr FieldPlan plan(int f) {
  return f == F_W     ? FieldPlan{S_DW, 1, 1, S_DDW, 1}
         : f <= F_GZZ ? FieldPlan{S_DGT + (f - F_GXX), 6, 2, S_LGT + (f - F_GXX), 0}
         : f == F_KH  ? FieldPlan{S_DKH, 1, 0, 0, 1}
         : f == F_TH  ? FieldPlan{S_DTH, 1, 0, 0, 1}
         : f <= F_AZZ ? FieldPlan{-1, 0, 0, 0, 1}
         : f <= F_GAMZ ? FieldPlan{S_DGAM + (f - F_GAMX), 3, 0, 0, 1}
         : f == F_ALP ? FieldPlan{S_DAL, 1, 1, S_DDAL, 1}
         : f <= F_BETZ ? FieldPlan{S_DBE + (f - F_BETX), 3, 3, S_LBE + (f - F_BETX), 0}
                       : FieldPlan{-1, 0, 0, 0, 1};
}

template <int TY, int TZ>
struct Cfg {
  static constexpr int NT = 32 * TY * TZ;
  static constexpr int BX = 38, BY = TY + 6, BZ = TZ + 6;
  static constexpr int SY = BX, SZ = BX * BY;  // strides in the box (pairs)
  static constexpr unsigned BYTES = BX * BY * BZ * 8;
  static constexpr int BUFB = (BYTES + 127) / 128 * 128;
  static constexpr int SMEM = 1024 + 2 * BUFB + NSLOT * NT * 4;
};

struct TileLoc {
  int slot;  // patch slot in the launch arguments
  int x0, y0, z0;
};

template <int TY, int TZ>
__device__ __forceinline__ TileLoc locate(const TmaStageArgs& A, int tile) {
  int s = 0;
#pragma unroll 1
  while (s + 1 < A.np && tile >= A.tstart[s + 1]) ++s;
  int r = tile - A.tstart[s];
  TileLoc L;
  L.slot = s;
  L.x0 = (r % A.ntx[s]) * 32;
  r /= A.ntx[s];
  L.y0 = (r % A.nty[s]) * TY;
  L.z0 = (r / A.nty[s]) * TZ;
  return L;
}

// ------------------------------------------------------------------ phase 1

// Where a stencil value comes from: the staged box in shared memory (offsets
// are compile-time constants) or the stage state in global memory through
// the L1 cache.
template <int SY, int SZ>
struct SmemAcc {
  const float2* __restrict__ T;
  int c;  // this thread's point in the box
  __device__ __forceinline__ float2 operator()(int dx, int dy, int dz) const {
    return T[c + dx + dy * SY + dz * SZ];
  }
};
struct GlobalAcc {
  const float2* __restrict__ F;  // the field at this thread's point
  long long sy, sz;
  __device__ __forceinline__ float2 operator()(int dx, int dy, int dz) const {
    return __ldg(F + dx + dy * sy + dz * sz);
  }
};

// One field, values from `at`: forms the plan's derivatives into the slots
// (NT columns), the advection + dissipation sum into S_AK + F, and returns
// the centre value.
// The unscaled first difference 8 (f_1 - f_-1) - (f_2 - f_-2) along B at the
// point `at` + k e_A, summed from its hi/lo pair (the inner derivative of the
// nested mixed derivative D_A (D_B f)).
template <class Acc>
__device__ __forceinline__ float inner_d1(const Acc& at, int A, int B, int k) {
  auto pt = [&](int kb) {
    return at((A == 0 ? k : 0) + (B == 0 ? kb : 0), (A == 1 ? k : 0) + (B == 1 ? kb : 0),
              (A == 2 ? k : 0) + (B == 2 ? kb : 0));
  };
  return hsum(fma2s(sub2(pt(1), pt(-1)), 8.0f, sub2(pt(-2), pt(2))));
}

// D_A (D_B f) * 144 h^2 from the inner differences at A-offsets +1, -1, +2, -2
__device__ __forceinline__ float outer_d1(float gp1, float gm1, float gp2, float gm2) {
  return __fmaf_rn(__fsub_rn(gp1, gm1), 8.0f, __fsub_rn(gm2, gp2));
}

template <bool SPLIT, class Acc, class Slots, bool SHF = false>
__device__ __forceinline__ float field_pass_p(const Acc& at, const FieldPlan P, const int F, const Slots& SD,
                                              const float wko[3], const float wup[3], float c1, float c2,
                                              float c11, const float gtu[6], bool full = false) {
#define AT(d, k) at((d) == 0 ? (k) : 0, (d) == 1 ? (k) : 0, (d) == 2 ? (k) : 0)
  const float2 c0 = at(0, 0, 0);
  float2 acc = make_float2(0.0f, 0.0f);
  float dd[6];  // second derivatives, symmetric index
  float g1[3];  // unscaled first differences at the point (the inner ones of D_x D_y, D_x D_z)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float2 m3 = AT(d, -3), m2 = AT(d, -2), m1 = AT(d, -1);
    const float2 p1 = AT(d, 1), p2 = AT(d, 2), p3 = AT(d, 3);
    // centre-referenced sums (symmetric stencils) ...
    const float2 a = add2(sub2(m3, c0), sub2(p3, c0));
    const float2 b = add2(sub2(m2, c0), sub2(p2, c0));
    const float2 cc = add2(sub2(m1, c0), sub2(p1, c0));
    const float2 ko = fma2s(cc, 15.0f, fma2s(b, -6.0f, a));  // Delta^6 along d
    // ... and pair differences (antisymmetric stencils)
    const float2 e1 = sub2(p1, m1), e2n = sub2(m2, p2), e3 = sub2(p3, m3);
    const float2 as = fma2s(e1, 21.0f, fma2s(e2n, 6.0f, e3));
    acc = fma2s(ko, wko[d], acc);
    acc = fma2s(as, wup[d], acc);
    g1[d] = hsum(fma2s(e1, 8.0f, e2n));
    if (P.d1 >= 0) SD(P.d1 + P.d1s * d) = g1[d] * c1;
    if (P.d2 != 0) dd[d == 0 ? 0 : (d == 1 ? 3 : 5)] = hsum(fma2s(cc, 16.0f, neg2(b))) * c2;
  }
  if (P.d2 != 0) {
    // nested D_a (D_b f) from pair differences, (a, b) = (x, y), (x, z), (y, z)
    constexpr int PA[3] = {0, 0, 1}, PB[3] = {1, 2, 2}, PS[3] = {1, 2, 4};
    int m0 = 0;
    if (SHF) {
      // (x, y) and (x, z): the inner differences at the x neighbours are the
      // lanes' own g1 (a warp is 32 consecutive x); the four outside the warp
      // (x0 - 2, x0 - 1, x0 + 32, x0 + 33) come from lanes 0..3.  A warp that
      // does not fill its 32 x loads them all, in the same arithmetic.
      const int lane = threadIdx.x & 31;
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int B = PB[m];
        float gp1, gm1, gp2, gm2;
        if (full) {
          float hg = 0.0f;
          if (lane < 4) hg = inner_d1(at, 0, B, lane < 2 ? -2 : 30);
          auto nb = [&](int k) {
            const int src = lane + k;
            const float v = __shfl_sync(0xffffffffu, g1[B], src & 31);
            const float hv = __shfl_sync(0xffffffffu, hg, (src < 0 ? src + 2 : src - 30) & 3);
            return (src >= 0 && src < 32) ? v : hv;
          };
          gp1 = nb(1);
          gm1 = nb(-1);
          gp2 = nb(2);
          gm2 = nb(-2);
        } else {
          gp1 = inner_d1(at, 0, B, 1);
          gm1 = inner_d1(at, 0, B, -1);
          gp2 = inner_d1(at, 0, B, 2);
          gm2 = inner_d1(at, 0, B, -2);
        }
        dd[PS[m]] = outer_d1(gp1, gm1, gp2, gm2) * c11;
      }
      m0 = 2;
    }
#pragma unroll
    for (int m = m0; m < 3; ++m) {
      const int A = PA[m], B = PB[m];
      float2 inner[4];
      constexpr int KA[4] = {1, -1, 2, -2};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int ka = KA[u];
        auto pt = [&](int kb) {
          return at((A == 0 ? ka : 0) + (B == 0 ? kb : 0), (A == 1 ? ka : 0) + (B == 1 ? kb : 0),
                    (A == 2 ? ka : 0) + (B == 2 ? kb : 0));
        };
        inner[u] = fma2s(sub2(pt(1), pt(-1)), 8.0f, sub2(pt(-2), pt(2)));
      }
      dd[PS[m]] = hsum(fma2s(sub2(inner[0], inner[1]), 8.0f, sub2(inner[3], inner[2]))) * c11;
    }
    if (P.d2 == 1) {
#pragma unroll
      for (int q = 0; q < 6; ++q) SD(P.d2slot + q) = dd[q];
    } else {
      SD(P.d2slot) = symc(gtu, dd);
      if (P.d2 == 3) {
        const int I = F - F_BETX;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float v = dd[S2(j, I)];
          if (SPLIT)
            SD(S_DVB + 3 * I + j) = v;
          else if (I == 0)
            SD(S_DVB + j) = v;
          else
            SD(S_DVB + j) += v;
        }
      }
    }
  }
  SD((SPLIT ? S_AK_SPLIT : S_AK) + F) = hsum(acc);
#undef AT
  return c0.x + c0.y;
}


// ------------------------------------------------------------------ phase 2

// Curvature, gauge and Z4c sources from the slots and the centre values;
// r[f] = sources + advection + dissipation.
template <bool SPLIT, class Slots>
__device__ __forceinline__ void sources(const Slots& SD, const float cen[NF], const float gt[6],
                                        const float gtu[6], const DevParams& prm, float r[NF]) {
  const float W = cen[F_W], al = cen[F_ALP], Kh = cen[F_KH], Th = cen[F_TH];
  float At[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) At[a] = cen[F_AXX + a];
  float Gl[3][6], Gu[3][6], Gd[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = j; k < 3; ++k)
        Gl[i][S2(j, k)] = 0.5f * (SD(S_DGT + 6 * j + S2(i, k)) + SD(S_DGT + 6 * k + S2(i, j)) -
                                  SD(S_DGT + 6 * i + S2(j, k)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 6; ++a)
      Gu[i][a] = gtu[S2(i, 0)] * Gl[0][a] + gtu[S2(i, 1)] * Gl[1][a] + gtu[S2(i, 2)] * Gl[2][a];
#pragma unroll
  for (int i = 0; i < 3; ++i) Gd[i] = symc(gtu, Gu[i]);

  float Ric[6];
  {
    float X[3][3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
          X[j][k][l] = gtu[S2(l, 0)] * Gl[j][S2(k, 0)] + gtu[S2(l, 1)] * Gl[j][S2(k, 1)] +
                       gtu[S2(l, 2)] * Gl[j][S2(k, 2)];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int ij = S2(i, j);
        const float rr = -0.5f * SD(S_LGT + ij);
        float t2 = 0.0f, t3 = 0.0f, t4 = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          t2 += gt[S2(k, i)] * SD(S_DGAM + 3 * j + k) + gt[S2(k, j)] * SD(S_DGAM + 3 * i + k);
          t3 += Gd[k] * (Gl[i][S2(j, k)] + Gl[j][S2(i, k)]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l)
            t4 += Gu[k][S2(l, i)] * X[j][k][l] + Gu[k][S2(l, j)] * X[i][k][l] + Gu[k][S2(i, l)] * X[k][j][l];
        Ric[ij] = rr + 0.5f * t2 + 0.5f * t3 + t4;
      }
  }
  float dW[3], dal[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dW[d] = SD(S_DW + d);
    dal[d] = SD(S_DAL + d);
  }
  const float iW = 1.0f / W;
  float DDa[6], trDDa, dWda;
  {
    float DDW[6], DDal[6], dWW[6], dWa[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      DDW[a] = SD(S_DDW + a) - (Gu[0][a] * dW[0] + Gu[1][a] * dW[1] + Gu[2][a] * dW[2]);
      DDal[a] = SD(S_DDAL + a) - (Gu[0][a] * dal[0] + Gu[1][a] * dal[1] + Gu[2][a] * dal[2]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        dWW[S2(i, j)] = dW[i] * dW[j];
        dWa[S2(i, j)] = dW[i] * dal[j] + dW[j] * dal[i];
      }
    const float trDDW = symc(gtu, DDW);
    const float dWdW = symc(gtu, dWW);
    dWda = 0.5f * symc(gtu, dWa);
    trDDa = symc(gtu, DDal);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      Ric[a] += (DDW[a] + gt[a] * trDDW) * iW - 2.0f * gt[a] * dWdW * (iW * iW);
      DDa[a] = DDal[a] + (dWa[a] - gt[a] * dWda) * iW;
    }
  }
  const float Rsc = W * W * symc(gtu, Ric);
  const float Lapa = W * W * trDDa - W * dWda;

  const float K = Kh + 2.0f * Th;
  float dbe[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int i = 0; i < 3; ++i) dbe[d][i] = SD(S_DBE + 3 * d + i);
  const float divb = dbe[0][0] + dbe[1][1] + dbe[2][2];
  float Am[3][3], Atu[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Am[i][j] = gtu[S2(i, 0)] * At[S2(0, j)] + gtu[S2(i, 1)] * At[S2(1, j)] + gtu[S2(i, 2)] * At[S2(2, j)];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j)
      Atu[S2(i, j)] = Am[i][0] * gtu[S2(0, j)] + Am[i][1] * gtu[S2(1, j)] + Am[i][2] * gtu[S2(2, j)];
  const float AA = symc(At, Atu);

  r[F_W] = W * (1.0f / 3.0f) * (al * K - divb);
  {
    float X2[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) X2[a] = al * Ric[a] - DDa[a];
    const float trX3 = symc(gtu, X2) * (1.0f / 3.0f);
    const float W2 = W * W;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int ij = S2(i, j);
        float s = -2.0f * al * At[ij];
        float sA = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          s += gt[S2(i, k)] * dbe[j][k] + gt[S2(j, k)] * dbe[i][k];
          sA += At[S2(i, k)] * dbe[j][k] + At[S2(j, k)] * dbe[i][k];
        }
        r[F_GXX + ij] = s - (2.0f / 3.0f) * gt[ij] * divb;
        const float AikAkj = At[S2(i, 0)] * Am[0][j] + At[S2(i, 1)] * Am[1][j] + At[S2(i, 2)] * Am[2][j];
        r[F_AXX + ij] = sA - (2.0f / 3.0f) * At[ij] * divb + W2 * (X2[ij] - gt[ij] * trX3) +
                        al * (K * At[ij] - 2.0f * AikAkj);
      }
  }
  const float k1 = (float)prm.kappa1, k2 = (float)prm.kappa2;
  const float alk1 = al * k1;
  r[F_KH] = -Lapa + al * (AA + K * K * (1.0f / 3.0f)) + alk1 * (1.0f - k2) * Th;
  r[F_TH] = 0.5f * al * (Rsc - AA + (2.0f / 3.0f) * K * K) - alk1 * (2.0f + k2) * Th;
  {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float inner = symc(Gu[i], Atu);
      float s = 0.0f, tt = 0.0f, v = 0.0f;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        s += Atu[S2(i, j)] * dal[j];
        tt += Atu[S2(i, j)] * dW[j];
        v += gtu[S2(i, j)] * (2.0f * SD(S_DKH + j) + SD(S_DTH + j));
      }
      inner -= 3.0f * tt * iW + v * (1.0f / 3.0f);
      float g = -2.0f * s + 2.0f * al * inner;
      g += SD(S_LBE + i);
      float dvb[3];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dvb[j] = SPLIT ? SD(S_DVB + j) + SD(S_DVB + 3 + j) + SD(S_DVB + 6 + j) : SD(S_DVB + j);
      g += (gtu[S2(i, 0)] * dvb[0] + gtu[S2(i, 1)] * dvb[1] + gtu[S2(i, 2)] * dvb[2]) * (1.0f / 3.0f);
      g += (2.0f / 3.0f) * Gd[i] * divb;
      g -= Gd[0] * dbe[0][i] + Gd[1] * dbe[1][i] + Gd[2] * dbe[2][i];
      g -= 2.0f * alk1 * (cen[F_GAMX + i] - Gd[i]);
      r[F_GAMX + i] = g;
    }
  }
  if (prm.lapse == 1)
    r[F_ALP] = -al * al * K;
  else
    r[F_ALP] = -2.0f * al * (prm.lapse_uses_khat ? Kh : K);
  const float eta = (float)prm.eta;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float Bv = cen[F_BX + i];
    r[F_BETX + i] = 0.75f * Bv;
    r[F_BX + i] = r[F_GAMX + i] - eta * Bv;
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) r[f] += SD((SPLIT ? S_AK_SPLIT : S_AK) + f);
  if (prm.shift == 1) {
#pragma unroll
    for (int f = F_BETX; f < NF; ++f) r[f] = 0.0f;
  }
}

// Centre values needed before phase 1 -- gt (for the contractions) and beta
// (for the advection weights) -- the inverse metric, the stencil scales and
// the per-direction weights of Delta^6 and of the antisymmetric upwind part.
__device__ __forceinline__ void point_setup(const float2* __restrict__ U, long long q, long long fs, bool valid,
                                            double dx, double sigma_ko, float gt[6], float be[3], float gtu[6],
                                            float wko[3], float wup[3], float& c1, float& c2, float& c11) {
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const float2 v = valid ? __ldg(U + (F_GXX + a) * fs + q) : make_float2((a == 0 || a == 3 || a == 5), 0.f);
    gt[a] = v.x + v.y;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float2 v = valid ? __ldg(U + (F_BETX + d) * fs + q) : make_float2(0.f, 0.f);
    be[d] = v.x + v.y;
  }
  sym_inv_f(gt, gtu);
  const float h = (float)dx;
  c1 = 1.0f / (12.0f * h);
  c2 = c1 / h;
  c11 = c1 * c1;
  const float cko = (float)(sigma_ko / (64.0 * dx));
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    wko[d] = 0.5f * fabsf(be[d]) * c1 + cko;
    wup[d] = 0.5f * be[d] * c1;
  }
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ------------------------------------------------------------------ kernel

struct Pipe {
  uint64_t* bar;   // bar[0], bar[1]
  float2* buf[2];
  int* abort;      // shared flag: a wait ran out
};

template <int TY, int TZ>
__device__ __forceinline__ void issue_load(const TmaStageArgs& A, const Pipe& p, unsigned g, int tile, int f,
                                           int which) {
  const TileLoc L = locate<TY, TZ>(A, tile);
  uint64_t* bar = p.bar + (g & 1);
  mbar_expect_tx(bar, Cfg<TY, TZ>::BYTES);
  tma_load_3d(p.buf[g & 1], &A.map[L.slot][which], bar, 2 * L.x0, L.y0, f * A.nz[L.slot] + L.z0);
}

// wait for copy g; on time-out flag the CTA (the caller stops after the next barrier)
__device__ __forceinline__ void wait_copy(const Pipe& p, unsigned g, unsigned* err) {
  if (!mbar_wait_bounded(p.bar + (g & 1), (g >> 1) & 1)) {
    *p.abort = 1;
    atomicOr(err, (unsigned)ERR_TIMEOUT);
  }
}

template <int TY, int TZ, int MODE>
__global__ void __launch_bounds__(32 * TY * TZ, (TY * TZ <= 4) ? 2 : 1)
    z4c_stage_tma_kernel(const __grid_constant__ TmaStageArgs A) {
  using C = Cfg<TY, TZ>;
  extern __shared__ __align__(1024) unsigned char smem[];
  Pipe p;
  p.bar = reinterpret_cast<uint64_t*>(smem);
  p.abort = reinterpret_cast<int*>(smem + 64);
  p.buf[0] = reinterpret_cast<float2*>(smem + 1024);
  p.buf[1] = reinterpret_cast<float2*>(smem + 1024 + C::BUFB);
  float* sd = reinterpret_cast<float*>(smem + 1024 + 2 * C::BUFB);
  const int t = threadIdx.x;
  if ((int)blockIdx.x >= A.ntiles) return;
  if (t == 0) {
    mbar_init(p.bar, 1);
    mbar_init(p.bar + 1, 1);
    *p.abort = 0;
    mbar_fence_init();
  }
  __syncthreads();

  const StageArgs& S = A.st;
  const int ring = S.lev->ring;
  const int s = S.stage;
  // tensor map of the stage input: hl[0..2] (time levels), sa (3), sb (4)
  const int which = (MODE == 1 || s == 1) ? ring : (s == 3 ? 4 : 3);
  const int lx = t & 31, ly = (t >> 5) % TY, lz = (t >> 5) / TY;
  const int c = ((lz + 3) * C::BY + (ly + 3)) * C::BX + (lx + 3);

  unsigned g = 0;
  bool stop = false;
  if (t == 0) issue_load<TY, TZ>(A, p, 0, blockIdx.x, 0, which);

  for (int tile = blockIdx.x; tile < A.ntiles && !stop; tile += gridDim.x) {
    const TileLoc L = locate<TY, TZ>(A, tile);
    const DevPatch* P = S.patches + A.pid[L.slot];
    const int i = L.x0 + lx, j = L.y0 + ly, k = L.z0 + lz;
    const bool valid = i < P->n[0] && j < P->n[1] && k < P->n[2];
    const long long sy = P->px, sz = P->plane, fs = P->fstride;
    const long long q = (i + GH) + (long long)(j + GH) * sy + (long long)(k + GH) * sz;
    const float2* __restrict__ U = (MODE == 1) ? P->hl[ring] : mixed_in(P, s, ring);
    float gt[6], be[3], gtu[6], wko[3], wup[3], c1, c2, c11;
    point_setup(U, q, fs, valid, P->dx, S.prm.sigma_ko, gt, be, gtu, wko, wup, c1, c2, c11);
    if (valid && MODE == 0) {
      // the epilogue's streaming reads start their way from HBM into L2
      const double* ya = (s == 1) ? P->buf[ring] : P->buf[B_Y];
#pragma unroll 5
      for (int f = 0; f < NF; ++f) {
        prefetch_l2(ya + f * fs + q);
        if (s < 4) prefetch_l2(P->hl[ring] + f * fs + q);
      }
    }
    // the fields one after another (a loop: unrolled, the 25 passes overflow
    // the instruction cache)
#pragma unroll 1
    for (int f = 0; f < NF; ++f) {
      // the copy after this one: next field of this tile, or the first field
      // of the CTA's next tile; its buffer was released by the barrier that
      // ended copy g - 1
      if (t == 0) {
        if (f + 1 < NF)
          issue_load<TY, TZ>(A, p, g + 1, tile, f + 1, which);
        else if (tile + (int)gridDim.x < A.ntiles)
          issue_load<TY, TZ>(A, p, g + 1, tile + gridDim.x, 0, which);
      }
      wait_copy(p, g, S.err);
      const SmemAcc<C::SY, C::SZ> at{p.buf[g & 1], c};
      field_pass_p<false>(at, plan(f), f, SmemSlots<C::NT>{sd, t}, wko, wup, c1, c2, c11, gtu);
      __syncthreads();
      ++g;
      if (*p.abort) {
        stop = true;
        break;
      }
    }
    if (stop) break;
    if (!valid) continue;
    float cen[NF], r[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float2 v = __ldg(U + (long long)f * fs + q);
      cen[f] = v.x + v.y;
    }
    sources<false>(SmemSlots<C::NT>{sd, t}, cen, gt, gtu, S.prm, r);
    if (MODE == 1) {
      double* out = P->buf[B_S1];
#pragma unroll
      for (int f = 0; f < NF; ++f) out[f * fs + q] = (double)r[f];
    } else {
      rk_update_mixed(P, s, ring, S.dt, q, r, S.prm.w_floor, S.err);
    }
  }
  if (stop && t == 0) {
    // a wait ran out: let the copy still in flight (if any) land before the
    // shared memory is released, within the same bound
    mbar_wait_bounded(p.bar + (g & 1), (g >> 1) & 1);
  }
}

template <int TY, int TZ>
void launch_variant(const TmaStageArgs& a, int grid, cudaStream_t st) {
  const int smem = Cfg<TY, TZ>::SMEM;
  if (a.st.stage == 0)
    z4c_stage_tma_kernel<TY, TZ, 1><<<grid, Cfg<TY, TZ>::NT, smem, st>>>(a);
  else
    z4c_stage_tma_kernel<TY, TZ, 0><<<grid, Cfg<TY, TZ>::NT, smem, st>>>(a);
}

template <int TY, int TZ>
int setup_variant() {
  const int smem = Cfg<TY, TZ>::SMEM;
  if (cudaFuncSetAttribute(z4c_stage_tma_kernel<TY, TZ, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(z4c_stage_tma_kernel<TY, TZ, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, z4c_stage_tma_kernel<TY, TZ, 0>, Cfg<TY, TZ>::NT, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

// ------------------------------------------------------------------ L1 path

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
// PF: 0 no prefetching, 1 the next field's star and mixed-derivative rows,
// 2 its star rows only, 3 its z-arm rows only, 4 none of its rows (only the
// epilogue's streaming reads into L2)
template <int MINB, int MODE, int PF, bool SHF = false>
__global__ void __launch_bounds__(128, MINB) z4c_stage_ldg_kernel(StageArgs S) {
  extern __shared__ float sd[];
  const Tile tl = S.tiles[blockIdx.x];
  const DevPatch* P = S.patches + tl.patch;
  const int t = threadIdx.x;
  const int i = tl.x0 + (t & 31), j = tl.y0 + (t >> 5), k = tl.z0;
  if (i >= P->n[0] || j >= P->n[1] || k >= P->n[2]) return;
  // every lane of the warp is alive (its row is inside the patch, and so are
  // all 32 x of the tile): the x-neighbour exchange by shuffles is allowed
  const bool full = tl.x0 + 32 <= P->n[0];
  const int ring = S.lev->ring, s = S.stage;
  const long long sy = P->px, sz = P->plane, fs = P->fstride;
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
    const GlobalAcc at{U + (long long)f * fs + q, sy, sz};
    field_pass_p<false, GlobalAcc, SmemSlots<128>, SHF>(at, plan(f), f, SmemSlots<128>{sd, t}, wko, wup, c1, c2,
                                                         c11, gtu, full);
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

template <int MINB, int PF, bool SHF = false>
bool setup_ldg() {
  const int smem = NSLOT * 128 * 4;
  return cudaFuncSetAttribute(z4c_stage_ldg_kernel<MINB, 0, PF, SHF>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
         cudaFuncSetAttribute(z4c_stage_ldg_kernel<MINB, 1, PF, SHF>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
}

template <int MINB, int PF, bool SHF = false>
void launch_ldg(const StageArgs& a, cudaStream_t st) {
  const int smem = NSLOT * 128 * 4;
  if (a.stage == 0)
    z4c_stage_ldg_kernel<MINB, 1, PF, SHF><<<a.ntiles, 128, smem, st>>>(a);
  else
    z4c_stage_ldg_kernel<MINB, 0, PF, SHF><<<a.ntiles, 128, smem, st>>>(a);
}

// ------------------------------------------------------------------ split path

// The stage in two launches.  The derivative kernel forms, for FG fields per
// thread and one point, the same slot values as phase 1 and stores them as
// planes of FP32 in global memory; with no curvature algebra it needs few
// registers and no shared memory, so many warps hide the stencil latency.
// The algebra kernel then reads a point's slots (coalesced, one plane per
// slot), forms the sources and applies the RK4 update.  Point p of a launch
// is thread t of tile b: p = 128 b + t.
constexpr int FG = 5;  // fields per derivative thread

template <int MODE>
__global__ void __launch_bounds__(128) z4c_deriv_kernel(StageArgs S, float* __restrict__ dslot, long long npts) {
  const Tile tl = S.tiles[blockIdx.x];
  const DevPatch* P = S.patches + tl.patch;
  const int t = threadIdx.x;
  const int i = tl.x0 + (t & 31), j = tl.y0 + (t >> 5), k = tl.z0;
  if (i >= P->n[0] || j >= P->n[1] || k >= P->n[2]) return;
  const int ring = S.lev->ring, s = S.stage;
  const long long sy = P->px, sz = P->plane, fs = P->fstride;
  const long long q = (i + GH) + (long long)(j + GH) * sy + (long long)(k + GH) * sz;
  const float2* __restrict__ U = (MODE == 1) ? P->hl[ring] : mixed_in(P, s, ring);
  float gt[6], be[3], gtu[6], wko[3], wup[3], c1, c2, c11;
  point_setup(U, q, fs, true, P->dx, S.prm.sigma_ko, gt, be, gtu, wko, wup, c1, c2, c11);
  const GlobalSlots slots{dslot, npts, (long long)blockIdx.x * 128 + t};
  const int f0 = blockIdx.y * FG;
#pragma unroll 1
  for (int f = f0; f < f0 + FG; ++f) {
    if (f + 1 < f0 + FG) prefetch_field(U + (long long)(f + 1) * fs + q, sy, sz, plan(f + 1).d2 != 0);
    field_pass_p<true>(GlobalAcc{U + (long long)f * fs + q, sy, sz}, plan(f), f, slots, wko, wup, c1, c2, c11,
                       gtu);
  }
}

template <int MODE>
__global__ void __launch_bounds__(128, 3) z4c_algebra_kernel(StageArgs S, const float* __restrict__ dslot,
                                                             long long npts) {
  const Tile tl = S.tiles[blockIdx.x];
  const DevPatch* P = S.patches + tl.patch;
  const int t = threadIdx.x;
  const int i = tl.x0 + (t & 31), j = tl.y0 + (t >> 5), k = tl.z0;
  if (i >= P->n[0] || j >= P->n[1] || k >= P->n[2]) return;
  const int ring = S.lev->ring, s = S.stage;
  const long long sy = P->px, sz = P->plane, fs = P->fstride;
  const long long q = (i + GH) + (long long)(j + GH) * sy + (long long)(k + GH) * sz;
  const float2* __restrict__ U = (MODE == 1) ? P->hl[ring] : mixed_in(P, s, ring);
  if (MODE == 0) {
    const double* ya = (s == 1) ? P->buf[ring] : P->buf[B_Y];
#pragma unroll 5
    for (int f = 0; f < NF; ++f) {
      prefetch_l2(ya + f * fs + q);
      if (s < 4) prefetch_l2(P->hl[ring] + f * fs + q);
    }
  }
  float cen[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const float2 v = __ldg(U + (long long)f * fs + q);
    cen[f] = v.x + v.y;
  }
  float gt[6], gtu[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) gt[a] = cen[F_GXX + a];
  sym_inv_f(gt, gtu);
  float r[NF];
  sources<true>(GlobalSlotsIn{dslot, npts, (long long)blockIdx.x * 128 + t}, cen, gt, gtu, S.prm, r);
  if (MODE == 1) {
    double* out = P->buf[B_S1];
#pragma unroll
    for (int f = 0; f < NF; ++f) out[f * fs + q] = (double)r[f];
  } else {
    rk_update_mixed(P, s, ring, S.dt, q, r, S.prm.w_floor, S.err);
  }
}

}  // namespace

// tile shape (TY, TZ) of each TMA variant
static const int kShape[TMA_NVARIANTS][2] = {{4, 1}, {2, 2}, {4, 2}, {8, 1}};

void tma_variant_shape(int v, int* ty, int* tz) {
  const bool ok = v >= 0 && v < TMA_NVARIANTS;
  *ty = ok ? kShape[v][0] : 0;
  *tz = ok ? kShape[v][1] : 0;
}

int tma_box_bytes(int v) {
  return (v >= 0 && v < TMA_NVARIANTS) ? 38 * (kShape[v][0] + 6) * (kShape[v][1] + 6) * 8 : 0;
}

int tma_setup_variant(int v) {
  switch (v) {
    case 0: return setup_variant<4, 1>();
    case 1: return setup_variant<2, 2>();
    case 2: return setup_variant<4, 2>();
    case 3: return setup_variant<8, 1>();
  }
  return 0;
}

void launch_stage_tma(int v, const TmaStageArgs& a, int grid, cudaStream_t st) {
  switch (v) {
    case 0: launch_variant<4, 1>(a, grid, st); break;
    case 1: launch_variant<2, 2>(a, grid, st); break;
    case 2: launch_variant<4, 2>(a, grid, st); break;
    case 3: launch_variant<8, 1>(a, grid, st); break;
  }
}

// variant v: 0 (3 CTAs/SM, no prefetch), 1 (3, prefetch), 2 (4, prefetch),
// 3 (3, prefetch of the star rows only), 4 (3, z-arm rows only), 5 (3, the
// epilogue's reads only), 6 (as 4, the x-neighbour inner differences of the
// mixed derivatives exchanged by warp shuffles), 7 (as 6 with 4 CTAs/SM),
// 8 (as 4 with 4 CTAs/SM, 128 registers)
int ldg_setup(int v) {
  switch (v) {
    case 0: return setup_ldg<3, 0>();
    case 1: return setup_ldg<3, 1>();
    case 2: return setup_ldg<4, 1>();
    case 3: return setup_ldg<3, 2>();
    case 4: return setup_ldg<3, 3>();
    case 5: return setup_ldg<3, 4>();
    case 6: return setup_ldg<3, 3, true>();
    case 7: return setup_ldg<4, 3, true>();
    case 8: return setup_ldg<4, 3>();
  }
  return 0;
}

void launch_stage_ldg(int v, const StageArgs& a, cudaStream_t st) {
  if (a.ntiles == 0) return;
  switch (v) {
    case 0: launch_ldg<3, 0>(a, st); break;
    case 1: launch_ldg<3, 1>(a, st); break;
    case 2: launch_ldg<4, 1>(a, st); break;
    case 3: launch_ldg<3, 2>(a, st); break;
    case 4: launch_ldg<3, 3>(a, st); break;
    case 5: launch_ldg<3, 4>(a, st); break;
    case 6: launch_ldg<3, 3, true>(a, st); break;
    case 7: launch_ldg<4, 3, true>(a, st); break;
    case 8: launch_ldg<4, 3>(a, st); break;
  }
}

long long split_slot_floats(long long ntiles) { return (long long)NSLOT_SPLIT * ntiles * 128; }

void launch_stage_split(const StageArgs& a, float* dslot, cudaStream_t st) {
  if (a.ntiles == 0) return;
  const long long npts = (long long)a.ntiles * 128;
  const dim3 gd(a.ntiles, NF / FG);
  if (a.stage == 0) {
    z4c_deriv_kernel<1><<<gd, 128, 0, st>>>(a, dslot, npts);
    z4c_algebra_kernel<1><<<a.ntiles, 128, 0, st>>>(a, dslot, npts);
  } else {
    z4c_deriv_kernel<0><<<gd, 128, 0, st>>>(a, dslot, npts);
    z4c_algebra_kernel<0><<<a.ntiles, 128, 0, st>>>(a, dslot, npts);
  }
}

}  // namespace sacrak
