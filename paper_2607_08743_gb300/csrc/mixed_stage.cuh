// Device code shared by the mixed-precision stage kernels that work on the
// hi/lo pair buffers (z4c_mixed_tma.cu: TMA-staged, L1 path and split
// kernels; z4c_mixed_pair.cu: two points per thread with 128-bit loads):
// packed FP32x2 arithmetic on (hi, lo) pairs, the per-point layout of the
// derivative slots between the stencil pass and the curvature algebra, the
// plan of what each field's pass forms, the per-field stencil pass
// (Sec. 2.2: 4th-order centred first and second derivatives, nested mixed
// derivatives, lopsided upwind advection as |beta|/2 Delta^6 plus the
// antisymmetric part, 6th-order Kreiss-Oliger) and the Z4c sources
// (Sec. 2.1.1) in FP32.
#pragma once
#include <math.h>

#include "mixed_common.cuh"
#include "sacrak_dev.cuh"

namespace sacrak {
namespace mixed {
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

// The same with the row and plane pitches (pairs) fixed at compile time: the
// offset of every stencil value is a constant folded into the load
template <int SY, int SZ>
struct FixedAcc {
  const float2* __restrict__ F;
  __device__ __forceinline__ float2 operator()(int dx, int dy, int dz) const {
    return __ldg(F + (dx + dy * SY + dz * SZ));
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
          // compile-time indices (a runtime index would put dd in local memory)
          const float v = I == 0 ? dd[S2(j, 0)] : (I == 1 ? dd[S2(j, 1)] : dd[S2(j, 2)]);
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

}  // namespace mixed
}  // namespace sacrak
