// Mixed-precision Z4c RHS fused with the RK4 stage update.
//
// Every time level is kept in FP64 and, beside it, split into two FP32 arrays
// hi + lo (hi = the FP32 rounding of the value, lo = the FP32 rounding of the
// rest): hi + lo carries ~48 bits.  A stage state is represented as
// u_s = hi_n + lo_s with lo_s = lo_n + c_s dt k (FP32), so no stage ever
// converts from FP64.  Derivatives, advection, dissipation and the Z4c
// sources run in FP32 on differences against the centre value,
// (hi_k - hi_0) + (lo_k - lo_0): exact in hi for nearby values and accurate to
// FP32 relative to the difference itself, so 1e-10 perturbations of O(1)
// fields survive.  FP64 is kept for the RK4 accumulator y, the new time level
// u_{n+1} = y + dt/6 k4 and its algebraic constraints (det gt = 1, trace-free
// At, W floor); the intermediate stage states are enforced in FP32 on the
// deviations from the flat metric.
//
// The same equations as z4c_fp64.cu (Sec. 2.1.1, 2.2 of the SACRA-K paper).
#include <math.h>

#include "mixed_common.cuh"
#include "sacrak_dev.cuh"

namespace sacrak {
namespace {

using namespace mixed;

// ------------------------------------------------------------------ stencils

__device__ __forceinline__ float pdiff(const float2* __restrict__ F, long long a, long long b) {
  const float2 x = __ldg(F + a), y = __ldg(F + b);
  return (x.x - y.x) + (x.y - y.y);
}
__device__ __forceinline__ float cdiff(const float2* __restrict__ F, long long a, float h0, float l0) {
  const float2 x = __ldg(F + a);
  return (x.x - h0) + (x.y - l0);
}
// 8 (f1 - f-1) - (f2 - f-2); times 1/(12 h)
__device__ __forceinline__ float d1f(const float2* F, long long q, long long s) {
  return 8.0f * pdiff(F, q + s, q - s) - pdiff(F, q + 2 * s, q - 2 * s);
}
// 16 (f1 + f-1) - (f2 + f-2) - 30 f0 on centre differences; times 1/(12 h^2)
__device__ __forceinline__ float d2f(const float2* F, long long q, long long s, float h0, float l0) {
  float a = cdiff(F, q + s, h0, l0) + cdiff(F, q - s, h0, l0);
  float b = cdiff(F, q + 2 * s, h0, l0) + cdiff(F, q - 2 * s, h0, l0);
  return 16.0f * a - b;
}
// nested D_a(D_b f); times 1/(144 h^2)
__device__ __forceinline__ float d11f(const float2* F, long long q, long long sa, long long sb) {
  float p1 = d1f(F, q + sa, sb), m1 = d1f(F, q - sa, sb);
  float p2 = d1f(F, q + 2 * sa, sb), m2 = d1f(F, q - 2 * sa, sb);
  return 8.0f * (p1 - m1) - (p2 - m2);
}
// lopsided upwind on centre differences; times 1/(12 h)
__device__ __forceinline__ float dupf(const float2* F, long long q, long long st, float b, float h0,
                                      float l0) {
  long long s = b > 0.0f ? st : -st;
  float v = -3.0f * cdiff(F, q - s, h0, l0) + 18.0f * cdiff(F, q + s, h0, l0) -
            6.0f * cdiff(F, q + 2 * s, h0, l0) + cdiff(F, q + 3 * s, h0, l0);
  return b > 0.0f ? v : -v;
}
__device__ __forceinline__ float delta6f(const float2* F, long long q, long long st, float h0, float l0) {
  float a = cdiff(F, q + 3 * st, h0, l0) + cdiff(F, q - 3 * st, h0, l0);
  float b = cdiff(F, q + 2 * st, h0, l0) + cdiff(F, q - 2 * st, h0, l0);
  float c = cdiff(F, q + st, h0, l0) + cdiff(F, q - st, h0, l0);
  return (a - 6.0f * b) + 15.0f * c;
}

// ------------------------------------------------------------------ the RHS

// The 114 first and second derivatives a point needs are formed first and
// parked in shared memory (one column per thread, no sharing, so no barrier);
// the curvature algebra then reads them back as it goes.  Splitting the two
// phases this way keeps the algebra's register demand well below what holding
// every derivative in registers needed (255 registers with spills, 8 warps per
// SM), so more warps hide the latency of the stencil loads.
constexpr int MIX_THREADS = 128;
constexpr int ND = 139;  // values kept per point
// slots: dgt[d][a] 0..17, dW 18..20, dal 21..23, dGam[d][i] 24..32,
// dbe[d][i] 33..41, dKh 42..44, dTh 45..47, ddgt[a][lm] 48..83, ddW 84..89,
// ddal 90..95, ddbe[i][lm] 96..113, advection + dissipation of field f 114 + f
enum {
  K_DGT = 0, K_DW = 18, K_DAL = 21, K_DGAM = 24, K_DBE = 33, K_DKH = 42, K_DTH = 45,
  K_DDGT = 48, K_DDW = 84, K_DDAL = 90, K_DDBE = 96, K_AK = 114
};
// per field: slot of its x first derivative and the stride to y, z (-1: not
// needed), and the first of its six second-derivative slots (-1: not needed)
__constant__ int c_d1base[NF] = {K_DW, K_DGT + 0, K_DGT + 1, K_DGT + 2, K_DGT + 3, K_DGT + 4, K_DGT + 5,
                                 K_DKH, K_DTH, -1, -1, -1, -1, -1, -1, K_DGAM + 0, K_DGAM + 1, K_DGAM + 2,
                                 K_DAL, K_DBE + 0, K_DBE + 1, K_DBE + 2, -1, -1, -1};
__constant__ int c_d1stride[NF] = {1, 6, 6, 6, 6, 6, 6, 1, 1, 0, 0, 0, 0, 0, 0, 3, 3, 3, 1, 3, 3, 3, 0, 0, 0};
__constant__ int c_d2base[NF] = {K_DDW, K_DDGT + 0, K_DDGT + 6, K_DDGT + 12, K_DDGT + 18, K_DDGT + 24,
                                 K_DDGT + 30, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                                 K_DDAL, K_DDBE + 0, K_DDBE + 6, K_DDBE + 12, -1, -1, -1};

// Z4c RHS of one point in FP32 from the split state U (hi, lo interleaved);
// r[f] gets the full RHS (sources + advection + dissipation).  sd: this CTA's
// ND x MIX_THREADS shared-memory derivative slots.
__device__ __forceinline__ void z4c_rhs_point_mixed(const float2* __restrict__ U, long long q,
                                                    long long sy, long long sz, long long fs,
                                                    float h, const DevParams& prm, float* sd,
                                                    float r[NF]) {
  const long long st[3] = {1, sy, sz};
  const float c1 = 1.0f / (12.0f * h);
  const float c2 = c1 / h;
  const float c11 = c1 * c1;
  const int t = threadIdx.x;
#define HF(f) (U + (long long)(f) * fs)
#define SD(k) sd[(k) * MIX_THREADS + t]
  auto CV = [&](int f) {
    const float2 v = __ldg(HF(f) + q);
    return v.x + v.y;
  };

  // ---- phase 1: one pass over the fields: the 7-point star along each axis
  // gives the first and second derivatives, the lopsided advection and the
  // Kreiss-Oliger term from the same six differences; the mixed second
  // derivatives add the off-axis points.  Everything goes to shared memory.
  float be[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) be[i] = CV(F_BETX + i);
  const float cko = (float)(prm.sigma_ko / (64.0 * (double)h));
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    const float2* F = HF(f);
    const float2 c0 = __ldg(F + q);
    const float h0 = c0.x, l0 = c0.y;
    const int s1 = c_d1base[f], s1d = c_d1stride[f], s2 = c_d2base[f];
    float ko = 0.0f, adv = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long o = st[d];
      const float cm3 = cdiff(F, q - 3 * o, h0, l0), cm2 = cdiff(F, q - 2 * o, h0, l0);
      const float cm1 = cdiff(F, q - o, h0, l0), cp1 = cdiff(F, q + o, h0, l0);
      const float cp2 = cdiff(F, q + 2 * o, h0, l0), cp3 = cdiff(F, q + 3 * o, h0, l0);
      ko += (cm3 + cp3) - 6.0f * (cm2 + cp2) + 15.0f * (cm1 + cp1);
      // lopsided: one point behind and three ahead along the shift; the
      // mirrored branch is the same expression on mirrored points, negated
      const bool pos = be[d] > 0.0f;
      const float ua = pos ? cm1 : cp1, ub = pos ? cp1 : cm1, uc = pos ? cp2 : cm2, ud = pos ? cp3 : cm3;
      const float v = -3.0f * ua + 18.0f * ub - 6.0f * uc + ud;
      adv += be[d] * (pos ? v : -v);
      if (s1 >= 0) SD(s1 + s1d * d) = (8.0f * (cp1 - cm1) - (cp2 - cm2)) * c1;
      if (s2 >= 0) SD(s2 + (d == 0 ? 0 : (d == 1 ? 3 : 5))) = (16.0f * (cp1 + cm1) - (cp2 + cm2)) * c2;
    }
    if (s2 >= 0) {
      SD(s2 + 1) = d11f(F, q, st[0], st[1]) * c11;
      SD(s2 + 2) = d11f(F, q, st[0], st[2]) * c11;
      SD(s2 + 4) = d11f(F, q, st[1], st[2]) * c11;
    }
    SD(K_AK + f) = adv * c1 + ko * cko;
  }

  // ---- phase 2: curvature and sources
  const float W = CV(F_W), al = CV(F_ALP);
  const float Kh = CV(F_KH), Th = CV(F_TH);
  float gt[6], At[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    gt[a] = CV(F_GXX + a);
    At[a] = CV(F_AXX + a);
  }
  float gtu[6];
  sym_inv_f(gt, gtu);
  float Gl[3][6], Gu[3][6], Gd[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = j; k < 3; ++k)
        Gl[i][S2(j, k)] = 0.5f * (SD(K_DGT + 6 * j + S2(i, k)) + SD(K_DGT + 6 * k + S2(i, j)) -
                                  SD(K_DGT + 6 * i + S2(j, k)));
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
        float dd[6];
#pragma unroll
        for (int b = 0; b < 6; ++b) dd[b] = SD(K_DDGT + 6 * ij + b);
        float rr = -0.5f * symc(gtu, dd);
        float t2 = 0.0f, t3 = 0.0f, t4 = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          t2 += gt[S2(k, i)] * SD(K_DGAM + 3 * j + k) + gt[S2(k, j)] * SD(K_DGAM + 3 * i + k);
          t3 += Gd[k] * (Gl[i][S2(j, k)] + Gl[j][S2(i, k)]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l)
            t4 += Gu[k][S2(l, i)] * X[j][k][l] + Gu[k][S2(l, j)] * X[i][k][l] +
                  Gu[k][S2(i, l)] * X[k][j][l];
        Ric[ij] = rr + 0.5f * t2 + 0.5f * t3 + t4;
      }
  }
  float dW[3], dal[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dW[d] = SD(K_DW + d);
    dal[d] = SD(K_DAL + d);
  }
  const float iW = 1.0f / W;
  float DDa[6], trDDa, dWda;
  {
    float DDW[6], DDal[6], dWW[6], dWa[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      DDW[a] = SD(K_DDW + a) - (Gu[0][a] * dW[0] + Gu[1][a] * dW[1] + Gu[2][a] * dW[2]);
      DDal[a] = SD(K_DDAL + a) - (Gu[0][a] * dal[0] + Gu[1][a] * dal[1] + Gu[2][a] * dal[2]);
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
    for (int i = 0; i < 3; ++i) dbe[d][i] = SD(K_DBE + 3 * d + i);
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
        float AikAkj = At[S2(i, 0)] * Am[0][j] + At[S2(i, 1)] * Am[1][j] + At[S2(i, 2)] * Am[2][j];
        r[F_AXX + ij] = sA - (2.0f / 3.0f) * At[ij] * divb + W2 * (X2[ij] - gt[ij] * trX3) +
                        al * (K * At[ij] - 2.0f * AikAkj);
      }
  }
  const float k1 = (float)prm.kappa1, k2 = (float)prm.kappa2;
  const float alk1 = al * k1;
  r[F_KH] = -Lapa + al * (AA + K * K * (1.0f / 3.0f)) + alk1 * (1.0f - k2) * Th;
  r[F_TH] = 0.5f * al * (Rsc - AA + (2.0f / 3.0f) * K * K) - alk1 * (2.0f + k2) * Th;
  {
    float ddivb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      ddivb[j] = SD(K_DDBE + 0 + S2(j, 0)) + SD(K_DDBE + 6 + S2(j, 1)) + SD(K_DDBE + 12 + S2(j, 2));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float inner = symc(Gu[i], Atu);
      float s = 0.0f, tt = 0.0f, v = 0.0f;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        s += Atu[S2(i, j)] * dal[j];
        tt += Atu[S2(i, j)] * dW[j];
        v += gtu[S2(i, j)] * (2.0f * SD(K_DKH + j) + SD(K_DTH + j));
      }
      inner -= 3.0f * tt * iW + v * (1.0f / 3.0f);
      float g = -2.0f * s + 2.0f * al * inner;
      float ddb[6];
#pragma unroll
      for (int b = 0; b < 6; ++b) ddb[b] = SD(K_DDBE + 6 * i + b);
      g += symc(gtu, ddb);
      g += (gtu[S2(i, 0)] * ddivb[0] + gtu[S2(i, 1)] * ddivb[1] + gtu[S2(i, 2)] * ddivb[2]) * (1.0f / 3.0f);
      g += (2.0f / 3.0f) * Gd[i] * divb;
      g -= Gd[0] * dbe[0][i] + Gd[1] * dbe[1][i] + Gd[2] * dbe[2][i];
      g -= 2.0f * alk1 * (CV(F_GAMX + i) - Gd[i]);
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
    const float Bv = CV(F_BX + i);
    r[F_BETX + i] = 0.75f * Bv;
    r[F_BX + i] = r[F_GAMX + i] - eta * Bv;
  }

  // advection and dissipation from phase 1
#pragma unroll
  for (int f = 0; f < NF; ++f) r[f] += SD(K_AK + f);
  if (prm.shift == 1) {
#pragma unroll
    for (int f = F_BETX; f < NF; ++f) r[f] = 0.0f;
  }
#undef HF
#undef SD
}

template <int MODE>  // 0: RK stage, 1: RHS only (FP64 output in S1)
__global__ void __launch_bounds__(MIX_THREADS, 3) z4c_stage_mixed_kernel(StageArgs A) {
  extern __shared__ float sd[];  // ND x MIX_THREADS derivative slots
  const Tile tl = A.tiles[blockIdx.x];
  const DevPatch* P = A.patches + tl.patch;
  const int i = tl.x0 + (threadIdx.x & 31);
  const int j = tl.y0 + (threadIdx.x >> 5);
  const int k = tl.z0;
  if (i >= P->n[0] || j >= P->n[1] || k >= P->n[2]) return;
  const int ring = A.lev->ring;
  const int s = A.stage;
  const long long sy = P->px, sz = P->plane, fs = P->fstride;
  const long long q = (i + GH) + (long long)(j + GH) * sy + (long long)(k + GH) * sz;
  const float2* __restrict__ U = MODE ? P->hl[ring] : mixed_in(P, s, ring);
  float r[NF];
  z4c_rhs_point_mixed(U, q, sy, sz, fs, (float)P->dx, A.prm, sd, r);
  if (MODE == 1) {
    double* out = P->buf[B_S1];
#pragma unroll
    for (int f = 0; f < NF; ++f) out[f * fs + q] = (double)r[f];
    return;
  }
  rk_update_mixed(P, s, ring, A.dt, q, r, A.prm.w_floor, A.err);
}

// Sommerfeld ghosts of level-0 patches in the split representation
__global__ void __launch_bounds__(128) sommerfeld_mixed_kernel(GhostArgs A) {
  const DevPatch* P = A.patches + A.patch_ids[blockIdx.y];
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= shell_count(P->NX, P->NY, P->NZ)) return;
  int i, j, k;
  shell_ijk(id, P->NX, P->NY, P->NZ, i, j, k);
  const int ring = A.lev->ring;
  const int s = A.stage;
  const long long sy = P->px, sz = P->plane, fs = P->fstride;
  const long long q = i + (long long)j * sy + (long long)k * sz;
  const float2* __restrict__ U = mixed_in(P, s, ring);
  const double h = P->dx;
  const int idx[3] = {i, j, k};
  const long long st[3] = {1, sy, sz};
  float x[3];
  double xd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    xd[d] = P->origin[d] + (idx[d] - GH + 0.5) * h;
    x[d] = (float)xd[d];
  }
  const float ir = (float)(1.0 / sqrt(xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]));
  const float c = (float)(1.0 / (2.0 * h));
  float kk[NF];
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    const float2* F = U + (long long)f * fs;
    const float2 c0 = F[q];
    const float h0 = c0.x, l0 = c0.y;
    float acc = ((h0 - (float)flat_value(f)) + l0) * ir;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long o = xd[d] > 0.0 ? -st[d] : st[d];
      // (3 f0 - 4 f1 + f2) on centre differences
      const float2 a1 = F[q + o], a2 = F[q + 2 * o];
      float v = (-4.0f * ((a1.x - h0) + (a1.y - l0)) + ((a2.x - h0) + (a2.y - l0))) * c;
      float dfd = xd[d] > 0.0 ? v : -v;
      acc += (x[d] * ir) * dfd;
    }
    kk[f] = -acc;
  }
  rk_update_mixed(P, s, ring, A.dt, q, kk, A.prm.w_floor, A.err);
}

// split the current time level of one patch (all points) into hi + lo
__global__ void split_kernel(const DevPatch* patches, const DevLevel* levels, int patch) {
  const DevPatch* P = patches + patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long pts = (long long)P->NX * P->NY * P->NZ;
  if (id >= pts) return;
  const int I = id % P->NX, J = (id / P->NX) % P->NY, K = id / ((long long)P->NX * P->NY);
  const long long q = I + (long long)J * P->px + (long long)K * P->plane;
  const int ring = levels[P->level].ring;
  for (int f = 0; f < NF; ++f) P->hl[ring][f * P->fstride + q] = split2(P->buf[ring][f * P->fstride + q]);
}

}  // namespace

void launch_stage_mixed(const StageArgs& a, cudaStream_t st) {
  if (a.ntiles == 0) return;
  const size_t smem = sizeof(float) * ND * MIX_THREADS;
  // opt in to more than 48 KB of dynamic shared memory, once per device
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaFuncSetAttribute(z4c_stage_mixed_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(z4c_stage_mixed_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set[dev] = true;
  }
  if (a.stage == 0)
    z4c_stage_mixed_kernel<1><<<a.ntiles, MIX_THREADS, smem, st>>>(a);
  else
    z4c_stage_mixed_kernel<0><<<a.ntiles, MIX_THREADS, smem, st>>>(a);
}

void launch_sommerfeld_mixed(const GhostArgs& a, int npatches, long long max_shell, cudaStream_t st) {
  if (npatches == 0 || max_shell == 0) return;
  dim3 grid((unsigned)((max_shell + 127) / 128), npatches);
  sommerfeld_mixed_kernel<<<grid, 128, 0, st>>>(a);
}

void launch_split(const DevPatch* patches, const DevLevel* levels, int patch, long long tot,
                  cudaStream_t st) {
  split_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(patches, levels, patch);
}

}  // namespace sacrak
