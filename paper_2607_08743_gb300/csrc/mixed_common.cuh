// Device helpers shared by the mixed-precision stage kernels (z4c_mixed.cu,
// z4c_mixed_tma.cu): FP32 symmetric-tensor algebra, the hi/lo split of an
// FP64 value, the algebraic constraints of a stage state (FP32, on the
// deviation from the flat metric) and of a new time level (FP64), and the
// RK4 stage update with its FP64 accumulator.
#pragma once
#include <math.h>

#include "sacrak_dev.cuh"

namespace sacrak {
namespace mixed {

__device__ __forceinline__ void sym_inv_f(const float g[6], float gu[6]) {
  float c0 = g[3] * g[5] - g[4] * g[4];
  float c1 = g[2] * g[4] - g[1] * g[5];
  float c2 = g[1] * g[4] - g[2] * g[3];
  float id = 1.0f / (g[0] * c0 + g[1] * c1 + g[2] * c2);
  gu[0] = c0 * id;
  gu[1] = c1 * id;
  gu[2] = c2 * id;
  gu[3] = (g[0] * g[5] - g[2] * g[2]) * id;
  gu[4] = (g[1] * g[2] - g[0] * g[4]) * id;
  gu[5] = (g[0] * g[3] - g[1] * g[1]) * id;
}
__device__ __forceinline__ float symc(const float S[6], const float T[6]) {
  return S[0] * T[0] + S[3] * T[3] + S[5] * T[5] + 2.0f * (S[1] * T[1] + S[2] * T[2] + S[4] * T[4]);
}


// ------------------------------------------------------------------ epilogue

__device__ __forceinline__ float2 split2(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

// FP64 algebraic constraints of the new time level (same as the FP64 path)
__device__ __forceinline__ void enforce_point_d(double v[NF], double w_floor) {
  double g[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) g[a] = v[F_GXX + a];
  double det = g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) +
               g[2] * (g[1] * g[4] - g[3] * g[2]);
  // fac = det^(-1/3): an FP32 seed refined by two Newton steps for
  // y^-3 = det, y <- y (4 - det y^3) / 3 (quadratic convergence: a 1e-7
  // seed reaches FP64 rounding), instead of an FP64 cube root and division
  double fac = (double)rcbrtf((float)det);
#pragma unroll
  for (int it = 0; it < 2; ++it) fac *= (4.0 - det * (fac * fac * fac)) * (1.0 / 3.0);
#pragma unroll
  for (int a = 0; a < 6; ++a) g[a] *= fac;
  double c0 = g[3] * g[5] - g[4] * g[4], c1 = g[2] * g[4] - g[1] * g[5], c2 = g[1] * g[4] - g[2] * g[3];
  // the rescaled metric has det = 1 up to rounding, so one Newton step for
  // 1/x from 1, 2 - x, gives its inverse determinant to FP64 rounding
  double id = 2.0 - (g[0] * c0 + g[1] * c1 + g[2] * c2);
  double gu[6] = {c0 * id, c1 * id, c2 * id, (g[0] * g[5] - g[2] * g[2]) * id,
                  (g[1] * g[2] - g[0] * g[4]) * id, (g[0] * g[3] - g[1] * g[1]) * id};
  const double* A = v + F_AXX;
  double tr3 = (gu[0] * A[0] + gu[3] * A[3] + gu[5] * A[5] + 2.0 * (gu[1] * A[1] + gu[2] * A[2] + gu[4] * A[4])) *
               (1.0 / 3.0);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    v[F_GXX + a] = g[a];
    v[F_AXX + a] -= g[a] * tr3;
  }
  if (v[F_W] < w_floor) v[F_W] = w_floor;
}

// FP32 algebraic constraints of a stage state u = hi + lo, applied to lo:
// det gt = 1 through the deviation h = gt - 1 (det - 1 = tr h + second and
// third invariants, so small deviations keep their precision), trace-free At,
// W floor.
__device__ __forceinline__ void enforce_stage_f(const float hi[NF], float lo[NF], float w_floor) {
  float hd[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const bool diag = (a == 0 || a == 3 || a == 5);
    hd[a] = (diag ? hi[F_GXX + a] - 1.0f : hi[F_GXX + a]) + lo[F_GXX + a];
  }
  const float tr = hd[0] + hd[3] + hd[5];
  const float q2 = hd[0] * hd[3] + hd[0] * hd[5] + hd[3] * hd[5] - hd[1] * hd[1] - hd[2] * hd[2] -
                   hd[4] * hd[4];
  const float q3 = hd[0] * (hd[3] * hd[5] - hd[4] * hd[4]) - hd[1] * (hd[1] * hd[5] - hd[4] * hd[2]) +
                   hd[2] * (hd[1] * hd[4] - hd[3] * hd[2]);
  const float fm1 = expm1f(-log1pf(tr + q2 + q3) * (1.0f / 3.0f));  // det^(-1/3) - 1
  float g[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const float gv = hi[F_GXX + a] + lo[F_GXX + a];
    lo[F_GXX + a] += gv * fm1;
    g[a] = gv * (1.0f + fm1);
  }
  float gu[6], A[6];
  sym_inv_f(g, gu);
#pragma unroll
  for (int a = 0; a < 6; ++a) A[a] = hi[F_AXX + a] + lo[F_AXX + a];
  const float tr3 = symc(gu, A) * (1.0f / 3.0f);
#pragma unroll
  for (int a = 0; a < 6; ++a) lo[F_AXX + a] -= g[a] * tr3;
  if (hi[F_W] + lo[F_W] < w_floor) lo[F_W] = w_floor - hi[F_W];
}

__device__ __forceinline__ void rk_update_mixed(const DevPatch* P, int s, int ring, double dt,
                                                long long q, const float k[NF], double w_floor,
                                                unsigned* err) {
  const long long fs = P->fstride;
  const float2* __restrict__ Hn = P->hl[ring];
  double* __restrict__ y = P->buf[B_Y];
  bool bad = false;
  if (s < 4) {
    const double bw = (s == 1) ? (1.0 / 6.0) : (1.0 / 3.0);
    const double bdt = bw * dt;
    const float cdt = (float)((s == 3 ? 1.0 : 0.5) * dt);
    const double* __restrict__ Un = P->buf[ring];
    float2* __restrict__ out = mixed_out(P, s);
    float hi[NF], lo[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const long long o = f * fs + q;
      const double yn = (s == 1 ? Un[o] : y[o]) + bdt * (double)k[f];
      y[o] = yn;
      const float2 n = Hn[o];
      hi[f] = n.x;
      lo[f] = n.y + cdt * k[f];
      bad |= !isfinite(k[f]);  // (FP32 test: a non-finite RHS is what can enter)
    }
    enforce_stage_f(hi, lo, (float)w_floor);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      out[f * fs + q] = make_float2(hi[f], lo[f]);
      bad |= !isfinite(lo[f]);
    }
  } else {
    const double bdt = dt / 6.0;
    const int nx = (ring + 1) % 3;
    double* __restrict__ Un1 = P->buf[nx];
    float2* __restrict__ Hx = P->hl[nx];
    double v[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) v[f] = y[f * fs + q] + bdt * (double)k[f];
    enforce_point_d(v, w_floor);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const long long o = f * fs + q;
      Un1[o] = v[f];
      const float2 h = split2(v[f]);
      Hx[o] = h;
      bad |= !isfinite(h.x);  // the FP32 rounding of a non-finite value is non-finite
    }
  }
  if (bad) atomicOr(err, (unsigned)ERR_NONFINITE);
}

}  // namespace mixed
}  // namespace sacrak
