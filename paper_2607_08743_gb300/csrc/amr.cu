// Ghost zones and Berger-Oliger inter-level operators (Sec. 2.2.1, 2.2.2):
// periodic and frozen ghost fills, 6th-order Lagrange prolongation of child
// ghosts with quadratic (linear on the first step) time interpolation between
// parent time levels, 4th-order Lagrange restriction, same-level exchange.
#include "sacrak_dev.cuh"

namespace sacrak {

__device__ __forceinline__ long long nshell(const DevPatch* P) {
  return (long long)P->NX * P->NY * P->NZ -
         (long long)(P->NX - 2 * GH) * (P->NY - 2 * GH) * (P->NZ - 2 * GH);
}

// slot selector for ghost fills: which buffer of the patch receives ghosts
// mode: 0 = stage input of stage s, 1 = current time level, 2 = next time level
__device__ __forceinline__ int fill_slot(int mode, int s, int ring) {
  return mode == 0 ? stage_in_slot(s, ring) : (mode == 1 ? ring : (ring + 1) % 3);
}

__device__ __forceinline__ void split_to(double v, float2* hl, long long o) {
  const float hi = __double2float_rn(v);
  hl[o] = make_float2(hi, __double2float_rn(v - (double)hi));
}

// periodic: every ghost takes the value of the active point congruent modulo n
// (mixed precision: the split buffers the stage reads are copied as well)
__global__ void periodic_fill_kernel(FillArgs A) {
  const DevPatch* P = A.patches + A.patch_ids[blockIdx.y];
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nshell(P)) return;
  int i, j, k;
  shell_ijk(id, P->NX, P->NY, P->NZ, i, j, k);
  const int si = GH + ((i - GH) % P->n[0] + P->n[0]) % P->n[0];
  const int sj = GH + ((j - GH) % P->n[1] + P->n[1]) % P->n[1];
  const int sk = GH + ((k - GH) % P->n[2] + P->n[2]) % P->n[2];
  const int ring = A.lev->ring;
  const long long q = i + (long long)j * P->px + (long long)k * P->plane;
  const long long qs = si + (long long)sj * P->px + (long long)sk * P->plane;
  const long long fs = P->fstride;
  if (!A.mixed) {
    double* u = P->buf[fill_slot(A.mode, A.stage, ring)];
    for (int f = 0; f < NF; ++f) u[f * fs + q] = u[f * fs + qs];
    return;
  }
  if (A.mode == 0 && A.stage > 1) {
    float2* in = mixed_in(P, A.stage, ring);
    for (int f = 0; f < NF; ++f) in[f * fs + q] = in[f * fs + qs];
    return;
  }
  const int slot = A.mode == 2 ? (ring + 1) % 3 : ring;
  double* u = P->buf[slot];
  float2* hl = P->hl[slot];
  for (int f = 0; f < NF; ++f) {
    u[f * fs + q] = u[f * fs + qs];
    hl[f * fs + q] = hl[f * fs + qs];
  }
}

// frozen: ghosts of the target buffer take the ghosts of the current level
__global__ void frozen_fill_kernel(FillArgs A) {
  const DevPatch* P = A.patches + A.patch_ids[blockIdx.y];
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nshell(P)) return;
  int i, j, k;
  shell_ijk(id, P->NX, P->NY, P->NZ, i, j, k);
  const int ring = A.lev->ring;
  const long long q = i + (long long)j * P->px + (long long)k * P->plane;
  const long long fs = P->fstride;
  if (!A.mixed) {
    const int dst = fill_slot(A.mode, A.stage, ring);
    if (dst == ring) return;
    for (int f = 0; f < NF; ++f) P->buf[dst][f * fs + q] = P->buf[ring][f * fs + q];
    return;
  }
  if (A.mode == 0) {
    if (A.stage == 1) return;
    float2* in = mixed_in(P, A.stage, ring);
    for (int f = 0; f < NF; ++f) in[f * fs + q] = P->hl[ring][f * fs + q];
    return;
  }
  if (A.mode != 2) return;
  const int nx = (ring + 1) % 3;
  for (int f = 0; f < NF; ++f) {
    P->buf[nx][f * fs + q] = P->buf[ring][f * fs + q];
    P->hl[nx][f * fs + q] = P->hl[ring][f * fs + q];
  }
}

// 6-point Lagrange weights at +1/4 (nodes -2..3) and -1/4 (nodes -3..2), /8192
__constant__ double c_wp[6] = {77.0 / 8192, -693.0 / 8192, 6930.0 / 8192,
                               2310.0 / 8192, -495.0 / 8192, 63.0 / 8192};
__constant__ double c_wm[6] = {63.0 / 8192, -495.0 / 8192, 2310.0 / 8192,
                               6930.0 / 8192, -693.0 / 8192, 77.0 / 8192};

__device__ __forceinline__ int floor_half(int i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

// Spatial prolongation of one parent time level onto the ghost shell of each
// child (Sec. 2.2.1, 6th-order Lagrange, tensor product).  The result is
// cached per parent ring slot in the child's gsh[slot]; the per-stage ghost
// fill then only combines the cached slots in time (ghost_time_fill_kernel),
// so the 6^3 stencils run twice per parent step instead of at every child
// stage.  One thread computes one field of the 2x2x2 children of one parent
// cell from its 7^3 neighbourhood with separable x, y, z passes (the even
// child sits at -1/4 of the parent cell, nodes -3..2; the odd one at +1/4,
// nodes -2..3).
struct ProlongArgs {
  const DevPatch* patches;
  const int* patch_ids;   // children (one level)
  const DevLevel* plev;   // parent level: slot = its current ring slot
};

__device__ __forceinline__ void box_shell_ijk(long long id, int m0, int m1, int m2, int w, int& a,
                                              int& b, int& c) {
  // shell of width w of an m0 x m1 x m2 box: two z slabs, two y slabs, two x slabs
  const long long zs = (long long)w * m1 * m0;
  const int n2 = m2 - 2 * w, n1 = m1 - 2 * w;
  const long long ys = (long long)w * m0 * n2;
  if (id < 2 * zs) {
    int side = id >= zs;
    long long r = id - side * zs;
    a = (int)(r % m0);
    r /= m0;
    b = (int)(r % m1);
    c = (int)(r / m1) + (side ? m2 - w : 0);
    return;
  }
  id -= 2 * zs;
  if (id < 2 * ys) {
    int side = id >= ys;
    long long r = id - side * ys;
    a = (int)(r % m0);
    r /= m0;
    b = (int)(r % w) + (side ? m1 - w : 0);
    c = (int)(r / w) + w;
    return;
  }
  id -= 2 * ys;
  const long long xs = (long long)w * n1 * n2;
  int side = id >= xs;
  long long r = id - side * xs;
  a = (int)(r % w) + (side ? m0 - w : 0);
  r /= w;
  b = (int)(r % n1) + w;
  c = (int)(r / n1) + w;
}

__global__ void __launch_bounds__(128) prolong_space_kernel(ProlongArgs A, long long max_work) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= max_work) return;
  const DevPatch* C = A.patches + A.patch_ids[blockIdx.y];
  // parent cells whose children touch the ghost shell: the box
  // [off-2, off+n/2+1] minus its interior [off, off+n/2-1] (a shell of width 2)
  const int m0 = C->n[0] / 2 + 4, m1 = C->n[1] / 2 + 4, m2 = C->n[2] / 2 + 4;
  const long long ncl = (long long)m0 * m1 * m2 - (long long)(m0 - 4) * (m1 - 4) * (m2 - 4);
  const int f = (int)(tid % NF);
  const long long cl = tid / NF;
  if (cl >= ncl) return;
  int a, b, c;
  box_shell_ijk(cl, m0, m1, m2, 2, a, b, c);
  const DevPatch* P = A.patches + C->parent;
  const int slot = A.plev->ring;
  const double* __restrict__ up = P->buf[slot] + (long long)f * P->fstride;
  // parent array index of the cell and of its 7^3 neighbourhood origin
  const int pi = C->off[0] - 2 + a + GH, pj = C->off[1] - 2 + b + GH, pk = C->off[2] - 2 + c + GH;
  const long long q0 = (pi - 3) + (long long)(pj - 3) * P->px + (long long)(pk - 3) * P->plane;
  // weights over offsets -3..3 for the even (-1/4) and odd (+1/4) child
  double we[7], wo[7];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    we[t] = c_wm[t];
    wo[t + 1] = c_wp[t];
  }
  we[6] = 0.0;
  wo[0] = 0.0;
  // Only parent cells off-4 .. off+n/2+3 (parent active cells, by the nesting
  // margin) are read: the children that are kept need no others, and cells
  // outside that range (possibly never written) would turn a zero weight into
  // NaN.  Valid stencil offsets t along each axis: [t_lo, t_hi].
  const int xlo = max(0, 1 - a), xhi = min(6, C->n[0] / 2 + 8 - a);
  const int ylo = max(0, 1 - b), yhi = min(6, C->n[1] / 2 + 8 - b);
  const int zlo = max(0, 1 - c), zhi = min(6, C->n[2] / 2 + 8 - c);
  double acc[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};  // [z][y][x] parity
#pragma unroll 1
  for (int kz = zlo; kz <= zhi; ++kz) {
    double vy[2][2] = {{0, 0}, {0, 0}};
#pragma unroll
    for (int jy = 0; jy < 7; ++jy) {
      if (jy < ylo || jy > yhi) continue;
      const double* row = up + q0 + (long long)kz * P->plane + (long long)jy * P->px;
      double xe = 0.0, xo = 0.0;
#pragma unroll
      for (int ix = 0; ix < 7; ++ix) {
        const double v = (ix >= xlo && ix <= xhi) ? __ldg(row + ix) : 0.0;
        xe += we[ix] * v;
        xo += wo[ix] * v;
      }
      vy[0][0] += we[jy] * xe;
      vy[0][1] += we[jy] * xo;
      vy[1][0] += wo[jy] * xe;
      vy[1][1] += wo[jy] * xo;
    }
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        acc[0][y][x] += we[kz] * vy[y][x];
        acc[1][y][x] += wo[kz] * vy[y][x];
      }
  }
  // child indices of the even child along each axis
  const int c0 = 2 * (a - 2), c1 = 2 * (b - 2), c2 = 2 * (c - 2);
  double* __restrict__ g = C->gsh[slot] + (long long)f * C->fstride;
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const int i = c0 + x, j = c1 + y, k = c2 + z;
        if (i < -GH || j < -GH || k < -GH || i >= C->n[0] + GH || j >= C->n[1] + GH || k >= C->n[2] + GH)
          continue;
        const bool active = i >= 0 && j >= 0 && k >= 0 && i < C->n[0] && j < C->n[1] && k < C->n[2];
        if (active) continue;
        g[(i + GH) + (long long)(j + GH) * C->px + (long long)(k + GH) * C->plane] = acc[z][y][x];
      }
}

// Mixed precision: the same interpolant in FP32 on differences against the
// parent cell's value, from the parent's hi/lo split, added to that value in
// FP64 (the weights sum to one along every axis, so subtracting the reference
// changes nothing but the rounding).
__global__ void __launch_bounds__(128) prolong_space_mixed_kernel(ProlongArgs A, long long max_work) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= max_work) return;
  const DevPatch* C = A.patches + A.patch_ids[blockIdx.y];
  const int m0 = C->n[0] / 2 + 4, m1 = C->n[1] / 2 + 4, m2 = C->n[2] / 2 + 4;
  const long long ncl = (long long)m0 * m1 * m2 - (long long)(m0 - 4) * (m1 - 4) * (m2 - 4);
  const int f = (int)(tid % NF);
  const long long cl = tid / NF;
  if (cl >= ncl) return;
  int a, b, c;
  box_shell_ijk(cl, m0, m1, m2, 2, a, b, c);
  const DevPatch* P = A.patches + C->parent;
  const int slot = A.plev->ring;
  const long long fo = (long long)f * P->fstride;
  const float2* __restrict__ hp = P->hl[slot] + fo;
  const int pi = C->off[0] - 2 + a + GH, pj = C->off[1] - 2 + b + GH, pk = C->off[2] - 2 + c + GH;
  // reference: the parent cell itself when it is readable, else the nearest
  // readable cell along each axis
  const int xlo = max(0, 1 - a), xhi = min(6, C->n[0] / 2 + 8 - a);
  const int ylo = max(0, 1 - b), yhi = min(6, C->n[1] / 2 + 8 - b);
  const int zlo = max(0, 1 - c), zhi = min(6, C->n[2] / 2 + 8 - c);
  const int ri = pi - 3 + min(max(3, xlo), xhi), rj = pj - 3 + min(max(3, ylo), yhi),
            rk = pk - 3 + min(max(3, zlo), zhi);
  const long long qr = ri + (long long)rj * P->px + (long long)rk * P->plane;
  const float2 ref = hp[qr];
  const float h0 = ref.x, l0 = ref.y;
  const double u0 = P->buf[slot][fo + qr];
  const long long q0 = (pi - 3) + (long long)(pj - 3) * P->px + (long long)(pk - 3) * P->plane;
  float we[7], wo[7];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    we[t] = (float)c_wm[t];
    wo[t + 1] = (float)c_wp[t];
  }
  we[6] = 0.0f;
  wo[0] = 0.0f;
  float acc[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
#pragma unroll 1
  for (int kz = zlo; kz <= zhi; ++kz) {
    float vy[2][2] = {{0, 0}, {0, 0}};
#pragma unroll
    for (int jy = 0; jy < 7; ++jy) {
      if (jy < ylo || jy > yhi) continue;
      const long long row = q0 + (long long)kz * P->plane + (long long)jy * P->px;
      float xe = 0.0f, xo = 0.0f;
#pragma unroll
      for (int ix = 0; ix < 7; ++ix) {
        float v = 0.0f;
        if (ix >= xlo && ix <= xhi) {
          const float2 w = __ldg(hp + row + ix);
          v = (w.x - h0) + (w.y - l0);
        }
        xe += we[ix] * v;
        xo += wo[ix] * v;
      }
      vy[0][0] += we[jy] * xe;
      vy[0][1] += we[jy] * xo;
      vy[1][0] += wo[jy] * xe;
      vy[1][1] += wo[jy] * xo;
    }
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        acc[0][y][x] += we[kz] * vy[y][x];
        acc[1][y][x] += wo[kz] * vy[y][x];
      }
  }
  const int c0 = 2 * (a - 2), c1 = 2 * (b - 2), c2 = 2 * (c - 2);
  double* __restrict__ g = C->gsh[slot] + (long long)f * C->fstride;
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const int i = c0 + x, j = c1 + y, k = c2 + z;
        if (i < -GH || j < -GH || k < -GH || i >= C->n[0] + GH || j >= C->n[1] + GH || k >= C->n[2] + GH)
          continue;
        const bool active = i >= 0 && j >= 0 && k >= 0 && i < C->n[0] && j < C->n[1] && k < C->n[2];
        if (active) continue;
        g[(i + GH) + (long long)(j + GH) * C->px + (long long)(k + GH) * C->plane] = u0 + (double)acc[z][y][x];
      }
}

// Ghosts of the child's target buffer = time combination of the cached
// spatial prolongations of the parent's (oldest, middle, newest) slots.
__global__ void ghost_time_fill_kernel(FillArgs A) {
  const DevPatch* C = A.patches + A.patch_ids[blockIdx.y];
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nshell(C)) return;
  int i, j, k;
  shell_ijk(id, C->NX, C->NY, C->NZ, i, j, k);
  const int pr = A.plev->ring;
  const bool q3 = A.plev->nvalid >= 3;
  const double w0 = q3 ? A.wq[0] : 0.0, w1 = q3 ? A.wq[1] : A.wl[1], w2 = q3 ? A.wq[2] : A.wl[2];
  const double* __restrict__ g0 = C->gsh[(pr + 1) % 3];
  const double* __restrict__ g1 = C->gsh[(pr + 2) % 3];
  const double* __restrict__ g2 = C->gsh[pr];
  const int ring = A.lev->ring;
  const long long q = i + (long long)j * C->px + (long long)k * C->plane;
  if (!A.mixed) {
    double* __restrict__ dst = C->buf[fill_slot(A.mode, A.stage, ring)];
    for (int f = 0; f < NF; ++f) {
      const long long o = f * C->fstride + q;
      double v = w1 * g1[o] + w2 * g2[o];
      if (q3) v += w0 * g0[o];
      dst[o] = v;
    }
    return;
  }
  // mixed precision: stage 1 (and the fill of the current level) sets the
  // FP64 ghost and its hi/lo split; later stages set lo_s = v - hi_n
  const bool later = (A.mode == 0 && A.stage > 1);
  float2* __restrict__ in = later ? mixed_in(C, A.stage, ring) : nullptr;
  for (int f = 0; f < NF; ++f) {
    const long long o = f * C->fstride + q;
    double v = w1 * g1[o] + w2 * g2[o];
    if (q3) v += w0 * g0[o];
    if (later) {
      const float hi = C->hl[ring][o].x;
      in[o] = make_float2(hi, __double2float_rn(v - (double)hi));
    } else {
      C->buf[ring][o] = v;
      split_to(v, C->hl[ring], o);
    }
  }
}

// Restriction: every parent cell covered by the child's active region takes
// the tensor-product 4-point Lagrange interpolant of the child's current time
// level at the parent cell centre, weights (-1, 9, 9, -1)/16 on child cells
// 2m-1 .. 2m+2.
__global__ void __launch_bounds__(128) restrict_kernel(FillArgs A) {
  const DevPatch* C = A.patches + A.patch_ids[blockIdx.y];
  const DevPatch* P = A.patches + C->parent;
  const int mx = C->n[0] / 2, my = C->n[1] / 2, mz = C->n[2] / 2;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)mx * my * mz) return;
  const int I = id % mx;
  const int J = (id / mx) % my;
  const int K = id / ((long long)mx * my);
  const double* __restrict__ uc = C->buf[A.lev->ring];
  double* __restrict__ up = P->buf[A.plev->ring];
  const double w[4] = {-1.0 / 16, 9.0 / 16, 9.0 / 16, -1.0 / 16};
  const long long q0 = (2 * I - 1 + GH) + (long long)(2 * J - 1 + GH) * C->px +
                       (long long)(2 * K - 1 + GH) * C->plane;
  const long long qp = (I + C->off[0] + GH) + (long long)(J + C->off[1] + GH) * P->px +
                       (long long)(K + C->off[2] + GH) * P->plane;
  for (int f = 0; f < NF; ++f) {
    const double* src = uc + f * C->fstride + q0;
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double vy = 0.0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double* row = src + (long long)c * C->plane + (long long)b * C->px;
        double vx = w[0] * __ldg(row) + w[1] * __ldg(row + 1) + w[2] * __ldg(row + 2) +
                    w[3] * __ldg(row + 3);
        vy += w[b] * vx;
      }
      v += w[c] * vy;
    }
    up[f * P->fstride + qp] = v;
    if (A.mixed) split_to(v, P->hl[A.plev->ring], f * P->fstride + qp);
  }
}

// Same-level exchange between patch a and patch b (aligned, same spacing):
// a's ghosts over b's active region take b's values, b's ghosts over a's
// active region take a's values, points active in both take the average.
__global__ void exchange_kernel(ExchArgs E) {
  const DevPatch* Pa = E.patches + E.a;
  const DevPatch* Pb = E.patches + E.b;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)Pa->NX * Pa->NY * Pa->NZ;
  if (id >= tot) return;
  const int I = id % Pa->NX, J = (id / Pa->NX) % Pa->NY, K = id / ((long long)Pa->NX * Pa->NY);
  const int i = I - GH, j = J - GH, k = K - GH;
  const int ib = i + E.off[0], jb = j + E.off[1], kb = k + E.off[2];
  const bool b_in = ib >= -GH && ib < Pb->n[0] + GH && jb >= -GH && jb < Pb->n[1] + GH &&
                    kb >= -GH && kb < Pb->n[2] + GH;
  if (!b_in) return;
  const bool a_act = i >= 0 && i < Pa->n[0] && j >= 0 && j < Pa->n[1] && k >= 0 && k < Pa->n[2];
  const bool b_act = ib >= 0 && ib < Pb->n[0] && jb >= 0 && jb < Pb->n[1] && kb >= 0 && kb < Pb->n[2];
  if (!a_act && !b_act) return;
  const int ring = E.lev->ring;
  const long long qa = I + (long long)J * Pa->px + (long long)K * Pa->plane;
  const long long qb = (ib + GH) + (long long)(jb + GH) * Pb->px + (long long)(kb + GH) * Pb->plane;
  if (E.mixed && E.mode == 0 && E.stage > 1) {
    // stage state hi_n + lo_s: move lo_s (and average the stage values)
    float2* ia = mixed_in(Pa, E.stage, ring);
    float2* ib = mixed_in(Pb, E.stage, ring);
    for (int f = 0; f < NF; ++f) {
      const long long oa = f * Pa->fstride + qa, ob = f * Pb->fstride + qb;
      const float2 a = ia[oa], b = ib[ob];
      if (a_act && b_act) {
        const float m = 0.5f * ((a.x + a.y) + (b.x + b.y));
        ia[oa] = make_float2(a.x, m - a.x);
        ib[ob] = make_float2(b.x, m - b.x);
      } else if (b_act) {
        ia[oa] = make_float2(a.x, (b.x - a.x) + b.y);
      } else {
        ib[ob] = make_float2(b.x, (a.x - b.x) + a.y);
      }
    }
    return;
  }
  const int slot = E.mixed ? ring : fill_slot(E.mode, E.stage, ring);
  double* ua = Pa->buf[slot];
  double* ub = Pb->buf[slot];
  for (int f = 0; f < NF; ++f) {
    const long long oa = f * Pa->fstride + qa, ob = f * Pb->fstride + qb;
    double* pa = ua + oa;
    double* pb = ub + ob;
    if (a_act && b_act) {
      double m = 0.5 * (*pa + *pb);
      *pa = m;
      *pb = m;
    } else if (b_act) {
      *pa = *pb;
    } else {
      *pb = *pa;
    }
    if (E.mixed) {
      split_to(*pa, Pa->hl[slot], oa);
      split_to(*pb, Pb->hl[slot], ob);
    }
  }
}

// level bookkeeping after a completed RK4 step: advance the ring, count valid
// time levels, advance the time
__global__ void level_advance_kernel(DevLevel* L, double dt) {
  L->ring = (L->ring + 1) % 3;
  L->nvalid = L->nvalid < 3 ? L->nvalid + 1 : 3;
  L->steps += 1;
  L->t += dt;
}

// ----------------------------------------------------------------------------

void launch_fill(int kind, const FillArgs& a, int npatches, long long maxpts, cudaStream_t st) {
  if (npatches == 0 || maxpts == 0) return;
  dim3 grid((unsigned)((maxpts + 127) / 128), npatches);
  switch (kind) {
    case 0: periodic_fill_kernel<<<grid, 128, 0, st>>>(a); break;
    case 1: frozen_fill_kernel<<<grid, 128, 0, st>>>(a); break;
    case 2: ghost_time_fill_kernel<<<grid, 128, 0, st>>>(a); break;
    case 3: restrict_kernel<<<grid, 128, 0, st>>>(a); break;
  }
}

void launch_prolong_space(const DevPatch* patches, const int* ids, const DevLevel* plev, int nchildren,
                          long long max_clusters, int mixed, cudaStream_t st) {
  if (nchildren == 0 || max_clusters == 0) return;
  ProlongArgs a;
  a.patches = patches;
  a.patch_ids = ids;
  a.plev = plev;
  const long long work = max_clusters * NF;
  dim3 grid((unsigned)((work + 127) / 128), nchildren);
  if (mixed)
    prolong_space_mixed_kernel<<<grid, 128, 0, st>>>(a, work);
  else
    prolong_space_kernel<<<grid, 128, 0, st>>>(a, work);
}

void launch_exchange(const ExchArgs& e, long long tot, cudaStream_t st) {
  exchange_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(e);
}

void launch_level_advance(DevLevel* L, double dt, cudaStream_t st) {
  level_advance_kernel<<<1, 1, 0, st>>>(L, dt);
}

}  // namespace sacrak
