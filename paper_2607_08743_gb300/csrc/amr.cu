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

// periodic: every ghost takes the value of the active point congruent modulo n
__global__ void periodic_fill_kernel(FillArgs A) {
  const DevPatch* P = A.patches + A.patch_ids[blockIdx.y];
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nshell(P)) return;
  int i, j, k;
  shell_ijk(id, P->NX, P->NY, P->NZ, i, j, k);
  const int si = GH + ((i - GH) % P->n[0] + P->n[0]) % P->n[0];
  const int sj = GH + ((j - GH) % P->n[1] + P->n[1]) % P->n[1];
  const int sk = GH + ((k - GH) % P->n[2] + P->n[2]) % P->n[2];
  double* u = P->buf[fill_slot(A.mode, A.stage, A.lev->ring)];
  const long long q = i + (long long)j * P->px + (long long)k * P->plane;
  const long long qs = si + (long long)sj * P->px + (long long)sk * P->plane;
  for (int f = 0; f < NF; ++f) u[f * P->fstride + q] = u[f * P->fstride + qs];
}

// frozen: ghosts of the target buffer take the ghosts of the current level
__global__ void frozen_fill_kernel(FillArgs A) {
  const DevPatch* P = A.patches + A.patch_ids[blockIdx.y];
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nshell(P)) return;
  int i, j, k;
  shell_ijk(id, P->NX, P->NY, P->NZ, i, j, k);
  const int ring = A.lev->ring;
  const int dst = fill_slot(A.mode, A.stage, ring);
  if (dst == ring) return;
  const long long q = i + (long long)j * P->px + (long long)k * P->plane;
  for (int f = 0; f < NF; ++f) P->buf[dst][f * P->fstride + q] = P->buf[ring][f * P->fstride + q];
}

// 6-point Lagrange weights at +1/4 (nodes -2..3) and -1/4 (nodes -3..2), /8192
__constant__ double c_wp[6] = {77.0 / 8192, -693.0 / 8192, 6930.0 / 8192,
                               2310.0 / 8192, -495.0 / 8192, 63.0 / 8192};
__constant__ double c_wm[6] = {63.0 / 8192, -495.0 / 8192, 2310.0 / 8192,
                               6930.0 / 8192, -693.0 / 8192, 77.0 / 8192};

__device__ __forceinline__ int floor_half(int i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

// Child ghosts from the parent: a combination of the parent's time levels
// (oldest, middle, newest; the host computes the weights: quadratic once three
// levels exist, linear before) interpolated in space with the tensor-product
// 6-point Lagrange interpolant.
__global__ void __launch_bounds__(128) prolong_kernel(FillArgs A) {
  const DevPatch* C = A.patches + A.patch_ids[blockIdx.y];
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nshell(C)) return;
  int i, j, k;
  shell_ijk(id, C->NX, C->NY, C->NZ, i, j, k);
  const DevPatch* P = A.patches + C->parent;
  const int pr = A.plev->ring;
  const int nv = A.plev->nvalid;
  const bool q3 = nv >= 3;
  const double wt[3] = {q3 ? A.wq[0] : 0.0, q3 ? A.wq[1] : A.wl[1], q3 ? A.wq[2] : A.wl[2]};
  const double* __restrict__ t0 = P->buf[(pr + 1) % 3];  // oldest
  const double* __restrict__ t1 = P->buf[(pr + 2) % 3];  // middle
  const double* __restrict__ t2 = P->buf[pr];            // newest
  const int ci[3] = {i - GH, j - GH, k - GH};
  int base[3];
  const double* w[3];
  int lo[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int odd = ci[d] & 1;
    base[d] = C->off[d] + floor_half(ci[d]) + GH;
    w[d] = odd ? c_wp : c_wm;
    lo[d] = odd ? -2 : -3;
  }
  double* __restrict__ dst = C->buf[fill_slot(A.mode, A.stage, A.lev->ring)];
  const long long qc = i + (long long)j * C->px + (long long)k * C->plane;
  const long long q0 = (base[0] + lo[0]) + (long long)(base[1] + lo[1]) * P->px +
                       (long long)(base[2] + lo[2]) * P->plane;
  const bool quad = nv >= 3;
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    const long long fo = f * P->fstride + q0;
    double v = 0.0;
#pragma unroll 1
    for (int c = 0; c < 6; ++c) {
      double vy = 0.0;
#pragma unroll 1
      for (int b = 0; b < 6; ++b) {
        const long long o = fo + (long long)c * P->plane + (long long)b * P->px;
        double vx = 0.0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          double val = wt[1] * __ldg(t1 + o + a) + wt[2] * __ldg(t2 + o + a);
          if (quad) val += wt[0] * __ldg(t0 + o + a);
          vx += w[0][a] * val;
        }
        vy += w[1][b] * vx;
      }
      v += w[2][c] * vy;
    }
    dst[f * C->fstride + qc] = v;
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
  const int slot = fill_slot(E.mode, E.stage, ring);
  double* ua = Pa->buf[slot];
  double* ub = Pb->buf[slot];
  const long long qa = I + (long long)J * Pa->px + (long long)K * Pa->plane;
  const long long qb = (ib + GH) + (long long)(jb + GH) * Pb->px + (long long)(kb + GH) * Pb->plane;
  for (int f = 0; f < NF; ++f) {
    double* pa = ua + f * Pa->fstride + qa;
    double* pb = ub + f * Pb->fstride + qb;
    if (a_act && b_act) {
      double m = 0.5 * (*pa + *pb);
      *pa = m;
      *pb = m;
    } else if (b_act) {
      *pa = *pb;
    } else {
      *pb = *pa;
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
    case 2: prolong_kernel<<<grid, 128, 0, st>>>(a); break;
    case 3: restrict_kernel<<<grid, 128, 0, st>>>(a); break;
  }
}

void launch_exchange(const ExchArgs& e, long long tot, cudaStream_t st) {
  exchange_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(e);
}

void launch_level_advance(DevLevel* L, double dt, cudaStream_t st) {
  level_advance_kernel<<<1, 1, 0, st>>>(L, dt);
}

}  // namespace sacrak
