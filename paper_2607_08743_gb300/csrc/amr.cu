// Ghost zones and Berger-Oliger inter-level operators (Sec. 2.2.1, 2.2.2):
// periodic and frozen ghost fills, 6th-order Lagrange prolongation of child
// ghosts with quadratic (linear on the first step) time interpolation between
// parent time levels, 4th-order Lagrange restriction, same-level exchange.
#include <type_traits>

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
// so the spatial stencils run twice per parent step instead of at every child
// stage.
//
// The parent cells whose children reach the child's ghost shell form a shell
// of width 2 around the parent cells under the child's active region: the
// box of m = n/2 + 4 cells per axis (parent cells off-2 .. off+n/2+1) minus
// its interior.  That shell is cut into six slabs (two per axis, 2 cells
// thick) and each slab into bricks of at most 8 x 8 cells in its two long
// directions.  One CTA takes one field of one brick: it stages the brick's
// parent cells plus a 3-cell halo in shared memory and applies the 6-point
// interpolant as three separable passes (x, then y, then z), each child at
// -1/4 (nodes -3..2) or +1/4 (nodes -2..3) of its parent cell.  The passes
// run in FP64, or in mixed precision in double-float FP32 pairs from the
// parent's hi/lo split, stored as the split of the result.  (A plain FP32
// version on differences from one reference per brick spread its rounding
// over the brick's variation, up to 14 parent cells; the refinement-boundary
// ghosts it produced made the Gamma-driver fields of the finest levels drift
// about five times further from the FP64 run over 64 coarse steps.)
struct ProlongArgs {
  const DevPatch* patches;
  const int* patch_ids;   // children (one level)
  const DevLevel* plev;   // parent level: slot = its current ring slot - back
  int back;
};

constexpr int PB = 8;          // brick edge along a slab's long directions
constexpr int PB_THREADS = 256;
constexpr int PB_S = 14 * 14 * 8;   // staged parent cells: (8+6) x (8+6) x (2+6)
constexpr int PB_X1 = 16 * 14 * 8;  // after the x pass, largest orientation
constexpr int PB_X2 = 16 * 16 * 8;  // after the y pass

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// bricks of one slab: s = 0,1 z slabs, 2,3 y slabs, 4,5 x slabs
__host__ __device__ inline void slab_bricks(int s, int m0, int m1, int m2, int nb[3]) {
  const int ax = 2 - s / 2;  // thin axis: z, y, x
  const int len[3] = {m0, m1, m2};
  for (int d = 0; d < 3; ++d) {
    int l = len[d];
    if (d == ax) {
      nb[d] = 1;
      continue;
    }
    // z slabs cover everything in x and y; y slabs the middle (2 .. m-3) in
    // z; x slabs the middle in y and z
    if (d > ax) l -= 4;
    nb[d] = cdiv(l, PB);
  }
}

__host__ __device__ inline int slab_count(int s, int m0, int m1, int m2) {
  int nb[3];
  slab_bricks(s, m0, m1, m2, nb);
  return nb[0] * nb[1] * nb[2];
}

int prolong_bricks(int n0, int n1, int n2) {
  const int m0 = n0 / 2 + 4, m1 = n1 / 2 + 4, m2 = n2 / 2 + 4;
  int tot = 0;
  for (int s = 0; s < 6; ++s) tot += slab_count(s, m0, m1, m2);
  return tot;
}

// Arithmetic of the passes: FP64, or (mixed precision) double-float pairs
// (hi, lo) of FP32 with error-free products and sums, which keep about 44
// bits at FP32 instruction rates.  The weights are exact in FP32.
__device__ __forceinline__ void p_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void p_zero(float2& a) { a = make_float2(0.0f, 0.0f); }
__device__ __forceinline__ void p_fma(double& acc, double w, double x) { acc = fma(w, x, acc); }
// (explicitly rounded intrinsics: a contraction into an FMA would break the
// error-free transformations)
__device__ __forceinline__ void p_fma(float2& acc, double wd, float2 x) {
  const float w = (float)wd;
  const float p = __fmul_rn(w, x.x);
  const float pe = fmaf(w, x.x, -p);  // p + pe = w x.hi exactly
  const float sh = __fadd_rn(acc.x, p);  // two-sum of acc.hi and p
  const float bb = __fsub_rn(sh, acc.x);
  const float e = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(sh, bb)), __fsub_rn(p, bb));
  acc.y = __fadd_rn(acc.y, fmaf(w, x.y, __fadd_rn(e, pe)));
  acc.x = sh;
}
__device__ __forceinline__ void p_norm(double&) {}
__device__ __forceinline__ void p_norm(float2& a) {  // two-sum: hi = RN(hi + lo)
  const float sh = __fadd_rn(a.x, a.y);
  const float bb = __fsub_rn(sh, a.x);
  a.y = __fadd_rn(__fsub_rn(a.x, __fsub_rn(sh, bb)), __fsub_rn(a.y, bb));
  a.x = sh;
}

template <bool MIXED>
__global__ void __launch_bounds__(PB_THREADS) prolong_brick_kernel(ProlongArgs A) {
  typedef typename std::conditional<MIXED, float2, double>::type T;
  __shared__ T S[PB_S];
  __shared__ T X1[PB_X1];
  __shared__ T X2[PB_X2];
  const DevPatch* C = A.patches + A.patch_ids[blockIdx.z];
  const int f = blockIdx.y;
  const int m[3] = {C->n[0] / 2 + 4, C->n[1] / 2 + 4, C->n[2] / 2 + 4};
  // which slab and which brick of it
  int b = blockIdx.x, s = 0;
  for (; s < 6; ++s) {
    const int c = slab_count(s, m[0], m[1], m[2]);
    if (b < c) break;
    b -= c;
  }
  if (s == 6) return;
  int nb[3];
  slab_bricks(s, m[0], m[1], m[2], nb);
  const int ax = 2 - s / 2;
  const int bi[3] = {b % nb[0], (b / nb[0]) % nb[1], b / (nb[0] * nb[1])};
  int lo[3], B[3];
  for (int d = 0; d < 3; ++d) {
    if (d == ax) {
      lo[d] = (s & 1) ? m[d] - 2 : 0;
      B[d] = 2;
      continue;
    }
    const int base = d > ax ? 2 : 0;  // slab range along d starts here
    const int len = d > ax ? m[d] - 4 : m[d];
    lo[d] = base + bi[d] * PB;
    B[d] = min(PB, base + len - lo[d]);
  }
  const int Sx = B[0] + 6, Sy = B[1] + 6, Sz = B[2] + 6;
  const int Cx = 2 * B[0], Cy = 2 * B[1], Cz = 2 * B[2];
  const DevPatch* P = A.patches + C->parent;
  const int slot = (A.plev->ring + 3 - A.back) % 3;
  const long long fo = (long long)f * P->fstride;
  // parent array index of shell cell a along d: off[d] - 2 + a + GH
  auto pq = [&](int a, int bb, int c) {
    return (long long)(C->off[0] - 2 + a + GH) + (long long)(C->off[1] - 2 + bb + GH) * P->px +
           (long long)(C->off[2] - 2 + c + GH) * P->plane;
  };
  // Only parent cells -2 .. m+1 (parent active cells off-4 .. off+n/2+3, by
  // the nesting margin) are read: the children that are kept need no others,
  // and cells outside that range (possibly never written) would turn a zero
  // weight into NaN.  They are staged as 0.
  // threads as a 16 x 16 sheet (x, y); every pass loops over its third axis
  // (every extent is at most 16)
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (tx < Sx && ty < Sy) {
    const int a = lo[0] - 3 + tx, bb = lo[1] - 3 + ty;
    const bool inxy = a >= -2 && a <= m[0] + 1 && bb >= -2 && bb <= m[1] + 1;
    for (int z = 0; z < Sz; ++z) {
      const int c = lo[2] - 3 + z;
      T v;
      p_zero(v);
      // (with equatorial symmetry a child on z = 0 has no parent margin
      // below: parent cells outside the parent array are staged as 0; they
      // only reach children at z < 0, which the reflection overwrites)
      const int pk = C->off[2] - 2 + c + GH;
      if (inxy && c >= -2 && c <= m[2] + 1 && pk >= 0 && pk < P->NZ) {
        if (MIXED)
          v = *reinterpret_cast<const T*>(P->hl[slot] + fo + pq(a, bb, c));
        else
          v = *reinterpret_cast<const T*>(P->buf[slot] + fo + pq(a, bb, c));
      }
      S[(z * Sy + ty) * Sx + tx] = v;
    }
  }
  __syncthreads();
  // x pass: X1[z][y][cx]
  if (tx < Cx && ty < Sy) {
    const int p = tx >> 1, od = tx & 1;
    for (int z = 0; z < Sz; ++z) {
      const T* row = S + (z * Sy + ty) * Sx + p + od;
      T acc;
      p_zero(acc);
#pragma unroll
      for (int t = 0; t < 6; ++t) p_fma(acc, od ? c_wp[t] : c_wm[t], row[t]);
      p_norm(acc);
      X1[(z * Sy + ty) * Cx + tx] = acc;
    }
  }
  __syncthreads();
  // y pass: X2[z][cy][cx]
  if (tx < Cx && ty < Cy) {
    const int p = ty >> 1, od = ty & 1;
    for (int z = 0; z < Sz; ++z) {
      const T* col = X1 + (z * Sy + p + od) * Cx + tx;
      T acc;
      p_zero(acc);
#pragma unroll
      for (int t = 0; t < 6; ++t) p_fma(acc, od ? c_wp[t] : c_wm[t], col[t * Cx]);
      p_norm(acc);
      X2[(z * Cy + ty) * Cx + tx] = acc;
    }
  }
  __syncthreads();
  // z pass and store of the children in the ghost shell (mixed precision:
  // stored as hi/lo pairs in the same 8-byte entries)
  double* __restrict__ g = C->gsh[slot] + (long long)f * C->fstride;
  float2* __restrict__ g2 = reinterpret_cast<float2*>(g);
  if (tx < Cx && ty < Cy) {
    const int i = 2 * lo[0] - 4 + tx, j = 2 * lo[1] - 4 + ty;
    if (i < -GH || j < -GH || i >= C->n[0] + GH || j >= C->n[1] + GH) return;
    const bool actxy = i >= 0 && j >= 0 && i < C->n[0] && j < C->n[1];
    for (int cz = 0; cz < Cz; ++cz) {
      const int k = 2 * lo[2] - 4 + cz;
      if (k < -GH || k >= C->n[2] + GH) continue;
      if (actxy && k >= 0 && k < C->n[2]) continue;
      const int p = cz >> 1, od = cz & 1;
      const T* col = X2 + ((p + od) * Cy + ty) * Cx + tx;
      T acc;
      p_zero(acc);
#pragma unroll
      for (int t = 0; t < 6; ++t) p_fma(acc, od ? c_wp[t] : c_wm[t], col[t * Cx * Cy]);
      p_norm(acc);  // mixed precision: (RN(v), v - RN(v)), the split of the value
      const long long o = (i + GH) + (long long)(j + GH) * C->px + (long long)(k + GH) * C->plane;
      *reinterpret_cast<T*>(MIXED ? (void*)(g2 + o) : (void*)(g + o)) = acc;
    }
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
  // at a parent time level (the start of the first child step, the end of
  // the second) only one weight is non-zero: the other slots are not read
  const bool u0 = q3 && w0 != 0.0, u1 = w1 != 0.0, u2 = w2 != 0.0;
  const double* __restrict__ g0 = C->gsh[(pr + 1) % 3];
  const double* __restrict__ g1 = C->gsh[(pr + 2) % 3];
  const double* __restrict__ g2 = C->gsh[pr];
  const int ring = A.lev->ring;
  const long long q = i + (long long)j * C->px + (long long)k * C->plane;
  // this block's five fields (gridDim.z = 5 groups)
  const int f0 = blockIdx.z * (NF / 5);
  const bool dual = A.dual && A.mode == 0 && A.stage == 2;
  if (!A.mixed) {
    double* __restrict__ dst = C->buf[fill_slot(A.mode, A.stage, ring)];
    double* __restrict__ dst3 = C->buf[fill_slot(0, 3, ring)];
#pragma unroll
    for (int f = f0; f < f0 + NF / 5; ++f) {
      const long long o = f * C->fstride + q;
      // (a zero weight times a finite cached value adds exactly nothing)
      double v = (u1 && u2) ? w1 * g1[o] + w2 * g2[o] : (u1 ? w1 * g1[o] : w2 * g2[o]);
      if (u0) v += w0 * g0[o];
      dst[o] = v;
      if (dual) dst3[o] = v;
    }
    return;
  }
  // mixed precision: the cached slots hold hi/lo pairs.  Stage 1 (and the
  // fill of the current level) sets the FP64 ghost and its split; later
  // stages set lo_s = v - hi_n.  The time weights sum to one and are exact
  // in FP32, so both are formed in FP32 on differences from a nearby hi.
  const bool later = (A.mode == 0 && A.stage > 1);
  float2* __restrict__ in = later ? mixed_in(C, A.stage, ring) : nullptr;
  float2* __restrict__ in3 = mixed_in(C, 3, ring);
  const float2* __restrict__ h0 = reinterpret_cast<const float2*>(g0);
  const float2* __restrict__ h1 = reinterpret_cast<const float2*>(g1);
  const float2* __restrict__ h2 = reinterpret_cast<const float2*>(g2);
  const float w0f = (float)w0, w1f = (float)w1, w2f = (float)w2;
#pragma unroll
  for (int f = f0; f < f0 + NF / 5; ++f) {
    const long long o = f * C->fstride + q;
    const float2 z = make_float2(0.0f, 0.0f);
    const float2 a1 = u1 ? h1[o] : z, a2 = u2 ? h2[o] : z;
    const float2 a0 = u0 ? h0[o] : z;
    if (later) {
      const float hi = C->hl[ring][o].x;
      float lo = w1f * ((a1.x - hi) + a1.y) + w2f * ((a2.x - hi) + a2.y);
      if (u0) lo += w0f * ((a0.x - hi) + a0.y);
      in[o] = make_float2(hi, lo);
      if (dual) in3[o] = make_float2(hi, lo);
    } else {
      // differences from the hi part of the first slot read
      const float r = u1 ? a1.x : a2.x;
      float d = u1 ? w1f * a1.y + w2f * ((a2.x - r) + a2.y) : w2f * a2.y;
      if (u0) d += w0f * ((a0.x - r) + a0.y);
      const double v = (double)r + (double)d;
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
  if (A.mixed) {
    // mixed precision: the interpolant in FP32 on the child's hi/lo split,
    // as differences from the fine cell (2I, 2J, 2K), added back to that
    // cell's FP64 value (the weights sum to one along every axis)
    const float2* __restrict__ hc = C->hl[A.lev->ring];
    const long long qr = q0 + 1 + C->px + C->plane;
    const float wf[4] = {-1.0f / 16, 9.0f / 16, 9.0f / 16, -1.0f / 16};
    for (int f = 0; f < NF; ++f) {
      const long long o = f * C->fstride;
      const float2 r = hc[o + qr];
      const float2* src = hc + o + q0;
      float v = 0.0f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float vy = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float2* row = src + (long long)c * C->plane + (long long)b * C->px;
          float vx = 0.0f;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float2 x = __ldg(row + a);
            vx += wf[a] * ((x.x - r.x) + (x.y - r.y));
          }
          vy += wf[b] * vx;
        }
        v += wf[c] * vy;
      }
      const double res = uc[o + qr] + (double)v;
      up[f * P->fstride + qp] = res;
      split_to(res, P->hl[A.plev->ring], f * P->fstride + qp);
    }
    return;
  }
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

// Equatorial reflection symmetry (Sec. 2.2.2): the z < 0 ghost layers of a
// patch whose lower z face is z = 0 take f(x, y, -z) = s_z f(x, y, z);
// s_z = -1 for the fields with an odd number of z indices.  Ghost layer k
// (array index) mirrors active layer 2 GH - 1 - k, over the whole x-y extent.
__device__ __forceinline__ int zparity(int f) {
  const unsigned odd = (1u << F_GXZ) | (1u << F_GYZ) | (1u << F_AXZ) | (1u << F_AYZ) | (1u << F_GAMZ) |
                       (1u << F_BETZ) | (1u << F_BZ);
  return (odd >> f) & 1u ? -1 : 1;
}

__global__ void zreflect_kernel(FillArgs A) {
  const DevPatch* P = A.patches + A.patch_ids[blockIdx.y];
  if (!P->zrefl) return;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long slab = (long long)GH * P->NY * P->NX;
  if (id >= slab) return;
  const int i = (int)(id % P->NX);
  const int j = (int)((id / P->NX) % P->NY);
  const int k = (int)(id / ((long long)P->NX * P->NY));
  const int ring = A.lev->ring;
  const long long q = i + (long long)j * P->px + (long long)k * P->plane;
  const long long qm = i + (long long)j * P->px + (long long)(2 * GH - 1 - k) * P->plane;
  const long long fs = P->fstride;
  if (A.mixed && A.mode == 0 && A.stage > 1) {
    float2* in = mixed_in(P, A.stage, ring);  // the split stage state (hi, lo): both change sign
    for (int f = 0; f < NF; ++f) {
      const float2 v = in[f * fs + qm];
      const float sg = (float)zparity(f);
      in[f * fs + q] = make_float2(sg * v.x, sg * v.y);
    }
    return;
  }
  const int slot = fill_slot(A.mode, A.stage, ring);
  double* u = P->buf[slot];
  for (int f = 0; f < NF; ++f) u[f * fs + q] = zparity(f) * u[f * fs + qm];
  if (A.mixed && slot < 3) {  // a time level: its split as well
    float2* hl = P->hl[slot];
    for (int f = 0; f < NF; ++f) {
      const float2 v = hl[f * fs + qm];
      const float sg = (float)zparity(f);
      hl[f * fs + q] = make_float2(sg * v.x, sg * v.y);
    }
  }
}

void launch_zreflect(const FillArgs& a, int npatches, long long maxpts, cudaStream_t st) {
  if (npatches == 0 || maxpts == 0) return;
  zreflect_kernel<<<dim3((unsigned)((maxpts + 127) / 128), npatches), 128, 0, st>>>(a);
}

// Copy between a patch buffer (rows of px doubles) and a contiguous patch
// array (rows of NX doubles): host transfers then move one contiguous block.
__global__ void repack_kernel(double* __restrict__ dst, const double* __restrict__ src, long long rows, int NX,
                              int px, int to_pitched) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  for (long long r = blockIdx.y; r < rows; r += gridDim.y) {
    if (to_pitched)
      dst[r * px + x] = src[r * NX + x];
    else
      dst[r * NX + x] = src[r * px + x];
  }
}

void launch_repack(double* dst, const double* src, long long rows, int NX, int px, int to_pitched,
                   cudaStream_t st) {
  const unsigned gy = (unsigned)(rows < 65535 ? rows : 65535);
  repack_kernel<<<dim3((NX + 127) / 128, gy), 128, 0, st>>>(dst, src, rows, NX, px, to_pitched);
}

// level bookkeeping after a completed RK4 step: advance the ring, count valid
// time levels, advance the time
__global__ void level_advance_kernel(DevLevel* L, double dt) {
  L->ring = (L->ring + 1) % 3;
  L->nvalid = L->nvalid < 3 ? L->nvalid + 1 : 3;
  L->steps += 1;
  L->t += dt;
}

__global__ void set_nvalid_kernel(DevLevel* L, int nvalid) { L->nvalid = nvalid; }

// ---------------------------------------------------------------------------
// Moving boxes (Sec. 2.2.1)

// beta^i at x: tricubic Lagrange from the 4 nearest cell centres per axis,
// all of them active cells (false otherwise)
__device__ bool interp_shift(const DevPatch* P, const double* __restrict__ u, const double x[3],
                             double b[3]) {
  int i0[3];
  double w[3][4];
  const int n[3] = {P->n[0], P->n[1], P->n[2]};
  for (int d = 0; d < 3; ++d) {
    const double t = (x[d] - P->origin[d]) / P->dx - 0.5 + GH;  // array coordinate
    if (!(t >= GH + 1.0 && t < GH + n[d] - 2.0)) return false;
    i0[d] = (int)floor(t) - 1;
    const double s = t - i0[d], s1 = s - 1.0, s2 = s - 2.0, s3 = s - 3.0;
    w[d][0] = -s1 * s2 * s3 / 6.0;
    w[d][1] = s * s2 * s3 / 2.0;
    w[d][2] = -s * s1 * s3 / 2.0;
    w[d][3] = s * s1 * s2 / 6.0;
  }
  for (int c = 0; c < 3; ++c) {
    const double* f = u + (long long)(F_BETX + c) * P->fstride;
    double v = 0.0;
    for (int k = 0; k < 4; ++k)
      for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i)
          v += w[0][i] * w[1][j] * w[2][k] *
               f[(i0[0] + i) + (long long)(i0[1] + j) * P->px + (long long)(i0[2] + k) * P->plane];
    b[c] = v;
  }
  return true;
}

// one thread per puncture: x <- x - dt/2 (beta_old(x) + beta_new(x - dt beta_old(x)))
__global__ void track_kernel(TrackArgs A) {
  const int p = threadIdx.x;
  if (p >= A.np) return;
  DevPunct* q = A.punct + p;
  if (q->level != A.level) return;
  const DevPatch* P = A.patches + q->patch;
  const int ring = A.levels[A.level].ring;
  double x[3], b0[3], b1[3], xs[3];
  for (int d = 0; d < 3; ++d) x[d] = q->x[d];
  if (!interp_shift(P, P->buf[ring], x, b0)) {
    atomicOr(A.err, ERR_TRACK);
    return;
  }
  for (int d = 0; d < 3; ++d) xs[d] = __dsub_rn(x[d], __dmul_rn(A.dt, b0[d]));
  if (!interp_shift(P, P->buf[(ring + 1) % 3], xs, b1)) {
    atomicOr(A.err, ERR_TRACK);
    return;
  }
  const double h = __dmul_rn(0.5, A.dt);
  for (int d = 0; d < 3; ++d) q->x[d] = __dsub_rn(x[d], __dmul_rn(h, __dadd_rn(b0[d], b1[d])));
}

__global__ void move_patch_kernel(MoveArgs A) {
  const DevPatch* C = A.patches + A.patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)C->NX * C->NY * C->NZ;
  if (id >= tot) return;
  const int i = (int)(id % C->NX), j = (int)((id / C->NX) % C->NY), k = (int)(id / ((long long)C->NX * C->NY));
  const long long q = i + (long long)j * C->px + (long long)k * C->plane;
  const int io = i + A.sh[0], jo = j + A.sh[1], ko = k + A.sh[2];
  const double* __restrict__ src = C->buf[A.levels[C->level].ring];
  if (io >= GH && io < GH + C->n[0] && jo >= GH && jo < GH + C->n[1] && ko >= GH && ko < GH + C->n[2]) {
    const long long qo = io + (long long)jo * C->px + (long long)ko * C->plane;
    for (int f = 0; f < NF; ++f) A.dst[f * C->fstride + q] = src[f * C->fstride + qo];
    return;
  }
  if (A.skip_zlower && k < GH) return;  // the reflection fills these
  const DevPatch* P = A.patches + C->parent;
  const double* __restrict__ up = P->buf[A.levels[P->level].ring];
  // parent array index of the first stencil point and the weights along each
  // axis: child cell c (active index) lies at parent cell off + floor(c/2)
  // +- 1/4; odd c: nodes -2..3 (c_wp), even c: nodes -3..2 (c_wm)
  const int ci[3] = {i - GH, j - GH, k - GH};
  const int Pd[3] = {P->NX, P->NY, P->NZ};
  int lo[3];
  const double* w[3];
  for (int d = 0; d < 3; ++d) {
    const int odd = ci[d] & 1;
    lo[d] = A.noff[d] + floor_half(ci[d]) + GH - (odd ? 2 : 3);
    w[d] = odd ? c_wp : c_wm;
    if (lo[d] < 0 || lo[d] + 5 >= Pd[d]) {
      atomicOr(A.err, ERR_BOUNDS);
      return;
    }
  }
  for (int f = 0; f < NF; ++f) {
    const double* fp = up + (long long)f * P->fstride;
    double v = 0.0;
    for (int c = 0; c < 6; ++c)
      for (int b = 0; b < 6; ++b)
        for (int a = 0; a < 6; ++a)
          v += w[0][a] * w[1][b] * w[2][c] *
               fp[(lo[0] + a) + (long long)(lo[1] + b) * P->px + (long long)(lo[2] + c) * P->plane];
    A.dst[f * C->fstride + q] = v;
  }
}

// ----------------------------------------------------------------------------

void launch_fill(int kind, const FillArgs& a, int npatches, long long maxpts, cudaStream_t st) {
  if (npatches == 0 || maxpts == 0) return;
  dim3 grid((unsigned)((maxpts + 127) / 128), npatches);
  switch (kind) {
    case 0: periodic_fill_kernel<<<grid, 128, 0, st>>>(a); break;
    case 1: frozen_fill_kernel<<<grid, 128, 0, st>>>(a); break;
    case 2: ghost_time_fill_kernel<<<dim3(grid.x, grid.y, 5), 128, 0, st>>>(a); break;
    case 3: restrict_kernel<<<grid, 128, 0, st>>>(a); break;
  }
}

void launch_prolong_space(const DevPatch* patches, const int* ids, const DevLevel* plev, int nchildren,
                          long long max_bricks, int mixed, cudaStream_t st, int back) {
  if (nchildren == 0 || max_bricks == 0) return;
  ProlongArgs a;
  a.patches = patches;
  a.patch_ids = ids;
  a.plev = plev;
  a.back = back;
  dim3 grid((unsigned)max_bricks, NF, nchildren);
  if (mixed)
    prolong_brick_kernel<true><<<grid, PB_THREADS, 0, st>>>(a);
  else
    prolong_brick_kernel<false><<<grid, PB_THREADS, 0, st>>>(a);
}

void launch_exchange(const ExchArgs& e, long long tot, cudaStream_t st) {
  exchange_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(e);
}

void launch_set_nvalid(DevLevel* L, int nvalid, cudaStream_t st) { set_nvalid_kernel<<<1, 1, 0, st>>>(L, nvalid); }

void launch_track(const TrackArgs& a, cudaStream_t st) { track_kernel<<<1, 32, 0, st>>>(a); }

void launch_move(const MoveArgs& a, long long tot, cudaStream_t st) {
  move_patch_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(a);
}

void launch_level_advance(DevLevel* L, double dt, cudaStream_t st) {
  level_advance_kernel<<<1, 1, 0, st>>>(L, dt);
}

}  // namespace sacrak
