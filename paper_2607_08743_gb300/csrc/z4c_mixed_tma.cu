// Mixed-precision Z4c RHS + RK4 stage kernel with TMA-staged field tiles.
//
// Same equations and precision split as z4c_mixed.cu (Sec. 2.1.1, 2.2 of the
// SACRA-K paper: 4th-order centred derivatives, lopsided upwind advection,
// 6th-order Kreiss-Oliger dissipation, classical RK4), organised for the
// memory system of sm_103a:
//
//  - A CTA owns a tile of 32 x TY x TZ points (one thread per point, x along
//    the lanes).  For every field it needs the tile plus a 3-cell halo, a box
//    of 38 x (TY+6) x (TZ+6) hi/lo pairs (copied as 40 pairs per row from one
//    cell before the halo, so that the copy starts on a 16-byte boundary of
//    the buffer), which one elected thread copies into
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
#include "mixed_stage.cuh"
#include "ldg_stage.cuh"
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

// bounded wait: at most `limit` cycles of SM clock
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

template <int TY, int TZ>
struct Cfg {
  static constexpr int NT = 32 * TY * TZ;
  static constexpr int BX = 40, BY = TY + 6, BZ = TZ + 6;  // box row: cells x0-4 .. x0+35
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

// wait for copy g within `limit` cycles (limit < 0: run out at once); on
// time-out flag the CTA (the caller stops after the next barrier)
__device__ __forceinline__ void wait_copy(const Pipe& p, unsigned g, long long limit, unsigned* err) {
  if (limit < 0 || !mbar_wait_bounded(p.bar + (g & 1), (g >> 1) & 1, limit)) {
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
  const int c = ((lz + 3) * C::BY + (ly + 3)) * C::BX + (lx + 4);

  unsigned g = 0;
  unsigned issued = 0;  // copies issued by thread 0
  bool stop = false;
  if (t == 0) {
    issue_load<TY, TZ>(A, p, 0, blockIdx.x, 0, which);
    issued = 1;
  }

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
        if (f + 1 < NF) {
          issue_load<TY, TZ>(A, p, g + 1, tile, f + 1, which);
          issued = g + 2;
        } else if (tile + (int)gridDim.x < A.ntiles) {
          issue_load<TY, TZ>(A, p, g + 1, tile + gridDim.x, 0, which);
          issued = g + 2;
        }
      }
      wait_copy(p, g, A.wait_cycles, S.err);
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
    // a wait ran out: every copy that may still be in flight (the one whose
    // wait ran out and the one issued after it; all earlier ones were waited
    // for) lands before the CTA exits and its shared memory is released,
    // each within the full bound
    for (unsigned c = issued >= 2 ? issued - 2 : 0; c < issued; ++c)
      mbar_wait_bounded(p.bar + (c & 1), (c >> 1) & 1, TMA_WAIT_CYCLES);
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

// one CTA per tile, or (PERS) a grid of resident CTAs that walks the level's
// tiles with a static stride (one persistent launch per level)
template <int MINB, int MODE, int PF, bool SHF, bool PERS>
__global__ void __launch_bounds__(128, MINB) z4c_stage_ldg_kernel(StageArgs S) {
  extern __shared__ float sd[];
  if constexpr (!PERS) {
    ldg_tile<MINB, MODE, PF, SHF>(S, blockIdx.x, sd);
  } else {
    for (int tile = blockIdx.x; tile < S.ntiles; tile += gridDim.x) ldg_tile<MINB, MODE, PF, SHF>(S, tile, sd);
  }
}

// resident CTAs of the persistent variant per device (0: not set up)
int g_pers_grid[64] = {};

template <int MINB, int PF, bool SHF = false, bool PERS = false>
bool setup_ldg() {
  const int smem = NSLOT * 128 * 4;
  bool ok = cudaFuncSetAttribute(z4c_stage_ldg_kernel<MINB, 0, PF, SHF, PERS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
            cudaFuncSetAttribute(z4c_stage_ldg_kernel<MINB, 1, PF, SHF, PERS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
  if (ok && PERS) {
    int dev = 0, nsm = 0, nb = 0;
    ok = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 &&
         cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
         cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, z4c_stage_ldg_kernel<MINB, 0, PF, SHF, PERS>, 128,
                                                       smem) == cudaSuccess &&
         nb > 0;
    if (ok) g_pers_grid[dev] = nsm * nb;
  }
  return ok;
}

template <int MINB, int PF, bool SHF = false, bool PERS = false>
void launch_ldg(const StageArgs& a, cudaStream_t st) {
  const int smem = NSLOT * 128 * 4;
  int grid = a.ntiles;
  if (PERS) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int res = (dev >= 0 && dev < 64) ? g_pers_grid[dev] : 0;
    if (res > 0 && res < grid) grid = res;
  }
  if (a.stage == 0)
    z4c_stage_ldg_kernel<MINB, 1, PF, SHF, PERS><<<grid, 128, smem, st>>>(a);
  else
    z4c_stage_ldg_kernel<MINB, 0, PF, SHF, PERS><<<grid, 128, smem, st>>>(a);
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
  return (v >= 0 && v < TMA_NVARIANTS) ? 40 * (kShape[v][0] + 6) * (kShape[v][1] + 6) * 8 : 0;
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
// 8 (as 4 with 4 CTAs/SM, 128 registers), 9 (as 4, persistent: resident
// CTAs walk the level's tiles)
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
    case 9: return setup_ldg<3, 3, false, true>();
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
    case 9: launch_ldg<3, 3, false, true>(a, st); break;
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
