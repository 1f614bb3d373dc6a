// C ABI of the Z4c hot path: grid creation over a caller-owned device arena,
// data movement, RK4 stages, Berger-Oliger subcycling (captured as a CUDA
// graph) and diagnostics.  Host code only issues launches; every step of the
// path runs in the kernels of z4c_fp64.cu, z4c_mixed.cu, amr.cu and
// diagnostics.cu.
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sacrak.h"
#include "sacrak_dev.cuh"
#include "grhd.h"
#include "stage_tma.h"

using namespace sacrak;

namespace {

constexpr int TILE_X = 32, TILE_Y = 4;
enum { FILL_PERIODIC = 0, FILL_FROZEN = 1, FILL_PROLONG = 2, FILL_RESTRICT = 3 };

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
  // byte offsets inside the arena
  size_t patches, levels, ids, tiles, err, results, punct, scratch, dslot, states, total;
  std::vector<size_t> patch_state;  // offset of each patch's first buffer
  std::vector<size_t> matter_state; // offset of each patch's matter arrays (fluid grids)
  std::vector<long long> fstride;
  std::vector<int> px;
  size_t ntiles = 0, scratch_doubles = 0;
};

// fields of the matter arrays of a patch: conserved variables in the six
// state slots, primitives + Lorentz factor, face fluxes, Z4c matter terms,
// the cached prolongations of the parent's three time levels, and the
// RK4-weighted face fluxes of the last step and of the last two steps
constexpr int MATTER_FIELDS = NBUF * NM + NMP + 3 * NM + NZSRC + 3 * NM + 3 * NM + 3 * NM;

bool describe(int nlevels, int npatches, const sacrak_patch_desc* pd, int mixed, int matter, Layout& L,
              std::string& why) {
  if (matter && mixed) {
    why = "a fluid needs FP64";
    return false;
  }
  if (nlevels < 1 || npatches < 1 || !pd) {
    why = "need at least one level and one patch";
    return false;
  }
  std::vector<int> count(nlevels, 0);
  for (int p = 0; p < npatches; ++p) {
    if (pd[p].level < 0 || pd[p].level >= nlevels) {
      why = "patch level out of range";
      return false;
    }
    for (int d = 0; d < 3; ++d)
      if (pd[p].n[d] < 4 || pd[p].n[d] > 4096) {
        why = "patch size out of range (4..4096 cells per axis)";
        return false;
      }
    count[pd[p].level]++;
  }
  for (int l = 0; l < nlevels; ++l)
    if (count[l] == 0) {
      why = "every level needs a patch";
      return false;
    }
  size_t off = 0;
  L.patches = off;
  off = align_up(off + sizeof(DevPatch) * npatches, 256);
  L.levels = off;
  off = align_up(off + sizeof(DevLevel) * nlevels, 256);
  L.ids = off;
  off = align_up(off + sizeof(int) * npatches, 256);
  size_t ntiles = 0, maxtiles_level = 0, maxpts = 0;
  std::vector<size_t> lt(nlevels, 0);
  for (int p = 0; p < npatches; ++p) {
    size_t t = (size_t)((pd[p].n[0] + TILE_X - 1) / TILE_X) * ((pd[p].n[1] + TILE_Y - 1) / TILE_Y) *
               pd[p].n[2];
    ntiles += t;
    lt[pd[p].level] += t;
    size_t pts = (size_t)(pd[p].n[0] + 2 * GH) * (pd[p].n[1] + 2 * GH) * (pd[p].n[2] + 2 * GH);
    maxpts = pts > maxpts ? pts : maxpts;
  }
  for (int l = 0; l < nlevels; ++l) maxtiles_level = lt[l] > maxtiles_level ? lt[l] : maxtiles_level;
  L.ntiles = ntiles;
  L.tiles = off;
  off = align_up(off + sizeof(Tile) * ntiles, 256);
  L.err = off;
  off = align_up(off + 16, 256);
  L.results = off;
  off = align_up(off + 64 * sizeof(double), 256);
  L.punct = off;
  off = align_up(off + MAX_PUNCT * sizeof(DevPunct), 256);
  L.scratch_doubles = maxtiles_level * 5 > maxpts / 256 + 1 ? maxtiles_level * 5 : maxpts / 256 + 1;
  if (L.scratch_doubles < 6 * (size_t)ADM_MAX_THETA) L.scratch_doubles = 6 * (size_t)ADM_MAX_THETA;
  L.scratch = off;
  off = align_up(off + L.scratch_doubles * sizeof(double), 256);
  // mixed precision: FP32 derivative planes of the split stage kernel, for
  // the level with the most tiles
  L.dslot = off;
  if (mixed) off = align_up(off + (size_t)split_slot_floats((long long)maxtiles_level) * sizeof(float), 256);
  L.states = off;
  L.patch_state.resize(npatches);
  L.matter_state.assign(npatches, 0);
  L.fstride.resize(npatches);
  L.px.resize(npatches);
  for (int p = 0; p < npatches; ++p) {
    int NX = pd[p].n[0] + 2 * GH, NY = pd[p].n[1] + 2 * GH, NZ = pd[p].n[2] + 2 * GH;
    // row pitch: at least one spare element per row, rounded to 8 (the
    // buffers start one element past their 256-byte boundary, so that cells
    // 2m, 2m+1 of a row share a 16-byte line; see the patch table below)
    int px = (int)align_up(NX + 1, 8);
    long long fs = (long long)px * NY * NZ;
    L.px[p] = px;
    L.fstride[p] = fs;
    L.patch_state[p] = off;
    const int nbuf = NBUF + (pd[p].level > 0 ? 3 : 0);  // + cached prolongation slots
    off = align_up(off + (size_t)nbuf * NF * fs * sizeof(double), 256);
    if (mixed) off = align_up(off + (size_t)5 * NF * fs * sizeof(float2), 256);  // hl[3] sa sb
    if (matter) {
      L.matter_state[p] = off;
      off = align_up(off + (size_t)MATTER_FIELDS * fs * sizeof(double), 256);
    }
  }
  // whole-buffer copies and fills from the shifted bases reach one element
  // past the last buffer
  L.total = off + 256;
  return true;
}

}  // namespace

struct sacrak_grid {
  sacrak_params prm;
  cudaStream_t stream;
  char* arena;
  size_t arena_bytes;
  int nlevels, npatches;
  double dx0;
  Layout L;
  std::vector<DevPatch> hp;                // host copy of the patch table
  std::vector<std::vector<int>> lvl_ids;   // patch ids per level
  std::vector<int> lvl_id_off;             // offset of each level's ids in the device id array
  std::vector<size_t> lvl_tile_off, lvl_ntiles;
  std::vector<long long> lvl_max_shell, lvl_max_restrict, lvl_max_clusters;  // clusters: prolongation bricks
  std::vector<long long> lvl_max_zslab;  // points of the z < 0 ghost slab
  bool shells_dirty = true;
  bool split_dirty = true;  // mixed precision: hi/lo of the current levels stale
  DevPatch* d_patches;
  DevLevel* d_levels;
  int* d_ids;
  Tile* d_tiles;
  unsigned* d_err;
  double* d_results;
  double* d_scratch;
  float* d_dslot;  // mixed precision: derivative planes of the split stage kernel
  // moving boxes: tracked punctures (positions on the device), the puncture
  // each patch follows (-1: none), the levels a tracker runs on
  DevPunct* d_punct;
  int npunct = 0;
  std::vector<int> follow;
  // fluid grids: the star each patch follows (-1: none), located by the
  // density maximum of the finest patch that follows it
  std::vector<int> follow_star;
  int nstars = 0;
  std::vector<DevPunct> hpunct;  // tracking patch and level of each puncture
  bool invalid = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // second stream for the refinement-boundary time fills and the parent's
  // prolongation, which run beside the stage kernels (sacrak_set_overlap);
  // side_live: work on it that the main stream has not waited for yet
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool side_live = false;
  bool overlap = true;
  std::string last_error;
  // profiling of the fused stage kernel
  bool prof = false;
  long long tma_wait_cycles = 0;  // 0: TMA_WAIT_CYCLES (sacrak_set_wait_limit)
  // fluid (params.matter): EOS and atmosphere
  DevEOS eos = {};
  bool eos_set = false;
  bool matter_ready = false;  // primitives uploaded
  bool matter_shells_dirty = true;  // the children's fluid caches predate the last upload
  double rho_atm = 0.0, r_atm = 0.0;
  int riemann = 0;  // face flux of the fluid: 0 HLLC in the face tetrad, 1 HLLE (sacrak_set_riemann)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t ev_used = 0;
  long long prof_zones = 0;
  std::vector<long long> lvl_zones;
  // stage kernel per level: 0 the direct kernel, 1..TMA_NVARIANTS the TMA
  // variant (id - 1); chosen by default, by sacrak_set_stage_kernel or by
  // sacrak_autotune
  std::vector<int> lvl_kernel;
  // TMA descriptors per variant and patch (built on first use of a variant)
  std::vector<std::array<CUtensorMap, 5>> maps[TMA_NVARIANTS];
  int tma_blocks[TMA_NVARIANTS] = {};  // resident CTAs per SM, 0 = not set up
  int nsm = 0;
};

namespace {

sacrak_status fail(sacrak_grid* g, sacrak_status s, const char* fmt, ...) {
  if (g) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g->last_error = buf;
    if (s == SACRAK_ECUDA || s == SACRAK_ENONFINITE || s == SACRAK_ETIMEOUT) g->invalid = true;
  }
  return s;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(g, SACRAK_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));           \
  } while (0)

DevParams dev_params(const sacrak_params& p) {
  DevParams d;
  d.kappa1 = p.kappa1;
  d.kappa2 = p.kappa2;
  d.eta = p.eta;
  d.sigma_ko = p.sigma_ko;
  d.w_floor = p.w_floor;
  d.lapse = p.lapse;
  d.shift = p.shift;
  d.lapse_uses_khat = p.lapse_uses_khat;
  d.matter = p.matter;
  return d;
}

double level_dt(const sacrak_grid* g, int l) { return g->prm.courant * g->dx0 / std::ldexp(1.0, l); }

sacrak_status check_launch(sacrak_grid* g) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(g, SACRAK_ECUDA, "launch: %s", cudaGetErrorString(e));
  return SACRAK_OK;
}

// read the device error flag (synchronises the stream)
sacrak_status sync_and_check(sacrak_grid* g) {
  unsigned flag = 0;
  CK(cudaMemcpyAsync(&flag, g->d_err, sizeof flag, cudaMemcpyDeviceToHost, g->stream));
  CK(cudaStreamSynchronize(g->stream));
  // a wait that ran out or a failed bounds check skipped writes, so later
  // non-finite values may be their consequence: they are reported first
  if (flag & ERR_TIMEOUT) return fail(g, SACRAK_ETIMEOUT, "bounded device wait ran out");
  if (flag & ERR_BOUNDS) return fail(g, SACRAK_ECUDA, "device bounds check failed");
  if (flag & ERR_NONFINITE) return fail(g, SACRAK_ENONFINITE, "non-finite value in a stage update");
  if (flag & ERR_TRACK) {  // reported once; the grid stays usable
    const unsigned rest = flag & ~(unsigned)ERR_TRACK;
    CK(cudaMemcpy(g->d_err, &rest, sizeof rest, cudaMemcpyHostToDevice));
    return fail(g, SACRAK_EINVAL, "a puncture's interpolation stencil left its tracking patch (regrid)");
  }
  return SACRAK_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// Can TMA variant v run the patches `pids` in one launch?  Every box must fit
// in its patch array (32 x TY x TZ active cells at least) and the launch
// arguments hold TMA_MAXP patches.
bool tma_eligible(const sacrak_grid* g, int v, const std::vector<int>& pids) {
  if (g->prm.precision != 1 || v < 0 || v >= TMA_NVARIANTS || pids.empty() || (int)pids.size() > TMA_MAXP)
    return false;
  int ty, tz;
  tma_variant_shape(v, &ty, &tz);
  for (int pid : pids) {
    const DevPatch& P = g->hp[pid];
    if (P.n[0] < 32 || P.n[1] < ty || P.n[2] < tz) return false;
  }
  return true;
}

// kernel ids: 0 direct, 1..TMA_NVARIANTS TMA variant id-1, then the two
// L1-path kernels with packed pair arithmetic (without and with prefetching)
constexpr int K_LDG3 = TMA_NVARIANTS + 1, K_LDG4 = TMA_NVARIANTS + 2, K_SPLIT = TMA_NVARIANTS + 3,
              K_LDG_PF4 = TMA_NVARIANTS + 4, K_LDG_PFS = TMA_NVARIANTS + 5, K_LDG_PFZ = TMA_NVARIANTS + 6,
              K_LDG_PFE = TMA_NVARIANTS + 7, K_LDG_SHF = TMA_NVARIANTS + 8, K_LDG_SHF4 = TMA_NVARIANTS + 9,
              K_LDG_PFZ4 = TMA_NVARIANTS + 10, K_PAIR = TMA_NVARIANTS + 11, K_PAIR_PFZ = TMA_NVARIANTS + 12,
              K_PAIR_PFZ3 = TMA_NVARIANTS + 13, K_LDG_PFZ_PERS = TMA_NVARIANTS + 14,
              K_LDG_FIX = TMA_NVARIANTS + 15, K_LDG_FIX4 = TMA_NVARIANTS + 16, K_COUNT = TMA_NVARIANTS + 17;

// pair-kernel variant of a kernel id (-1 for others)
int pair_variant(int k) { return k == K_PAIR ? 0 : k == K_PAIR_PFZ ? 1 : k == K_PAIR_PFZ3 ? 2 : -1; }

// L1-path variant of a kernel id (-1 for others)
int ldg_variant(int k) {
  return k == K_LDG3 ? 0 : k == K_LDG4 ? 1 : k == K_LDG_PF4 ? 2 : k == K_LDG_PFS ? 3 : k == K_LDG_PFZ ? 4
         : k == K_LDG_PFE ? 5 : k == K_LDG_SHF ? 6 : k == K_LDG_SHF4 ? 7 : k == K_LDG_PFZ4 ? 8
         : k == K_LDG_PFZ_PERS ? 9 : -1;
}

bool kernel_eligible(const sacrak_grid* g, int k, const std::vector<int>& pids) {
  if (k == 0) return true;
  if (k >= 1 && k <= TMA_NVARIANTS) return tma_eligible(g, k - 1, pids);
  if (pair_variant(k) >= 0) {
    if (g->prm.precision != 1) return false;
    for (int pid : pids)  // 32-bit element offsets
      if ((long long)NF * g->hp[pid].fstride >= (1LL << 31)) return false;
    return true;
  }
  return (ldg_variant(k) >= 0 || k == K_SPLIT || k == K_LDG_FIX || k == K_LDG_FIX4) && g->prm.precision == 1;
}

// the row and plane pitches shared by every patch of a level (-1 if they differ)
void level_pitches(const sacrak_grid* g, const std::vector<int>& pids, long long* sy, long long* sz) {
  *sy = *sz = -1;
  for (size_t i = 0; i < pids.size(); ++i) {
    const DevPatch& P = g->hp[pids[i]];
    if (i == 0) {
      *sy = P.px;
      *sz = P.plane;
    } else if (P.px != *sy || P.plane != *sz) {
      *sy = *sz = -1;
      return;
    }
  }
}

// tensor maps of variant v for every patch: the five split buffers viewed as
// 3D arrays of floats [NF*NZ][NY][2*(NX+1)] from their 256-byte aligned slot
// (element 0 of a row is the spare element before ghost cell -3; row pitch
// px pairs), box 80 x (TY+6) x (TZ+6) floats: 40 pairs from cell x0 - 4, so
// that the box's x coordinate 2*x0 floats is a multiple of 16 bytes
sacrak_status ensure_maps(sacrak_grid* g, int v) {
  if (!g->maps[v].empty() && g->tma_blocks[v] > 0) return SACRAK_OK;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(g, SACRAK_ECUDA, "cuTensorMapEncodeTiled is not available");
  int ty, tz;
  tma_variant_shape(v, &ty, &tz);
  std::vector<std::array<CUtensorMap, 5>> maps(g->npatches);
  for (int p = 0; p < g->npatches; ++p) {
    const DevPatch& P = g->hp[p];
    float2* bufs[5] = {P.hl[0], P.hl[1], P.hl[2], P.sa, P.sb};
    const cuuint64_t dims[3] = {(cuuint64_t)2 * (P.NX + 1), (cuuint64_t)P.NY, (cuuint64_t)NF * P.NZ};
    const cuuint64_t strides[2] = {(cuuint64_t)P.px * 8, (cuuint64_t)P.plane * 8};
    const cuuint32_t box[3] = {80, (cuuint32_t)(ty + 6), (cuuint32_t)(tz + 6)};
    const cuuint32_t es[3] = {1, 1, 1};
    for (int b = 0; b < 5; ++b) {
      CUresult r = enc(&maps[p][b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)(bufs[b] - 1), dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(g, SACRAK_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
  }
  const int nb = tma_setup_variant(v);
  if (nb <= 0) {
    cudaGetLastError();
    return fail(g, SACRAK_ECUDA, "TMA stage kernel %d cannot be resident", v + 1);
  }
  if (g->nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g->nsm <= 0)
      return fail(g, SACRAK_ECUDA, "cannot read the SM count");
  }
  g->maps[v] = std::move(maps);
  g->tma_blocks[v] = nb;
  return SACRAK_OK;
}

void launch_stage(sacrak_grid* g, const StageArgs& a, long long zones, const std::vector<int>& pids,
                  int kernel) {
  if (g->prof) {
    if (g->ev_used == g->ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> p;
      cudaEventCreate(&p.first);
      cudaEventCreate(&p.second);
      g->ev.push_back(p);
    }
    cudaEventRecord(g->ev[g->ev_used].first, g->stream);
  }
  if (g->prm.precision == 1 && kernel >= 1 && kernel <= TMA_NVARIANTS) {
    const int v = kernel - 1;
    int ty, tz;
    tma_variant_shape(v, &ty, &tz);
    TmaStageArgs t;
    std::memset(&t, 0, sizeof t);
    t.st = a;
    t.np = (int)pids.size();
    int acc = 0;
    for (int i = 0; i < t.np; ++i) {
      const DevPatch& P = g->hp[pids[i]];
      t.pid[i] = pids[i];
      t.tstart[i] = acc;
      t.ntx[i] = (P.n[0] + 31) / 32;
      t.nty[i] = (P.n[1] + ty - 1) / ty;
      t.nz[i] = P.NZ;
      acc += t.ntx[i] * t.nty[i] * ((P.n[2] + tz - 1) / tz);
      for (int b = 0; b < 5; ++b) t.map[i][b] = g->maps[v][pids[i]][b];
    }
    t.tstart[t.np] = acc;
    t.ntiles = acc;
    t.wait_cycles = g->tma_wait_cycles != 0 ? g->tma_wait_cycles : TMA_WAIT_CYCLES;
    const long long res = (long long)g->nsm * g->tma_blocks[v];
    const int grid = (int)(acc < res ? acc : res);
    if (grid > 0) launch_stage_tma(v, t, grid, g->stream);
  } else if (g->prm.precision == 1 && ldg_variant(kernel) >= 0) {
    launch_stage_ldg(ldg_variant(kernel), a, g->stream);
  } else if (g->prm.precision == 1 && (kernel == K_LDG_FIX || kernel == K_LDG_FIX4)) {
    // the instance of the level's pitches, else the same kernel with runtime pitches
    const bool four = kernel == K_LDG_FIX4;
    long long sy, sz;
    level_pitches(g, pids, &sy, &sz);
    if (!launch_stage_fixed(a, sy, sz, four ? 4 : 3, g->stream)) launch_stage_ldg(ldg_variant(K_LDG_PFZ), a, g->stream);
  } else if (g->prm.precision == 1 && pair_variant(kernel) >= 0) {
    launch_stage_pair(pair_variant(kernel), a, g->stream);
  } else if (g->prm.precision == 1 && kernel == K_SPLIT) {
    launch_stage_split(a, g->d_dslot, g->stream);
  } else if (g->prm.precision == 1) {
    launch_stage_mixed(a, g->stream);
  } else {
    launch_stage_fp64(a, g->stream);
  }
  if (g->prof) {
    cudaEventRecord(g->ev[g->ev_used].second, g->stream);
    g->ev_used++;
    g->prof_zones += zones;
  }
}

// select the stage kernel of a level (0 direct, 1.. TMA variant + 1)
// forget the captured coarse step (its launches no longer match the grid)
void drop_graph(sacrak_grid* g) {
  if (!g->graph_exec) return;
  cudaGraphExecDestroy(g->graph_exec);
  cudaGraphDestroy(g->graph);
  g->graph_exec = nullptr;
  g->graph = nullptr;
}

sacrak_status select_kernel(sacrak_grid* g, int l, int kernel) {
  if (!kernel_eligible(g, kernel, g->lvl_ids[l]))
    return fail(g, SACRAK_EINVAL, "kernel %d not usable on level %d", kernel, l);
  if (kernel >= 1 && kernel <= TMA_NVARIANTS) {
    sacrak_status st = ensure_maps(g, kernel - 1);
    if (st != SACRAK_OK) return st;
  }
  if (kernel == K_LDG_FIX || kernel == K_LDG_FIX4) {
    static bool done[64][2] = {};  // shared-memory opt-in of the instances and of their fallback, once per device
    const bool four = kernel == K_LDG_FIX4;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done[dev][four]) {
      if (!fixed_setup(four ? 4 : 3) || !ldg_setup(ldg_variant(K_LDG_PFZ)))
        return fail(g, SACRAK_ECUDA, "stage kernel %d setup failed", kernel);
      if (dev >= 0 && dev < 64) done[dev][four] = true;
    }
  }
  if (ldg_variant(kernel) >= 0) {
    static bool done[64][10] = {};  // shared-memory opt-in (and resident grid), once per device
    const int v = ldg_variant(kernel);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done[dev][v]) {
      if (!ldg_setup(v)) return fail(g, SACRAK_ECUDA, "stage kernel %d setup failed", kernel);
      if (dev >= 0 && dev < 64) done[dev][v] = true;
    }
  }
  if (pair_variant(kernel) >= 0) {
    static bool done[64][3] = {};  // shared-memory opt-in, once per device
    const int v = pair_variant(kernel);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done[dev][v]) {
      if (!pair_setup(v)) return fail(g, SACRAK_ECUDA, "stage kernel %d setup failed", kernel);
      if (dev >= 0 && dev < 64) done[dev][v] = true;
    }
  }
  if (g->lvl_kernel[l] != kernel) drop_graph(g);  // the captured coarse step used the old kernel
  g->lvl_kernel[l] = kernel;
  return SACRAK_OK;
}

// Time weights of the parent's (oldest, middle, newest) levels for the ghost
// data of child RK stage `stage` (1..4) of a child step that starts at
// fraction s0 of the parent's last step and lasts ds: the parent's time
// interpolant -- quadratic through s = -1, 0, 1 once three levels exist,
// linear through s = 0, 1 before (Sec. 2.2.1) -- evaluated at the stage time
// s0 + c_s ds, c = (0, 1/2, 1/2, 1).  stage 0 asks for s0 itself.
void ghost_time_weights(double s0, double ds, int stage, double wq[3], double wl[3]) {
  static const double cf[5] = {0.0, 0.0, 0.5, 0.5, 1.0};
  const double s = s0 + cf[stage] * ds;
  wq[0] = s * (s - 1.0) * 0.5;
  wq[1] = (1.0 - s) * (1.0 + s);
  wq[2] = s * (s + 1.0) * 0.5;
  wl[0] = 0.0;
  wl[1] = 1.0 - s;
  wl[2] = s;
}

FillArgs fill_args(sacrak_grid* g, int l, int mode, int stage, double s0, double ds = 0.0) {
  FillArgs a;
  a.patches = g->d_patches;
  a.patch_ids = g->d_ids + g->lvl_id_off[l];
  a.lev = g->d_levels + l;
  a.plev = l > 0 ? g->d_levels + (l - 1) : nullptr;
  a.mode = mode;
  a.stage = stage;
  ghost_time_weights(s0, ds, mode == 0 ? stage : 0, a.wq, a.wl);
  a.mixed = g->prm.precision == 1;
  a.dual = 0;
  return a;
}

void release_side(sacrak_grid* g) {
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  if (g->side) cudaStreamDestroy(g->side);
  g->ev_fork = g->ev_join = nullptr;
  g->side = nullptr;
}

// The main stream hands work to the side stream (fork) and waits for all of
// it (join).  Both are stream-ordered event operations, so they become graph
// edges under capture.
void fork_side(sacrak_grid* g) {
  cudaEventRecord(g->ev_fork, g->stream);
  cudaStreamWaitEvent(g->side, g->ev_fork, 0);
  g->side_live = true;
}
void join_side(sacrak_grid* g) {
  if (!g->side_live) return;
  cudaEventRecord(g->ev_join, g->side);
  cudaStreamWaitEvent(g->stream, g->ev_join, 0);
  g->side_live = false;
}

// time fill of a refined level's ghosts from the cached prolongations, for
// the buffer given by (mode, stage); the child step starts at fraction s0 of
// the parent step and lasts ds; dual: the stage-2 input and the stage-3
// input together (stages 2 and 3 share their time)
void time_fill(sacrak_grid* g, int l, int mode, int stage, double s0, double ds, bool dual, cudaStream_t st) {
  FillArgs fa = fill_args(g, l, mode, stage, s0, ds);
  fa.dual = dual;
  launch_fill(FILL_PROLONG, fa, (int)g->lvl_ids[l].size(), g->lvl_max_shell[l], st);
}

// same-level exchange between every overlapping pair of level l
void exchange_level(sacrak_grid* g, int l, int mode, int stage) {
  const auto& ids = g->lvl_ids[l];
  for (size_t a = 0; a < ids.size(); ++a)
    for (size_t b = a + 1; b < ids.size(); ++b) {
      const DevPatch& A = g->hp[ids[a]];
      const DevPatch& B = g->hp[ids[b]];
      int off[3];
      bool touch = true;
      for (int d = 0; d < 3; ++d) {
        off[d] = (int)std::llround((A.origin[d] - B.origin[d]) / A.dx);
        // index ranges incl. ghosts overlap?
        int alo = -GH + off[d], ahi = A.n[d] + GH - 1 + off[d];
        int blo = -GH, bhi = B.n[d] + GH - 1;
        if (ahi < blo || bhi < alo) touch = false;
      }
      if (!touch) continue;
      ExchArgs e;
      e.patches = g->d_patches;
      e.lev = g->d_levels + l;
      e.a = ids[a];
      e.b = ids[b];
      for (int d = 0; d < 3; ++d) e.off[d] = off[d];
      e.mode = mode;
      e.stage = stage;
      e.mixed = g->prm.precision == 1;
      launch_exchange(e, (long long)A.NX * A.NY * A.NZ, g->stream);
    }
}

// ghost fill of level l for the buffer given by (mode, stage); for levels
// > 0 the child step starts at fraction s0 of the parent step and lasts ds
// prolong: 0 skip the time fill (exchange only), 1 fill, 2 fill the stage-2
// input and the stage-3 input together (stages 2 and 3 share their time)
void fill_ghosts(sacrak_grid* g, int l, int mode, int stage, double s0, double ds, int prolong = 1) {
  const int np = (int)g->lvl_ids[l].size();
  if (l == 0) {
    if (g->prm.bc == 1)
      launch_fill(FILL_PERIODIC, fill_args(g, l, mode, stage, 0.0), np, g->lvl_max_shell[l], g->stream);
    else if (g->prm.bc == 2)
      launch_fill(FILL_FROZEN, fill_args(g, l, mode, stage, 0.0), np, g->lvl_max_shell[l], g->stream);
    return;
  }
  if (prolong) time_fill(g, l, mode, stage, s0, ds, prolong == 2, g->stream);
  exchange_level(g, l, mode, stage);
}

// equatorial reflection of the level's z < 0 ghosts in the (mode, stage) buffer
void zreflect(sacrak_grid* g, int l, int mode, int stage) {
  if (!g->prm.zsym) return;
  launch_zreflect(fill_args(g, l, mode, stage, 0.0), (int)g->lvl_ids[l].size(), g->lvl_max_zslab[l], g->stream);
}

MatterAmrArgs matter_amr_args(const sacrak_grid* g, int l) {
  MatterAmrArgs a;
  a.patches = g->d_patches;
  a.child_ids = g->d_ids + g->lvl_id_off[l];
  a.plev = g->d_levels + (l - 1);
  a.clev = g->d_levels + l;
  a.dt_parent = level_dt(g, l - 1);
  return a;
}

// the fluid of level l-1's current slot prolonged onto level l's ghost shells
void refresh_matter_shells(sacrak_grid* g, int l) {
  if (!g->prm.matter || l <= 0 || l >= g->nlevels) return;
  launch_matter_prolong(matter_amr_args(g, l), (int)g->lvl_ids[l].size(), g->lvl_max_shell[l], g->stream);
}

// spatial prolongation of level l-1's current slot onto level l's shells
// (on the side stream with overlap: the children's first stage-2 fill, also
// on the side stream, is the first reader of the new slot's cache)
void refresh_shells(sacrak_grid* g, int l, bool side = false) {
  if (l <= 0 || l >= g->nlevels) return;
  if (side) fork_side(g);
  launch_prolong_space(g->d_patches, g->d_ids + g->lvl_id_off[l], g->d_levels + (l - 1),
                       (int)g->lvl_ids[l].size(), g->lvl_max_clusters[l], g->prm.precision == 1,
                       side ? g->side : g->stream);
}

MatterArgs matter_args(const sacrak_grid* g, int pid, int stage, double dt, double s0, double ds, int wstage);

// after new data: every child level's cache for its parent's current slot,
// and (mixed precision) the hi/lo split of every current level
void refresh_all_shells(sacrak_grid* g) {
  if (g->prm.zsym && (g->split_dirty || g->shells_dirty))  // new data: mirror it first
    for (int l = 0; l < g->nlevels; ++l) zreflect(g, l, 1, 0);
  if (g->prm.precision == 1 && g->split_dirty) {
    for (int p = 0; p < g->npatches; ++p) {
      const DevPatch& P = g->hp[p];
      launch_split(g->d_patches, g->d_levels, p, (long long)P.NX * P.NY * P.NZ, g->stream);
    }
    g->split_dirty = false;
  }
  if (g->prm.matter && g->matter_ready && g->matter_shells_dirty) {
    if (g->prm.zsym)  // new fluid data: mirror it first
      for (int p = 0; p < g->npatches; ++p) launch_matter_zreflect(matter_args(g, p, 0, 0.0, 1.0, 0.0, 0), g->stream);
    for (int l = 1; l < g->nlevels; ++l) refresh_matter_shells(g, l);
    g->matter_shells_dirty = false;
  }
  if (!g->shells_dirty) return;
  for (int l = 1; l < g->nlevels; ++l) refresh_shells(g, l);
  g->shells_dirty = false;
}

// the fluid of patch pid at RK stage `stage`; levels > 0 take their ghost
// cells from the parent at the time s0 + c ds (c = 0, 1/2, 1/2, 1 for the
// stage `wstage` = 1..4; 0 for wstage 0), s0 and ds locating the call in the
// parent's last step
MatterArgs matter_args(const sacrak_grid* g, int pid, int stage, double dt, double s0 = 1.0, double ds = 0.0,
                       int wstage = 0) {
  const DevPatch& P = g->hp[pid];
  MatterArgs a;
  std::memset(&a, 0, sizeof a);
  a.P = g->d_patches + pid;
  a.lev = g->d_levels + P.level;
  a.plev = P.level > 0 ? g->d_levels + (P.level - 1) : nullptr;
  ghost_time_weights(s0, ds, wstage, a.wq, a.wl);
  a.first_substep = s0 == 0.0;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = P.n[d];
    a.origin[d] = P.origin[d];
  }
  a.NX = P.NX;
  a.NY = P.NY;
  a.NZ = P.NZ;
  a.sy = P.px;
  a.sz = P.plane;
  a.fs = P.fstride;
  a.dx = P.dx;
  a.eos = g->eos;
  a.rho_atm = g->rho_atm;
  a.r_atm = g->r_atm;
  a.periodic = g->prm.bc == 1;
  a.stage = stage;
  a.coupled = 1;
  a.riemann = g->riemann;
  a.dt = dt;
  a.out = nullptr;
  a.err = g->d_err;
  return a;
}

// fluid of level l at RK stage s (0: the current level, 5: the new level):
// recovery (atmosphere, Z4c matter terms) and the primitives' ghost cells
// (levels > 0: from the parent at time s0 + c(wstage) ds of its last step)
void matter_recover(sacrak_grid* g, int l, int s, double dt, double s0 = 1.0, double ds = 0.0, int wstage = 0) {
  for (int pid : g->lvl_ids[l]) {
    const MatterArgs a = matter_args(g, pid, s, dt, s0, ds, wstage);
    launch_matter_prep(a, g->stream);
    if (l == 0)
      launch_matter_ghosts(a, g->stream);
    else
      launch_matter_child_ghosts(a, g->stream);
    // equatorial symmetry: after the other ghost treatments (patches on z = 0)
    if (g->prm.zsym) launch_matter_zreflect(a, g->stream);
  }
}

// face fluxes and the stage update of the fluid (s = 0: d_t into out)
void matter_advance(sacrak_grid* g, int l, int s, double dt, double* out = nullptr, double s0 = 1.0) {
  for (int pid : g->lvl_ids[l]) {
    MatterArgs a = matter_args(g, pid, s, dt, s0);
    a.out = out;
    for (int d = 0; d < 3; ++d) launch_matter_flux(a, d, g->stream);
    launch_matter_update(a, g->stream);
  }
}

void rk4_level(sacrak_grid* g, int l, double dt, double frac0, double dfrac) {
  const int np = (int)g->lvl_ids[l].size();
  // refined levels with overlap: the time fill of stage 2 (with stage 3's)
  // runs on the side stream beside the stage-1 kernel, the one of stage 4
  // beside the stage-3 kernel.  Each writes only ghost cells, of buffers that
  // the concurrent kernel neither reads nor writes (stage kernels write
  // active cells only); the same-level exchange, which reads active cells of
  // the stage input, follows the join on the main stream.
  const bool ov = g->overlap && l > 0;
  for (int s = 1; s <= 4; ++s) {
    if (!(l == 0 && (g->prm.bc == 0 || (g->prm.bc == 2 && s == 1)))) {
      if (ov && (s == 2 || s == 4)) {
        join_side(g);
        exchange_level(g, l, 0, s);
      } else {
        fill_ghosts(g, l, 0, s, frac0, dfrac, l > 0 ? (s == 2 ? 2 : (s == 3 ? 0 : 1)) : 1);
      }
    }
    zreflect(g, l, 0, s);  // equatorial symmetry: after every other ghost treatment
    // the fluid of this stage: primitives and the Z4c matter terms first
    if (g->prm.matter) matter_recover(g, l, s, dt, frac0, dfrac, s);
    StageArgs a;
    a.tiles = g->d_tiles + g->lvl_tile_off[l];
    a.ntiles = (int)g->lvl_ntiles[l];
    a.patches = g->d_patches;
    a.lev = g->d_levels + l;
    a.stage = s;
    a.dt = dt;
    a.prm = dev_params(g->prm);
    a.err = g->d_err;
    const bool fill_next = ov && (s == 1 || s == 3);
    if (fill_next) fork_side(g);  // recorded before the stage kernel: the fill does not wait for it
    launch_stage(g, a, g->lvl_zones[l], g->lvl_ids[l], g->lvl_kernel[l]);
    if (fill_next) time_fill(g, l, 0, s + 1, frac0, dfrac, s == 1, g->side);
    if (l == 0 && g->prm.bc == 0) {
      GhostArgs ga;
      ga.patches = g->d_patches;
      ga.patch_ids = g->d_ids + g->lvl_id_off[l];
      ga.lev = g->d_levels + l;
      ga.stage = s;
      ga.dt = dt;
      ga.prm = a.prm;
      ga.err = g->d_err;
      if (g->prm.precision == 1)
        launch_sommerfeld_mixed(ga, np, g->lvl_max_shell[l], g->stream);
      else
        launch_sommerfeld(ga, np, g->lvl_max_shell[l], g->stream);
    }
    if (g->prm.matter) matter_advance(g, l, s, dt, nullptr, frac0);  // on this stage's metric
  }
  if (g->prm.matter) matter_recover(g, l, 5, dt, frac0, dfrac, 4);  // primitives of the new level
  // ghosts of the new time level for periodic / frozen outer boundaries
  if (l == 0 && g->prm.bc == 1)
    launch_fill(FILL_PERIODIC, fill_args(g, l, 2, 4, 0.0), np, g->lvl_max_shell[l], g->stream);
  if (l == 0 && g->prm.bc == 2)
    launch_fill(FILL_FROZEN, fill_args(g, l, 2, 4, 0.0), np, g->lvl_max_shell[l], g->stream);
  // the new level's z < 0 ghosts mirror its new values (the children's
  // prolongation reads those parent cells)
  zreflect(g, l, 2, 4);
  for (int p = 0; p < g->npunct; ++p)
    if (g->hpunct[p].level == l) {  // the punctures tracked on this level
      TrackArgs ta;
      ta.patches = g->d_patches;
      ta.levels = g->d_levels;
      ta.punct = g->d_punct;
      ta.np = g->npunct;
      ta.level = l;
      ta.dt = dt;
      ta.err = g->d_err;
      launch_track(ta, g->stream);
      break;
    }
  // work on the side stream reads this level's ring index (the prolongation
  // of its restricted slot): it ends before the ring advances
  join_side(g);
  launch_level_advance(g->d_levels + l, dt, g->stream);
  refresh_shells(g, l + 1, g->overlap);  // the children's cache of this level's new slot
  refresh_matter_shells(g, l + 1);
}

// do two patches of level l share active cells (the exchange then averages
// them, changing active data that the next level's prolongation reads)?
bool active_overlap(const sacrak_grid* g, int l) {
  const auto& ids = g->lvl_ids[l];
  for (size_t a = 0; a < ids.size(); ++a)
    for (size_t b = a + 1; b < ids.size(); ++b) {
      const DevPatch& A = g->hp[ids[a]];
      const DevPatch& B = g->hp[ids[b]];
      bool ov = true;
      for (int d = 0; d < 3; ++d) {
        const int off = (int)std::llround((A.origin[d] - B.origin[d]) / A.dx);
        if (!(off < B.n[d] && off + A.n[d] > 0)) ov = false;
      }
      if (ov) return true;
    }
  return false;
}

void level_step_rec(sacrak_grid* g, int l, double frac0, double dfrac) {
  rk4_level(g, l, level_dt(g, l), frac0, dfrac);
  if (l + 1 < g->nlevels) {
    level_step_rec(g, l + 1, 0.0, 0.5);
    level_step_rec(g, l + 1, 0.5, 0.5);
    const int nc = (int)g->lvl_ids[l + 1].size();
    fill_ghosts(g, l + 1, 1, 0, 1.0, 0.0);  // prolongation (unrestricted parent) + exchange
    zreflect(g, l + 1, 1, 0);
    // the exchange averaged shared active cells of level l+1: its children
    // cache that slot again
    if (l + 2 < g->nlevels && active_overlap(g, l + 1)) refresh_shells(g, l + 2);
    launch_fill(FILL_RESTRICT, fill_args(g, l + 1, 1, 0, 0.0), nc, g->lvl_max_restrict[l + 1],
                g->stream);
    if (g->prm.matter) {
      // the fluid (Sec. 2.2.1): volume-averaged restriction, reflux (one child
      // at a time), the parent's primitives of the corrected level, and the
      // children's cache of it
      const MatterAmrArgs ma = matter_amr_args(g, l + 1);
      launch_matter_restrict(ma, nc, g->lvl_max_restrict[l + 1], g->stream);
      for (int c = 0; c < nc; ++c) {
        MatterAmrArgs one = ma;
        one.child_ids = ma.child_ids + c;
        const DevPatch& C = g->hp[g->lvl_ids[l + 1][c]];
        const long long nf = 2LL * ((long long)(C.n[1] / 2) * (C.n[2] / 2) + (long long)(C.n[0] / 2) * (C.n[2] / 2) +
                                    (long long)(C.n[0] / 2) * (C.n[1] / 2));
        launch_matter_reflux(one, 1, nf, g->stream);
      }
      matter_recover(g, l, 0, 0.0, frac0, dfrac, 4);
      refresh_matter_shells(g, l + 1);
    }
    zreflect(g, l, 1, 0);      // restricted cells next to z = 0 have mirrors among the ghosts
    // the restricted slot, for the next parent step: with overlap on the side
    // stream, beside the parent's next step, joined before that step
    // advances the parent's ring (the kernel reads the ring); it reads only
    // the parent's active cells, which that step does not change, and its
    // readers, the children's time fills, come later.  Not under equatorial
    // symmetry: there it also reads the parent's reflected z < 0 ghosts,
    // which the parent's next stage-1 time fill rewrites before reflecting.
    refresh_shells(g, l + 1, g->overlap && !g->prm.zsym);
  }
}

// ---- moving boxes (Sec. 2.2.1) ----

int floor_div2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

// smallest offset (parent cells) of child c along d inside par: 4, or 0 for
// a child that starts on the equator with its parent under equatorial symmetry
int nest_lo(const sacrak_grid* g, const DevPatch& c, const DevPatch& par, int d, int off) {
  return (g->prm.zsym && d == 2 && c.zrefl && par.zrefl && off == 0) ? 0 : 4;
}

std::vector<int> children_of(const sacrak_grid* g, int pid, bool only_fixed) {
  std::vector<int> k;
  for (int q = 0; q < g->npatches; ++q)
    if (g->hp[q].parent == pid && (!only_fixed || (g->follow[q] < 0 && g->follow_star[q] < 0))) k.push_back(q);
  return k;
}

// the shifts (parent cells) per axis that keep patch pid (geometry geo[pid])
// nested in geo[parent] and the children kids nested in it; no z shifts
// under equatorial symmetry (punctures on the equator stay there)
void shift_range(const sacrak_grid* g, int pid, const std::vector<DevPatch>& geo, const std::vector<int>& kids,
                 int lo[3], int hi[3]) {
  const DevPatch& c = geo[pid];
  const DevPatch& par = geo[c.parent];
  for (int d = 0; d < 3; ++d) {
    const int off = (int)std::llround((c.origin[d] - par.origin[d]) / par.dx);
    int a = nest_lo(g, c, par, d, off) - off;
    int b = par.n[d] - 4 - c.n[d] / 2 - off;
    for (int kid : kids) {
      const DevPatch& k = geo[kid];
      const int koff = (int)std::llround((k.origin[d] - c.origin[d]) / c.dx);
      // the child's offset becomes koff - 2 s
      a = std::max(a, -floor_div2(c.n[d] - 4 - k.n[d] / 2 - koff));
      b = std::min(b, floor_div2(koff - nest_lo(g, k, c, d, koff)));
    }
    if (g->prm.zsym && d == 2) a = b = 0;
    lo[d] = a;
    hi[d] = b;
  }
}

// all levels at the same time (after whole coarse steps); lv gets the levels
sacrak_status synchronised(sacrak_grid* g, std::vector<DevLevel>& lv) {
  lv.resize(g->nlevels);
  CK(cudaMemcpyAsync(lv.data(), g->d_levels, sizeof(DevLevel) * g->nlevels, cudaMemcpyDeviceToHost, g->stream));
  CK(cudaStreamSynchronize(g->stream));
  for (int l = 1; l < g->nlevels; ++l)
    if ((long long)lv[l].steps != ((long long)lv[0].steps << l))
      return fail(g, SACRAK_EINVAL, "levels not synchronised (move patches between coarse steps)");
  return SACRAK_OK;
}

// shift patch pid by s parent cells: its current time level into the stage
// buffer (old active cells copied, the rest prolonged from the parent), back
// into the ring slot, then the geometry; the level's time-level history
// restarts
void apply_move(sacrak_grid* g, int pid, const int s[3], const std::vector<DevLevel>& lv) {
  DevPatch& C = g->hp[pid];
  MoveArgs a;
  a.patches = g->d_patches;
  a.levels = g->d_levels;
  a.patch = pid;
  for (int d = 0; d < 3; ++d) {
    a.sh[d] = 2 * s[d];
    a.noff[d] = C.off[d] + s[d];
  }
  a.skip_zlower = g->prm.zsym && C.zrefl;
  a.dst = C.buf[B_S0];
  a.err = g->d_err;
  launch_move(a, (long long)C.NX * C.NY * C.NZ, g->stream);
  cudaMemcpyAsync(C.buf[lv[C.level].ring], C.buf[B_S0], sizeof(double) * NF * C.fstride,
                  cudaMemcpyDeviceToDevice, g->stream);
  for (int d = 0; d < 3; ++d) {
    C.origin[d] = C.origin[d] + (2 * s[d]) * C.dx;
    C.off[d] += s[d];
  }
  for (int k : children_of(g, pid, false))
    for (int d = 0; d < 3; ++d) g->hp[k].off[d] -= 2 * s[d];
  cudaMemcpyAsync(g->d_patches, g->hp.data(), sizeof(DevPatch) * g->npatches, cudaMemcpyHostToDevice,
                  g->stream);
  launch_set_nvalid(g->d_levels + C.level, 1, g->stream);
  // where the parent level's patches share active cells, the exchange at the
  // start of each of its steps averaged them in place in its stored time
  // levels: caches of its older slots rebuilt now would differ from those
  // its children used, so its history restarts too.  With a fluid it
  // restarts as well: the fluid's primitives exist for the current time
  // level only, so the moved patch's cached prolongations of the parent's
  // older levels cannot be rebuilt
  if (active_overlap(g, C.level - 1) || g->prm.matter) launch_set_nvalid(g->d_levels + C.level - 1, 1, g->stream);
  zreflect(g, C.level, 1, 0);
  if (g->prm.matter) {
    // the fluid (Sec. 2.2.1): kept where active before and after, the
    // parent's prolongation elsewhere, into the face-flux arrays, then back
    MatterMoveArgs m;
    m.patches = g->d_patches;
    m.patch = pid;
    m.ring = lv[C.level].ring;
    m.pring = lv[C.level - 1].ring;
    for (int d = 0; d < 3; ++d) m.sh[d] = 2 * s[d];
    m.eos = g->eos;
    m.err = g->d_err;
    launch_matter_move(m, (long long)C.NX * C.NY * C.NZ, g->stream);
    cudaMemcpyAsync(C.mcons[m.ring], C.mflux, sizeof(double) * NM * C.fstride, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(C.mprim, C.mflux + NM * C.fstride, sizeof(double) * NMP * C.fstride, cudaMemcpyDeviceToDevice,
                    g->stream);
    if (g->prm.zsym) launch_matter_zreflect(matter_args(g, pid, 0, 0.0, 1.0, 0.0, 0), g->stream);
  }
  if (g->prm.precision == 1)
    launch_split(g->d_patches, g->d_levels, pid, (long long)C.NX * C.NY * C.NZ, g->stream);
}

// after moves: every child level's cache of all three parent slots (the
// fluid's: of the parent's current slot, the only valid one after a move),
// and no captured coarse step
void refresh_after_move(sacrak_grid* g) {
  for (int l = 1; l < g->nlevels; ++l)
    for (int back = 0; back < 3; ++back)
      launch_prolong_space(g->d_patches, g->d_ids + g->lvl_id_off[l], g->d_levels + (l - 1),
                           (int)g->lvl_ids[l].size(), g->lvl_max_clusters[l], g->prm.precision == 1,
                           g->stream, back);
  if (g->prm.matter)
    for (int l = 1; l < g->nlevels; ++l) refresh_matter_shells(g, l);
  drop_graph(g);
}

sacrak_status not_capturing(sacrak_grid* g) {
  cudaStreamCaptureStatus cs;
  CK(cudaStreamIsCapturing(g->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(g, SACRAK_ESTATE, "stream is being captured");
  return SACRAK_OK;
}

sacrak_status reset_levels(sacrak_grid* g) {
  std::vector<DevLevel> lv(g->nlevels);
  for (auto& x : lv) {
    x.ring = 0;
    x.nvalid = 1;
    x.steps = 0;
    x.pad_ = 0;
    x.t = 0.0;
  }
  CK(cudaMemcpyAsync(g->d_levels, lv.data(), sizeof(DevLevel) * g->nlevels, cudaMemcpyHostToDevice,
                     g->stream));
  CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), g->stream));
  g->invalid = false;
  return SACRAK_OK;
}

sacrak_status read_level(sacrak_grid* g, int l, DevLevel* out) {
  CK(cudaMemcpyAsync(out, g->d_levels + l, sizeof(DevLevel), cudaMemcpyDeviceToHost, g->stream));
  CK(cudaStreamSynchronize(g->stream));
  return SACRAK_OK;
}

}  // namespace

extern "C" {

size_t sacrak_arena_bytes(int nlevels, int npatches, const sacrak_patch_desc* patches,
                          const sacrak_params* params) {
  Layout L;
  std::string why;
  const int mixed = params ? (params->precision == 1) : 0;
  const int matter = params ? (params->matter != 0) : 0;
  if (!describe(nlevels, npatches, patches, mixed, matter, L, why)) return 0;
  return L.total;
}

sacrak_status sacrak_grid_create(int nlevels, double dx0, int npatches,
                                 const sacrak_patch_desc* pd, const sacrak_params* params,
                                 void* cuda_stream, void* device_arena, size_t arena_bytes,
                                 sacrak_grid** out) {
  if (!out || !params || !device_arena || !(dx0 > 0.0)) return SACRAK_EINVAL;
  *out = nullptr;
  Layout L;
  std::string why;
  if (params->matter < 0 || params->matter > 1) return SACRAK_EINVAL;
  if (!describe(nlevels, npatches, pd, params->precision == 1, params->matter, L, why)) return SACRAK_EINVAL;
  if (arena_bytes < L.total || ((uintptr_t)device_arena % 256) != 0) return SACRAK_EINVAL;
  const sacrak_params& p = *params;
  if (p.lapse < 0 || p.lapse > 1 || p.shift < 0 || p.shift > 1 || p.bc < 0 || p.bc > 2 ||
      p.precision < 0 || p.precision > 1 || !(p.courant > 0.0) || !(p.sigma_ko >= 0.0) || p.zsym < 0 ||
      p.zsym > 1 || (p.zsym && p.bc == 1))
    return SACRAK_EINVAL;

  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, device_arena) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return SACRAK_EINVAL;
  }

  sacrak_grid* g = new sacrak_grid();
  g->prm = p;
  g->stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    release_side(g);
    delete g;
    return SACRAK_ECUDA;
  }
  g->arena = (char*)device_arena;
  g->arena_bytes = arena_bytes;
  g->nlevels = nlevels;
  g->npatches = npatches;
  g->dx0 = dx0;
  g->L = L;
  g->hp.resize(npatches);
  g->lvl_ids.assign(nlevels, {});
  for (int i = 0; i < npatches; ++i) {
    DevPatch& P = g->hp[i];
    std::memset(&P, 0, sizeof P);
    for (int d = 0; d < 3; ++d) {
      P.n[d] = pd[i].n[d];
      P.origin[d] = pd[i].origin[d];
    }
    P.NX = P.n[0] + 2 * GH;
    P.NY = P.n[1] + 2 * GH;
    P.NZ = P.n[2] + 2 * GH;
    P.px = L.px[i];
    P.plane = (long long)P.px * P.NY;
    P.fstride = L.fstride[i];
    P.level = pd[i].level;
    P.dx = dx0 / std::ldexp(1.0, P.level);
    P.zrefl = (p.zsym && std::fabs(P.origin[2]) <= 1e-12 * P.dx) ? 1 : 0;
    P.parent = -1;
    // Every state buffer starts one element (8 bytes) past its 256-byte
    // aligned slot: active cell i of a row is then at element i + 4 of the
    // slot, so the pair of cells (2m, 2m+1) is one aligned 16-byte vector
    // (the pair stage kernels load them with 128-bit loads).  The row pitch
    // keeps a spare element, so every row stays inside its own pitch.
    for (int b = 0; b < NBUF; ++b)
      P.buf[b] = (double*)(g->arena + L.patch_state[i] + (size_t)b * NF * P.fstride * sizeof(double)) + 1;
    for (int b = 0; b < 3; ++b)
      P.gsh[b] = P.level > 0 ? (double*)(g->arena + L.patch_state[i] +
                                        (size_t)(NBUF + b) * NF * P.fstride * sizeof(double)) + 1
                             : nullptr;
    if (p.precision == 1) {
      const size_t nb = (size_t)(NBUF + (P.level > 0 ? 3 : 0)) * NF * P.fstride * sizeof(double);
      float2* m0 = (float2*)(g->arena + align_up(L.patch_state[i] + nb, 256));
      const size_t fl = (size_t)NF * P.fstride;
      for (int b = 0; b < 3; ++b) P.hl[b] = m0 + (size_t)b * fl + 1;
      P.sa = m0 + 3 * fl + 1;
      P.sb = m0 + 4 * fl + 1;
    }
    if (p.matter) {
      double* m0 = (double*)(g->arena + L.matter_state[i]);
      const size_t fl = (size_t)P.fstride;
      for (int b = 0; b < NBUF; ++b) P.mcons[b] = m0 + (size_t)b * NM * fl;
      P.mprim = m0 + (size_t)NBUF * NM * fl;
      P.mflux = P.mprim + (size_t)NMP * fl;
      P.mzsrc = P.mflux + (size_t)3 * NM * fl;
      for (int b = 0; b < 3; ++b) P.mgsh[b] = P.mzsrc + (size_t)(NZSRC + b * NM) * fl;
      P.mfs = P.mzsrc + (size_t)(NZSRC + 3 * NM) * fl;
      P.mfa = P.mfs + (size_t)3 * NM * fl;
    }
    g->lvl_ids[P.level].push_back(i);
  }
  // parents: the patch of the level above containing the child with margin
  for (int i = 0; i < npatches; ++i) {
    DevPatch& C = g->hp[i];
    if (C.level == 0) continue;
    for (int d = 0; d < 3; ++d)
      if (C.n[d] % 2) {
        release_side(g);
        delete g;
        return SACRAK_EINVAL;
      }
    for (int j : g->lvl_ids[C.level - 1]) {
      const DevPatch& P = g->hp[j];
      bool ok = true;
      int off[3];
      for (int d = 0; d < 3; ++d) {
        double t = (C.origin[d] - P.origin[d]) / P.dx;
        double r = std::floor(t + 0.5);
        if (std::fabs(t - r) > 1e-9) ok = false;
        off[d] = (int)r;
        // prolongation stencils need parent cells off-4 .. off+n/2+3 inside the
        // active region; with equatorial symmetry a child and its parent may
        // both start at z = 0 (the parent's reflected ghosts serve below)
        const bool zlow = d == 2 && C.zrefl && P.zrefl && off[d] == 0;
        if ((!zlow && off[d] - 4 < 0) || off[d] + C.n[d] / 2 + 3 > P.n[d] - 1) ok = false;
      }
      if (ok) {
        C.parent = j;
        for (int d = 0; d < 3; ++d) C.off[d] = off[d];
        break;
      }
    }
    if (C.parent < 0) {
      release_side(g);
      delete g;
      return SACRAK_EINVAL;
    }
  }
  // Sommerfeld ghosts use one-sided differences toward the origin: the
  // origin must lie inside every level-0 patch so that they stay in the array
  if (p.bc == 0)
    for (int i : g->lvl_ids[0])
      for (int d = 0; d < 3; ++d) {
        const DevPatch& P = g->hp[i];
        if (!((P.origin[d] < 0.0 || (d == 2 && P.zrefl)) && P.origin[d] + P.n[d] * P.dx > 0.0)) {
          release_side(g);
          delete g;
          return SACRAK_EINVAL;
        }
      }
  // a fluid on several levels: the patches of a level share no cells (each
  // parent cell is restricted from one child and refluxed once per face)
  if (p.matter)
    for (int l = 1; l < nlevels; ++l)
      if (active_overlap(g, l)) {
        release_side(g);
        delete g;
        return SACRAK_EINVAL;
      }
  g->d_patches = (DevPatch*)(g->arena + L.patches);
  g->d_levels = (DevLevel*)(g->arena + L.levels);
  g->d_ids = (int*)(g->arena + L.ids);
  g->d_tiles = (Tile*)(g->arena + L.tiles);
  g->d_err = (unsigned*)(g->arena + L.err);
  g->d_results = (double*)(g->arena + L.results);
  g->d_scratch = (double*)(g->arena + L.scratch);
  g->d_dslot = (float*)(g->arena + L.dslot);
  g->d_punct = (DevPunct*)(g->arena + L.punct);
  g->follow.assign(npatches, -1);
  g->follow_star.assign(npatches, -1);
  std::vector<int> ids;
  std::vector<Tile> tiles;
  g->lvl_id_off.resize(nlevels);
  g->lvl_tile_off.resize(nlevels);
  g->lvl_ntiles.resize(nlevels);
  g->lvl_max_shell.assign(nlevels, 0);
  g->lvl_zones.assign(nlevels, 0);
  g->lvl_max_clusters.assign(nlevels, 0);
  g->lvl_max_restrict.assign(nlevels, 0);
  g->lvl_max_zslab.assign(nlevels, 0);
  for (int l = 0; l < nlevels; ++l) {
    g->lvl_id_off[l] = (int)ids.size();
    g->lvl_tile_off[l] = tiles.size();
    for (int pid : g->lvl_ids[l]) {
      ids.push_back(pid);
      const DevPatch& P = g->hp[pid];
      for (int z = 0; z < P.n[2]; ++z)
        for (int y = 0; y < P.n[1]; y += TILE_Y)
          for (int x = 0; x < P.n[0]; x += TILE_X) tiles.push_back(Tile{pid, x, y, z});
      const long long zs = (long long)GH * P.NX * P.NY;
      if (zs > g->lvl_max_zslab[l]) g->lvl_max_zslab[l] = zs;
      long long sh = (long long)P.NX * P.NY * P.NZ - (long long)P.n[0] * P.n[1] * P.n[2];
      if (sh > g->lvl_max_shell[l]) g->lvl_max_shell[l] = sh;
      g->lvl_zones[l] += (long long)P.n[0] * P.n[1] * P.n[2];
      if (P.level > 0) {
        const long long nb = prolong_bricks(P.n[0], P.n[1], P.n[2]);
        if (nb > g->lvl_max_clusters[l]) g->lvl_max_clusters[l] = nb;
      }
      long long rs = (long long)(P.n[0] / 2) * (P.n[1] / 2) * (P.n[2] / 2);
      if (rs > g->lvl_max_restrict[l]) g->lvl_max_restrict[l] = rs;
    }
    g->lvl_ntiles[l] = tiles.size() - g->lvl_tile_off[l];
  }
  cudaStream_t s = g->stream;
  sacrak_status st = SACRAK_OK;
  if (cudaMemcpyAsync(g->d_patches, g->hp.data(), sizeof(DevPatch) * npatches,
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(g->d_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(g->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    st = SACRAK_ECUDA;
  if (st == SACRAK_OK) st = reset_levels(g);
  if (st == SACRAK_OK) {
    // tables must be on the device before the host vectors go away
    if (cudaStreamSynchronize(s) != cudaSuccess) st = SACRAK_ECUDA;
  }
  if (st == SACRAK_OK) st = sacrak_set_initial_data(g, 0, 0, nullptr, nullptr, 0, 1, 0, 0, 0);
  // default stage kernel (mixed precision): the L1-path kernel with packed
  // pair arithmetic that prefetches the next field's z arms and the RK
  // update's streaming reads, with the patch pitches fixed at compile time
  // and 4 CTAs per SM where the level's patches have an instance, else with
  // runtime pitches and 3 CTAs per SM
  g->lvl_kernel.assign(nlevels, 0);
  for (int l = 0; st == SACRAK_OK && l < nlevels; ++l)
    if (p.precision == 1) st = select_kernel(g, l, K_LDG_FIX4);
  if (st != SACRAK_OK) {
    cudaGetLastError();
    release_side(g);
    delete g;
    return st;
  }
  *out = g;
  return SACRAK_OK;
}

sacrak_status sacrak_grid_destroy(sacrak_grid* g) {
  if (!g) return SACRAK_EINVAL;
  release_side(g);
  for (auto& p : g->ev) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  if (g->graph_exec) cudaGraphExecDestroy(g->graph_exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return SACRAK_OK;
}

sacrak_status sacrak_set_initial_data(sacrak_grid* g, int kind, int npunct, const double* m,
                                      const double* pos, double gw_amp, double gw_len,
                                      double noise_amp, uint64_t seed, int symmetrise_pi) {
  if (!g) return SACRAK_EINVAL;
  if (kind < 0 || kind > 2 || npunct < 0 || npunct > 8 || (kind == 1 && (!m || !pos)) ||
      (kind == 2 && !(gw_len > 0.0)) || !(noise_amp >= 0.0))
    return fail(g, SACRAK_EINVAL, "invalid initial-data arguments");
  if (symmetrise_pi) {
    for (const DevPatch& P : g->hp)
      for (int d = 0; d < 2; ++d)
        if (std::fabs(P.origin[d] + 0.5 * P.n[d] * P.dx) > 1e-12 * P.dx)
          return fail(g, SACRAK_EINVAL, "pi symmetrisation needs patches centred on x = y = 0");
  }
  sacrak_status st = reset_levels(g);
  if (st != SACRAK_OK) return st;
  g->shells_dirty = true;
  g->split_dirty = true;
  InitArgs a;
  std::memset(&a, 0, sizeof a);
  a.patches = g->d_patches;
  a.levels = g->d_levels;
  a.kind = kind;
  a.npunct = kind == 1 ? npunct : 0;
  for (int i = 0; i < a.npunct; ++i) {
    a.m[i] = m[i];
    for (int d = 0; d < 3; ++d) a.pos[3 * i + d] = pos[3 * i + d];
  }
  a.gw_amp = gw_amp;
  a.gw_len = gw_len;
  a.noise_amp = noise_amp;
  a.seed = seed;
  for (int d = 0; d < 3; ++d) a.lo[d] = g->hp[g->lvl_ids[0][0]].origin[d];
  for (int p = 0; p < g->npatches; ++p) {
    const DevPatch& P = g->hp[p];
    launch_init(a, p, (long long)P.NX * P.NY * P.NZ, g->stream);
    if (symmetrise_pi) launch_symmetrise(g->d_patches, g->d_levels, p, (long long)(P.NX / 2) * P.NY * P.NZ, g->stream);
  }
  return check_launch(g);
}

static sacrak_status copy_patch(sacrak_grid* g, int patch, double* dst_dev_slot, const double* src,
                                double* dst, bool upload, int nfields = NF) {
  const DevPatch& P = g->hp[patch];
  size_t width = (size_t)P.NX * sizeof(double);
  size_t rows = (size_t)nfields * P.NY * P.NZ;
  cudaPointerAttributes at;
  const void* host_side = upload ? (const void*)src : (const void*)dst;
  const bool is_host = cudaPointerGetAttributes(&at, host_side) != cudaSuccess ||
                       at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
  cudaGetLastError();
  if (is_host) {
    // one contiguous host transfer through a free stage buffer of the patch,
    // repacked to / from the padded rows on the device
    double* stage = (dst_dev_slot == P.buf[B_S1]) ? P.buf[B_S0] : P.buf[B_S1];
    if (upload) {
      CK(cudaMemcpyAsync(stage, src, width * rows, cudaMemcpyHostToDevice, g->stream));
      launch_repack(dst_dev_slot, stage, (long long)rows, P.NX, P.px, 1, g->stream);
    } else {
      launch_repack(stage, dst_dev_slot, (long long)rows, P.NX, P.px, 0, g->stream);
      CK(cudaMemcpyAsync(dst, stage, width * rows, cudaMemcpyDeviceToHost, g->stream));
    }
    return check_launch(g);
  }
  if (upload)
    CK(cudaMemcpy2DAsync(dst_dev_slot, P.px * sizeof(double), src, width, width, rows,
                         cudaMemcpyDefault, g->stream));
  else
    CK(cudaMemcpy2DAsync(dst, width, dst_dev_slot, P.px * sizeof(double), width, rows,
                         cudaMemcpyDefault, g->stream));
  return SACRAK_OK;
}

sacrak_status sacrak_upload_fields(sacrak_grid* g, int patch, const double* src) {
  if (!g) return SACRAK_EINVAL;
  if (patch < 0 || patch >= g->npatches || !src) return fail(g, SACRAK_EINVAL, "bad patch or pointer");
  const DevPatch& P = g->hp[patch];
  DevLevel lv;
  sacrak_status st = read_level(g, P.level, &lv);
  if (st != SACRAK_OK) return st;
  st = copy_patch(g, patch, P.buf[lv.ring], src, nullptr, true);
  if (st != SACRAK_OK) return st;
  lv.nvalid = 1;
  g->shells_dirty = true;
  g->split_dirty = true;
  CK(cudaMemcpyAsync(&g->d_levels[P.level], &lv, sizeof lv, cudaMemcpyHostToDevice, g->stream));
  CK(cudaStreamSynchronize(g->stream));  // lv is a host stack variable
  g->invalid = false;
  CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), g->stream));
  return SACRAK_OK;
}

sacrak_status sacrak_download_fields(sacrak_grid* g, int patch, double* dst) {
  if (!g) return SACRAK_EINVAL;
  if (patch < 0 || patch >= g->npatches || !dst) return fail(g, SACRAK_EINVAL, "bad patch or pointer");
  const DevPatch& P = g->hp[patch];
  DevLevel lv;
  sacrak_status st = read_level(g, P.level, &lv);
  if (st != SACRAK_OK) return st;
  st = copy_patch(g, patch, P.buf[lv.ring], nullptr, dst, false);
  if (st != SACRAK_OK) return st;
  return sync_and_check(g);
}

sacrak_status sacrak_rhs(sacrak_grid* g, int patch, double* dst) {
  if (!g) return SACRAK_EINVAL;
  if (patch < 0 || patch >= g->npatches || !dst) return fail(g, SACRAK_EINVAL, "bad patch or pointer");
  if (g->invalid) return fail(g, SACRAK_ESTATE, "grid state invalid after an earlier error");
  const DevPatch& P = g->hp[patch];
  refresh_all_shells(g);
  CK(cudaMemsetAsync(P.buf[B_S1], 0, (size_t)NF * P.fstride * sizeof(double), g->stream));
  // launch over this patch's tiles only
  const int l = P.level;
  size_t first = g->lvl_tile_off[l], count = 0;
  {
    size_t acc = 0;
    for (int pid : g->lvl_ids[l]) {
      const DevPatch& Q = g->hp[pid];
      size_t t = (size_t)((Q.n[0] + TILE_X - 1) / TILE_X) * ((Q.n[1] + TILE_Y - 1) / TILE_Y) * Q.n[2];
      if (pid == patch) {
        first += acc;
        count = t;
        break;
      }
      acc += t;
    }
  }
  StageArgs a;
  a.tiles = g->d_tiles + first;
  a.ntiles = (int)count;
  a.patches = g->d_patches;
  a.lev = g->d_levels + l;
  a.stage = 0;
  a.dt = 0.0;
  a.prm = dev_params(g->prm);
  a.err = g->d_err;
  if (g->prm.matter) {
    if (!g->matter_ready) return fail(g, SACRAK_ESTATE, "no fluid uploaded (sacrak_upload_matter)");
    matter_recover(g, l, 0, 0.0);
  }
  launch_stage(g, a, (long long)P.n[0] * P.n[1] * P.n[2], std::vector<int>{patch}, g->lvl_kernel[l]);
  sacrak_status st = check_launch(g);
  if (st != SACRAK_OK) return st;
  st = copy_patch(g, patch, P.buf[B_S1], nullptr, dst, false);
  if (st != SACRAK_OK) return st;
  return sync_and_check(g);
}

sacrak_status sacrak_rk4_step(sacrak_grid* g, int level, double dt) {
  if (!g) return SACRAK_EINVAL;
  if (level < 0 || level >= g->nlevels) return fail(g, SACRAK_EINVAL, "bad level");
  if (g->invalid) return fail(g, SACRAK_ESTATE, "grid state invalid after an earlier error");
  if (g->prm.matter && !g->matter_ready) return fail(g, SACRAK_ESTATE, "no fluid uploaded (sacrak_upload_matter)");
  refresh_all_shells(g);
  rk4_level(g, level, dt > 0.0 ? dt : level_dt(g, level), 0.0, 0.5);
  join_side(g);
  return check_launch(g);
}

sacrak_status sacrak_level_step(sacrak_grid* g, int level) {
  if (!g) return SACRAK_EINVAL;
  if (level < 0 || level >= g->nlevels) return fail(g, SACRAK_EINVAL, "bad level");
  if (g->invalid) return fail(g, SACRAK_ESTATE, "grid state invalid after an earlier error");
  if (g->prm.matter && !g->matter_ready) return fail(g, SACRAK_ESTATE, "no fluid uploaded (sacrak_upload_matter)");
  refresh_all_shells(g);  // eager, outside any graph
  if (level > 0 || g->stream == nullptr || g->prof) {
    level_step_rec(g, level, 0.0, 0.5);
    join_side(g);
    return check_launch(g);
  }
  if (!g->graph_exec) {
    cudaStreamCaptureStatus cs;
    CK(cudaStreamIsCapturing(g->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) {  // caller is capturing: just record launches
      level_step_rec(g, 0, 0.0, 1.0);
      join_side(g);
      return check_launch(g);
    }
    CK(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    level_step_rec(g, 0, 0.0, 1.0);
    join_side(g);
    cudaGraph_t graph;
    cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
    if (e != cudaSuccess) return fail(g, SACRAK_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&g->graph_exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return fail(g, SACRAK_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    g->graph = graph;
  }
  CK(cudaGraphLaunch(g->graph_exec, g->stream));
  return SACRAK_OK;
}

// ---- matter (Sec. 2.1.2, 2.2) ----

sacrak_status sacrak_set_eos(sacrak_grid* g, int npieces, double K0, const double* gammas, const double* rho_bounds,
                             double gamma_th) {
  if (!g) return SACRAK_EINVAL;
  if (!g->prm.matter) return fail(g, SACRAK_EINVAL, "grid created without a fluid (params.matter = 0)");
  if (npieces < 1 || npieces > MAX_PIECES || !gammas || (npieces > 1 && !rho_bounds) || !(K0 >= 0.0) ||
      !(gamma_th > 1.0) || !std::isfinite(K0) || !std::isfinite(gamma_th))
    return fail(g, SACRAK_EINVAL, "bad EOS parameters");
  DevEOS e;
  std::memset(&e, 0, sizeof e);
  e.n = npieces;
  e.gth = gamma_th;
  for (int i = 0; i < npieces; ++i) {
    if (!(gammas[i] > 1.0) || !std::isfinite(gammas[i])) return fail(g, SACRAK_EINVAL, "polytrope index <= 1");
    e.G[i] = gammas[i];
  }
  for (int i = 0; i + 1 < npieces; ++i) {
    if (!(rho_bounds[i] > 0.0) || (i > 0 && !(rho_bounds[i] > rho_bounds[i - 1])))
      return fail(g, SACRAK_EINVAL, "piece boundaries must be positive and increasing");
    e.rb[i] = rho_bounds[i];
  }
  // continuity of P and eps_cold at the boundaries fixes K_i and a_i
  e.K[0] = K0;
  e.a[0] = 0.0;
  for (int i = 1; i < npieces; ++i) {
    const double rb = e.rb[i - 1], g0 = e.G[i - 1], g1 = e.G[i];
    e.K[i] = e.K[i - 1] * std::pow(rb, g0 - g1);
    const double eprev = e.a[i - 1] + e.K[i - 1] * std::pow(rb, g0 - 1.0) / (g0 - 1.0);
    e.a[i] = eprev - e.K[i] * std::pow(rb, g1 - 1.0) / (g1 - 1.0);
  }
  g->eos = e;
  g->eos_set = true;
  drop_graph(g);  // the captured launches hold the old EOS
  return SACRAK_OK;
}

sacrak_status sacrak_set_atmosphere(sacrak_grid* g, double rho_atm, double r_atm) {
  if (!g) return SACRAK_EINVAL;
  if (!g->prm.matter) return fail(g, SACRAK_EINVAL, "grid created without a fluid (params.matter = 0)");
  if (!(rho_atm > 0.0) || !(r_atm > 0.0) || !std::isfinite(rho_atm) || !std::isfinite(r_atm))
    return fail(g, SACRAK_EINVAL, "atmosphere density and radius must be positive");
  g->rho_atm = rho_atm;
  g->r_atm = r_atm;
  drop_graph(g);
  return SACRAK_OK;
}

sacrak_status sacrak_set_riemann(sacrak_grid* g, int solver) {
  if (!g) return SACRAK_EINVAL;
  if (!g->prm.matter) return fail(g, SACRAK_EINVAL, "grid created without a fluid (params.matter = 0)");
  if (solver != 0 && solver != 1) return fail(g, SACRAK_EINVAL, "Riemann solver must be 0 (HLLC) or 1 (HLLE)");
  g->riemann = solver;
  drop_graph(g);
  return SACRAK_OK;
}

sacrak_status sacrak_upload_matter(sacrak_grid* g, int patch, const double* prim) {
  if (!g) return SACRAK_EINVAL;
  if (!g->prm.matter) return fail(g, SACRAK_EINVAL, "grid created without a fluid (params.matter = 0)");
  if (patch < 0 || patch >= g->npatches || !prim) return fail(g, SACRAK_EINVAL, "bad patch or pointer");
  if (!g->eos_set || !(g->rho_atm > 0.0)) return fail(g, SACRAK_ESTATE, "set the EOS and the atmosphere first");
  const DevPatch& P = g->hp[patch];
  sacrak_status st = copy_patch(g, patch, P.mprim, prim, nullptr, true, NM);
  if (st != SACRAK_OK) return st;
  launch_matter_prim2con(matter_args(g, patch, 0, 0.0), g->stream);
  st = check_launch(g);
  if (st != SACRAK_OK) return st;
  g->matter_ready = true;
  g->matter_shells_dirty = true;
  drop_graph(g);
  return sync_and_check(g);
}

sacrak_status sacrak_download_matter(sacrak_grid* g, int patch, double* prim) {
  if (!g) return SACRAK_EINVAL;
  if (!g->prm.matter) return fail(g, SACRAK_EINVAL, "grid created without a fluid (params.matter = 0)");
  if (patch < 0 || patch >= g->npatches || !prim) return fail(g, SACRAK_EINVAL, "bad patch or pointer");
  if (!g->matter_ready) return fail(g, SACRAK_ESTATE, "no fluid uploaded (sacrak_upload_matter)");
  const DevPatch& P = g->hp[patch];
  sacrak_status st = copy_patch(g, patch, P.mprim, nullptr, prim, false, NM);
  if (st != SACRAK_OK) return st;
  return sync_and_check(g);
}

sacrak_status sacrak_matter_rhs(sacrak_grid* g, int patch, double* rhs) {
  if (!g) return SACRAK_EINVAL;
  if (!g->prm.matter) return fail(g, SACRAK_EINVAL, "grid created without a fluid (params.matter = 0)");
  if (patch < 0 || patch >= g->npatches || !rhs) return fail(g, SACRAK_EINVAL, "bad patch or pointer");
  if (!g->matter_ready) return fail(g, SACRAK_ESTATE, "no fluid uploaded (sacrak_upload_matter)");
  if (g->invalid) return fail(g, SACRAK_ESTATE, "grid state invalid after an earlier error");
  const DevPatch& P = g->hp[patch];
  refresh_all_shells(g);  // (levels > 0: the fluid's ghost cells come from the parent's cache)
  CK(cudaMemsetAsync(P.buf[B_S1], 0, (size_t)NM * P.fstride * sizeof(double), g->stream));
  matter_recover(g, P.level, 0, 0.0);
  matter_advance(g, P.level, 0, 0.0, P.buf[B_S1]);
  sacrak_status st = check_launch(g);
  if (st != SACRAK_OK) return st;
  st = copy_patch(g, patch, P.buf[B_S1], nullptr, rhs, false, NM);
  if (st != SACRAK_OK) return st;
  return sync_and_check(g);
}

sacrak_status sacrak_constraints(sacrak_grid* g, int level, double w_excise, double out_l2[4]) {
  if (!g) return SACRAK_EINVAL;
  if (level < 0 || level >= g->nlevels || !out_l2) return fail(g, SACRAK_EINVAL, "bad arguments");
  ConsArgs a;
  a.tiles = g->d_tiles + g->lvl_tile_off[level];
  a.patches = g->d_patches;
  a.lev = g->d_levels + level;
  a.w_excise = w_excise;
  a.partial = g->d_scratch;
  launch_constraints(a, (int)g->lvl_ntiles[level], g->d_results, g->stream);
  sacrak_status st = check_launch(g);
  if (st != SACRAK_OK) return st;
  double sums[5];
  CK(cudaMemcpyAsync(sums, g->d_results, sizeof sums, cudaMemcpyDeviceToHost, g->stream));
  st = sync_and_check(g);
  if (st != SACRAK_OK) return st;
  for (int c = 0; c < 4; ++c) out_l2[c] = sums[4] > 0 ? std::sqrt(sums[c] / sums[4]) : 0.0;
  return SACRAK_OK;
}

sacrak_status sacrak_adm_integrals(sacrak_grid* g, int patch, const double centre[3], double radius,
                                   int ntheta, int nphi, double out[5]) {
  if (!g) return SACRAK_EINVAL;
  if (patch < 0 || patch >= g->npatches || !centre || !out || !(radius > 0.0) || !std::isfinite(radius) ||
      ntheta < 1 || ntheta > ADM_MAX_THETA || nphi < 1 || nphi > (1 << 20) || !std::isfinite(centre[0]) ||
      !std::isfinite(centre[1]) || !std::isfinite(centre[2]))
    return fail(g, SACRAK_EINVAL, "bad arguments");
  AdmArgs a;
  a.patches = g->d_patches;
  a.levels = g->d_levels;
  a.patch = patch;
  a.ntheta = ntheta;
  a.nphi = nphi;
  for (int d = 0; d < 3; ++d) a.c[d] = centre[d];
  a.r = radius;
  a.ring = g->d_scratch;
  launch_adm(a, g->d_results, g->stream);
  sacrak_status st = check_launch(g);
  if (st != SACRAK_OK) return st;
  double v[6];
  CK(cudaMemcpyAsync(v, g->d_results, sizeof v, cudaMemcpyDeviceToHost, g->stream));
  st = sync_and_check(g);
  if (st != SACRAK_OK) return st;
  if (v[5] != 0.0)
    return fail(g, SACRAK_EINVAL, "%.0f sphere points within 2 cells of the edge of patch %d", v[5], patch);
  for (int c = 0; c < 5; ++c) out[c] = v[c];
  return SACRAK_OK;
}

sacrak_status sacrak_track_punctures(sacrak_grid* g, int npunct, const double* pos, const int* follow) {
  if (!g) return SACRAK_EINVAL;
  if (npunct < 0 || npunct > MAX_PUNCT || (npunct > 0 && (!pos || !follow)))
    return fail(g, SACRAK_EINVAL, "bad arguments");
  std::vector<DevPunct> hp(npunct);
  for (int p = 0; p < npunct; ++p) {
    for (int d = 0; d < 3; ++d) {
      if (!std::isfinite(pos[3 * p + d])) return fail(g, SACRAK_EINVAL, "puncture position not finite");
      hp[p].x[d] = pos[3 * p + d];
    }
    hp[p].patch = -1;
    hp[p].level = -1;
  }
  std::vector<int> fl(g->npatches, -1);
  if (npunct > 0)
    for (int q = 0; q < g->npatches; ++q) {
      if (follow[q] < -1 || follow[q] >= npunct) return fail(g, SACRAK_EINVAL, "follow[%d] out of range", q);
      if (follow[q] >= 0 && g->hp[q].level == 0)
        return fail(g, SACRAK_EINVAL, "level-0 patch %d cannot move", q);
      if (follow[q] >= 0 && g->follow_star[q] >= 0)
        return fail(g, SACRAK_EINVAL, "patch %d follows a star", q);
      fl[q] = follow[q];
      if (fl[q] >= 0 && g->hp[q].level > hp[fl[q]].level) {  // the finest patch tracks
        hp[fl[q]].patch = q;
        hp[fl[q]].level = g->hp[q].level;
      }
    }
  for (int p = 0; p < npunct; ++p)
    if (hp[p].patch < 0) return fail(g, SACRAK_EINVAL, "puncture %d is followed by no patch", p);
  sacrak_status st = not_capturing(g);
  if (st != SACRAK_OK) return st;
  if (npunct > 0)
    CK(cudaMemcpyAsync(g->d_punct, hp.data(), sizeof(DevPunct) * npunct, cudaMemcpyHostToDevice, g->stream));
  st = sync_and_check(g);  // (also keeps hp alive until the copy is done)
  if (st != SACRAK_OK) return st;
  g->npunct = npunct;
  g->hpunct = hp;
  g->follow = fl;
  drop_graph(g);  // the captured coarse step has no (or other) trackers
  return SACRAK_OK;
}

sacrak_status sacrak_get_punctures(sacrak_grid* g, double* pos) {
  if (!g) return SACRAK_EINVAL;
  if (g->npunct > 0 && !pos) return fail(g, SACRAK_EINVAL, "bad arguments");
  std::vector<DevPunct> hp(g->npunct);
  if (g->npunct > 0)
    CK(cudaMemcpyAsync(hp.data(), g->d_punct, sizeof(DevPunct) * g->npunct, cudaMemcpyDeviceToHost, g->stream));
  sacrak_status st = sync_and_check(g);
  if (st != SACRAK_OK) return st;
  for (int p = 0; p < g->npunct; ++p)
    for (int d = 0; d < 3; ++d) pos[3 * p + d] = hp[p].x[d];
  return SACRAK_OK;
}

// the largest rest-mass density over the patch's active cells and the centre
// of the first cell (z, y, x order) that holds it
sacrak_status density_maximum(sacrak_grid* g, int patch, double out[4]) {
  const DevPatch& P = g->hp[patch];
  const int maxb = (int)std::min<size_t>(g->L.scratch_doubles / 2, 152 * 16);
  launch_density_max(g->d_patches, patch, (long long)P.n[0] * P.n[1] * P.n[2], g->d_scratch, maxb, g->stream);
  double r[2];
  CK(cudaMemcpyAsync(r, g->d_scratch, sizeof r, cudaMemcpyDeviceToHost, g->stream));
  sacrak_status st = sync_and_check(g);
  if (st != SACRAK_OK) return st;
  const long long id = (long long)r[1];
  if (id < 0) return fail(g, SACRAK_ENONFINITE, "no finite density on patch %d", patch);
  const long long i = id % P.n[0], j = (id / P.n[0]) % P.n[1], k = id / ((long long)P.n[0] * P.n[1]);
  out[0] = r[0];
  out[1] = P.origin[0] + (i + 0.5) * P.dx;
  out[2] = P.origin[1] + (j + 0.5) * P.dx;
  out[3] = P.origin[2] + (k + 0.5) * P.dx;
  return SACRAK_OK;
}

sacrak_status sacrak_density_maximum(sacrak_grid* g, int patch, double out[4]) {
  if (!g) return SACRAK_EINVAL;
  if (!g->prm.matter) return fail(g, SACRAK_EINVAL, "grid created without a fluid (params.matter = 0)");
  if (patch < 0 || patch >= g->npatches || !out) return fail(g, SACRAK_EINVAL, "bad arguments");
  if (!g->matter_ready) return fail(g, SACRAK_ESTATE, "no fluid uploaded (sacrak_upload_matter)");
  sacrak_status st = not_capturing(g);
  if (st != SACRAK_OK) return st;
  return density_maximum(g, patch, out);
}

sacrak_status sacrak_track_stars(sacrak_grid* g, int nstars, const int* follow) {
  if (!g) return SACRAK_EINVAL;
  if (!g->prm.matter) return fail(g, SACRAK_EINVAL, "grid created without a fluid (params.matter = 0)");
  if (nstars < 0 || nstars > g->npatches || (nstars > 0 && !follow)) return fail(g, SACRAK_EINVAL, "bad arguments");
  std::vector<int> fl(g->npatches, -1), count(nstars, 0);
  if (nstars > 0)
    for (int q = 0; q < g->npatches; ++q) {
      if (follow[q] < -1 || follow[q] >= nstars) return fail(g, SACRAK_EINVAL, "follow[%d] out of range", q);
      if (follow[q] >= 0 && g->hp[q].level == 0)
        return fail(g, SACRAK_EINVAL, "level-0 patch %d cannot move", q);
      if (follow[q] >= 0 && g->follow[q] >= 0) return fail(g, SACRAK_EINVAL, "patch %d follows a puncture", q);
      fl[q] = follow[q];
      if (fl[q] >= 0) count[fl[q]]++;
    }
  for (int sidx = 0; sidx < nstars; ++sidx)
    if (count[sidx] == 0) return fail(g, SACRAK_EINVAL, "star %d is followed by no patch", sidx);
  g->follow_star = fl;
  g->nstars = nstars;
  return SACRAK_OK;
}

sacrak_status sacrak_move_patch(sacrak_grid* g, int patch, const int shift[3]) {
  if (!g) return SACRAK_EINVAL;
  if (g->prm.matter && !g->matter_ready) return fail(g, SACRAK_ESTATE, "no fluid uploaded (sacrak_upload_matter)");
  if (patch < 0 || patch >= g->npatches || !shift) return fail(g, SACRAK_EINVAL, "bad arguments");
  if (g->hp[patch].level == 0) return fail(g, SACRAK_EINVAL, "level-0 patches do not move");
  if (g->invalid) return fail(g, SACRAK_ESTATE, "grid holds invalid data");
  sacrak_status st = not_capturing(g);
  if (st != SACRAK_OK) return st;
  std::vector<DevLevel> lv;
  st = synchronised(g, lv);
  if (st != SACRAK_OK) return st;
  int lo[3], hi[3];
  shift_range(g, patch, g->hp, children_of(g, patch, false), lo, hi);
  for (int d = 0; d < 3; ++d)
    if (shift[d] < lo[d] || shift[d] > hi[d])
      return fail(g, SACRAK_EINVAL, "shift %d along axis %d outside %d..%d (nesting)", shift[d], d, lo[d], hi[d]);
  if (shift[0] == 0 && shift[1] == 0 && shift[2] == 0) return SACRAK_OK;
  apply_move(g, patch, shift, lv);
  refresh_after_move(g);
  st = check_launch(g);
  if (st != SACRAK_OK) return st;
  return sync_and_check(g);
}

sacrak_status sacrak_patch_origin(sacrak_grid* g, int patch, double origin[3]) {
  if (!g) return SACRAK_EINVAL;
  if (patch < 0 || patch >= g->npatches || !origin) return fail(g, SACRAK_EINVAL, "bad arguments");
  for (int d = 0; d < 3; ++d) origin[d] = g->hp[patch].origin[d];
  return SACRAK_OK;
}

sacrak_status sacrak_regrid(sacrak_grid* g, int* moved) {
  if (!g) return SACRAK_EINVAL;
  if (!moved) return fail(g, SACRAK_EINVAL, "bad arguments");
  *moved = 0;
  if (g->npunct == 0 && g->nstars == 0) return SACRAK_OK;
  if (g->prm.matter && !g->matter_ready) return fail(g, SACRAK_ESTATE, "no fluid uploaded (sacrak_upload_matter)");
  if (g->invalid) return fail(g, SACRAK_ESTATE, "grid holds invalid data");
  sacrak_status st = not_capturing(g);
  if (st != SACRAK_OK) return st;
  std::vector<DevLevel> lv;
  st = synchronised(g, lv);
  if (st != SACRAK_OK) return st;
  std::vector<DevPunct> hx(g->npunct);
  if (g->npunct > 0)
    CK(cudaMemcpyAsync(hx.data(), g->d_punct, sizeof(DevPunct) * g->npunct, cudaMemcpyDeviceToHost, g->stream));
  st = sync_and_check(g);
  if (st != SACRAK_OK) return st;
  // the stars: the density maximum of the finest patch that follows each
  std::vector<std::array<double, 3>> xs(g->nstars);
  for (int sidx = 0; sidx < g->nstars; ++sidx) {
    int best = -1;
    for (int q = 0; q < g->npatches; ++q)
      if (g->follow_star[q] == sidx && (best < 0 || g->hp[q].level > g->hp[best].level)) best = q;
    double r[4];
    st = density_maximum(g, best, r);
    if (st != SACRAK_OK) return st;
    xs[sidx] = {r[1], r[2], r[3]};
  }
  // plan coarse to fine on copies of the geometry, check it, then move
  std::vector<DevPatch> geo = g->hp;
  std::vector<std::pair<int, std::array<int, 3>>> plan;
  for (int l = 1; l < g->nlevels; ++l)
    for (int pid : g->lvl_ids[l]) {
      const int p = g->follow[pid], sp = g->follow_star[pid];
      if (p < 0 && sp < 0) continue;
      const double* target = p >= 0 ? hx[p].x : xs[sp].data();
      DevPatch& c = geo[pid];
      const double dxp = 2.0 * c.dx;
      std::array<int, 3> s;
      for (int d = 0; d < 3; ++d)
        s[d] = (int)std::trunc((target[d] - (c.origin[d] + 0.5 * c.n[d] * c.dx)) / dxp);
      int lo[3], hi[3];
      shift_range(g, pid, geo, children_of(g, pid, true), lo, hi);
      for (int d = 0; d < 3; ++d) {
        if (lo[d] > hi[d]) return fail(g, SACRAK_EINVAL, "patch %d cannot stay nested", pid);
        s[d] = std::min(std::max(s[d], lo[d]), hi[d]);
      }
      if (s[0] || s[1] || s[2]) {
        for (int d = 0; d < 3; ++d) c.origin[d] = c.origin[d] + (2 * s[d]) * c.dx;
        plan.push_back({pid, s});
      }
    }
  for (int pid = 0; pid < g->npatches; ++pid) {
    if (geo[pid].parent < 0) continue;
    int lo[3], hi[3];
    shift_range(g, pid, geo, children_of(g, pid, false), lo, hi);
    for (int d = 0; d < 3; ++d)
      if (lo[d] > 0 || hi[d] < 0) return fail(g, SACRAK_EINVAL, "regrid would break the nesting of patch %d", pid);
  }
  if (plan.empty()) return SACRAK_OK;
  for (auto& m : plan) apply_move(g, m.first, m.second.data(), lv);
  refresh_after_move(g);
  st = check_launch(g);
  if (st != SACRAK_OK) return st;
  *moved = (int)plan.size();
  return sync_and_check(g);
}

sacrak_status sacrak_psi4_modes(sacrak_grid* g, int patch, const double centre[3], double radius, int ntheta,
                                int nphi, int lmax, double* out) {
  if (!g) return SACRAK_EINVAL;
  if (patch < 0 || patch >= g->npatches || !centre || !out || !(radius > 0.0) || !std::isfinite(radius) ||
      ntheta < 1 || ntheta > ADM_MAX_THETA || nphi < 1 || nphi > (1 << 20) || lmax < 2 || lmax > PSI4_MAX_L ||
      !std::isfinite(centre[0]) || !std::isfinite(centre[1]) || !std::isfinite(centre[2]))
    return fail(g, SACRAK_EINVAL, "bad arguments");
  const DevPatch& P = g->hp[patch];
  const int nm = (lmax + 1) * (lmax + 1) - 4;
  // the sphere values go to the patch's first RK stage buffer, the per-cell
  // Weyl parts to its second (both dead between steps)
  if (2.0 * ntheta * (double)nphi > (double)NF * P.fstride)
    return fail(g, SACRAK_EINVAL, "ntheta x nphi too large for the patch's stage buffer");
  if ((size_t)(3 * ntheta + 2 * nm) > g->L.scratch_doubles) return fail(g, SACRAK_EINVAL, "ntheta too large");
  Psi4Args a;
  a.patches = g->d_patches;
  a.levels = g->d_levels;
  a.patch = patch;
  a.ntheta = ntheta;
  a.nphi = nphi;
  a.lmax = lmax;
  for (int d = 0; d < 3; ++d) a.c[d] = centre[d];
  a.r = radius;
  a.psi = P.buf[B_S0];
  a.cells = P.buf[B_S1];
  a.ring = g->d_scratch;
  a.out = g->d_scratch + 3 * ntheta;
  launch_psi4(a, (long long)P.NX * P.NY * P.NZ, g->stream);
  sacrak_status st = check_launch(g);
  if (st != SACRAK_OK) return st;
  std::vector<double> v(3 * ntheta + 2 * nm);
  CK(cudaMemcpyAsync(v.data(), g->d_scratch, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, g->stream));
  st = sync_and_check(g);
  if (st != SACRAK_OK) return st;
  double bad = 0.0;
  for (int i = 0; i < ntheta; ++i) bad += v[2 * ntheta + i];
  if (bad != 0.0)
    return fail(g, SACRAK_EINVAL, "%.0f sphere points within 2 cells of the edge of patch %d", bad, patch);
  for (int k = 0; k < 2 * nm; ++k) out[k] = v[3 * ntheta + k];
  return SACRAK_OK;
}

sacrak_status sacrak_pi_symmetry(sacrak_grid* g, int patch, double* out) {
  if (!g) return SACRAK_EINVAL;
  if (patch < 0 || patch >= g->npatches || !out) return fail(g, SACRAK_EINVAL, "bad arguments");
  const DevPatch& P = g->hp[patch];
  for (int d = 0; d < 2; ++d)
    if (std::fabs(P.origin[d] + 0.5 * P.n[d] * P.dx) > 1e-12 * P.dx)
      return fail(g, SACRAK_EINVAL, "patch not centred on x = y = 0");
  launch_pi_symmetry(g->d_patches, g->d_levels, patch, (long long)P.NX * P.NY * P.NZ, g->d_scratch,
                     g->d_results, g->stream);
  sacrak_status st = check_launch(g);
  if (st != SACRAK_OK) return st;
  double v;
  CK(cudaMemcpyAsync(&v, g->d_results, sizeof v, cudaMemcpyDeviceToHost, g->stream));
  st = sync_and_check(g);
  if (st != SACRAK_OK) return st;
  *out = v;
  return SACRAK_OK;
}

sacrak_status sacrak_profile_enable(sacrak_grid* g, int enable) {
  if (!g) return SACRAK_EINVAL;
  g->prof = enable != 0;
  g->ev_used = 0;
  g->prof_zones = 0;
  return SACRAK_OK;
}

sacrak_status sacrak_profile_read(sacrak_grid* g, double* ms, long long* launches, long long* zones) {
  if (!g || !ms || !launches || !zones) return SACRAK_EINVAL;
  CK(cudaStreamSynchronize(g->stream));
  double tot = 0.0;
  for (size_t i = 0; i < g->ev_used; ++i) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, g->ev[i].first, g->ev[i].second));
    tot += t;
  }
  *ms = tot;
  *launches = (long long)g->ev_used;
  *zones = g->prof_zones;
  return SACRAK_OK;
}

sacrak_status sacrak_set_stage_kernel(sacrak_grid* g, int level, int kernel) {
  if (!g) return SACRAK_EINVAL;
  if (level < 0 || level >= g->nlevels || kernel < 0 || kernel >= K_COUNT ||
      !kernel_eligible(g, kernel, g->lvl_ids[level]))
    return fail(g, SACRAK_EINVAL, "stage kernel %d not usable on level %d", kernel, level);
  return select_kernel(g, level, kernel);
}

sacrak_status sacrak_set_wait_limit(sacrak_grid* g, long long cycles) {
  if (!g) return SACRAK_EINVAL;
  if (g->tma_wait_cycles != cycles) drop_graph(g);  // the captured launches hold the old bound
  g->tma_wait_cycles = cycles;
  return SACRAK_OK;
}

sacrak_status sacrak_set_overlap(sacrak_grid* g, int on) {
  if (!g) return SACRAK_EINVAL;
  if (on != 0 && on != 1) return fail(g, SACRAK_EINVAL, "overlap must be 0 or 1");
  if (g->overlap != (on == 1)) drop_graph(g);  // the captured coarse step has the other schedule
  g->overlap = on == 1;
  return SACRAK_OK;
}

sacrak_status sacrak_get_stage_kernel(sacrak_grid* g, int level, int* kernel) {
  if (!g) return SACRAK_EINVAL;
  if (level < 0 || level >= g->nlevels || !kernel) return fail(g, SACRAK_EINVAL, "bad arguments");
  *kernel = g->lvl_kernel[level];
  return SACRAK_OK;
}

// Process-wide cache of autotuning results: the fastest stage kernel for a
// level, keyed by device, precision and the level's patch shapes.
static std::mutex g_tune_mu;
static std::map<std::vector<int>, int> g_tune_cache;

sacrak_status sacrak_autotune(sacrak_grid* g, int reps, int use_cache, double* us_out) {
  if (!g) return SACRAK_EINVAL;
  if (reps < 1 || reps > 1000) return fail(g, SACRAK_EINVAL, "reps must be 1..1000");
  if (g->invalid) return fail(g, SACRAK_ESTATE, "grid state invalid after an earlier error");
  cudaStreamCaptureStatus cs;
  CK(cudaStreamIsCapturing(g->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(g, SACRAK_ESTATE, "autotuning needs a stream that is not capturing");
  if (us_out)
    for (int i = 0; i < g->nlevels * K_COUNT; ++i) us_out[i] = -1.0;
  refresh_all_shells(g);  // the split of the current levels must be valid
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  sacrak_status st = SACRAK_OK;
  // levels of identical shape in this call share one timing (and so one
  // choice, as the process-wide cache would give them)
  std::map<std::vector<int>, std::pair<int, std::vector<double>>> now;
  for (int l = 0; l < g->nlevels && st == SACRAK_OK; ++l) {
    std::vector<int> key = {dev, g->prm.precision};
    for (int pid : g->lvl_ids[l]) key.insert(key.end(), g->hp[pid].n, g->hp[pid].n + 3);
    {
      auto it = now.find(key);
      if (it != now.end()) {
        if (us_out)
          for (int k = 0; k < K_COUNT; ++k) us_out[l * K_COUNT + k] = it->second.second[k];
        st = select_kernel(g, l, it->second.first);
        continue;
      }
    }
    if (use_cache) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        st = select_kernel(g, l, it->second);
        continue;
      }
    }
    // time stage 1 of the level with every usable kernel: it reads the
    // current time level and writes only the RK accumulator and the first
    // stage buffer, so repeating it leaves the state as it was
    StageArgs a;
    a.tiles = g->d_tiles + g->lvl_tile_off[l];
    a.ntiles = (int)g->lvl_ntiles[l];
    a.patches = g->d_patches;
    a.lev = g->d_levels + l;
    a.stage = 1;
    a.dt = level_dt(g, l);
    a.prm = dev_params(g->prm);
    a.err = g->d_err;
    int best = g->lvl_kernel[l];
    float best_ms = 0.0f, keep_ms = 0.0f;
    const int nk = g->prm.precision == 1 ? K_COUNT : 1;
    const int keep = g->lvl_kernel[l];
    for (int k = 0; k < nk && st == SACRAK_OK; ++k) {
      if (!kernel_eligible(g, k, g->lvl_ids[l])) continue;
      if ((st = select_kernel(g, l, k)) != SACRAK_OK) break;  // one-time set-up of kernel k
      const bool prof = g->prof;
      g->prof = false;
      launch_stage(g, a, 0, g->lvl_ids[l], k);  // warm-up
      cudaEventRecord(e0, g->stream);
      for (int r = 0; r < reps; ++r) launch_stage(g, a, 0, g->lvl_ids[l], k);
      cudaEventRecord(e1, g->stream);
      g->prof = prof;
      if ((st = check_launch(g)) != SACRAK_OK) break;
      if ((st = sync_and_check(g)) != SACRAK_OK) break;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (us_out) us_out[l * K_COUNT + k] = 1e3 * ms;
      if (k == keep) keep_ms = ms;
      if (k == 0 || ms < best_ms) {
        best = k;
        best_ms = ms;
      }
    }
    if (st != SACRAK_OK) {
      select_kernel(g, l, keep);
      break;
    }
    // stage 1 stands in for all four stages: a kernel replaces the level's
    // current one only when it is more than 2% faster (kernel 11 led kernel
    // 10 by 1% on stage 1 of the 64^3 levels and lost over whole steps)
    if (best != keep && keep_ms > 0.0f && best_ms >= 0.98f * keep_ms) best = keep;
    st = select_kernel(g, l, best);
    {
      std::vector<double> row(K_COUNT, -1.0);
      if (us_out)
        for (int k = 0; k < K_COUNT; ++k) row[k] = us_out[l * K_COUNT + k];
      now[key] = std::make_pair(best, row);
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

sacrak_status sacrak_level_time(sacrak_grid* g, int level, double* t) {
  if (!g) return SACRAK_EINVAL;
  if (level < 0 || level >= g->nlevels || !t) return fail(g, SACRAK_EINVAL, "bad arguments");
  DevLevel lv;
  sacrak_status st = read_level(g, level, &lv);
  if (st != SACRAK_OK) return st;
  *t = lv.t;
  return SACRAK_OK;
}

const char* sacrak_last_error(const sacrak_grid* g) { return g ? g->last_error.c_str() : "null grid"; }

}  // extern "C"
