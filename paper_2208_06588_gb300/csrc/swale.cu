// Host side and C ABI (include/swale.h) of the GB300 (sm_103a) FP64 solver for the
// well-balanced ALE-WENO hybrid scheme (Zhang, Xia & Xu, arXiv 2208.06588). The kernels are in
// swale_kernels.cuh, the per-cell arithmetic in swale_cell.cuh.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/swale.h"
#include "swale_kernels.cuh"
#include "swale_adjoint_kernels.cuh"

using namespace swale_dev;

struct swale_ctx {
  swale_config cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t B = 0, Ntot = 0;        // instances, total cells
  std::vector<int64_t> off;       // B + 1 cell offsets
  DevState D{};
  int Tr = 128, Tu = 128;         // tile sizes of the reconstruction / update kernels
  int grid_r = 0, grid_u = 0;     // 0: one block per tile, else a persistent grid of that size
  double gauss_wsum = 1.0;
  std::vector<void*> allocs;      // state
  std::vector<void*> tile_allocs; // work lists (rebuilt when the tile sizes change)
  uint8_t* flag_buf = nullptr;    // dense classes of a batch
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  std::string err;
  // Kernel timing (swale_set_timing): event pairs around every launch, by kernel family.
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_family;
  size_t ev_used = 0;
  // Stage-viscosity log (swale_alpha_log): device array of 3 values per step and instance.
  double* alpha_log = nullptr;
  int64_t alpha_cap = 0, alpha_base = 0;
  int32_t alpha_mode = 0;
  // L2-projection bottom (swale_set_bottom_function); part of the state allocations.
  int32_t bot_pieces = 0, bot_deg = 0;
  double *bot_breaks = nullptr, *bot_coef = nullptr;
  // Epoch of the mesh geometry cache; bumped whenever the state is set or restored, so that a
  // cache entry written before is never taken for the restored state.
  uint32_t geo_epoch = 1;
  // swale_adjoint: keep every step's stage data from the segment recompute (1) instead of
  // recomputing each step before its reverse sweep (0).
  int32_t adjoint_tape = 0;
  // swale_set_wait_test: polls of the bulk-copy waits (0: the default) and extra bytes they
  // expect (0).
  int32_t wait_tries = 0;
  uint32_t tx_pad = 0;
};

namespace {

// NVTX range over a host call (a no-op unless a profiling tool is attached): the step loops,
// graph replays, the adjoint's phases and the autotuner show up by name on a timeline.
struct NvtxRange {
  explicit NvtxRange(const char* m) { nvtxRangePushA(m); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

swale_status fail(swale_ctx* ctx, swale_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

#define SW_CUDA(ctx, call)                                                                          \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail(ctx, SWALE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copies n values from caller memory (host or device) into a host vector.
template <class T>
swale_status fetch(swale_ctx* ctx, const T* src, size_t n, std::vector<T>& dst) {
  dst.resize(n);
  if (is_device_ptr(src)) {
    SW_CUDA(ctx, cudaMemcpyAsync(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
    SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  } else {
    std::memcpy(dst.data(), src, n * sizeof(T));
  }
  return SWALE_OK;
}

swale_status put_out(swale_ctx* ctx, void* dst, const void* dev_src, size_t bytes) {
  if (!dst) return SWALE_OK;
  SW_CUDA(ctx, cudaMemcpyAsync(dst, dev_src, bytes, cudaMemcpyDefault, ctx->stream));
  return SWALE_OK;
}

StepConst step_const(const swale_ctx* ctx) {
  StepConst K;
  K.sc.g = ctx->cfg.g;
  K.sc.eps_weno = ctx->cfg.eps_weno;
  K.sc.eps_pp = ctx->cfg.eps_pp;
  K.sc.h_dry = ctx->cfg.h_dry;
  K.sc.beta_dx_global = ctx->cfg.beta_dx_global;
  K.sc.limit_hu = ctx->cfg.limit_hu;
  K.t_end = ctx->cfg.t_end;
  K.dt_fixed = ctx->cfg.dt_fixed;
  K.mesh_T = ctx->cfg.mesh_T;
  K.gauss_wsum = ctx->gauss_wsum;
  K.gauss_iwsum = 1.0 / ctx->gauss_wsum;
  K.bc = ctx->cfg.bc;
  K.mesh = ctx->cfg.mesh;
  K.gauss_half = ctx->cfg.gauss_half;
  K.B = (int32_t)ctx->B;
  K.alpha_log = ctx->alpha_log;
  K.alpha_cap = ctx->alpha_cap;
  K.alpha_base = ctx->alpha_base;
  K.alpha_mode = ctx->alpha_mode;
  K.scheme = ctx->cfg.scheme;
  K.geo_epoch = ctx->geo_epoch;
  K.bot_pieces = ctx->bot_pieces;
  K.bot_deg = ctx->bot_deg;
  K.bot_breaks = ctx->bot_breaks;
  K.bot_coef = ctx->bot_coef;
  K.wait_tries = ctx->wait_tries > 0 ? ctx->wait_tries : kWaitTries;
  K.tx_pad = ctx->tx_pad;
  K.wave_rel = ctx->cfg.alpha_bound ? 0 : 1;
  return K;
}

// Whether stage 1's alpha can use the node velocities (Eq. alpha2D as written): they are known
// before the stage runs, except for the secant speeds of the profile motion, which depend on dt.
int stage1_wave_rel(const swale_config& c) { return (!c.alpha_bound && c.mesh != SWALE_MESH_PROFILE) ? 1 : 0; }

void drop_graph(swale_ctx* ctx);

// The state was set or restored: invalidate the mesh geometry cache (and the captured steps,
// which carry the epoch).
void bump_geo(swale_ctx* ctx) {
  ++ctx->geo_epoch;
  drop_graph(ctx);
}

void drop_graph(swale_ctx* ctx) {
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
}

void free_tiles(swale_ctx* ctx) {
  for (void* p : ctx->tile_allocs) cudaFree(p);
  ctx->tile_allocs.clear();
  ctx->D.rtiles = ctx->D.utiles = ctx->D.mtiles = ctx->D.ftiles = nullptr;
}

void free_alpha_log(swale_ctx* ctx) {
  if (ctx->alpha_log) cudaFree(ctx->alpha_log);
  ctx->alpha_log = nullptr;
  ctx->alpha_cap = 0;
  ctx->alpha_mode = 0;
}

void free_state(swale_ctx* ctx) {
  drop_graph(ctx);
  free_tiles(ctx);
  free_alpha_log(ctx);
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  ctx->D = DevState{};
  ctx->B = ctx->Ntot = 0;
  ctx->off.clear();
  ctx->flag_buf = nullptr;
  ctx->bot_pieces = ctx->bot_deg = 0;
  ctx->bot_breaks = ctx->bot_coef = nullptr;
}

template <class T>
swale_status dalloc(swale_ctx* ctx, std::vector<void*>& list, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T) + 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SWALE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  list.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return SWALE_OK;
}

// Device arrays of B instances with Ntot cells in total.
swale_status alloc_state(swale_ctx* ctx, int64_t B, int64_t Ntot, DevState& D) {
  const size_t nc = (size_t)Ntot, nn = nc + B, ne = nc + 2 * B;
  double** cells[] = {&D.E0, &D.M0, &D.B0, &D.Ea, &D.Ma, &D.Ba, &D.Eb, &D.Mb, &D.Bb,
                      &D.YE, &D.YM, &D.YB, &D.J0, &D.J1, &D.J2, &D.bE, &D.bM, &D.bB, &D.bJ};
  for (double** p : cells)
    if (swale_status s = dalloc(ctx, ctx->allocs, p, nc)) return s;
  double** nodes[] = {&D.x, &D.w, &D.P, &D.bx};
  for (double** p : nodes)
    if (swale_status s = dalloc(ctx, ctx->allocs, p, nn)) return s;
  double** edges[] = {&D.eEL, &D.eER, &D.eBL, &D.eBR, &D.ehL, &D.ehR, &D.euL, &D.euR, &D.ipair, &D.itri};
  for (double** p : edges)
    if (swale_status s = dalloc(ctx, ctx->allocs, p, ne)) return s;
  if (ctx->cfg.scheme == SWALE_SCHEME_SPECIAL) {
    if (swale_status s = dalloc(ctx, ctx->allocs, &D.eG1, ne)) return s;
    if (swale_status s = dalloc(ctx, ctx->allocs, &D.eG2, ne)) return s;
  }
  if (swale_status s = dalloc(ctx, ctx->allocs, &D.geo, (size_t)SWALE_GEO_ARRAYS * ne)) return s;
  D.geo_stride = (int64_t)ne;
  if (swale_status s = dalloc(ctx, ctx->allocs, &D.flags, ne)) return s;
  if (swale_status s = dalloc(ctx, ctx->allocs, &D.IC, (size_t)B)) return s;
  if (swale_status s = dalloc(ctx, ctx->allocs, &D.S, (size_t)B)) return s;
  return SWALE_OK;
}

swale_status check_config(const swale_config* c, std::string& why) {
  if (!(c->g > 0) || !(c->eps_weno > 0) || !(c->eps_pp >= 0) || !(c->h_dry >= 0)) {
    why = "g, eps_weno must be > 0 and eps_pp, h_dry >= 0";
    return SWALE_EINVAL;
  }
  if (!(c->dt_fixed > 0) && !(c->cfl > 0)) {
    why = "cfl must be > 0 unless dt_fixed > 0";
    return SWALE_EINVAL;
  }
  if (c->bc < 0 || c->bc > 2) {
    why = "bc must be 0 (periodic), 1 (transmissive) or 2 (reflective)";
    return SWALE_EINVAL;
  }
  if (c->mesh < 0 || c->mesh > 3) {
    why = "mesh must be 0 (static), 1 (profile), 2 (fluid_gauss) or 3 (linear)";
    return SWALE_EINVAL;
  }
  if (c->alpha_bound != 0 && c->alpha_bound != 1) {
    why = "alpha_bound must be 0 or 1";
    return SWALE_EINVAL;
  }
  if (c->limit_hu != 0 && c->limit_hu != 1) {
    why = "limit_hu must be 0 or 1";
    return SWALE_EINVAL;
  }
  if (c->scheme < 0 || c->scheme > 2) {
    why = "scheme must be 0 (hydrostatic), 1 (nonwb) or 2 (special)";
    return SWALE_EINVAL;
  }
  if (c->mesh == SWALE_MESH_PROFILE && !(c->mesh_T > 0)) {
    why = "mesh_T must be > 0 for profile motion";
    return SWALE_EINVAL;
  }
  if (c->mesh == SWALE_MESH_FLUID_GAUSS) {
    if (c->gauss_half < 0 || c->gauss_half > kMaxGaussHalf || !(c->gauss_sigma > 0)) {
      why = "fluid_gauss needs gauss_sigma > 0 and 0 <= gauss_half <= 64";
      return SWALE_EINVAL;
    }
    if (c->bc == SWALE_BC_PERIODIC) {
      why = "fluid_gauss motion fixes the end nodes and needs a non-periodic domain";
      return SWALE_EINVAL;
    }
  }
  return SWALE_OK;
}

bool valid_tile(int T) { return T == 64 || T == 128 || T == 256; }

// Builds the work lists for the current tile sizes (implicit for one instance) and the
// per-instance tile counts; uploads the instance constants.
swale_status build_tiles(swale_ctx* ctx, std::vector<InstConst>& ic) {
  drop_graph(ctx);
  free_tiles(ctx);
  const int64_t B = ctx->B;
  const int Tr = ctx->Tr, Tu = ctx->Tu, Tm = kMeshNodes;
  const int Tf = Tu - 1;  // cells of a forward update tile (its Tu interfaces take one pass)
  std::vector<Tile> rt, ut, mt, ft;
  for (int64_t i = 0; i < B; ++i) {
    const int64_t N = ic[i].N;
    const int64_t nr = (N + 2 + Tr - 1) / Tr, nu = (N + Tu - 1) / Tu, nm = (N + 1 + Tm - 1) / Tm;
    const int64_t nf = (N + Tf - 1) / Tf;
    ic[i].ntiles_r = (int32_t)nr;
    if (B > 1) {
      for (int64_t t = 0; t < nr; ++t) rt.push_back(Tile{(int32_t)i, (int32_t)(t * Tr - 1)});
      for (int64_t t = 0; t < nu; ++t) ut.push_back(Tile{(int32_t)i, (int32_t)(t * Tu)});
      for (int64_t t = 0; t < nm; ++t) mt.push_back(Tile{(int32_t)i, (int32_t)(t * Tm)});
      for (int64_t t = 0; t < nf; ++t) ft.push_back(Tile{(int32_t)i, (int32_t)(t * Tf)});
    } else {
      ctx->D.nr = (int32_t)nr;
      ctx->D.nu = (int32_t)nu;
      ctx->D.nm = (int32_t)nm;
      ctx->D.nf = (int32_t)nf;
    }
  }
  if (B > 1) {
    Tile *dr, *du, *dm, *df;
    if (swale_status s = dalloc(ctx, ctx->tile_allocs, &dr, rt.size())) return s;
    if (swale_status s = dalloc(ctx, ctx->tile_allocs, &du, ut.size())) return s;
    if (swale_status s = dalloc(ctx, ctx->tile_allocs, &dm, mt.size())) return s;
    if (swale_status s = dalloc(ctx, ctx->tile_allocs, &df, ft.size())) return s;
    SW_CUDA(ctx, cudaMemcpyAsync(dr, rt.data(), rt.size() * sizeof(Tile), cudaMemcpyHostToDevice, ctx->stream));
    SW_CUDA(ctx, cudaMemcpyAsync(du, ut.data(), ut.size() * sizeof(Tile), cudaMemcpyHostToDevice, ctx->stream));
    SW_CUDA(ctx, cudaMemcpyAsync(dm, mt.data(), mt.size() * sizeof(Tile), cudaMemcpyHostToDevice, ctx->stream));
    SW_CUDA(ctx, cudaMemcpyAsync(df, ft.data(), ft.size() * sizeof(Tile), cudaMemcpyHostToDevice, ctx->stream));
    ctx->D.rtiles = dr;
    ctx->D.utiles = du;
    ctx->D.mtiles = dm;
    ctx->D.ftiles = df;
    ctx->D.nr = (int32_t)rt.size();
    ctx->D.nu = (int32_t)ut.size();
    ctx->D.nm = (int32_t)mt.size();
    ctx->D.nf = (int32_t)ft.size();
  }
  SW_CUDA(ctx, cudaMemcpyAsync(ctx->D.IC, ic.data(), B * sizeof(InstConst), cudaMemcpyHostToDevice, ctx->stream));
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SWALE_OK;
}

// Re-reads the instance constants from the device, rebuilds the work lists.
swale_status rebuild_tiles(swale_ctx* ctx) {
  std::vector<InstConst> ic(ctx->B);
  SW_CUDA(ctx, cudaMemcpyAsync(ic.data(), ctx->D.IC, ctx->B * sizeof(InstConst), cudaMemcpyDeviceToHost,
                               ctx->stream));
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return build_tiles(ctx, ic);
}

enum { FAM_PROLOGUE = 0, FAM_MESH = 1, FAM_RECON = 2, FAM_UPDATE = 3, FAM_COUNT = 4 };

// Runs launch() on the context's stream; with timing enabled, brackets it by two events.
template <class F>
swale_status timed_launch(swale_ctx* ctx, int family, F&& launch) {
  if (!ctx->timing) {
    launch();
    return SWALE_OK;
  }
  while (ctx->ev_pool.size() < ctx->ev_used + 2) {
    cudaEvent_t e;
    SW_CUDA(ctx, cudaEventCreate(&e));
    ctx->ev_pool.push_back(e);
  }
  SW_CUDA(ctx, cudaEventRecord(ctx->ev_pool[ctx->ev_used], ctx->stream));
  launch();
  SW_CUDA(ctx, cudaEventRecord(ctx->ev_pool[ctx->ev_used + 1], ctx->stream));
  ctx->ev_family.push_back(family);
  ctx->ev_used += 2;
  return SWALE_OK;
}

template <int STAGE>
void launch_recon(const StepConst& K, const DevState& D, int T, unsigned grid, cudaStream_t s, const double* E,
                  const double* M, const double* B, const double* J) {
  if (K.scheme == SWALE_SCHEME_NONWB) {
    if (T == 64) k_recon<STAGE, 64, 1><<<grid, 64, 0, s>>>(K, D, E, M, B, J);
    else if (T == 256) k_recon<STAGE, 256, 1><<<grid, 256, 0, s>>>(K, D, E, M, B, J);
    else k_recon<STAGE, 128, 1><<<grid, 128, 0, s>>>(K, D, E, M, B, J);
    return;
  }
  if (K.scheme == SWALE_SCHEME_SPECIAL) {
    if (T == 64) k_recon<STAGE, 64, 2><<<grid, 64, 0, s>>>(K, D, E, M, B, J);
    else if (T == 256) k_recon<STAGE, 256, 2><<<grid, 256, 0, s>>>(K, D, E, M, B, J);
    else k_recon<STAGE, 128, 2><<<grid, 128, 0, s>>>(K, D, E, M, B, J);
    return;
  }
  if (D.gK) {  // the adjoint's recomputes: also store the smooth-class linear form
    if (T == 64) k_recon<STAGE, 64, 0, false, true><<<grid, 64, 0, s>>>(K, D, E, M, B, J);
    else if (T == 256) k_recon<STAGE, 256, 0, false, true><<<grid, 256, 0, s>>>(K, D, E, M, B, J);
    else k_recon<STAGE, 128, 0, false, true><<<grid, 128, 0, s>>>(K, D, E, M, B, J);
    return;
  }
  if constexpr (STAGE == 1) {
    if (D.geo) {  // stage 1 reads the cached geometry: more resident warps
      if (T == 64) k_recon<STAGE, 64, 0, true><<<grid, 64, 0, s>>>(K, D, E, M, B, J);
      else if (T == 256) k_recon<STAGE, 256, 0, true><<<grid, 256, 0, s>>>(K, D, E, M, B, J);
      else k_recon<STAGE, 128, 0, true><<<grid, 128, 0, s>>>(K, D, E, M, B, J);
      return;
    }
  }
  if (T == 64) k_recon<STAGE, 64><<<grid, 64, 0, s>>>(K, D, E, M, B, J);
  else if (T == 256) k_recon<STAGE, 256><<<grid, 256, 0, s>>>(K, D, E, M, B, J);
  else k_recon<STAGE, 128><<<grid, 128, 0, s>>>(K, D, E, M, B, J);
}

template <int STAGE, int MODE>
void launch_update(const StepConst& K, const DevState& D, int T, unsigned grid, cudaStream_t s, const double* E,
                   const double* M, const double* B, const double* J, RhsOut ro) {
  if (MODE == 0 && K.scheme == SWALE_SCHEME_HYDROSTATIC && K.bot_pieces == 0 && D.gK) {
    // the adjoint's recomputes: also store the source form's entries
    if (T == 64) k_update<STAGE, MODE, 64, true, true><<<grid, 64, 0, s>>>(K, D, E, M, B, J, ro);
    else if (T == 256) k_update<STAGE, MODE, 256, true, true><<<grid, 256, 0, s>>>(K, D, E, M, B, J, ro);
    else k_update<STAGE, MODE, 128, true, true><<<grid, 128, 0, s>>>(K, D, E, M, B, J, ro);
    return;
  }
  if (MODE == 0 && K.scheme == SWALE_SCHEME_HYDROSTATIC && K.bot_pieces == 0) {
    if (T == 64) k_update<STAGE, MODE, 64, true><<<grid, 64, 0, s>>>(K, D, E, M, B, J, ro);
    else if (T == 256) k_update<STAGE, MODE, 256, true><<<grid, 256, 0, s>>>(K, D, E, M, B, J, ro);
    else k_update<STAGE, MODE, 128, true><<<grid, 128, 0, s>>>(K, D, E, M, B, J, ro);
    return;
  }
  if (T == 64) k_update<STAGE, MODE, 64><<<grid, 64, 0, s>>>(K, D, E, M, B, J, ro);
  else if (T == 256) k_update<STAGE, MODE, 256><<<grid, 256, 0, s>>>(K, D, E, M, B, J, ro);
  else k_update<STAGE, MODE, 128><<<grid, 128, 0, s>>>(K, D, E, M, B, J, ro);
}

unsigned grid_of(int32_t ntiles, int persistent) {
  if (persistent > 0 && persistent < ntiles) return (unsigned)persistent;
  return (unsigned)std::max(ntiles, 1);
}

// Enqueues one step of the state D on stream s with geometry-cache epoch `epoch`. stageD
// (optional, 3 entries): the device state each stage's kernels use; copies of D that differ only
// in their edge arrays keep every stage's edge values (the adjoint's recompute of a step).
swale_status enqueue_step_on(swale_ctx* ctx, const DevState& D, cudaStream_t s, const DevState* stageD,
                             uint32_t epoch) {
  StepConst K = step_const(ctx);
  K.geo_epoch = epoch;
  const DevState& D1 = stageD ? stageD[0] : D;
  const DevState& D2 = stageD ? stageD[1] : D;
  const DevState& D3 = stageD ? stageD[2] : D;
  const unsigned gr = grid_of(D.nr, ctx->grid_r), gu = grid_of(D.nf, ctx->grid_u);
  const int Tr = ctx->Tr, Tu = ctx->Tu;
  const RhsOut none{nullptr, nullptr, nullptr, 0.0};
  swale_status st = SWALE_OK;
  auto L = [&](int fam, auto&& f) {
    if (st == SWALE_OK) st = timed_launch(ctx, fam, f);
  };
  L(FAM_PROLOGUE, [&] { k_prologue<<<(unsigned)((ctx->B + 127) / 128), 128, 0, s>>>(K, D); });
  if (K.mesh == SWALE_MESH_FLUID_GAUSS) {
    const size_t shm = (size_t)(3 * kMeshThreads + 4 * K.gauss_half + 4) * sizeof(double);
    L(FAM_MESH, [&] { k_mesh_gauss<<<(unsigned)std::max(D.nm, 1), kMeshThreads, shm, s>>>(K, D); });
  }
  StepConst K1 = K;
  K1.wave_rel = stage1_wave_rel(ctx->cfg);
  L(FAM_RECON, [&] { launch_recon<1>(K1, D1, Tr, gr, s, D.E0, D.M0, D.B0, D.J0); });
  L(FAM_UPDATE, [&] { launch_update<1, 0>(K1, D1, Tu, gu, s, D.E0, D.M0, D.B0, D.J0, none); });
  L(FAM_RECON, [&] { launch_recon<2>(K, D2, Tr, gr, s, D.Ea, D.Ma, D.Ba, D.J1); });
  L(FAM_UPDATE, [&] { launch_update<2, 0>(K, D2, Tu, gu, s, D.Ea, D.Ma, D.Ba, D.J1, none); });
  L(FAM_RECON, [&] { launch_recon<3>(K, D3, Tr, gr, s, D.Eb, D.Mb, D.Bb, D.J2); });
  L(FAM_UPDATE, [&] { launch_update<3, 0>(K, D3, Tu, gu, s, D.Eb, D.Mb, D.Bb, D.J2, none); });
  L(FAM_PROLOGUE, [&] { k_commit<<<(unsigned)std::min<int64_t>(ctx->B, 1024), 256, 0, s>>>(K, D); });
  if (st) return st;
  SW_CUDA(ctx, cudaGetLastError());
  return SWALE_OK;
}

// Enqueues one step of the context's state on its stream.
swale_status enqueue_step(swale_ctx* ctx, const DevState* stageD = nullptr) {
  return enqueue_step_on(ctx, ctx->D, ctx->stream, stageD, ctx->geo_epoch);
}

// Enqueues n steps: whole graphs of kGraphSteps steps, then single steps (graphs are not used
// while kernel timing is on).
swale_status enqueue_steps(swale_ctx* ctx, int64_t n) {
  constexpr int kGraphSteps = 8;
  if (!ctx->timing && n >= kGraphSteps) {
    if (!ctx->graph) {
      cudaGraph_t g;
      SW_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      swale_status cs = SWALE_OK;
      for (int i = 0; i < kGraphSteps && cs == SWALE_OK; ++i) cs = enqueue_step(ctx);
      cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
      if (cs) return cs;
      if (e != cudaSuccess) return fail(ctx, SWALE_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&ctx->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(ctx, SWALE_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
      ctx->graph_steps = kGraphSteps;
    }
    while (n >= ctx->graph_steps) {
      NvtxRange r("swale graph replay (8 steps)");
      SW_CUDA(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
      n -= ctx->graph_steps;
    }
  }
  for (; n > 0; --n)
    if (swale_status s = enqueue_step(ctx)) return s;
  return SWALE_OK;
}

// Common set-up of B instances from host vectors.
swale_status set_instances(swale_ctx* ctx, const std::vector<int64_t>& off, const std::vector<double>& x,
                           const std::vector<double>& q, const std::vector<double>& m, const std::vector<double>& bb,
                           const std::vector<double>& P, const std::vector<double>& cfl, bool q0_is_eta,
                           bool check_depth = true) {
  const int64_t B = (int64_t)off.size() - 1;
  const int64_t Ntot = off[B];
  std::vector<double> E(Ntot), J(Ntot);
  std::vector<InstConst> ic(B);
  std::vector<DevScalars> S0(B);
  for (int64_t i = 0; i < B; ++i) {
    const int64_t c0 = off[i], N = off[i + 1] - off[i], n0 = c0 + i;
    if (N < 5) return fail(ctx, SWALE_EINVAL, "every instance needs N >= 5 cells");
    double jmax = 0.0, jmin = INFINITY, pmax = 0.0;
    for (int64_t k = 0; k <= N; ++k) {
      if (!std::isfinite(x[n0 + k]) || !std::isfinite(P[n0 + k]))
        return fail(ctx, SWALE_EINVAL, "non-finite node or profile");
      pmax = std::max(pmax, std::fabs(P[n0 + k]));
    }
    for (int64_t j = 0; j < N; ++j) {
      const int64_t g = c0 + j;
      J[g] = x[n0 + j + 1] - x[n0 + j];
      if (!(J[g] > 0.0)) return fail(ctx, SWALE_EINVAL, "nodes must be strictly increasing");
      jmax = std::max(jmax, J[g]);
      jmin = std::min(jmin, J[g]);
      if (!std::isfinite(q[g]) || !std::isfinite(m[g]) || !std::isfinite(bb[g]))
        return fail(ctx, SWALE_EINVAL, "non-finite cell average");
      E[g] = q0_is_eta ? q[g] : q[g] + bb[g];
      if (check_depth && E[g] - bb[g] < 0.0) return fail(ctx, SWALE_EINVAL, "negative depth in the initial data");
    }
    if (!(cfl[i] > 0.0) && !(ctx->cfg.dt_fixed > 0.0)) return fail(ctx, SWALE_EINVAL, "cfl must be > 0");
    ic[i].N = N;
    ic[i].coff = c0;
    ic[i].cfl = cfl[i];
    ic[i].Wbar_profile = (ctx->cfg.mesh == SWALE_MESH_PROFILE) ? kTwoPi / ctx->cfg.mesh_T * pmax
                         : (ctx->cfg.mesh == SWALE_MESH_LINEAR)  ? pmax
                                                                 : 0.0;
    ic[i].ntiles_r = 0;
    ic[i].pad_ = 0;
    std::memset(&S0[i], 0, sizeof(DevScalars));
    std::memcpy(&S0[i].JmaxN, &jmax, 8);
    std::memcpy(&S0[i].JminN, &jmin, 8);
    S0[i].Wbar = ic[i].Wbar_profile;
  }
  free_state(ctx);
  swale_status s = alloc_state(ctx, B, Ntot, ctx->D);
  if (s) {
    free_state(ctx);
    return s;
  }
  ctx->B = B;
  ctx->Ntot = Ntot;
  ctx->off = off;
  bump_geo(ctx);
  DevState& D = ctx->D;
  cudaStream_t st = ctx->stream;
  const size_t cb = Ntot * sizeof(double), nb = (Ntot + B) * sizeof(double);
  SW_CUDA(ctx, cudaMemcpyAsync(D.E0, E.data(), cb, cudaMemcpyHostToDevice, st));
  SW_CUDA(ctx, cudaMemcpyAsync(D.M0, m.data(), cb, cudaMemcpyHostToDevice, st));
  SW_CUDA(ctx, cudaMemcpyAsync(D.B0, bb.data(), cb, cudaMemcpyHostToDevice, st));
  SW_CUDA(ctx, cudaMemcpyAsync(D.J0, J.data(), cb, cudaMemcpyHostToDevice, st));
  SW_CUDA(ctx, cudaMemcpyAsync(D.x, x.data(), nb, cudaMemcpyHostToDevice, st));
  SW_CUDA(ctx, cudaMemcpyAsync(D.P, P.data(), nb, cudaMemcpyHostToDevice, st));
  SW_CUDA(ctx, cudaMemsetAsync(D.w, 0, nb, st));
  SW_CUDA(ctx, cudaMemsetAsync(D.flags, 0, Ntot + 2 * B, st));
  SW_CUDA(ctx, cudaMemcpyAsync(D.S, S0.data(), B * sizeof(DevScalars), cudaMemcpyHostToDevice, st));
  if (ctx->cfg.mesh == SWALE_MESH_FLUID_GAUSS) {
    const int H = ctx->cfg.gauss_half;
    std::vector<double> gw(2 * kMaxGaussHalf + 1, 0.0);
    for (int mm = -H; mm <= H; ++mm)
      gw[mm + H] = std::exp(-(double)(mm * mm) / (2.0 * ctx->cfg.gauss_sigma * ctx->cfg.gauss_sigma));
    double ws = 0.0;
    for (int mm = -H; mm <= H; ++mm) ws += gw[mm + H];
    ctx->gauss_wsum = ws;
    SW_CUDA(ctx, cudaMemcpyToSymbolAsync(c_gauss_w, gw.data(), gw.size() * sizeof(double), 0,
                                         cudaMemcpyHostToDevice, st));
  }
  return build_tiles(ctx, ic);
}

swale_status status_from_bits(swale_ctx* ctx, unsigned int bits) {
  if (bits & swale::ST_TIMEOUT)
    return fail(ctx, SWALE_ETIMEOUT, "a bounded wait for a bulk copy gave up; the stage was abandoned");
  if (bits & swale::ST_NODT)
    return fail(ctx, SWALE_ENONFINITE, "no finite time step: zero wave speed, no mesh motion and t_end = 0");
  if (bits & swale::ST_NONFINITE) return fail(ctx, SWALE_ENONFINITE, "non-finite value in a stage");
  if (bits & swale::ST_EMESH) return fail(ctx, SWALE_EMESH, "non-positive cell width");
  if (bits & swale::ST_EWEIGHT) return fail(ctx, SWALE_EWEIGHT, "non-positive linear weight");
  return SWALE_OK;
}

// Per-instance scalars to the host.
swale_status read_scalars(swale_ctx* ctx, std::vector<DevScalars>& S) {
  S.resize(ctx->B);
  SW_CUDA(ctx, cudaMemcpyAsync(S.data(), ctx->D.S, ctx->B * sizeof(DevScalars), cudaMemcpyDeviceToHost,
                               ctx->stream));
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SWALE_OK;
}

}  // namespace

extern "C" {

swale_status swale_create(swale_ctx** out, const swale_config* cfg, void* cuda_stream) {
  if (!out || !cfg) return SWALE_EINVAL;
  *out = nullptr;
  std::string why;
  if (check_config(cfg, why) != SWALE_OK) return SWALE_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return SWALE_EINVAL;
  }
  swale_ctx* ctx = new swale_ctx();
  ctx->cfg = *cfg;
  ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (!ctx->stream) {
    // The legacy default stream cannot be captured into a graph: use a private blocking
    // stream, which is still ordered with the legacy default stream.
    if (cudaStreamCreate(&ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return SWALE_ECUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return SWALE_OK;
}

swale_status swale_set_problem(swale_ctx* ctx, int64_t N, const double* x_nodes, const double* q0, const double* hu,
                               const double* b, const double* profile, int32_t q0_is_eta) {
  if (!ctx) return SWALE_EINVAL;
  if (N < 5) return fail(ctx, SWALE_EINVAL, "N must be >= 5");
  if (N > 0x7fffffffLL) return fail(ctx, SWALE_EINVAL, "N must be < 2^31");
  if (!x_nodes || !q0 || !hu || !b) return fail(ctx, SWALE_EINVAL, "x_nodes, q0, hu and b are required");
  if ((ctx->cfg.mesh == SWALE_MESH_PROFILE || ctx->cfg.mesh == SWALE_MESH_LINEAR) && !profile)
    return fail(ctx, SWALE_EINVAL, "profile and linear motion need the node profile");
  std::vector<double> x, q, m, bb, P;
  swale_status s;
  if ((s = fetch(ctx, x_nodes, N + 1, x)) || (s = fetch(ctx, q0, N, q)) || (s = fetch(ctx, hu, N, m)) ||
      (s = fetch(ctx, b, N, bb)))
    return s;
  if (profile) {
    if ((s = fetch(ctx, profile, N + 1, P))) return s;
  } else {
    P.assign(N + 1, 0.0);
  }
  return set_instances(ctx, {0, N}, x, q, m, bb, P, {ctx->cfg.cfl}, q0_is_eta != 0);
}

swale_status swale_batch_set_problem(swale_ctx* ctx, int64_t B, const int64_t* offsets, const double* x_nodes,
                                     const double* q0, const double* hu, const double* b, const double* profile,
                                     const double* cfl, int32_t q0_is_eta) {
  if (!ctx) return SWALE_EINVAL;
  if (B < 1 || B > 0x7fffffff) return fail(ctx, SWALE_EINVAL, "B must be >= 1");
  if (!offsets || !x_nodes || !q0 || !hu || !b)
    return fail(ctx, SWALE_EINVAL, "offsets, x_nodes, q0, hu and b are required");
  if ((ctx->cfg.mesh == SWALE_MESH_PROFILE || ctx->cfg.mesh == SWALE_MESH_LINEAR) && !profile)
    return fail(ctx, SWALE_EINVAL, "profile and linear motion need the node profile");
  std::vector<int64_t> off;
  swale_status s;
  if ((s = fetch(ctx, offsets, (size_t)B + 1, off))) return s;
  if (off[0] != 0) return fail(ctx, SWALE_EINVAL, "offsets[0] must be 0");
  for (int64_t i = 0; i < B; ++i)
    if (off[i + 1] - off[i] < 5) return fail(ctx, SWALE_EINVAL, "every instance needs N >= 5 cells");
  if (off[B] > 0x7fffffffLL) return fail(ctx, SWALE_EINVAL, "total cells must be < 2^31");
  const int64_t Ntot = off[B];
  std::vector<double> x, q, m, bb, P, c;
  if ((s = fetch(ctx, x_nodes, Ntot + B, x)) || (s = fetch(ctx, q0, Ntot, q)) || (s = fetch(ctx, hu, Ntot, m)) ||
      (s = fetch(ctx, b, Ntot, bb)))
    return s;
  if (profile) {
    if ((s = fetch(ctx, profile, Ntot + B, P))) return s;
  } else {
    P.assign(Ntot + B, 0.0);
  }
  if (cfl) {
    if ((s = fetch(ctx, cfl, (size_t)B, c))) return s;
  } else {
    c.assign(B, ctx->cfg.cfl);
  }
  return set_instances(ctx, off, x, q, m, bb, P, c, q0_is_eta != 0);
}

swale_status swale_step(swale_ctx* ctx, double* dt_out) {
  NvtxRange nvtx_range("swale_step");
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  if (swale_status s = enqueue_step(ctx)) return s;
  if (dt_out) {
    SW_CUDA(ctx, cudaMemcpyAsync(dt_out, &ctx->D.S->dt, sizeof(double), cudaMemcpyDefault, ctx->stream));
    SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return SWALE_OK;
}

swale_status swale_advance(swale_ctx* ctx, int64_t max_steps, int64_t* steps_done) {
  NvtxRange nvtx_range("swale_advance");
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  if (max_steps < 0) return fail(ctx, SWALE_EINVAL, "max_steps < 0");
  long long s0 = 0;
  SW_CUDA(ctx, cudaMemcpyAsync(&s0, &ctx->D.S->steps, sizeof(s0), cudaMemcpyDeviceToHost, ctx->stream));
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<DevScalars> S;
  const double t_end = ctx->cfg.t_end;
  if (t_end > 0.0) {
    // With an end time, the steps go out in chunks of growing length (64 .. 4096 steps); after
    // each, the host reads the instances' scalars and stops once every instance has reached
    // t_end or stopped on an error (the prologue's test), so that a generous max_steps does not
    // launch a long tail of no-op steps.
    int64_t left = max_steps, chunk = 64;
    while (left > 0) {
      const int64_t n = std::min(left, chunk);
      if (swale_status s = enqueue_steps(ctx, n)) return s;
      left -= n;
      if (left == 0) break;
      if (swale_status s = read_scalars(ctx, S)) return s;
      bool idle = true;
      for (const DevScalars& v : S)
        if (!((v.status & kErrBits) || v.t >= t_end)) {
          idle = false;
          break;
        }
      if (idle) break;
      chunk = std::min<int64_t>(2 * chunk, 4096);
    }
  } else {
    if (swale_status s = enqueue_steps(ctx, max_steps)) return s;
  }
  if (swale_status s = read_scalars(ctx, S)) return s;
  unsigned int bits = 0;
  for (const DevScalars& v : S) bits |= v.status;
  if (steps_done) *steps_done = S[0].steps - s0;
  return status_from_bits(ctx, bits);
}

swale_status swale_enqueue(swale_ctx* ctx, int64_t nsteps) {
  NvtxRange nvtx_range("swale_enqueue");
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  if (nsteps < 0) return fail(ctx, SWALE_EINVAL, "nsteps < 0");
  return enqueue_steps(ctx, nsteps);
}

swale_status swale_set_timing(swale_ctx* ctx, int32_t enable) {
  if (!ctx) return SWALE_EINVAL;
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->timing = enable != 0;
  ctx->ev_used = 0;
  ctx->ev_family.clear();
  return SWALE_OK;
}

swale_status swale_get_timing(swale_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx) return SWALE_EINVAL;
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double acc[FAM_COUNT] = {0, 0, 0, 0};
  int64_t cnt[FAM_COUNT] = {0, 0, 0, 0};
  for (size_t i = 0; i < ctx->ev_family.size(); ++i) {
    float m = 0.f;
    SW_CUDA(ctx, cudaEventElapsedTime(&m, ctx->ev_pool[2 * i], ctx->ev_pool[2 * i + 1]));
    acc[ctx->ev_family[i]] += m;
    cnt[ctx->ev_family[i]] += 1;
  }
  for (int f = 0; f < FAM_COUNT; ++f) {
    if (ms) ms[f] = acc[f];
    if (launches) launches[f] = cnt[f];
  }
  return SWALE_OK;
}

swale_status swale_get_state(swale_ctx* ctx, double* h, double* hu, double* b, double* eta, double* x_nodes,
                             double* t) {
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  if (ctx->B != 1) return fail(ctx, SWALE_EINVAL, "a batch: use swale_batch_get_state");
  const int64_t N = ctx->Ntot;
  const size_t cb = N * sizeof(double);
  swale_status s;
  if ((s = put_out(ctx, hu, ctx->D.M0, cb)) || (s = put_out(ctx, b, ctx->D.B0, cb)) ||
      (s = put_out(ctx, eta, ctx->D.E0, cb)) || (s = put_out(ctx, x_nodes, ctx->D.x, cb + sizeof(double))) ||
      (s = put_out(ctx, t, &ctx->D.S->t, sizeof(double))))
    return s;
  if (h) {
    std::vector<double> E(N), B(N);
    SW_CUDA(ctx, cudaMemcpyAsync(E.data(), ctx->D.E0, cb, cudaMemcpyDeviceToHost, ctx->stream));
    SW_CUDA(ctx, cudaMemcpyAsync(B.data(), ctx->D.B0, cb, cudaMemcpyDeviceToHost, ctx->stream));
    SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t j = 0; j < N; ++j) E[j] -= B[j];
    SW_CUDA(ctx, cudaMemcpyAsync(h, E.data(), cb, cudaMemcpyDefault, ctx->stream));
  }
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SWALE_OK;
}

swale_status swale_batch_get_state(swale_ctx* ctx, double* hu, double* b, double* eta, double* x_nodes, double* t,
                                   double* dt) {
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  const size_t cb = ctx->Ntot * sizeof(double), nb = (ctx->Ntot + ctx->B) * sizeof(double);
  swale_status s;
  if ((s = put_out(ctx, hu, ctx->D.M0, cb)) || (s = put_out(ctx, b, ctx->D.B0, cb)) ||
      (s = put_out(ctx, eta, ctx->D.E0, cb)) || (s = put_out(ctx, x_nodes, ctx->D.x, nb)))
    return s;
  if (t || dt) {
    std::vector<DevScalars> S;
    if ((s = read_scalars(ctx, S))) return s;
    std::vector<double> tv(ctx->B), dv(ctx->B);
    for (int64_t i = 0; i < ctx->B; ++i) {
      tv[i] = S[i].t;
      dv[i] = S[i].dt;
    }
    if (t) SW_CUDA(ctx, cudaMemcpyAsync(t, tv.data(), ctx->B * sizeof(double), cudaMemcpyDefault, ctx->stream));
    if (dt) SW_CUDA(ctx, cudaMemcpyAsync(dt, dv.data(), ctx->B * sizeof(double), cudaMemcpyDefault, ctx->stream));
  }
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SWALE_OK;
}

swale_status swale_get_flags(swale_ctx* ctx, uint8_t* flags) {
  if (!ctx || !flags) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  if (ctx->B == 1) {
    SW_CUDA(ctx, cudaMemcpyAsync(flags, ctx->D.flags + 1, ctx->Ntot, cudaMemcpyDefault, ctx->stream));
  } else {
    if (!ctx->flag_buf)
      if (swale_status s = dalloc(ctx, ctx->allocs, &ctx->flag_buf, (size_t)ctx->Ntot)) return s;
    k_gather_flags<<<(unsigned)std::min<int64_t>(ctx->B, 65535), 256, 0, ctx->stream>>>(ctx->D, (int32_t)ctx->B,
                                                                                        ctx->flag_buf);
    SW_CUDA(ctx, cudaGetLastError());
    SW_CUDA(ctx, cudaMemcpyAsync(flags, ctx->flag_buf, ctx->Ntot, cudaMemcpyDefault, ctx->stream));
  }
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SWALE_OK;
}

swale_status swale_get_status(swale_ctx* ctx, uint32_t* status_bits, int64_t* steps, double* last_dt) {
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  std::vector<DevScalars> S;
  if (swale_status s = read_scalars(ctx, S)) return s;
  unsigned int bits = 0;
  for (const DevScalars& v : S) bits |= v.status;
  if (status_bits) *status_bits = bits;
  if (steps) *steps = S[0].steps;
  if (last_dt) *last_dt = S[0].dt;
  return SWALE_OK;
}

namespace {
constexpr char kSaveMagic[8] = {'S', 'W', 'A', 'L', 'E', 'S', 'T', '1'};
constexpr uint32_t kSaveVersion = 2;
}  // namespace

swale_status swale_save(swale_ctx* ctx, const char* path) {
  if (!ctx || !path) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  const int64_t B = ctx->B, Nt = ctx->Ntot, NN = Nt + B;
  const DevState& D = ctx->D;
  std::vector<double> E(Nt), M(Nt), Bb(Nt), J(Nt), x(NN), P(NN), cfl(B), br, cf;
  std::vector<DevScalars> S(B);
  std::vector<InstConst> ic(B);
  cudaStream_t st = ctx->stream;
  SW_CUDA(ctx, cudaMemcpyAsync(E.data(), D.E0, Nt * 8, cudaMemcpyDeviceToHost, st));
  SW_CUDA(ctx, cudaMemcpyAsync(M.data(), D.M0, Nt * 8, cudaMemcpyDeviceToHost, st));
  SW_CUDA(ctx, cudaMemcpyAsync(Bb.data(), D.B0, Nt * 8, cudaMemcpyDeviceToHost, st));
  SW_CUDA(ctx, cudaMemcpyAsync(J.data(), D.J0, Nt * 8, cudaMemcpyDeviceToHost, st));
  SW_CUDA(ctx, cudaMemcpyAsync(x.data(), D.x, NN * 8, cudaMemcpyDeviceToHost, st));
  SW_CUDA(ctx, cudaMemcpyAsync(P.data(), D.P, NN * 8, cudaMemcpyDeviceToHost, st));
  SW_CUDA(ctx, cudaMemcpyAsync(S.data(), D.S, B * sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
  SW_CUDA(ctx, cudaMemcpyAsync(ic.data(), D.IC, B * sizeof(InstConst), cudaMemcpyDeviceToHost, st));
  if (ctx->bot_pieces > 0) {
    br.resize(ctx->bot_pieces + 1);
    cf.resize((size_t)ctx->bot_pieces * (ctx->bot_deg + 1));
    SW_CUDA(ctx, cudaMemcpyAsync(br.data(), ctx->bot_breaks, br.size() * 8, cudaMemcpyDeviceToHost, st));
    SW_CUDA(ctx, cudaMemcpyAsync(cf.data(), ctx->bot_coef, cf.size() * 8, cudaMemcpyDeviceToHost, st));
  }
  SW_CUDA(ctx, cudaStreamSynchronize(st));
  for (int64_t i = 0; i < B; ++i) cfl[i] = ic[i].cfl;
  std::ofstream f(path, std::ios::binary | std::ios::trunc);
  if (!f) return fail(ctx, SWALE_EINVAL, std::string("cannot open ") + path);
  auto put = [&](const void* p, size_t n) { f.write(reinterpret_cast<const char*>(p), (std::streamsize)n); };
  const uint32_t ver = kSaveVersion, ssz = (uint32_t)sizeof(DevScalars);
  put(kSaveMagic, 8);
  put(&ver, 4);
  put(&ssz, 4);
  put(&ctx->cfg, sizeof(swale_config));
  put(&B, 8);
  put(&Nt, 8);
  put(ctx->off.data(), (B + 1) * 8);
  put(cfl.data(), B * 8);
  for (const std::vector<double>* v : {&E, &M, &Bb, &J, &x, &P}) put(v->data(), v->size() * 8);
  put(S.data(), B * sizeof(DevScalars));
  const int32_t np = ctx->bot_pieces, deg = ctx->bot_deg;
  put(&np, 4);
  put(&deg, 4);
  if (np > 0) {
    put(br.data(), br.size() * 8);
    put(cf.data(), cf.size() * 8);
  }
  f.close();
  if (!f) return fail(ctx, SWALE_EINVAL, std::string("write failed: ") + path);
  return SWALE_OK;
}

swale_status swale_load(swale_ctx* ctx, const char* path) {
  if (!ctx || !path) return SWALE_EINVAL;
  std::ifstream f(path, std::ios::binary);
  if (!f) return fail(ctx, SWALE_EINVAL, std::string("cannot open ") + path);
  auto get = [&](void* p, size_t n) { return (bool)f.read(reinterpret_cast<char*>(p), (std::streamsize)n); };
  char magic[8];
  uint32_t ver = 0, ssz = 0;
  swale_config cfg;
  int64_t B = 0, Nt = 0;
  if (!get(magic, 8) || std::memcmp(magic, kSaveMagic, 8) != 0) return fail(ctx, SWALE_EINVAL, "not a state file");
  if (!get(&ver, 4) || ver != kSaveVersion || !get(&ssz, 4) || ssz != sizeof(DevScalars))
    return fail(ctx, SWALE_EINVAL, "state file of another version");
  if (!get(&cfg, sizeof(cfg)) || std::memcmp(&cfg, &ctx->cfg, sizeof(cfg)) != 0)
    return fail(ctx, SWALE_EINVAL, "the state file was written under another configuration");
  if (!get(&B, 8) || !get(&Nt, 8) || B < 1 || Nt < 5 * B || Nt > 0x7fffffffLL || B > Nt)
    return fail(ctx, SWALE_EINVAL, "bad sizes in the state file");
  const int64_t NN = Nt + B;
  std::vector<int64_t> off(B + 1);
  std::vector<double> cfl(B), E(Nt), M(Nt), Bb(Nt), J(Nt), x(NN), P(NN);
  std::vector<DevScalars> S(B);
  bool ok = get(off.data(), (B + 1) * 8) && get(cfl.data(), B * 8);
  for (std::vector<double>* v : {&E, &M, &Bb, &J, &x, &P}) ok = ok && get(v->data(), v->size() * 8);
  ok = ok && get(S.data(), B * sizeof(DevScalars));
  int32_t np = 0, deg = 0;
  ok = ok && get(&np, 4) && get(&deg, 4);
  std::vector<double> br, cf;
  if (ok && np > 0) {
    if (np > (1 << 20) || deg < 0 || deg > 8) return fail(ctx, SWALE_EINVAL, "bad bottom function in the state file");
    br.resize(np + 1);
    cf.resize((size_t)np * (deg + 1));
    ok = get(br.data(), br.size() * 8) && get(cf.data(), cf.size() * 8);
  }
  if (!ok) return fail(ctx, SWALE_EINVAL, "truncated state file");
  if (off[0] != 0 || off[B] != Nt) return fail(ctx, SWALE_EINVAL, "bad offsets in the state file");
  // (a saved run may hold rounding-level negative depths in dry cells: not re-checked)
  if (swale_status s = set_instances(ctx, off, x, E, M, Bb, P, cfl, true, false)) return s;
  // The state as it was: the widths of the GCL recursion and the per-instance scalars (time,
  // step count, extrema); no mesh geometry is cached for it.
  for (DevScalars& v : S) v.geo_tag = 0;
  SW_CUDA(ctx, cudaMemcpyAsync(ctx->D.J0, J.data(), Nt * 8, cudaMemcpyHostToDevice, ctx->stream));
  SW_CUDA(ctx, cudaMemcpyAsync(ctx->D.S, S.data(), B * sizeof(DevScalars), cudaMemcpyHostToDevice, ctx->stream));
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (np > 0) return swale_set_bottom_function(ctx, np, deg, br.data(), cf.data());
  return SWALE_OK;
}

swale_status swale_set_bottom_function(swale_ctx* ctx, int32_t npieces, int32_t degree, const double* breaks,
                                       const double* coef) {
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "set the problem first");
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  drop_graph(ctx);
  if (npieces == 0) {
    ctx->bot_pieces = 0;
    return SWALE_OK;
  }
  if (npieces < 0 || npieces > (1 << 20) || degree < 0 || degree > 8 || !breaks || !coef)
    return fail(ctx, SWALE_EINVAL, "need 1 <= npieces <= 2^20, 0 <= degree <= 8, breaks and coef");
  std::vector<double> br, cf, x;
  swale_status st;
  if ((st = fetch(ctx, breaks, (size_t)npieces + 1, br)) || (st = fetch(ctx, coef, (size_t)npieces * (degree + 1), cf)))
    return st;
  for (int32_t p = 0; p < npieces; ++p)
    if (!(br[p + 1] > br[p]) || !std::isfinite(br[p]) || !std::isfinite(br[p + 1]))
      return fail(ctx, SWALE_EINVAL, "breakpoints must be finite and increasing");
  for (double c : cf)
    if (!std::isfinite(c)) return fail(ctx, SWALE_EINVAL, "non-finite coefficient");
  if ((st = fetch(ctx, (const double*)ctx->D.x, (size_t)(ctx->Ntot + ctx->B), x))) return st;
  for (int64_t i = 0; i < ctx->B; ++i)
    if (x[ctx->off[i] + i] < br[0] || x[ctx->off[i + 1] + i] > br[npieces])
      return fail(ctx, SWALE_EINVAL, "the breakpoints must cover every instance's domain");
  double *dbr = nullptr, *dcf = nullptr;
  if ((st = dalloc(ctx, ctx->allocs, &dbr, br.size())) || (st = dalloc(ctx, ctx->allocs, &dcf, cf.size())))
    return st;
  if (!ctx->D.xn && (st = dalloc(ctx, ctx->allocs, &ctx->D.xn, (size_t)(ctx->Ntot + ctx->B)))) return st;
  SW_CUDA(ctx, cudaMemcpyAsync(dbr, br.data(), br.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  SW_CUDA(ctx, cudaMemcpyAsync(dcf, cf.data(), cf.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->bot_breaks = dbr;
  ctx->bot_coef = dcf;
  ctx->bot_pieces = npieces;
  ctx->bot_deg = degree;
  return SWALE_OK;
}

swale_status swale_set_tiles(swale_ctx* ctx, int32_t recon_tile, int32_t update_tile, int32_t recon_grid,
                             int32_t update_grid) {
  if (!ctx) return SWALE_EINVAL;
  if (!valid_tile(recon_tile) || !valid_tile(update_tile) || recon_grid < 0 || update_grid < 0)
    return fail(ctx, SWALE_EINVAL, "tiles must be 64, 128 or 256 and grids >= 0");
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const bool retile = (recon_tile != ctx->Tr || update_tile != ctx->Tu);
  ctx->Tr = recon_tile;
  ctx->Tu = update_tile;
  ctx->grid_r = recon_grid;
  ctx->grid_u = update_grid;
  drop_graph(ctx);
  if (retile && ctx->B > 0) return rebuild_tiles(ctx);
  return SWALE_OK;
}

swale_status swale_get_tiles(swale_ctx* ctx, int32_t* tiles) {
  if (!ctx || !tiles) return SWALE_EINVAL;
  tiles[0] = ctx->Tr;
  tiles[1] = ctx->Tu;
  tiles[2] = ctx->grid_r;
  tiles[3] = ctx->grid_u;
  return SWALE_OK;
}

swale_status swale_autotune(swale_ctx* ctx, int32_t steps, const char* cache_path, int32_t* tiles_out) {
  NvtxRange nvtx_range("swale_autotune");
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  if (steps < 1) return fail(ctx, SWALE_EINVAL, "steps must be >= 1");
  int dev = 0, sms = 0;
  SW_CUDA(ctx, cudaGetDevice(&dev));
  SW_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // Cache key: device size, batch shape (instances, log2 of the cells), mesh kind.
  std::ostringstream key;
  key << "sm" << sms << "_B" << ctx->B << "_N2^" << (int)std::lround(std::log2((double)ctx->Ntot)) << "_mesh"
      << ctx->cfg.mesh;
  if (cache_path && *cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      if (line.find("\"" + key.str() + "\"") == std::string::npos) continue;
      int v[4];
      const char* names[4] = {"\"recon_tile\":", "\"update_tile\":", "\"recon_grid\":", "\"update_grid\":"};
      bool ok = true;
      for (int k = 0; k < 4 && ok; ++k) {
        size_t p = line.find(names[k]);
        if (p == std::string::npos) ok = false;
        else v[k] = std::atoi(line.c_str() + p + std::strlen(names[k]));
      }
      if (ok && valid_tile(v[0]) && valid_tile(v[1])) {
        if (swale_status s = swale_set_tiles(ctx, v[0], v[1], v[2], v[3])) return s;
        if (tiles_out) swale_get_tiles(ctx, tiles_out);
        return SWALE_OK;
      }
    }
  }
  // Snapshot of the evolving state; every candidate runs from it and it is restored after.
  DevState& D = ctx->D;
  const size_t cb = ctx->Ntot * sizeof(double), nb = (ctx->Ntot + ctx->B) * sizeof(double);
  const size_t sb = ctx->B * sizeof(DevScalars);
  std::vector<void*> snap_allocs;
  double *sE = nullptr, *sM = nullptr, *sB = nullptr, *sJ = nullptr, *sx = nullptr;
  DevScalars* sS = nullptr;
  swale_status s = SWALE_OK;
  if (!s) s = dalloc(ctx, snap_allocs, &sE, ctx->Ntot);
  if (!s) s = dalloc(ctx, snap_allocs, &sM, ctx->Ntot);
  if (!s) s = dalloc(ctx, snap_allocs, &sB, ctx->Ntot);
  if (!s) s = dalloc(ctx, snap_allocs, &sJ, ctx->Ntot);
  if (!s) s = dalloc(ctx, snap_allocs, &sx, ctx->Ntot + ctx->B);
  if (!s) s = dalloc(ctx, snap_allocs, &sS, (size_t)ctx->B);
  auto release = [&](swale_status r) {
    cudaStreamSynchronize(ctx->stream);
    for (void* p : snap_allocs) cudaFree(p);
    return r;
  };
  if (s) return release(s);
  auto copy_state = [&](bool save) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    double* dst[5] = {sE, sM, sB, sJ, sx};
    double* src[5] = {D.E0, D.M0, D.B0, D.J0, D.x};
    const size_t sz[5] = {cb, cb, cb, cb, nb};
    for (int i = 0; i < 5 && !e; ++i)
      e = save ? cudaMemcpyAsync(dst[i], src[i], sz[i], k, ctx->stream)
               : cudaMemcpyAsync(src[i], dst[i], sz[i], k, ctx->stream);
    if (!e) e = save ? cudaMemcpyAsync(sS, D.S, sb, k, ctx->stream) : cudaMemcpyAsync(D.S, sS, sb, k, ctx->stream);
    return e;
  };
  if (cudaError_t e = copy_state(true)) return release(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
  const bool timing = ctx->timing;
  ctx->timing = false;
  const int occ_r = 6, occ_u = 8;  // resident 128-thread blocks per SM of the persistent candidates
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = INFINITY;
  int bt[4] = {ctx->Tr, ctx->Tu, ctx->grid_r, ctx->grid_u};
  const int tiles[3] = {64, 128, 256};
  for (int tr : tiles)
    for (int tu : tiles)
      for (int pers = 0; pers < 2 && !s; ++pers) {
        const int gr = pers ? sms * occ_r * 128 / tr : 0, gu = pers ? sms * occ_u * 128 / tu : 0;
        s = swale_set_tiles(ctx, tr, tu, gr, gu);
        if (s) break;
        float ms = 0.f;
        cudaError_t e = copy_state(false);
        bump_geo(ctx);
        // One untimed step, then the timed ones, three times: the candidate's time is the
        // fastest of the three (the top candidates lie within a per cent of each other, about
        // the spread of a single short timing).
        if (!e && !(s = enqueue_steps(ctx, 1))) {
          ms = INFINITY;
          for (int rep = 0; rep < 3 && !s && !e; ++rep) {
            float m = 0.f;
            cudaEventRecord(e0, ctx->stream);
            s = enqueue_steps(ctx, steps);
            cudaEventRecord(e1, ctx->stream);
            e = cudaEventSynchronize(e1);
            if (!e) e = cudaEventElapsedTime(&m, e0, e1);
            if (!e) ms = std::min(ms, m);
          }
        }
        if (e) s = fail(ctx, SWALE_ECUDA, cudaGetErrorString(e));
        if (!s && ms < best) {
          best = ms;
          bt[0] = tr;
          bt[1] = tu;
          bt[2] = gr;
          bt[3] = gu;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->timing = timing;
  if (!s) s = swale_set_tiles(ctx, bt[0], bt[1], bt[2], bt[3]);
  if (!s) {
    if (cudaError_t e = copy_state(false)) s = fail(ctx, SWALE_ECUDA, cudaGetErrorString(e));
    bump_geo(ctx);
  }
  if (!s && cache_path && *cache_path) {
    std::ofstream outf(cache_path, std::ios::app);
    outf << "{\"key\": \"" << key.str() << "\", \"recon_tile\": " << bt[0] << ", \"update_tile\": " << bt[1]
         << ", \"recon_grid\": " << bt[2] << ", \"update_grid\": " << bt[3] << ", \"ms_per_step\": "
         << best / steps << "}\n";
  }
  if (!s && tiles_out) swale_get_tiles(ctx, tiles_out);
  return release(s);
}

swale_status swale_rhs(swale_ctx* ctx, int64_t N, const double* E, const double* M, const double* B,
                       const double* J, const double* w, double alpha, double* RE, double* RM, double* RB,
                       double* A_out, uint8_t* flags, uint32_t* status_bits) {
  if (!ctx) return SWALE_EINVAL;
  if (N < 5) return fail(ctx, SWALE_EINVAL, "N must be >= 5");
  if (!E || !M || !B || !J || !w || !RE || !RM || !RB) return fail(ctx, SWALE_EINVAL, "null array");
  swale_ctx tmp;
  tmp.cfg = ctx->cfg;
  tmp.stream = ctx->stream;
  DevState& D = tmp.D;
  swale_status s = alloc_state(&tmp, 1, N, D);
  double* R3 = nullptr;
  if (!s) s = dalloc(&tmp, tmp.allocs, &R3, 3 * (size_t)N);
  auto cleanup = [&](swale_status r) {
    cudaStreamSynchronize(tmp.stream);
    free_state(&tmp);
    tmp.stream = nullptr;
    if (r != SWALE_OK && !tmp.err.empty()) ctx->err = tmp.err;
    return r;
  };
  if (s) return cleanup(s);
  tmp.B = 1;
  tmp.Ntot = N;
  const size_t cb = N * sizeof(double);
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMemcpyAsync(D.E0, E, cb, cudaMemcpyDefault, st);
  e = e ? e : cudaMemcpyAsync(D.M0, M, cb, cudaMemcpyDefault, st);
  e = e ? e : cudaMemcpyAsync(D.B0, B, cb, cudaMemcpyDefault, st);
  e = e ? e : cudaMemcpyAsync(D.J0, J, cb, cudaMemcpyDefault, st);
  e = e ? e : cudaMemcpyAsync(D.w, w, cb + sizeof(double), cudaMemcpyDefault, st);
  if (e) return cleanup(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
  std::vector<InstConst> ic(1);
  std::memset(ic.data(), 0, sizeof(InstConst));
  ic[0].N = N;
  ic[0].cfl = 1.0;
  DevScalars S0;
  std::memset(&S0, 0, sizeof(S0));
  S0.Jmin0 = 0x3ff0000000000000ull;  // 1.0: keeps the unused stage-1 dt arithmetic finite
  e = cudaMemcpyAsync(D.S, &S0, sizeof(S0), cudaMemcpyHostToDevice, st);
  if (e) return cleanup(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
  if ((s = build_tiles(&tmp, ic))) return cleanup(s);
  StepConst K = step_const(&tmp);
  K.t_end = 0.0;
  K.mesh = SWALE_MESH_STATIC;
  k_widths_max<<<64, 256, 0, st>>>(D.J0, N, D.S);
  launch_recon<1>(K, D, tmp.Tr, grid_of(D.nr, 0), st, D.E0, D.M0, D.B0, D.J0);
  unsigned long long Abits = 0;
  e = cudaGetLastError();
  e = e ? e : cudaMemcpyAsync(&Abits, &D.S->A[0], 8, cudaMemcpyDeviceToHost, st);
  e = e ? e : cudaStreamSynchronize(st);
  if (e) return cleanup(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
  double A;
  std::memcpy(&A, &Abits, 8);
  if (!(alpha > 0.0) && K.wave_rel) {
    alpha = A;  // Eq. alpha2D: the wave speeds were taken relative to w
  } else if (!(alpha > 0.0)) {
    std::vector<double> wh(N + 1);
    e = cudaMemcpy(wh.data(), w, (N + 1) * sizeof(double), cudaMemcpyDefault);
    if (e) return cleanup(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
    double wb = 0.0;
    for (double v : wh) wb = std::max(wb, std::fabs(v));
    alpha = A + wb;
  }
  RhsOut ro{R3, R3 + N, R3 + 2 * N, alpha};
  launch_update<2, 1>(K, D, tmp.Tu, grid_of(D.nf, 0), st, D.E0, D.M0, D.B0, D.J0, ro);
  e = cudaGetLastError();
  e = e ? e : cudaMemcpyAsync(RE, ro.RE, cb, cudaMemcpyDefault, st);
  e = e ? e : cudaMemcpyAsync(RM, ro.RM, cb, cudaMemcpyDefault, st);
  e = e ? e : cudaMemcpyAsync(RB, ro.RB, cb, cudaMemcpyDefault, st);
  if (flags) e = e ? e : cudaMemcpyAsync(flags, D.flags + 1, N, cudaMemcpyDefault, st);
  unsigned int bits = 0;
  e = e ? e : cudaMemcpyAsync(&bits, &D.S->status, sizeof(bits), cudaMemcpyDeviceToHost, st);
  e = e ? e : cudaStreamSynchronize(st);
  if (e) return cleanup(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
  if (A_out) *A_out = A;
  if (status_bits) *status_bits = bits;
  return cleanup(SWALE_OK);
}

const char* swale_last_error(const swale_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void swale_destroy(swale_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_state(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

}  // extern "C"

// ======================================================================================
// Stage-viscosity log and the discrete adjoint
// ======================================================================================
namespace {

long long device_steps(swale_ctx* ctx) {
  long long s = 0;
  cudaMemcpyAsync(&s, &ctx->D.S->steps, sizeof(s), cudaMemcpyDeviceToHost, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  return s;
}

template <int STAGE>
void launch_adj_stage(swale_ctx* ctx, const DevState& D, const StepConst& K, const AdjState& A, const double* E,
                      const double* M, const double* B, const double* J) {
  cudaStream_t s = ctx->stream;
  const unsigned gu = grid_of(D.nu, ctx->grid_u), gr = grid_of(D.nr, ctx->grid_r);
  const int Tu = ctx->Tu, Tr = ctx->Tr;
  if (Tu == 64) {
    k_adj_flux<STAGE, 64><<<gu, 64, 0, s>>>(K, D, A);
    k_adj_source<STAGE, 64><<<gu, 64, 0, s>>>(K, D, A, E, B, J);
  } else if (Tu == 256) {
    k_adj_flux<STAGE, 256><<<gu, 256, 0, s>>>(K, D, A);
    k_adj_source<STAGE, 256><<<gu, 256, 0, s>>>(K, D, A, E, B, J);
  } else {
    k_adj_flux<STAGE, 128><<<gu, 128, 0, s>>>(K, D, A);
    k_adj_source<STAGE, 128><<<gu, 128, 0, s>>>(K, D, A, E, B, J);
  }
  if (Tr == 64) k_adj_recon<STAGE, 64><<<gr, 64, 0, s>>>(K, D, A, E, M, B, J);
  else if (Tr == 256) k_adj_recon<STAGE, 256><<<gr, 256, 0, s>>>(K, D, A, E, M, B, J);
  else k_adj_recon<STAGE, 128><<<gr, 128, 0, s>>>(K, D, A, E, M, B, J);
}

template <int PH>
void launch_adj_rk(swale_ctx* ctx, const DevState& D, const AdjState& A) {
  const unsigned gu = grid_of(D.nu, ctx->grid_u);
  if (ctx->Tu == 64) k_adj_rk<PH, 64><<<gu, 64, 0, ctx->stream>>>(D, A);
  else if (ctx->Tu == 256) k_adj_rk<PH, 256><<<gu, 256, 0, ctx->stream>>>(D, A);
  else k_adj_rk<PH, 128><<<gu, 128, 0, ctx->stream>>>(D, A);
}


// Copies of the evolving state (q^n, J^n, nodes, per-instance scalars).
struct StateCopy {
  double *E, *M, *B, *J, *x;
  DevScalars* S;
};

// Bytes one array of swale_adjoint takes in its block: rounded up to 256 bytes, plus 256 bytes of
// slack as every device array of the library has.
uint64_t adj_block(uint64_t bytes) { return (bytes + 255) / 256 * 256 + 256; }

// Bytes of the device block swale_adjoint carves its arrays from; the list follows the arrays in
// swale_adjoint one for one.
uint64_t adjoint_bytes(int64_t B, int64_t Nt, int64_t nsteps, int64_t ckpt_every, int32_t G, int32_t tape) {
  const int64_t NN = Nt + B, NE = Nt + 2 * B;
  const int64_t C = std::min(ckpt_every, nsteps), nseg = (nsteps + C - 1) / C;
  auto a = [](uint64_t n, uint64_t size) { return adj_block(n * size); };
  const uint64_t copy = 4 * a(Nt, 8) + a(NN, 8) + a(B, sizeof(DevScalars));
  const uint64_t state_set = 15 * a(Nt, 8) + 2 * a(NN, 8) + 10 * a(NE, 8) + a(NE, 1) + a(B, sizeof(DevScalars));
  const uint64_t common = 15 * a(Nt, 8) + 8 * a(NE, 8) + state_set + 2 * a((uint64_t)B * G, 8) +
                          a((uint64_t)nsteps * B * G, 8) + a(B, 8) + a((uint64_t)nsteps * B * 3, 8);
  // Segment buffers (per-step snapshots, and the tape's slots): two, one being recomputed while
  // the other is reversed; one when a single segment covers every step.
  const uint64_t nb = nseg == 1 ? 1 : 2;
  if (tape) {
    // per step of a segment: three stage edge sets with their smooth-class linear and source
    // forms, q^(1), J^(1), q^(2), J^(2), node velocities
    const uint64_t slot = 30 * a(NE, 8) + 3 * a(14 * (uint64_t)NE, 8) + 8 * a(Nt, 8) + a(NN, 8);
    return common + (uint64_t)(nseg + nb * C + 1) * copy + (uint64_t)(nb * C) * slot;
  }
  // two state sets of the step recompute: four further stage edge sets and six sets of forms
  return common + state_set + 40 * a(NE, 8) + 6 * a(14 * (uint64_t)NE, 8) + (uint64_t)(nseg + nb * C + 3) * copy;
}

}  // namespace

namespace {
// The kernels' reciprocal (swale::recip) applied element-wise, grid-stride.
__global__ void k_check_recip(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = swale::recip(x[i]);
}
}  // namespace

extern "C" {

swale_status swale_alpha_log(swale_ctx* ctx, int32_t mode, int64_t nsteps, const double* log) {
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  if (mode < 0 || mode > 2 || (mode != 0 && nsteps < 1)) return fail(ctx, SWALE_EINVAL, "bad mode or nsteps");
  if (mode == 2 && !log) return fail(ctx, SWALE_EINVAL, "replay needs a log");
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  drop_graph(ctx);
  free_alpha_log(ctx);
  if (mode == 0) return SWALE_OK;
  const size_t n = (size_t)nsteps * ctx->B * 3;
  void* q = nullptr;
  if (cudaMalloc(&q, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SWALE_ENOMEM, "alpha log");
  }
  ctx->alpha_log = (double*)q;
  ctx->alpha_cap = nsteps;
  ctx->alpha_base = device_steps(ctx);
  ctx->alpha_mode = mode;
  if (mode == 2) SW_CUDA(ctx, cudaMemcpyAsync(ctx->alpha_log, log, n * sizeof(double), cudaMemcpyDefault, ctx->stream));
  else SW_CUDA(ctx, cudaMemsetAsync(ctx->alpha_log, 0, n * sizeof(double), ctx->stream));
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SWALE_OK;
}

swale_status swale_get_alpha_log(swale_ctx* ctx, double* log) {
  if (!ctx || !log) return SWALE_EINVAL;
  if (!ctx->alpha_log) return fail(ctx, SWALE_EINVAL, "no alpha log");
  SW_CUDA(ctx, cudaMemcpyAsync(log, ctx->alpha_log, (size_t)ctx->alpha_cap * ctx->B * 3 * sizeof(double),
                               cudaMemcpyDefault, ctx->stream));
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SWALE_OK;
}

swale_status swale_adjoint_bytes(int64_t B, int64_t Ntot, int64_t nsteps, int64_t ckpt_every, int32_t G,
                                 int32_t tape, uint64_t* bytes) {
  if (!bytes || B < 1 || Ntot < 1 || nsteps < 1 || ckpt_every < 1 || G < 1 || tape < 0 || tape > 1)
    return SWALE_EINVAL;
  *bytes = adjoint_bytes(B, Ntot, nsteps, ckpt_every, G, tape);
  return SWALE_OK;
}

swale_status swale_set_wait_test(swale_ctx* ctx, int32_t tries, uint32_t pad_bytes) {
  if (!ctx) return SWALE_EINVAL;
  if (tries < 0) return fail(ctx, SWALE_EINVAL, "tries must be >= 0");
  SW_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  drop_graph(ctx);
  ctx->wait_tries = tries;
  ctx->tx_pad = pad_bytes;
  return SWALE_OK;
}

swale_status swale_check_recip(void* cuda_stream, int64_t n, const double* x, double* y) {
  if (n < 0 || (n > 0 && (!x || !y))) return SWALE_EINVAL;
  if (n == 0) return SWALE_OK;
  cudaPointerAttributes ax{}, ay{};
  if (cudaPointerGetAttributes(&ax, x) != cudaSuccess || cudaPointerGetAttributes(&ay, y) != cudaSuccess) {
    cudaGetLastError();
    return SWALE_EINVAL;
  }
  if (ax.type != cudaMemoryTypeDevice || ay.type != cudaMemoryTypeDevice) return SWALE_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || ax.device != dev || ay.device != dev) {
    cudaGetLastError();
    return SWALE_EINVAL;  // the arrays must live on the current device (the stream's)
  }
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_check_recip<<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? SWALE_OK : SWALE_ECUDA;
}

swale_status swale_set_adjoint_tape(swale_ctx* ctx, int32_t enable) {
  if (!ctx) return SWALE_EINVAL;
  if (enable < 0 || enable > 1) return fail(ctx, SWALE_EINVAL, "enable must be 0 or 1");
  ctx->adjoint_tape = enable;
  return SWALE_OK;
}

swale_status swale_adjoint(swale_ctx* ctx, int64_t nsteps, int64_t ckpt_every, int32_t G, const double* gauges_x,
                           const double* h_obs, double* J, double* dJ_deta0, double* dJ_dhu0, double* dJ_db0) {
  if (!ctx) return SWALE_EINVAL;
  if (ctx->B == 0) return fail(ctx, SWALE_EINVAL, "no problem set");
  if (nsteps < 1 || ckpt_every < 1 || G < 1 || !gauges_x || !h_obs)
    return fail(ctx, SWALE_EINVAL, "nsteps, ckpt_every, G >= 1 and gauges, observations required");
  if (ctx->cfg.mesh == SWALE_MESH_FLUID_GAUSS)
    return fail(ctx, SWALE_EINVAL, "the adjoint needs a prescribed mesh (static, profile or linear motion)");
  if (ctx->cfg.t_end > 0.0) return fail(ctx, SWALE_EINVAL, "the adjoint runs a fixed number of steps: t_end = 0");
  if (ctx->bot_pieces > 0) return fail(ctx, SWALE_EINVAL, "the adjoint evolves the bottom (no L2-projection bottom)");
  if (ctx->cfg.scheme != SWALE_SCHEME_HYDROSTATIC)
    return fail(ctx, SWALE_EINVAL, "the adjoint differentiates the hydrostatic well-balanced scheme");
  const int64_t B = ctx->B, Nt = ctx->Ntot, NN = Nt + B, NE = Nt + 2 * B;
  const int64_t C = std::min(ckpt_every, nsteps), nseg = (nsteps + C - 1) / C;
  const bool tape = ctx->adjoint_tape != 0;
  cudaStream_t st = ctx->stream;
  std::vector<void*> mem;
  swale_status s = SWALE_OK;
  // All of the call's device arrays are carved from one block of exactly swale_adjoint_bytes
  // bytes: one cudaMalloc and one cudaFree per call, however many segment buffers and tape
  // slots it holds (at large checkpoint intervals the tape alone has tens of thousands of
  // arrays, whose separate allocations took longer than the gradient).
  const uint64_t arena_bytes = adjoint_bytes(B, Nt, nsteps, ckpt_every, G, tape ? 1 : 0);
  char* arena = nullptr;
  uint64_t arena_off = 0;
  if (cudaError_t e0 = cudaMalloc(&arena, arena_bytes)) {
    cudaGetLastError();
    return fail(ctx, SWALE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e0));
  }
  mem.push_back(arena);
  auto carve = [&](auto** p, size_t n) -> swale_status {
    const uint64_t need = adj_block(n * sizeof(**p));
    if (arena_off + need > arena_bytes) return fail(ctx, SWALE_ENOMEM, "adjoint: scratch layout exceeds its block");
    *p = reinterpret_cast<std::remove_reference_t<decltype(*p)>>(arena + arena_off);
    arena_off += need;
    return SWALE_OK;
  };
  auto alloc_copy = [&](StateCopy& c) {
    if (!s) s = carve(&c.E, (size_t)Nt);
    if (!s) s = carve(&c.M, (size_t)Nt);
    if (!s) s = carve(&c.B, (size_t)Nt);
    if (!s) s = carve(&c.J, (size_t)Nt);
    if (!s) s = carve(&c.x, (size_t)NN);
    if (!s) s = carve(&c.S, (size_t)B);
  };
  // Three streams: the context's (forward run, reverse kernels), st2 (segment recomputes, low
  // priority), st3 (the recompute of each step before its reverse sweep). Events: 0 forward
  // done; 1-2 segment buffer b filled; 3-4 segment buffer b read; 5-6 step recompute on state
  // set k done; 7-8 reverse sweep on state set k done.
  cudaStream_t st2 = nullptr, st3 = nullptr;
  cudaEvent_t ev[9] = {};
  auto release = [&](swale_status r) {
    cudaStreamSynchronize(st);
    if (st2) cudaStreamSynchronize(st2);
    if (st3) cudaStreamSynchronize(st3);
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    if (st2) cudaStreamDestroy(st2);
    if (st3) cudaStreamDestroy(st3);
    for (void* p : mem) cudaFree(p);
    return r;
  };
  AdjState A{};
  double** cellbufs[] = {&A.lE, &A.lM, &A.lB, &A.yE, &A.yM, &A.yB, &A.pE, &A.pM, &A.pB,
                         &A.aE, &A.aM, &A.aB, &A.rE, &A.rM, &A.rB};
  for (double** p : cellbufs)
    if (!s) s = carve(p, (size_t)Nt);
  for (int k = 0; k < 8 && !s; ++k) s = carve(&A.ab[k], (size_t)NE);
  // Every forward run of the adjoint (the forward with checkpoints, the segment and the step
  // recomputes) computes the mesh geometry in all three stages instead of taking stage 1's from
  // the cache: a run that starts from a checkpoint has no cache entry, so with the cache the
  // recomputed trajectory would differ from the forward one by rounding wherever a segment
  // starts, and near a detector or limiter threshold that can flip a frozen branch. Without it
  // the trajectory, and the gradient up to the order of atomic additions, is the same for every
  // checkpoint interval.
  DevState base = ctx->D;
  base.geo = nullptr;
  // The adjoint's forward runs check the status after the fact; they keep no roll-back copies
  // (the further state sets share nothing with the context's backups).
  base.bE = base.bM = base.bB = base.bJ = base.bx = nullptr;
  // A further set of state arrays: its own state, stage, edge and flag arrays and scalars
  // (instance constants, work lists and the motion profile are shared, read only).
  auto alloc_state_set = [&](DevState& X) {
    X = base;
    double** cells[] = {&X.E0, &X.M0, &X.B0, &X.Ea, &X.Ma, &X.Ba, &X.Eb, &X.Mb,
                        &X.Bb, &X.YE, &X.YM, &X.YB, &X.J0, &X.J1, &X.J2};
    for (double** p : cells)
      if (!s) s = carve(p, (size_t)Nt);
    if (!s) s = carve(&X.x, (size_t)NN);
    if (!s) s = carve(&X.w, (size_t)NN);
    double** edges[] = {&X.eEL, &X.eER, &X.eBL, &X.eBR, &X.ehL, &X.ehR, &X.euL, &X.euR, &X.ipair, &X.itri};
    for (double** p : edges)
      if (!s) s = carve(p, (size_t)NE);
    if (!s) s = carve(&X.flags, (size_t)NE);
    if (!s) s = carve(&X.S, (size_t)B);
  };
  // The step recomputes alternate between two state sets R[0] (the context's arrays) and R[1],
  // so that the recompute of step m - 1 (on st3) overlaps the reverse sweep of step m. Each set
  // keeps the edge values of stages 1 and 2 in sets of their own (stage 3 keeps the set's).
  auto alloc_edges = [&](DevState& d) {
    double** ed[] = {&d.eEL, &d.eER, &d.eBL, &d.eBR, &d.ehL, &d.ehR, &d.euL, &d.euR, &d.ipair, &d.itri};
    for (double** p : ed)
      if (!s) s = carve(p, (size_t)NE);
  };
  DevState R[2], Ds[2][3];
  if (!tape) {
    R[0] = base;
    alloc_state_set(R[1]);
    for (int k = 0; k < 2; ++k) {
      Ds[k][0] = Ds[k][1] = Ds[k][2] = R[k];
      for (int t = 0; t < 2; ++t) alloc_edges(Ds[k][t]);
      // each stage's smooth-class linear form and source form, for that stage's reverse kernels
      for (int t = 0; t < 3; ++t)
        if (!s) s = carve(&Ds[k][t].gK, (size_t)14 * NE);
    }
  }
  // Segment recomputes: a third state set D2 recomputes segment sg - 1 into one of two
  // snapshot buffers while segment sg is reversed from the other.
  DevState D2;
  alloc_state_set(D2);
  // Snapshot buffers of two segments (one when a single segment covers every step).
  const int64_t nbuf = nseg == 1 ? 1 : 2;
  std::vector<StateCopy> ckpt(nseg), seg(C), seg2(nbuf == 2 ? C : 0);
  StateCopy fin, snapR[2];
  for (auto& c : ckpt) alloc_copy(c);
  for (auto& c : seg) alloc_copy(c);
  for (auto& c : seg2) alloc_copy(c);
  // Tape mode: the segment recompute keeps every step's stage data in a slot of its own (two
  // segments' worth, like the snapshots): the edge values of the three stages, q^(1), J^(1),
  // q^(2), J^(2) and the node velocities; the reverse sweep reads them instead of recomputing.
  // slot[b][i][t] is state set D2 with stage t's edge arrays and the stage arrays of step i of
  // buffer b.
  std::vector<DevState> slot[2];
  if (tape) {
    for (int b = 0; b < nbuf; ++b) {
      slot[b].resize((size_t)(3 * C));
      for (int64_t i = 0; i < C; ++i) {
        DevState base_i = D2;
        double** st_arr[] = {&base_i.Ea, &base_i.Ma, &base_i.Ba, &base_i.J1,
                             &base_i.Eb, &base_i.Mb, &base_i.Bb, &base_i.J2};
        for (double** p : st_arr)
          if (!s) s = carve(p, (size_t)Nt);
        if (!s) s = carve(&base_i.w, (size_t)NN);
        for (int t = 0; t < 3; ++t) {
          slot[b][3 * i + t] = base_i;
          alloc_edges(slot[b][3 * i + t]);
          if (!s) s = carve(&slot[b][3 * i + t].gK, (size_t)14 * NE);
        }
      }
    }
  }
  alloc_copy(fin);
  if (!tape) {
    alloc_copy(snapR[0]);
    alloc_copy(snapR[1]);
  }
  double *gx = nullptr, *obs = nullptr, *Jacc = nullptr, *alog = nullptr;
  if (!s) s = carve(&gx, (size_t)B * G);
  if (!s) s = carve(&obs, (size_t)nsteps * B * G);
  if (!s) s = carve(&Jacc, (size_t)B);
  if (!s) s = carve(&alog, (size_t)nsteps * B * 3);
  int64_t* gcell = nullptr;  // last cell of each gauge (searched from, the mesh moves little per step)
  if (!s) s = carve(&gcell, (size_t)B * G);
  if (s) return release(s);
  // q^n and J^n of the step being reversed, per state set.
  AdjState AR[2] = {A, A};
  for (int k = 0; k < 2; ++k) {
    AR[k].sE = snapR[k].E;
    AR[k].sM = snapR[k].M;
    AR[k].sB = snapR[k].B;
    AR[k].sJ = snapR[k].J;
  }
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMemcpyAsync(gx, gauges_x, (size_t)B * G * sizeof(double), cudaMemcpyDefault, st);
  e = e ? e : cudaMemcpyAsync(obs, h_obs, (size_t)nsteps * B * G * sizeof(double), cudaMemcpyDefault, st);
  e = e ? e : cudaMemsetAsync(Jacc, 0, B * sizeof(double), st);
  e = e ? e : cudaMemsetAsync(gcell, 0xff, (size_t)B * G * sizeof(int64_t), st);  // -1: not yet located
  e = e ? e : cudaMemsetAsync(A.aE, 0, Nt * sizeof(double), st);
  e = e ? e : cudaMemsetAsync(A.aM, 0, Nt * sizeof(double), st);
  e = e ? e : cudaMemsetAsync(A.aB, 0, Nt * sizeof(double), st);
  e = e ? e : cudaMemsetAsync(A.lE, 0, Nt * sizeof(double), st);
  e = e ? e : cudaMemsetAsync(A.lM, 0, Nt * sizeof(double), st);
  e = e ? e : cudaMemsetAsync(A.lB, 0, Nt * sizeof(double), st);
  int prio_least = 0, prio_greatest = 0;
  e = e ? e : cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  e = e ? e : cudaStreamCreateWithPriority(&st2, cudaStreamNonBlocking, prio_least);
  if (!tape) e = e ? e : cudaStreamCreateWithFlags(&st3, cudaStreamNonBlocking);
  for (cudaEvent_t& x : ev) e = e ? e : cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  if (e) return release(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
  DevState& D = ctx->D;
  auto save_from = [&](StateCopy& c, const DevState& X, cudaStream_t q) {
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    cudaError_t r = cudaMemcpyAsync(c.E, X.E0, Nt * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(c.M, X.M0, Nt * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(c.B, X.B0, Nt * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(c.J, X.J0, Nt * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(c.x, X.x, NN * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(c.S, X.S, B * sizeof(DevScalars), k, q);
    return r;
  };
  auto load_into = [&](const StateCopy& c, const DevState& X, cudaStream_t q) {
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    cudaError_t r = cudaMemcpyAsync(X.E0, c.E, Nt * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(X.M0, c.M, Nt * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(X.B0, c.B, Nt * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(X.J0, c.J, Nt * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(X.x, c.x, NN * sizeof(double), k, q);
    r = r ? r : cudaMemcpyAsync(X.S, c.S, B * sizeof(DevScalars), k, q);
    return r;
  };
  auto save = [&](StateCopy& c) { return save_from(c, D, st); };
  auto load = [&](const StateCopy& c) {
    bump_geo(ctx);
    return load_into(c, D, st);
  };
  // The forward records the stage viscosities; every recomputation replays them.
  double* old_log = ctx->alpha_log;
  const int64_t old_cap = ctx->alpha_cap, old_base = ctx->alpha_base;
  const int32_t old_mode = ctx->alpha_mode;
  const bool old_timing = ctx->timing;
  ctx->timing = false;
  drop_graph(ctx);
  ctx->alpha_log = alog;
  ctx->alpha_cap = nsteps;
  ctx->alpha_base = device_steps(ctx);
  ctx->alpha_mode = 1;
  if (old_mode == 2 && old_log) {
    // A replay log is active: the forward replays its rows for these steps instead of
    // recording new values (the gradient is then that of the scheme with those alphas).
    const int64_t row0 = ctx->alpha_base - old_base;
    if (row0 < 0 || row0 + nsteps > old_cap) {
      ctx->alpha_log = old_log;
      ctx->alpha_cap = old_cap;
      ctx->alpha_base = old_base;
      ctx->alpha_mode = old_mode;
      ctx->timing = old_timing;
      return release(fail(ctx, SWALE_EINVAL, "the active alpha replay log does not cover the adjoint's steps"));
    }
    e = cudaMemcpyAsync(alog, old_log + row0 * B * 3, (size_t)nsteps * B * 3 * sizeof(double),
                        cudaMemcpyDeviceToDevice, st);
    if (e) {
      ctx->alpha_log = old_log;
      ctx->alpha_cap = old_cap;
      ctx->alpha_base = old_base;
      ctx->alpha_mode = old_mode;
      ctx->timing = old_timing;
      return release(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
    }
    ctx->alpha_mode = 2;
  }
  auto restore_ctx = [&]() {
    drop_graph(ctx);
    ctx->alpha_log = old_log;
    ctx->alpha_cap = old_cap;
    ctx->alpha_base = old_base;
    ctx->alpha_mode = old_mode;
    ctx->timing = old_timing;
  };
  const unsigned gg = (unsigned)((B * G + 127) / 128);
  NvtxRange nvtx_adjoint("swale_adjoint");
  nvtxRangePushA("adjoint forward");
  // ---- forward with checkpoints and the misfit ----
  // The last segment is the one the reverse sweep starts with: the forward keeps its per-step
  // snapshots (and in tape mode its stage data) itself, so that segment is not recomputed.
  const int64_t nlast = (nseg - 1) * C, blast = (nseg - 1) & 1;
  std::vector<StateCopy>& buf_last = blast ? seg2 : seg;
  for (int64_t n = 0; n < nsteps && !s; ++n) {
    if (n % C == 0 && (e = save(ckpt[n / C]))) break;
    if (n >= nlast) {
      if ((e = save(buf_last[n - nlast]))) break;
      if (tape) {  // the step's stage data into its slot; the state is the context's own
        DevState f3[3];
        for (int t = 0; t < 3; ++t) {
          f3[t] = slot[blast][(size_t)(3 * (n - nlast) + t)];
          f3[t].E0 = base.E0;
          f3[t].M0 = base.M0;
          f3[t].B0 = base.B0;
          f3[t].J0 = base.J0;
          f3[t].YE = base.YE;
          f3[t].YM = base.YM;
          f3[t].YB = base.YB;
          f3[t].x = base.x;
          f3[t].S = base.S;
          f3[t].flags = base.flags;
        }
        s = enqueue_step_on(ctx, f3[2], st, f3, 0);
      } else {
        s = enqueue_step_on(ctx, base, st, nullptr, 0);
      }
    } else {
      s = enqueue_step_on(ctx, base, st, nullptr, 0);
    }
    if (!s) k_misfit<0><<<gg, 128, 0, st>>>(D, A, (int32_t)B, G, gx, obs + n * B * G, Jacc, gcell);
  }
  if (!s && !e) e = save(fin);
  if (!s && !e) e = cudaGetLastError();
  ctx->alpha_mode = 2;
  StepConst K = step_const(ctx);
  nvtxRangePop();
  NvtxRange nvtx_reverse("adjoint reverse");
  // ---- reverse, segment by segment ----
  // The set D2 recomputes segment sg from its checkpoint on st2, a snapshot per step, into
  // buffer sg % 2.
  auto recompute_segment = [&](int64_t sg) {
    const int64_t n0 = sg * C, n1 = std::min(nsteps, n0 + C);
    std::vector<StateCopy>& buf = (sg & 1) ? seg2 : seg;
    e = load_into(ckpt[sg], D2, st2);
    for (int64_t m = n0; m < n1 && !s && !e; ++m) {
      e = save_from(buf[m - n0], D2, st2);
      if (e) break;
      if (tape) {  // every step, the last one of the segment included, into its slot
        const DevState* sl = &slot[sg & 1][(size_t)(3 * (m - n0))];
        s = enqueue_step_on(ctx, sl[2], st2, sl, 0);
      } else if (m + 1 < n1) {
        s = enqueue_step_on(ctx, D2, st2, nullptr, 0);
      }
    }
    if (!s && !e) e = cudaEventRecord(ev[1 + (sg & 1)], st2);
  };
  if (!s && !e) e = cudaEventRecord(ev[0], st);
  if (!s && !e) e = cudaStreamWaitEvent(st2, ev[0], 0);
  // The last segment's snapshots (and tape) came from the forward run itself.
  if (!s && !e) e = cudaEventRecord(ev[1 + blast], st);
  bool used[2] = {false, false};
  int64_t idx = 0;
  for (int64_t sg = nseg - 1; sg >= 0 && !s && !e; --sg) {
    const int64_t n0 = sg * C, n1 = std::min(nsteps, n0 + C);
    if (sg >= 1) {
      // Segment sg - 1 goes into the buffer whose snapshots of segment sg + 1 st3 has read.
      if (sg + 1 < nseg) e = cudaStreamWaitEvent(st2, ev[3 + ((sg + 1) & 1)], 0);
      if (!e) recompute_segment(sg - 1);
      if (s || e) break;
    }
    const std::vector<StateCopy>& buf = (sg & 1) ? seg2 : seg;
    if (tape) {
      // Reverse sweeps from the tape: step m reads its stage data from slot m - n0 and the state
      // after it (q^{n+1}, J^{n+1}, nodes, scalars with the step's dt and viscosities) from the
      // next snapshot, the next segment's checkpoint or the final state.
      e = cudaStreamWaitEvent(st, ev[1 + (sg & 1)], 0);
      for (int64_t m = n1 - 1; m >= n0 && !s && !e; --m) {
        const StateCopy& before = buf[m - n0];
        const StateCopy& after = (m + 1 < n1) ? buf[m + 1 - n0] : (sg + 1 < nseg ? ckpt[sg + 1] : fin);
        DevState X3[3];
        for (int t = 0; t < 3; ++t) {
          X3[t] = slot[sg & 1][(size_t)(3 * (m - n0) + t)];
          X3[t].E0 = after.E;
          X3[t].M0 = after.M;
          X3[t].B0 = after.B;
          X3[t].J0 = after.J;
          X3[t].x = after.x;
          X3[t].S = after.S;
        }
        const DevState& X = X3[2];
        AdjState At = A;
        At.sE = before.E;
        At.sM = before.M;
        At.sB = before.B;
        At.sJ = before.J;
        k_misfit<1><<<gg, 128, 0, st>>>(X, A, (int32_t)B, G, gx, obs + m * B * G, Jacc, gcell);
        launch_adj_rk<3>(ctx, X, At);
        launch_adj_stage<3>(ctx, X3[2], K, At, X.Eb, X.Mb, X.Bb, X.J2);
        launch_adj_rk<2>(ctx, X, At);
        launch_adj_stage<2>(ctx, X3[1], K, At, X.Ea, X.Ma, X.Ba, X.J1);
        launch_adj_rk<1>(ctx, X, At);
        launch_adj_stage<1>(ctx, X3[0], K, At, before.E, before.M, before.B, before.J);
        launch_adj_rk<0>(ctx, X, At);
        e = cudaGetLastError();
      }
      // The segment's snapshots and slots are free once its reverse sweep is done.
      if (!s && !e) e = cudaEventRecord(ev[3 + (sg & 1)], st);
      continue;
    }
    e = cudaStreamWaitEvent(st3, ev[1 + (sg & 1)], 0);
    for (int64_t m = n1 - 1; m >= n0 && !s && !e; --m, ++idx) {
      const int k = (int)(idx & 1);
      const DevState& X = R[k];
      const StateCopy& c = buf[m - n0];
      // Recompute step m on state set k (st3), once the reverse sweep that last used it is done:
      // q^(1), q^(2), the stage meshes and node velocities stay in the set's state arrays, each
      // stage's edge values in its own set; q^n, J^n go to the set's snapshot.
      if (used[k]) e = cudaStreamWaitEvent(st3, ev[7 + k], 0);
      used[k] = true;
      e = e ? e : load_into(c, X, st3);
      e = e ? e : cudaMemcpyAsync(snapR[k].E, c.E, Nt * sizeof(double), cudaMemcpyDeviceToDevice, st3);
      e = e ? e : cudaMemcpyAsync(snapR[k].M, c.M, Nt * sizeof(double), cudaMemcpyDeviceToDevice, st3);
      e = e ? e : cudaMemcpyAsync(snapR[k].B, c.B, Nt * sizeof(double), cudaMemcpyDeviceToDevice, st3);
      e = e ? e : cudaMemcpyAsync(snapR[k].J, c.J, Nt * sizeof(double), cudaMemcpyDeviceToDevice, st3);
      if (e) break;
      if ((s = enqueue_step_on(ctx, X, st3, Ds[k], 0))) break;
      if ((e = cudaEventRecord(ev[5 + k], st3))) break;
      // Reverse sweep of step m on the context's stream.
      if ((e = cudaStreamWaitEvent(st, ev[5 + k], 0))) break;
      k_misfit<1><<<gg, 128, 0, st>>>(X, A, (int32_t)B, G, gx, obs + m * B * G, Jacc, gcell);
      launch_adj_rk<3>(ctx, X, AR[k]);
      launch_adj_stage<3>(ctx, Ds[k][2], K, AR[k], X.Eb, X.Mb, X.Bb, X.J2);
      launch_adj_rk<2>(ctx, X, AR[k]);
      launch_adj_stage<2>(ctx, Ds[k][1], K, AR[k], X.Ea, X.Ma, X.Ba, X.J1);
      launch_adj_rk<1>(ctx, X, AR[k]);
      launch_adj_stage<1>(ctx, Ds[k][0], K, AR[k], snapR[k].E, snapR[k].M, snapR[k].B, snapR[k].J);
      launch_adj_rk<0>(ctx, X, AR[k]);
      e = cudaGetLastError();
      if (!e) e = cudaEventRecord(ev[7 + k], st);
    }
    if (!s && !e) e = cudaEventRecord(ev[3 + (sg & 1)], st3);
  }
  if (!s && !e) e = load(fin);
  restore_ctx();
  if (s) return release(s);
  if (e) return release(fail(ctx, SWALE_ECUDA, std::string("adjoint: ") + cudaGetErrorString(e)));
  e = cudaSuccess;
  if (J) e = cudaMemcpyAsync(J, Jacc, B * sizeof(double), cudaMemcpyDefault, st);
  if (!e && dJ_deta0) e = cudaMemcpyAsync(dJ_deta0, A.lE, Nt * sizeof(double), cudaMemcpyDefault, st);
  if (!e && dJ_dhu0) e = cudaMemcpyAsync(dJ_dhu0, A.lM, Nt * sizeof(double), cudaMemcpyDefault, st);
  if (!e && dJ_db0) e = cudaMemcpyAsync(dJ_db0, A.lB, Nt * sizeof(double), cudaMemcpyDefault, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return release(fail(ctx, SWALE_ECUDA, cudaGetErrorString(e)));
  std::vector<DevScalars> Sh;
  if ((s = read_scalars(ctx, Sh))) return release(s);
  unsigned int bits = 0;
  for (const DevScalars& v : Sh) bits |= v.status;
  return release(status_from_bits(ctx, bits));
}

}  // extern "C"

// ======================================================================================
// Allocation-free right-hand side (swale_rhs_noalloc)
// ======================================================================================
// Some callers cannot call cudaMalloc: code that runs inside another framework's memory pool
// (which owns the device memory and must see every allocation), or work whose device memory
// must not grow while it runs. For them swale_rhs_noalloc evaluates the same right-hand side as
// swale_rhs with its scratch (the edge values, shared reciprocals, interior point values of the
// special source scheme, detector classes and reduction scalars) in the fixed array below,
// which every GPU that loads this library holds until the process exits.
namespace {

constexpr int64_t kNoAllocMaxCells = 65536;
constexpr int kNoAllocMaxDevices = 64;
constexpr int kNoAllocTile = 128;

struct NoAllocScratch {
  double edges[12][kNoAllocMaxCells + 2];  // 8 edge arrays, 2 reciprocals, 2 point-value arrays
  uint8_t flags[kNoAllocMaxCells + 2];
  InstConst ic;
  DevScalars S;
};

// Resets the scratch scalars of one call; the values come in as kernel arguments, so the call
// copies nothing from host memory.
__global__ void k_noalloc_init(InstConst* ic, DevScalars* S, int64_t N, int32_t ntiles_r) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  InstConst c = {};
  c.N = N;
  c.cfl = 1.0;
  c.ntiles_r = ntiles_r;
  *ic = c;
  DevScalars z = {};
  z.Jmin0 = 0x3ff0000000000000ull;  // 1.0: the unused stage-1 dt arithmetic stays finite
  *S = z;
}

// Fixed scratch of the allocation-free entry point (about 6.3 MB per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Device address of g_noalloc_scratch per device, obtained once with that device current.
void* g_noalloc_addr[kNoAllocMaxDevices];
std::once_flag g_noalloc_once[kNoAllocMaxDevices];
cudaError_t g_noalloc_err[kNoAllocMaxDevices];

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

swale_status swale_rhs_noalloc(const swale_config* cfg, void* cuda_stream, int64_t N, const double* E,
                               const double* M, const double* B, const double* J, const double* w, double alpha,
                               double* RE, double* RM, double* RB, double* A_out, uint8_t* flags) {
  if (!cfg || !E || !M || !B || !J || !w || !RE || !RM || !RB) return SWALE_EINVAL;
  if (N < 5 || N > kNoAllocMaxCells || !(alpha > 0.0)) return SWALE_EINVAL;
  if (!(cfg->g > 0) || !(cfg->eps_weno > 0) || !(cfg->eps_pp >= 0) || !(cfg->h_dry >= 0) || cfg->bc < 0 ||
      cfg->bc > 2 || cfg->scheme < 0 || cfg->scheme > 2 || (cfg->alpha_bound != 0 && cfg->alpha_bound != 1) ||
      (cfg->limit_hu != 0 && cfg->limit_hu != 1))
    return SWALE_EINVAL;
  const void* dev_ptrs[] = {E, M, B, J, w, RE, RM, RB};
  for (const void* p : dev_ptrs)
    if (!on_device(p)) return SWALE_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return SWALE_ECUDA;
  }
  // The scratch address below is the current device's: the stream must belong to it.
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int sdev = dev;
  if (st && cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
    cudaGetLastError();
    return SWALE_EINVAL;
  }
  if (sdev != dev) return SWALE_EINVAL;
  // First call on this device: look up the device address of the scratch array.
  std::call_once(g_noalloc_once[dev], [dev] {
    g_noalloc_err[dev] = cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch);
  });
  if (g_noalloc_err[dev] != cudaSuccess || !g_noalloc_addr[dev]) return SWALE_ECUDA;
  NoAllocScratch* scr = reinterpret_cast<NoAllocScratch*>(g_noalloc_addr[dev]);

  DevState D{};
  D.eEL = scr->edges[0];
  D.eER = scr->edges[1];
  D.eBL = scr->edges[2];
  D.eBR = scr->edges[3];
  D.ehL = scr->edges[4];
  D.ehR = scr->edges[5];
  D.euL = scr->edges[6];
  D.euR = scr->edges[7];
  D.ipair = scr->edges[8];
  D.itri = scr->edges[9];
  if (cfg->scheme == SWALE_SCHEME_SPECIAL) {
    D.eG1 = scr->edges[10];
    D.eG2 = scr->edges[11];
  }
  D.flags = scr->flags;
  D.IC = &scr->ic;
  D.S = &scr->S;
  D.w = const_cast<double*>(w);
  D.nr = (int32_t)((N + 2 + kNoAllocTile - 1) / kNoAllocTile);
  D.nu = (int32_t)((N + kNoAllocTile - 1) / kNoAllocTile);
  D.nf = (int32_t)((N + kNoAllocTile - 2) / (kNoAllocTile - 1));
  StepConst K;
  K.sc.g = cfg->g;
  K.sc.eps_weno = cfg->eps_weno;
  K.sc.eps_pp = cfg->eps_pp;
  K.sc.h_dry = cfg->h_dry;
  K.sc.beta_dx_global = cfg->beta_dx_global;
  K.sc.limit_hu = cfg->limit_hu;
  K.t_end = 0.0;
  K.dt_fixed = 0.0;
  K.mesh_T = 1.0;
  K.gauss_wsum = 1.0;
  K.gauss_iwsum = 1.0;
  K.bc = cfg->bc;
  K.mesh = SWALE_MESH_STATIC;
  K.gauss_half = 0;
  K.B = 1;
  K.alpha_log = nullptr;
  K.alpha_cap = 0;
  K.alpha_base = 0;
  K.alpha_mode = 0;
  K.wait_tries = kWaitTries;
  K.tx_pad = 0;
  K.bot_pieces = K.bot_deg = 0;
  K.bot_breaks = K.bot_coef = nullptr;
  K.scheme = cfg->scheme;
  K.geo_epoch = 0;  // no geometry cache here (D.geo is null)
  K.wave_rel = cfg->alpha_bound ? 0 : 1;  // the largest |u - w| + sqrt(g h) (Eq. alpha2D) in A_out
  // The scalars keep the previous call's contents: start them from zero.
  k_noalloc_init<<<1, 32, 0, st>>>(&scr->ic, &scr->S, N, D.nr);
  k_widths_max<<<64, 256, 0, st>>>(J, N, &scr->S);
  if (cfg->scheme == SWALE_SCHEME_NONWB)
    k_recon<1, kNoAllocTile, 1><<<(unsigned)D.nr, kNoAllocTile, 0, st>>>(K, D, E, M, B, J);
  else if (cfg->scheme == SWALE_SCHEME_SPECIAL)
    k_recon<1, kNoAllocTile, 2><<<(unsigned)D.nr, kNoAllocTile, 0, st>>>(K, D, E, M, B, J);
  else
    k_recon<1, kNoAllocTile><<<(unsigned)D.nr, kNoAllocTile, 0, st>>>(K, D, E, M, B, J);
  RhsOut ro{RE, RM, RB, alpha};
  k_update<2, 1, kNoAllocTile><<<(unsigned)D.nf, kNoAllocTile, 0, st>>>(K, D, E, M, B, J, ro);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && flags) e = cudaMemcpyAsync(flags, scr->flags + 1, (size_t)N, cudaMemcpyDefault, st);
  if (e == cudaSuccess && A_out) {
    unsigned long long bits = 0;
    e = cudaMemcpyAsync(&bits, &scr->S.A[0], sizeof(bits), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) std::memcpy(A_out, &bits, sizeof(double));
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SWALE_ECUDA;
  }
  return SWALE_OK;
}

}  // extern "C"
