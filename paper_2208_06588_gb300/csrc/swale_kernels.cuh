// Device side of the GB300 (sm_103a) FP64 solver for the well-balanced ALE-WENO hybrid scheme
// (Zhang, Xia & Xu, arXiv 2208.06588): data layout and the stage kernels.
//
// One SSP-RK3 step (Eq. RK32D) is a fixed sequence of launches on one stream:
//   k_prologue                 per-instance scalar resets
//   [k_mesh_gauss]             fluid-driven node velocities
//   k_recon<1>, k_update<1>    stage 1 on the mesh at t_n
//   k_recon<2>, k_update<2>    stage 2 on the mesh at t_{n+1}
//   k_recon<3>, k_update<3>    stage 3 on the mesh at t_{n+1/2}
//   k_commit                   the step's time and step count, or its roll-back after an error
// Every launch serves all instances of a batch: blocks walk a work list of (instance, tile)
// entries in grid-stride order (one pass when the grid has one block per tile, a persistent
// loop when it is smaller). A single instance uses the implicit list t -> (0, t * T + first).
// The reconstruction also reduces the per-instance global wave speed of Eq. alpha2D (warp
// shuffle, shared memory, one atomicMax per tile on the order-preserving bit pattern of a
// non-negative double); in stage 1 the last tile of each instance computes that instance's
// dt, so dt, alpha and t never visit the host and steps replay as CUDA graphs.
//
// Error contract: an error bit (kErrBits) raised in a step stops the instance. Kernels skip an
// instance whose status holds one; the stage-3 update writes q^{n+1}, J^{n+1} and the nodes only
// if no error was raised before it (keeping q^n, J^n and x^n in backup arrays), and k_commit
// restores them if the stage-3 update itself raised one. The state is then that of the last
// good step; later steps (also inside a captured graph) are no-ops for the instance.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swale.h"
#include "swale_cell.cuh"

namespace swale_dev {

static_assert(sizeof(swale::CellGeom) == SWALE_GEOM_VALUES * sizeof(double), "CellGeom holds SWALE_GEOM_VALUES doubles");
static_assert(sizeof(swale::SourceGeom) == 6 * sizeof(double), "SourceGeom holds 6 doubles");
static_assert(sizeof(swale::SourceForm) == 6 * sizeof(double), "SourceForm holds 6 doubles");

using swale::EdgeState;
using swale::SchemeConst;

constexpr int kMaxGaussHalf = 64;
constexpr int kMeshThreads = 256;
constexpr int kMeshNodes = kMeshThreads - 1;  // nodes a mesh-velocity tile advances by
constexpr double kTwoPi = 6.283185307179586476925286766559;

// Per-instance device scalars. Maxima of non-negative doubles are kept as their bit patterns
// (unsigned order equals numeric order for non-negative IEEE doubles).
struct DevScalars {
  double t, dt, sdiff, Wbar, alpha1;
  unsigned int st3;                  // status bits raised by the stage-3 update (folded by k_commit)
  unsigned int pad_;
  unsigned long long A[3];           // max edge wave speed per stage
  unsigned long long Jmax[3];        // max width of the stage meshes J^n, J^(1), J^(2)
  unsigned long long Jmin0;          // min J^n
  unsigned long long JmaxN, JminN;   // of J^{n+1}, accumulated by stage 3
  unsigned long long Wabs, dWabs;    // fluid-driven motion: max |w|, max |w_{j+1} - w_j|
  long long steps;
  long long step_idx;                // index of the step in progress (set by the prologue)
  unsigned int status;
  unsigned int counter;              // reconstruction tiles finished in stage 1
  int done;
  int clipped;
  // Mesh geometry cache: stage 2 stores the per-cell reconstruction geometry of the t_{n+1} mesh,
  // which the next step's stage 1 reuses when the tag (context epoch, step index) matches.
  unsigned long long geo_tag;
};

// Per-instance constants.
struct InstConst {
  int64_t N;           // cells
  int64_t coff;        // first cell in the concatenated cell arrays (nodes: coff + i,
                       // edge arrays: coff + 2 i)
  double cfl;
  double Wbar_profile; // (2 pi / T) max |P| of the prescribed motion
  int32_t ntiles_r;    // reconstruction tiles of the instance
  int32_t pad_;
};

struct Tile {
  int32_t inst, c0;  // instance and first cell (reconstruction tiles start at cell -1)
};

// Constants of the whole launch.
struct StepConst {
  SchemeConst sc;
  double t_end, dt_fixed, mesh_T;
  double gauss_wsum;  // sum of the full Gaussian window, summed from -H to H
  double gauss_iwsum; // its reciprocal
  int32_t bc, mesh, gauss_half, B;
  // Stage viscosities: log of 3 values per step and instance (index (step * B + i) * 3 + s - 1);
  // alpha_mode 1 records the computed values, 2 replays the logged ones (the adjoint's and the
  // finite-difference checks' convention: alpha held fixed).
  double* alpha_log;
  int64_t alpha_cap;   // steps the log holds
  int64_t alpha_base;  // step counter value of log row 0
  int32_t alpha_mode;
  int32_t scheme;  // SWALE_SCHEME_*
  uint32_t geo_epoch;  // bumped by the host whenever the state is set or restored
  // Wave speeds of alpha (Eq. alpha2D): 1 = relative to the node velocity, |u - w| + sqrt(g h)
  // (w known when the stage runs), 0 = |u| + sqrt(g h), with the step bound Wbar of |w| added to
  // the maximum (stage 1 of the secant motion, whose w depends on dt; or on request).
  int32_t wave_rel;
  // L2-projection bottom (Eq. baverage); bot_pieces == 0: b evolves by Eq. bottomrk.
  int32_t bot_pieces, bot_deg;
  const double* bot_breaks;  // bot_pieces + 1 breakpoints
  const double* bot_coef;    // piece p: sum_k bot_coef[p (bot_deg + 1) + k] (x - break_p)^k
  // Bounded waits for bulk copies: polls before a wait gives up, and bytes expected beyond the
  // copies (0; swale_set_wait_test raises it so that the waits run out, to test that path).
  int32_t wait_tries;
  uint32_t tx_pad;
};

// Stage viscosity of instance i in stage s of step `step` (DevScalars::step_idx): the computed
// value, or the logged one in replay mode; recorded in record mode.
__device__ __forceinline__ double stage_alpha(const StepConst& K, int i, int s, double computed, long long step) {
  step -= K.alpha_base;
  if (K.alpha_mode == 0 || K.alpha_log == nullptr || step < 0 || step >= K.alpha_cap) return computed;
  double* slot = K.alpha_log + ((int64_t)step * K.B + i) * 3 + (s - 1);
  if (K.alpha_mode == 2) return *slot;
  *slot = computed;
  return computed;
}

// Device arrays of a batch (concatenated over instances).
struct DevState {
  double *E0, *M0, *B0;        // q^n (updated in place by stage 3)
  double *Ea, *Ma, *Ba;        // q^(1)
  double *Eb, *Mb, *Bb;        // q^(2)
  double *YE, *YM, *YB;        // running RK combination J q
  double *J0, *J1, *J2;        // J^n, J^(1), J^(2)
  double *x, *w, *P;           // nodes, node velocities, motion profile (N_i + 1 per instance)
  // Edge arrays hold cells -1..N_i of each instance (N_i + 2 per instance).
  double *eEL, *eER, *eBL, *eBR, *ehL, *ehR, *euL, *euR;
  double *ipair, *itri;        // 1/(J_c + J_{c+1}) and 1/(J_{c-1} + J_c + J_{c+1}) of the stage mesh
  double* xn;                  // nodes at t_{n+1}, written by stage 2 (L2-projection bottom only)
  // Backups of q^n, J^n (cells) and x^n (nodes) written by the stage-3 update before it commits
  // the step, restored by k_commit if that update raised an error (null: no roll-back).
  double *bE, *bM, *bB, *bJ, *bx;
  double *eG1, *eG2;           // eta at the interior Gauss-Lobatto points (special source scheme only)
  // Geometry cache: SWALE_GEOM_VALUES arrays in the edge layout, geo[k * geo_stride + idx].
  double* geo;
  int64_t geo_stride;
  // Per cell of the stage mesh, 14 arrays in the edge layout (gK[k * geo_stride + idx]): the
  // smooth class's linear form K[2][4] (k < 8), stored by the hydrostatic reconstruction, and the
  // source term's six form entries (k = 8..13), stored by the update; set only for the adjoint's
  // recomputes, whose reverse kernels read them instead of recomputing the mesh geometry.
  double* gK;
  uint8_t* flags;              // stage-1 classes, edge layout
  InstConst* IC;
  DevScalars* S;
  const Tile *rtiles, *utiles, *mtiles;  // work lists (null: one instance, implicit tiles)
  int32_t nr, nu, nm;                    // tiles in each list
  // The forward update's tiles: T - 1 cells for a block of T threads, so that its T interfaces
  // take one pass (utiles, of T cells, serve the adjoint's kernels).
  const Tile* ftiles;
  int32_t nf;
};

__constant__ double c_gauss_w[2 * kMaxGaussHalf + 1];

// Status bits that stop an instance (SWALE_BIT_NEGDEPTH is a warning).
constexpr unsigned int kErrBits =
    swale::ST_EWEIGHT | swale::ST_NONFINITE | swale::ST_EMESH | swale::ST_NODT | swale::ST_TIMEOUT;

// An instance takes no further part in the step: finished (t_end), or an error was raised.
__device__ __forceinline__ bool inst_idle(const DevScalars* S) {
  return S->done || (*(volatile const unsigned int*)&S->status & kErrBits);
}

// Node velocity array of a batch: the motion profile itself for the linear motion (constant
// node velocities), else the node-velocity array (zero for a static mesh).
__device__ __forceinline__ const double* node_velocities(const StepConst& K, const DevState& D) {
  return K.mesh == SWALE_MESH_LINEAR ? D.P : D.w;
}

__device__ __forceinline__ int64_t ghost(int64_t i, int64_t N, int bc) {
  if (bc == SWALE_BC_PERIODIC) {
    i %= N;
    return i < 0 ? i + N : i;
  }
  if (i < 0) return -1 - i;
  if (i >= N) return 2 * N - 1 - i;
  return i;
}

// L2 projection of the bottom onto one cell [a, c] (Eq. baverage): on each piece the cell
// overlaps (the first found by bisection of the breakpoints), the mean of the polynomial by the
// 5-point Gauss-Legendre rule, exact for degree <= 8 and divided by the sum of the weights so
// that constants come out exact; the cell average weights these means by the overlap lengths.
// (Differences of antiderivatives would cancel on short cells far from the breakpoint.)
__device__ __noinline__ double bottom_average(const StepConst& K, double a, double c) {
  const double xi[5] = {-0.9061798459386639928, -0.5384693101056830910, 0.0, 0.5384693101056830910,
                        0.9061798459386639928};
  const double wq[5] = {0.2369268850561890875, 0.4786286704993664680, 0.5688888888888888889, 0.4786286704993664680,
                        0.2369268850561890875};
  const double* br = K.bot_breaks;
  int lo = 0, hi = K.bot_pieces;  // the piece p with br[p] <= a < br[p + 1] (clamped)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (br[mid] <= a) lo = mid;
    else hi = mid;
  }
  double s = 0.0;
  for (int p = lo; p < K.bot_pieces && br[p] < c; ++p) {
    const double x0 = br[p], l = fmax(a, x0), h = fmin(c, br[p + 1]);
    if (!(h > l)) continue;
    const double* ck = K.bot_coef + p * (K.bot_deg + 1);
    const double m = 0.5 * (l + h), hw = 0.5 * (h - l);
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double t = m + hw * xi[q] - x0;
      double v = 0.0;
      for (int k = K.bot_deg; k >= 0; --k) v = v * t + ck[k];
      num += wq[q] * v;
      den += wq[q];
    }
    s += (h - l) * (num / den);
  }
  return s / (c - a);
}

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// Block-wide max / min of non-negative doubles, one atomicMax / atomicMin per block. The bit
// patterns of doubles >= +0 order like unsigned integers, so the reductions run on the integer
// pipe (the FP64 pipe is the bottleneck of the stage kernels). A NaN wins the max.
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }

__device__ __forceinline__ void block_max_to(unsigned long long* dst, double v) {
  __shared__ unsigned long long red[32];
  unsigned long long b = dbits(v);
  for (int o = 16; o > 0; o >>= 1) b = umax64(b, __shfl_xor_sync(0xffffffffu, b, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = b;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    b = lane < nw ? red[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) b = umax64(b, __shfl_xor_sync(0xffffffffu, b, o));
    if (lane == 0) atomicMax(dst, b);
  }
  __syncthreads();
}

__device__ __forceinline__ void block_min_to(unsigned long long* dst, double v) {
  __shared__ unsigned long long red[32];
  unsigned long long b = dbits(v);
  for (int o = 16; o > 0; o >>= 1) b = umin64(b, __shfl_xor_sync(0xffffffffu, b, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = b;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    b = lane < nw ? red[lane] : dbits(INFINITY);
    for (int o = 16; o > 0; o >>= 1) b = umin64(b, __shfl_xor_sync(0xffffffffu, b, o));
    if (lane == 0) atomicMin(dst, b);
  }
  __syncthreads();
}

// Exact maximum of the edge wave speeds (Eq. alpha2D) of a block's cells with few FP64
// operations: an FP32 estimate of every edge's |u| + sqrt(g h) (relative error below 2^-21)
// gives the block's FP32 maximum; only edges within 2^-16 of it can hold the exact maximum, and
// only those are evaluated in FP64 (in a warp, one edge per lane first, then the rare second
// one). When the FP32 maximum is below 1e-10 every edge is evaluated. Returns this thread's
// contribution to the exact block maximum (0 for non-candidates).
template <int T>
__device__ __forceinline__ double block_wave(double g, bool useL, bool useR, double hL, double uL, double hR,
                                             double uR) {
  __shared__ unsigned int wmax[T / 32];
  const float gf = swale::f32_trunc(g);
  const float fl = useL ? fabsf(swale::f32_trunc(uL)) + __fsqrt_rn(gf * fmaxf(swale::f32_trunc(hL), 0.0f)) : 0.0f;
  const float fr = useR ? fabsf(swale::f32_trunc(uR)) + __fsqrt_rn(gf * fmaxf(swale::f32_trunc(hR), 0.0f)) : 0.0f;
  const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fl, fr)));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  unsigned bm = 0;
#pragma unroll
  for (int w = 0; w < T / 32; ++w) bm = bm > wmax[w] ? bm : wmax[w];
  const float bmf = __uint_as_float(bm);
  const float thr = (bmf < 1e-10f) ? 0.0f : bmf * (1.0f - 1.0f / 65536.0f);
  const bool cl = useL && fl >= thr, cr = useR && fr >= thr;
  double wave = 0.0;
  const bool c1 = cl || cr;
  const unsigned cand = __ballot_sync(0xffffffffu, c1);
  if (cand) {
    // Flat water: when every candidate edge of the warp holds the same (h, u) bit for bit, one
    // evaluation gives the exact maximum of them all.
    const bool r0 = cr && !cl;
    const int src = __ffs(cand) - 1;
    const unsigned long long hb = dbits(__shfl_sync(0xffffffffu, r0 ? hR : hL, src));
    const unsigned long long ub = dbits(__shfl_sync(0xffffffffu, r0 ? uR : uL, src));
    const bool same = (!cl || (dbits(hL) == hb && dbits(uL) == ub)) && (!cr || (dbits(hR) == hb && dbits(uR) == ub));
    if (__all_sync(0xffffffffu, same)) {
      const double w0 = swale::wave_speed(g, bitsd(hb), bitsd(ub));
      return c1 ? w0 : 0.0;
    }
  }
  if (cand) {
    const bool right = cr && (!cl || fr > fl);
    const double w1 = swale::wave_speed(g, right ? hR : hL, right ? uR : uL);
    wave = c1 ? w1 : 0.0;
  }
  const bool c2 = cl && cr;
  if (__any_sync(0xffffffffu, c2)) {
    const bool right = !(fr > fl);  // the edge the first pass did not take
    const double w2 = swale::wave_speed(g, right ? hR : hL, right ? uR : uL);
    if (c2 && w2 > wave) wave = w2;
  }
  return wave;
}

__device__ __forceinline__ void block_or_status(unsigned int* dst, uint32_t st) {
  st = __reduce_or_sync(0xffffffffu, st);
  if ((threadIdx.x & 31) == 0 && st) atomicOr(dst, st);
}

// ------------------------------------------------------------------------------------
// Bulk (TMA) copies global -> shared, completed on an mbarrier. A copy needs 16-byte aligned
// source and destination and a size that is a multiple of 16 bytes (callers check all three).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
// Orders this thread's generic-proxy shared-memory accesses before later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase `parity` of bar to complete, at most `tries` polls (each poll itself
// blocks for a short hardware-defined time). Returns false if it gave up. kWaitTries bounds the
// wait for a tile's copies; when it runs out, the block waits kDrainTries more polls for those
// copies before it leaves (a block must not exit while its copies can still write its shared
// memory, which the SM hands to the next block).
constexpr int kWaitTries = 1 << 20;
constexpr int kDrainTries = 1 << 24;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int tries) {
  for (int i = 0; i < tries; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ------------------------------------------------------------------------------------
// Per-step prologue, one thread per instance: stage maxima reset, J^{n+1} statistics become
// those of J^n; an instance whose time reached t_end (t_end > 0) is marked done.
// ------------------------------------------------------------------------------------
__global__ void k_prologue(StepConst K, DevState D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K.B) return;
  DevScalars* S = D.S + i;
  // An error in an earlier step, or the end time reached: the instance is done.
  if ((S->status & kErrBits) || (K.t_end > 0.0 && S->t >= K.t_end)) {
    S->done = 1;
    return;
  }
  S->done = 0;
  S->clipped = 0;
  S->step_idx = S->steps;
  S->Jmax[0] = S->JmaxN;
  S->Jmin0 = S->JminN;
  S->JmaxN = 0ull;
  S->JminN = 0x7ff0000000000000ull;  // +inf
  S->A[0] = S->A[1] = S->A[2] = 0ull;
  S->Jmax[1] = S->Jmax[2] = 0ull;
  S->Wabs = S->dWabs = 0ull;
  S->counter = 0u;
  S->st3 = 0u;
  if (K.mesh != SWALE_MESH_FLUID_GAUSS) S->Wbar = D.IC[i].Wbar_profile;
}

// ------------------------------------------------------------------------------------
// Fluid-driven node velocity: raw_k = (u_{k-1} + u_k)/2 for k = 1..N-1 (u = hu/h, dry -> 0),
// truncated renormalised Gaussian filter, w_0 = w_N = 0. A block filters kMeshThreads nodes in
// one pass, one per thread, and tiles advance by kMeshNodes = kMeshThreads - 1 nodes: the last
// node of a tile is the next tile's first, filtered by both (the same sum in the same order),
// which gives the tile the right neighbour of its last node for max |w_{k+1} - w_k| without a
// second pass for one node. The block stages the cell velocities, the raw node velocities and
// its filtered nodes in shared memory (dynamic, 3 T + 4 H + 4 doubles).
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kMeshThreads) k_mesh_gauss(StepConst K, DevState D) {
  extern __shared__ double sh[];
  const int H = K.gauss_half, T = kMeshThreads, tid = threadIdx.x;
  const int nu = T + 2 * H + 2, nr = T + 2 * H + 1;
  double* su = sh;         // cell velocities, cells [k0 - H - 1, k0 + T + H]
  double* sraw = sh + nu;  // raw node velocities, nodes [k0 - H, k0 + T + H]
  double* sw = sraw + nr;  // filtered velocities, nodes [k0, k0 + T]
  for (int t = blockIdx.x; t < D.nm; t += gridDim.x) {
    const Tile tl = D.mtiles ? D.mtiles[t] : Tile{0, t * kMeshNodes};
    DevScalars* S = D.S + tl.inst;
    if (S->done) continue;
    const InstConst ic = D.IC[tl.inst];
    const int64_t N = ic.N, k0 = tl.c0;
    const double* E0 = D.E0 + ic.coff;
    const double* M0 = D.M0 + ic.coff;
    const double* B0 = D.B0 + ic.coff;
    double* w = D.w + ic.coff + tl.inst;
    __syncthreads();
    for (int i = tid; i < nu; i += T) {
      const int64_t c = k0 - H - 1 + i;
      double u = 0.0;
      if (c >= 0 && c < N) {
        const double h = E0[c] - B0[c];
        u = swale::dlt(K.sc.h_dry, h) ? M0[c] * swale::recip(h) : 0.0;
      }
      su[i] = u;
    }
    __syncthreads();
    for (int i = tid; i < nr; i += T) {
      const int64_t k = k0 - H + i;
      sraw[i] = (k >= 1 && k <= N - 1) ? 0.5 * (su[i] + su[i + 1]) : 0.0;
    }
    __syncthreads();
    {
      const int i = tid;
      const int64_t k = k0 + i;
      double v = 0.0;
      if (k >= 1 && k <= N - 1) {
        double acc = 0.0;
        if (k - H >= 1 && k + H <= N - 1) {
          for (int m = -H; m <= H; ++m) acc += c_gauss_w[m + H] * sraw[i + m + H];
          v = acc * K.gauss_iwsum;
        } else {
          double wsum = 0.0;
          for (int m = -H; m <= H; ++m) {
            const int64_t q = k + m;
            if (q < 1 || q > N - 1) continue;
            acc += c_gauss_w[m + H] * sraw[i + m + H];
            wsum += c_gauss_w[m + H];
          }
          v = acc / wsum;
        }
      }
      sw[i] = v;
    }
    __syncthreads();
    const int64_t k = k0 + tid;
    double wa = 0.0, dwa = 0.0;
    if (tid < kMeshNodes && k <= N) {
      w[k] = sw[tid];
      wa = fabs(sw[tid]);
      if (k < N) dwa = fabs(sw[tid + 1] - sw[tid]);
    }
    block_max_to(&S->Wabs, wa);
    block_max_to(&S->dWabs, dwa);
  }
}

// ------------------------------------------------------------------------------------
// Reconstruction + limiter of cells -1..N_i (rows a2-a7) for stage STAGE. A tile is T
// consecutive cells; the block stages their 5-cell stencils (tile plus a 2-cell halo each
// side) in shared memory, computes each pair's and each triple's reciprocal width and divided
// differences once, then reconstructs one cell per thread. It stores the pair / triple
// reciprocals for the update kernel of the same stage, reduces the wave speed, and in stage 1
// the instance's last tile computes its dt (and the secant factor of the prescribed motion).
// ------------------------------------------------------------------------------------
// A cell of the well-balanced scheme whose smooth class the FP32 test leaves open, out of line:
// the rest of its cached geometry (stage 1), the indicator factors and triple differences, the
// FP64 detector and the edge values of its class. A call, not inlined, so that this rare path's
// registers do not weigh on the smooth cells' code; its inputs are copies.
struct OpenCell {
  swale::CellGeom G;
  swale::StencilDD DD;
  double h[5], it[3], v0[3][3], dxe;
};
struct OpenOut {
  EdgeState o;
  uint32_t st;
  uint8_t flag;
};
__device__ __noinline__ OpenOut recon_open_cell(const SchemeConst P, OpenCell c, const double* geo, int64_t geo_stride,
                                                int64_t idx) {
  double* gv = reinterpret_cast<double*>(&c.G);
  constexpr int kF0 = offsetof(swale::CellGeom, F) / sizeof(double), kF1 = kF0 + 5;
  if (geo) {
#pragma unroll
    for (int k = 0; k < SWALE_GEOM_BASE; ++k)
      if (k < kF0 || k >= kF1) gv[k] = geo[k * geo_stride + idx];
  }
  swale::indicator_factors(c.h, c.dxe, c.G);
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int a = 0; a < 3; ++a) c.DD.D3[v][a] = swale::triple_dd(c.DD.D2[v][a], c.DD.D2[v][a + 1], c.it[a]);
  OpenOut r;
  r.st = 0;
  swale::recon_cell_g(P, c.G, c.v0, c.DD, r.o, r.flag, r.st, false);
  return r;
}

// Launch bounds (resident threads per SM): HIOCC, 8 blocks of 128 threads (64 registers), for
// stage 1 of the well-balanced scheme when it reads the cached mesh geometry: its per-cell work is
// light enough there that more resident warps win (measured: 0.8 % of the dam-break step), while
// every instantiation that computes the geometry itself spills heavily under that bound. The
// other well-balanced instantiations take 768 threads (6 blocks of 128, 80 registers, a few
// spilled doubles; 1.2 % faster per step than 4 blocks of 128 registers), the other schemes 512.
// STOREK: an instantiation of the hydrostatic scheme that also stores each cell's smooth-class
// linear form in D.gK (the adjoint's recomputes), so that the forward's own instantiations keep
// their registers.
template <int STAGE, int T, int SCHEME = 0, bool HIOCC = false, bool STOREK = false>
__global__ void __launch_bounds__(T, (HIOCC ? 1024 : (SCHEME == 0 ? 768 : 512)) / T) k_recon(StepConst K, DevState D, const double* __restrict__ Eg,
                                             const double* __restrict__ Mg, const double* __restrict__ Bg,
                                             const double* __restrict__ Jg) {
  __shared__ double sJ[T + 4], sV[3][T + 4];    // cells c0-2 .. c0+T+1
  __shared__ double sIP[T + 3], sD2[3][T + 3];  // pairs starting at those cells
  // Triples centred at cells c0-1 .. c0+T. The well-balanced scheme forms the second differences
  // per cell, and only where the FP32 smooth-class test cannot decide (the smooth class needs
  // none); the other schemes form them here.
  constexpr int TD3 = SCHEME == 0 ? 0 : T;
  __shared__ double sIT[T + 2], sD3[3][TD3 + 2];
  // FP32 copies of the pair differences (hu, h, and for the non-well-balanced scheme eta) and of
  // the triple reciprocals for the FP32 smooth-class tests
  constexpr int NV32 = SCHEME == 1 ? 3 : 2;
  __shared__ float sD2f[NV32][T + 3], sITf[T + 2];
  __shared__ __align__(16) double sRaw[4][T + 8];  // E, M, B, J of those cells as bulk-copied
  __shared__ __align__(8) uint64_t sBar;           // completion of the tile's bulk copies
  __shared__ __align__(8) uint64_t sPad;           // test hook: a barrier no copy completes
  __shared__ bool last;
  const int tid = threadIdx.x;
  const bool refl = (K.bc == SWALE_BC_REFLECTIVE);
  if (tid == 0) {
    mbar_init(&sBar);
    mbar_init(&sPad);
    fence_proxy_async();  // the initialised barriers, visible to the copy engine
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int t = blockIdx.x; t < D.nr; t += gridDim.x) {
    const Tile tl = D.rtiles ? D.rtiles[t] : Tile{0, t * T - 1};
    DevScalars* S = D.S + tl.inst;
    // every thread reads the flags once, then the block agrees (the status may change meanwhile)
    if (__syncthreads_or(inst_idle(S))) continue;
    const InstConst ic = D.IC[tl.inst];
    const int64_t N = ic.N, c0 = tl.c0;
    const double* E = Eg + ic.coff;
    const double* M = Mg + ic.coff;
    const double* B = Bg + ic.coff;
    const double* J = Jg + ic.coff;
    const int64_t eb = ic.coff + 2 * (int64_t)tl.inst;  // edge-array base of the instance
    __syncthreads();
    // The stencil cells of the tile that lie in the instance, [cs, ce], arrive by four bulk
    // copies (E, M, B, J). The copied span [ga, ge] (global element indices) is widened to
    // 16-byte boundaries: one element before cs where needed (it exists: ga >= 1), one after ce
    // when that element is in the arrays (the instance is not the last one, or ce < N - 1),
    // else one fewer (that cell is loaded directly). Shared rows are shifted by `off` so that
    // the first copied element lands on a 16-byte boundary as well. Ghost cells and anything
    // not copied take the direct loads below.
    const int64_t cs = c0 - 2 < 0 ? 0 : c0 - 2, ce = c0 + T + 1 < N - 1 ? c0 + T + 1 : N - 1;
    int64_t ga = (ic.coff + cs) & ~(int64_t)1, ge = ic.coff + ce;
    if (!(ge & 1)) ge += (ce + 1 < N || tl.inst + 1 < K.B) ? 1 : -1;
    const int rel = (int)(ga - ic.coff - (c0 - 2));  // shared index of ga before the shift
    const int off = 2 - (rel & 1);
    const uint32_t bytes = ge >= ga ? (uint32_t)((ge - ga + 1) * 8) : 0u;
    const bool bulk = bytes >= 16 && ((((uintptr_t)(Eg + ga)) | ((uintptr_t)(Mg + ga)) | ((uintptr_t)(Bg + ga)) |
                                       ((uintptr_t)(Jg + ga))) & 15) == 0;
    if (bulk) {
      if (tid == 0) {
        fence_proxy_async();  // the previous tile's reads of sRaw come before these writes
        mbar_arrive_expect_tx(&sBar, 4 * bytes);
        bulk_copy_g2s(&sRaw[0][rel + off], Eg + ga, bytes, &sBar);
        bulk_copy_g2s(&sRaw[1][rel + off], Mg + ga, bytes, &sBar);
        bulk_copy_g2s(&sRaw[2][rel + off], Bg + ga, bytes, &sBar);
        bulk_copy_g2s(&sRaw[3][rel + off], Jg + ga, bytes, &sBar);
        // Test hook: a second barrier expects bytes that no copy delivers.
        if (K.tx_pad) mbar_arrive_expect_tx(&sPad, K.tx_pad);
      }
      bool landed = mbar_wait_bounded(&sBar, phase, kWaitTries);
      bool ok = landed;
      if (!landed) landed = mbar_wait_bounded(&sBar, phase, kDrainTries);  // drain before leaving
      if (K.tx_pad && landed) ok = mbar_wait_bounded(&sPad, 0u, K.wait_tries > 0 ? K.wait_tries : kWaitTries);
      phase ^= 1u;
      // The copies did not complete in time (or the test barrier ran out): give the stage up.
      // Every copy of this block has landed here unless the drain wait ran out as well.
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(&S->status, (unsigned int)swale::ST_TIMEOUT);
        return;
      }
    }
    const int64_t gs = ga - ic.coff, gl = ge - ic.coff;  // copied cells (instance indices)
    for (int i = tid; i < T + 4; i += T) {
      const int64_t c = c0 - 2 + i;
      double jv = 1.0, ev = 0.0, mv = 0.0, bv = 0.0;  // filler beyond the last ghost cell
      if (bulk && c >= 0 && c < N && c >= gs && c <= gl) {
        const int k = i + off;
        ev = sRaw[0][k];
        mv = sRaw[1][k];
        bv = sRaw[2][k];
        jv = sRaw[3][k];
      } else if (c >= -3 && c <= N + 2) {
        const int64_t s = ghost(c, N, K.bc);
        jv = J[s];
        ev = E[s];
        bv = B[s];
        mv = M[s];
        if (refl && (c < 0 || c >= N)) mv = -mv;
      }
      sJ[i] = jv;
      sV[0][i] = ev;
      sV[1][i] = mv;
      sV[2][i] = ev - bv;  // the depth is reconstructed in place of the bottom
    }
    __syncthreads();
    for (int i = tid; i < T + 3; i += T) {
      const double ip = swale::pair_recip(sJ[i], sJ[i + 1]);
      sIP[i] = ip;
      double d2[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) sD2[v][i] = d2[v] = swale::pair_dd(sV[v][i], sV[v][i + 1], ip);
      sD2f[0][i] = swale::f32_trunc(d2[1]);
      sD2f[1][i] = swale::f32_trunc(d2[2]);
      if (SCHEME == 1) sD2f[NV32 - 1][i] = swale::f32_trunc(d2[0]);
    }
    __syncthreads();
    for (int i = tid; i < T + 2; i += T) {
      const double it = swale::triple_recip(sJ[i], sJ[i + 1], sJ[i + 2]);
      sIT[i] = it;
      if (SCHEME != 0) {
#pragma unroll
        for (int v = 0; v < 3; ++v) sD3[v][i] = swale::triple_dd(sD2[v][i], sD2[v][i + 1], it);
      }
      sITf[i] = swale::f32_trunc(it);
    }
    __syncthreads();
    const int64_t c = c0 + tid;
    const unsigned long long geo_now =
        ((unsigned long long)K.geo_epoch << 32) | (unsigned long long)(S->step_idx & 0xffffffffLL);
    const bool use_geo = STAGE == 1 && D.geo != nullptr && S->geo_tag == geo_now;
    if (STAGE == 2 && D.geo != nullptr && c0 == -1 && tid == 0)
      S->geo_tag = ((unsigned long long)K.geo_epoch << 32) | (unsigned long long)((S->step_idx + 1) & 0xffffffffLL);
    double wave = 0.0, ehL = 0.0, euL = 0.0, ehR = 0.0, euR = 0.0;
    bool useL = false, useR = false;
    uint32_t st = 0;
    if (c <= N) {
      double h[5], v0[3][3];
      swale::StencilDD DD;
#pragma unroll
      for (int k = 0; k < 5; ++k) h[k] = sJ[tid + k];
      // The well-balanced scheme reads its stencil data from shared memory where its class is
      // known (below): fewer values live across the mesh geometry.
      if (SCHEME != 0) {
#pragma unroll
        for (int v = 0; v < 3; ++v) {
#pragma unroll
          for (int a = 0; a < 3; ++a) v0[v][a] = sV[v][tid + a];
#pragma unroll
          for (int a = 0; a < 4; ++a) DD.D2[v][a] = sD2[v][tid + a];
#pragma unroll
          for (int a = 0; a < 3; ++a) DD.D3[v][a] = sD3[v][tid + a];
        }
      }
      const double dxmax = bitsd(S->Jmax[STAGE - 1]);
      const int64_t idx = eb + c + 1;
      // Mesh geometry of the cell: from the cache that the previous step's stage 2 filled on the
      // same mesh (t_{n+1}), else computed; stage 2 fills the cache.
      swale::CellGeom G;
      double* gv = reinterpret_cast<double*>(&G);
      constexpr int kGeo = SCHEME == 0 ? SWALE_GEOM_VALUES : SWALE_GEOM_BASE;  // values cached
      // The indicator factors (F, c4, c3) are not cached: they are formed below, in FP32 for the
      // smooth-class test and in FP64 only where that test cannot decide.
      constexpr int kF0 = offsetof(swale::CellGeom, F) / sizeof(double), kF1 = kF0 + 5;
      static_assert(offsetof(swale::CellGeom, c4) / sizeof(double) == kF0 + 4, "F, c3, c4 are adjacent");
      const double dxe = K.sc.beta_dx_global ? dxmax : h[2];
      // The well-balanced scheme reads only the smooth-class form K here; the rest of the cached
      // geometry (sub-stencil factors and linear weights) only for a cell whose class the FP32
      // test leaves open.
      constexpr int kLoad0 = SCHEME == 0 ? SWALE_GEOM_BASE : 0;
      if (use_geo) {
#pragma unroll
        for (int k = kLoad0; k < kGeo; ++k)
          if (k < kF0 || k >= kF1) gv[k] = D.geo[k * D.geo_stride + idx];
        if (!swale::gt0(h[2])) st |= swale::ST_EMESH;
      } else {
        swale::cell_geom(h, dxe, G, st, false);
        if (SCHEME == 0) {
          const double it3[3] = {sIT[tid], sIT[tid + 1], sIT[tid + 2]};
          swale::smooth_edge_coeffs(h, it3, G);
        }
      }
      if (STAGE == 2 && D.geo) {
#pragma unroll
        for (int k = 0; k < kGeo; ++k)
          if (k < kF0 || k >= kF1) D.geo[k * D.geo_stride + idx] = gv[k];
      }
      if (STOREK && SCHEME == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) D.gK[k * D.geo_stride + idx] = G.K[k >> 2][k & 3];
      }
      EdgeState o;
      uint8_t flag;
      double etaG[2] = {0.0, 0.0};
      // Indicator factors in FP32 from the FP32 widths.
      float F32[3], itf[3], c4f, c3f;
      swale::indicator_factors_f32(h, dxe, F32, c4f, c3f);
#pragma unroll
      for (int a = 0; a < 3; ++a) itf[a] = sITf[tid + a];
      const float epsf = swale::f32_trunc(K.sc.eps_weno);
      if (SCHEME == 1) {
        // Each characteristic field and the bottom: its smooth class in FP32 when that can be
        // told for sure, from the FP32 pair differences of eta, hu, h and the projection rows.
        const swale::NonwbProj pr = swale::nonwb_proj(K.sc, v0);
        const float a11 = swale::f32_trunc(pr.a11), a12 = swale::f32_trunc(pr.a12);
        const float a21 = swale::f32_trunc(pr.a21), a22 = swale::f32_trunc(pr.a22);
        float fd[3][4], fm[3][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float e2 = sD2f[NV32 - 1][tid + a], m2 = sD2f[0][tid + a], h2 = sD2f[1][tid + a];
          fd[0][a] = fmaf(a11, e2, a12 * m2);
          fm[0][a] = fmaf(fabsf(a11), fabsf(e2), fabsf(a12) * fabsf(m2));
          fd[1][a] = fmaf(a21, e2, a22 * m2);
          fm[1][a] = fmaf(fabsf(a21), fabsf(e2), fabsf(a22) * fabsf(m2));
          fd[2][a] = e2 - h2;
          fm[2][a] = fabsf(e2) + fabsf(h2);
        }
        bool known[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) known[f] = swale::sure_smooth1_f32(F32, c4f, c3f, fd[f], fm[f], itf, epsf);
        if (!(known[0] && known[1] && known[2])) swale::indicator_factors(h, dxe, G);
        swale::recon_cell_nonwb_g(K.sc, G, v0, DD, o, flag, st, pr, known);
      } else {
        // The smooth class, when FP32 can tell it for sure; else the FP64 detector decides.
        float d2h[4], d2m[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          d2h[a] = sD2f[1][tid + a];
          d2m[a] = sD2f[0][tid + a];
        }
        const bool smooth32 = swale::sure_smooth_f32(F32, c4f, c3f, d2h, d2m, itf, epsf);
        if (SCHEME == 0) {
          if (smooth32) {  // the cell's averages and pair differences are all the smooth class needs
#pragma unroll
            for (int v = 0; v < 3; ++v) {
              v0[v][2] = sV[v][tid + 2];
#pragma unroll
              for (int a = 0; a < 4; ++a) DD.D2[v][a] = sD2[v][tid + a];
            }
            swale::recon_cell_g(K.sc, G, v0, DD, o, flag, st, true);
          } else {  // the FP64 detector decides, out of line
            OpenCell oc;
            oc.G = G;
            oc.dxe = dxe;
#pragma unroll
            for (int k = 0; k < 5; ++k) oc.h[k] = h[k];
#pragma unroll
            for (int a = 0; a < 3; ++a) oc.it[a] = sIT[tid + a];
#pragma unroll
            for (int v = 0; v < 3; ++v) {
#pragma unroll
              for (int a = 0; a < 3; ++a) oc.v0[v][a] = sV[v][tid + a];
#pragma unroll
              for (int a = 0; a < 4; ++a) oc.DD.D2[v][a] = sD2[v][tid + a];
            }
            const OpenOut r = recon_open_cell(K.sc, oc, use_geo ? D.geo : nullptr, D.geo_stride, idx);
            o = r.o;
            flag = r.flag;
            st |= r.st;
          }
        } else {
          if (!smooth32) swale::indicator_factors(h, dxe, G);  // the FP64 detector needs them
          swale::recon_cell_special_g(K.sc, G, h, v0, DD, o, flag, st, etaG, smooth32);
        }
      }
      D.eEL[idx] = o.EL;
      D.eER[idx] = o.ER;
      D.eBL[idx] = o.BL;
      D.eBR[idx] = o.BR;
      D.ehL[idx] = o.hL;
      D.ehR[idx] = o.hR;
      D.euL[idx] = o.uL;
      D.euR[idx] = o.uR;
      if (SCHEME == 2) {
        D.eG1[idx] = etaG[0];
        D.eG2[idx] = etaG[1];
      }
      D.ipair[idx] = sIP[tid + 2];  // pair (c, c+1)
      D.itri[idx] = sIT[tid + 1];   // triple centred at c
      if (STAGE == 1) D.flags[idx] = flag;
      // Edges that touch interfaces 0..N only.
      useL = (c != -1);
      useR = (c != N);
      ehL = o.hL;
      euL = o.uL;
      ehR = o.hR;
      euR = o.uR;
      if (K.wave_rel) {  // Eq. alpha2D: speeds relative to the node (cell c spans nodes c, c+1)
        const double* wv = node_velocities(K, D) + ic.coff + tl.inst;
        if (useL) euL -= wv[c];
        if (useR) euR -= wv[c + 1];
      }
    }
    wave = block_wave<T>(K.sc.g, useL, useR, ehL, euL, ehR, euR);
    block_or_status(&S->status, st);
    block_max_to(&S->A[STAGE - 1], wave);
    if (STAGE == 1) {
      if (tid == 0) {
        __threadfence();
        const unsigned int ticket = atomicAdd(&S->counter, 1u);
        last = (ticket == (unsigned)ic.ntiles_r - 1u);
      }
      __syncthreads();
      if (last && tid == 0) {
        __threadfence();
        const double A1 = bitsd(atomicAdd(&S->A[0], 0ull));
        double Wbar = S->Wbar;
        double dwmax = 0.0;
        if (K.mesh == SWALE_MESH_FLUID_GAUSS) {
          Wbar = bitsd(atomicAdd(&S->Wabs, 0ull));
          dwmax = bitsd(atomicAdd(&S->dWabs, 0ull));
          S->Wbar = Wbar;
        }
        const double alpha1 = stage_alpha(K, tl.inst, 1, K.wave_rel ? A1 : A1 + Wbar, S->step_idx);
        const double tn = S->t;
        double dt;
        int clipped = 0;
        if (K.dt_fixed > 0.0) {
          dt = K.dt_fixed;
        } else {
          const double jmin = bitsd(S->Jmin0);
          dt = ic.cfl * jmin / alpha1;
          if (K.mesh == SWALE_MESH_FLUID_GAUSS && dwmax > 0.0) dt = fmin(dt, 0.5 * jmin / dwmax);
        }
        if (K.t_end > 0.0 && K.t_end - tn <= dt) {
          dt = K.t_end - tn;
          clipped = 1;
        }
        // alpha = 0 (a dry state at rest on a mesh that does not move) leaves the CFL condition
        // with no bound; without an end time there is no step to take: dt = 0, flagged.
        if (!(dt < INFINITY)) {
          dt = 0.0;
          atomicOr(&S->status, (unsigned int)swale::ST_NODT);
        }
        S->dt = dt;
        S->alpha1 = alpha1;
        S->clipped = clipped;
        if (K.mesh == SWALE_MESH_PROFILE) {
          const double s0 = sin(kTwoPi * tn / K.mesh_T);
          const double s1 = sin(kTwoPi * (tn + dt) / K.mesh_T);
          S->sdiff = dt > 0.0 ? (s1 - s0) / dt : 0.0;
        } else {
          S->sdiff = 0.0;
        }
        S->counter = 0u;
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// Fluxes, source and the RK combination of stage STAGE for cells 0..N_i-1 (rows a1, a8, a9;
// MODE 0), or the bare right-hand side of one instance (MODE 1, used by swale_rhs). A tile is
// T - 1 consecutive cells for a block of T threads: its T interfaces' fluxes are computed once,
// one per thread, into shared memory (a tile of T cells would leave its last interface to a
// second pass of a single thread); the widths, their reciprocals and the depth / bottom
// averages of the tile plus one halo cell each side are staged there too.
// ------------------------------------------------------------------------------------
struct RhsOut {
  double *RE, *RM, *RB;
  double alpha;
};

// PLAIN: an instantiation for the hydrostatic scheme without the L2-projection bottom (the
// common case), in which the other schemes' branches are compiled out; it is held to 64
// registers (8 blocks of 128 threads per SM: without the bound stage 1 takes 71 and 7 blocks,
// measured slower). STOREK: one that also stores the source form's entries in D.gK (the
// adjoint's recomputes).
template <int STAGE, int MODE, int T, bool PLAIN = false, bool STOREK = false>
__global__ void __launch_bounds__(T, PLAIN ? 1024 / T : 1) k_update(StepConst K, DevState D, const double* __restrict__ Eg,
                                              const double* __restrict__ Mg, const double* __restrict__ Bg,
                                              const double* __restrict__ Jsg, RhsOut ro) {
  __shared__ double sF[4][T], sW[T];                              // interfaces / nodes j0 .. j0+T-1
  __shared__ double sJ[T + 1], siJ[T + 1], sH[T + 1], sB[T + 1];  // cells j0-1 .. j0+T-1
  const int tid = threadIdx.x;
  (void)Mg;
  constexpr int TC = T - 1;  // cells of a tile; its T interfaces j0 .. j0 + TC, one per thread
  for (int t = blockIdx.x; t < D.nf; t += gridDim.x) {
    const Tile tl = D.ftiles ? D.ftiles[t] : Tile{0, t * TC};
    const int inst = tl.inst;
    DevScalars* S = D.S + inst;
    if (MODE == 0) {
      // Skip a finished instance and one whose step has failed. In stage 3 the status does not
      // change during the launch (this kernel raises its bits in st3), so every tile of an
      // instance decides alike: all commit the step or none does.
      if (__syncthreads_or(inst_idle(S))) continue;
    }
    const InstConst ic = D.IC[inst];
    const int64_t N = ic.N, j0 = tl.c0;
    const int64_t cb = ic.coff, nb = ic.coff + inst, eb = ic.coff + 2 * (int64_t)inst;
    const double* E = Eg + cb;
    const double* B = Bg + cb;
    const double* Js = Jsg + cb;
    double alpha, dt = 0.0;
    if (MODE == 1) {
      alpha = ro.alpha;
    } else {
      alpha = (STAGE == 1) ? S->alpha1 : bitsd(S->A[STAGE - 1]) + (K.wave_rel ? 0.0 : S->Wbar);
      if (STAGE > 1) {
        // Record / replay of stages 2 and 3 (stage 1 is handled where alpha1 is formed): every
        // tile computes the same value; the first tile of the instance records it.
        if (K.alpha_mode == 2) alpha = stage_alpha(K, inst, STAGE, alpha, S->step_idx);
        else if (K.alpha_mode == 1 && j0 == 0 && threadIdx.x == 0) stage_alpha(K, inst, STAGE, alpha, S->step_idx);
      }
      dt = S->dt;
    }
    const bool fresh_w = (MODE == 0 && STAGE == 1 && K.mesh == SWALE_MESH_PROFILE);
    // The source geometry of the cells (width ratios) is cached beside the reconstruction's
    // mesh geometry: stage 2 stores it and the next step's stage 1, on the same mesh, reads it
    // under the same tag.
    const unsigned long long geo_now =
        ((unsigned long long)K.geo_epoch << 32) | (unsigned long long)(S->step_idx & 0xffffffffLL);
    const bool use_sgeo = STAGE == 1 && MODE == 0 && D.geo != nullptr && S->geo_tag == geo_now;
    const double sdiff = fresh_w ? S->sdiff : 0.0;
    __syncthreads();
    {
      const int i = tid;
      const int64_t k = j0 + i;  // node / interface index
      if (k <= N) {
        double wk;
        if (fresh_w) {
          wk = D.P[nb + k] * sdiff;
          if (i < TC || k == N) D.w[nb + k] = wk;
        } else if (MODE == 0 && K.mesh == SWALE_MESH_STATIC) {
          wk = 0.0;
        } else if (MODE == 0 && K.mesh == SWALE_MESH_LINEAR) {
          wk = D.P[nb + k];  // constant node velocity (Eq. velocity)
          if (STAGE == 1 && (i < TC || k == N)) D.w[nb + k] = wk;
        } else {
          wk = D.w[nb + k];
        }
        sW[i] = wk;
        // Interface k: left state = right edge of cell k-1 (edge index k), right state = left
        // edge of cell k (edge index k+1).
        const int64_t el = eb + k, er = eb + k + 1;
        const swale::Flux F =
            (!PLAIN && K.scheme != 0) ? swale::interface_flux_plain(K.sc.g, alpha, wk, D.eER[el], D.eEL[er], D.eBR[el], D.eBL[er],
                                                        D.ehR[el], D.ehL[er], D.euR[el], D.euL[er])
                          : swale::interface_flux(K.sc.g, alpha, wk, D.eER[el], D.eEL[er], D.eBR[el], D.eBL[er],
                                                  D.ehR[el], D.ehL[er], D.euR[el], D.euL[er]);
        sF[0][i] = F.FE;
        sF[1][i] = F.FMm;
        sF[2][i] = F.FMp;
        sF[3][i] = F.FB;
      }
    }
    for (int i = tid; i < TC + 2; i += T) {
      const int64_t c = j0 - 1 + i;
      if (c >= -1 && c <= N) {
        const int64_t s = ghost(c, N, K.bc);
        const double jv = Js[s];
        sJ[i] = jv;
        if (!use_sgeo) siJ[i] = swale::recip(jv);  // only the source geometry needs it
        sH[i] = E[s] - B[s];
        sB[i] = B[s];
      }
    }
    __syncthreads();
    const int64_t j = j0 + tid;
    double jmaxa = 0.0, jmaxb = 0.0, jminb = INFINITY;
    uint32_t st = 0;
    if (tid < TC && j < N) {
      const swale::Flux Fl = {sF[0][tid], sF[1][tid], sF[2][tid], sF[3][tid]};
      const swale::Flux Fr = {sF[0][tid + 1], sF[1][tid + 1], sF[2][tid + 1], sF[3][tid + 1]};
      const int64_t ic_e = eb + j + 1;  // edge-array index of cell j
      const double hd[5] = {sH[tid], sH[tid + 1], sH[tid + 2], D.ehL[ic_e], D.ehR[ic_e]};
      const double bd[5] = {sB[tid], sB[tid + 1], sB[tid + 2], D.eBL[ic_e], D.eBR[ic_e]};
      // Six mesh-only values of the source per cell: the antisymmetric form (SourceForm), or the
      // width ratios (SourceGeom) for the special scheme's point-wise source.
      double Sj;
      if (!PLAIN && K.scheme == 2) {
        swale::SourceGeom sg;
        double* const src6 = reinterpret_cast<double*>(&sg);
        if (use_sgeo) {
#pragma unroll
          for (int k = 0; k < 6; ++k) src6[k] = D.geo[(SWALE_GEOM_VALUES + k) * D.geo_stride + ic_e];
        } else {
          sg = swale::source_geom(sJ[tid], sJ[tid + 1], siJ[tid], siJ[tid + 1], siJ[tid + 2], D.ipair[eb + j],
                                  D.ipair[eb + j + 1], D.itri[eb + j + 1]);
        }
        if (STAGE == 2 && MODE == 0 && D.geo) {
#pragma unroll
          for (int k = 0; k < 6; ++k) D.geo[(SWALE_GEOM_VALUES + k) * D.geo_stride + ic_e] = src6[k];
        }
        const double eta4[4] = {D.eEL[ic_e], D.eG1[ic_e], D.eG2[ic_e], D.eER[ic_e]};
        Sj = swale::source_cell_special(K.sc.g, E[j], eta4, bd, sg, D.eBR[ic_e - 1],
                                        D.eBL[ic_e + 1]);
      } else {
        swale::SourceForm sf;
        double* const src6 = reinterpret_cast<double*>(&sf);
        if (use_sgeo) {
#pragma unroll
          for (int k = 0; k < 6; ++k) src6[k] = D.geo[(SWALE_GEOM_VALUES + k) * D.geo_stride + ic_e];
        } else {
          sf = swale::source_form(sJ[tid], sJ[tid + 1], sJ[tid + 2], siJ[tid], siJ[tid + 1], siJ[tid + 2],
                                  D.ipair[eb + j], D.ipair[eb + j + 1], D.itri[eb + j + 1]);
        }
        if (STAGE == 2 && MODE == 0 && D.geo) {
#pragma unroll
          for (int k = 0; k < 6; ++k) D.geo[(SWALE_GEOM_VALUES + k) * D.geo_stride + ic_e] = src6[k];
        }
        if (STOREK) {
#pragma unroll
          for (int k = 0; k < 6; ++k) D.gK[(8 + k) * D.geo_stride + ic_e] = src6[k];
        }
        Sj = swale::source_cell_form(K.sc.g, hd, bd, sf);
      }
      const swale::CellRhs R = swale::cell_rhs(Fl, Fr, Sj);
      const double RE = R.RE, RM = R.RM, RB = R.RB;
      if (MODE == 1) {
        ro.RE[j] = RE;
        ro.RM[j] = RM;
        ro.RB[j] = RB;
      } else {
        const int64_t g = cb + j;  // global cell index
        const double wl = sW[tid], wr = sW[tid + 1];
        const double J0 = D.J0[g];
        const double dw = wr - wl;
        if (STAGE == 1) {
          const double J1 = J0 + dt * dw;
          const double J2 = 0.75 * J0 + 0.25 * J1 + 0.25 * dt * dw;
          // J^{n+1} of the recursion, checked here already so that a step that would invert a
          // cell fails before its stages run (stage 3 recomputes it from the stored J^(2)).
          const double J3c = (1.0 / 3.0) * J0 + (2.0 / 3.0) * J2 + (2.0 / 3.0) * dt * dw;
          D.J1[g] = J1;
          D.J2[g] = J2;
          jmaxa = J1;
          jmaxb = J2;
          if (!swale::gt0(J1) || !swale::gt0(J2) || !swale::gt0(J3c)) st |= swale::ST_EMESH;
          const double yE = J0 * D.E0[g] + dt * RE, yM = J0 * D.M0[g] + dt * RM, yB = J0 * D.B0[g] + dt * RB;
          D.YE[g] = yE;
          D.YM[g] = yM;
          D.YB[g] = yB;
          const double inv = swale::recip(J1);
          D.Ea[g] = yE * inv;
          D.Ma[g] = yM * inv;
          D.Ba[g] = yB * inv;
          if (!PLAIN && K.bot_pieces > 0)  // bottom of stage 2: projection onto the mesh at t_{n+1}
            D.Ba[g] = bottom_average(K, D.x[nb + j] + dt * wl, D.x[nb + j + 1] + dt * wr);
        } else if (STAGE == 2) {
          const double yE = 0.75 * (J0 * D.E0[g]) + 0.25 * (D.YE[g] + dt * RE);
          const double yM = 0.75 * (J0 * D.M0[g]) + 0.25 * (D.YM[g] + dt * RM);
          const double yB = 0.75 * (J0 * D.B0[g]) + 0.25 * (D.YB[g] + dt * RB);
          D.YE[g] = yE;
          D.YM[g] = yM;
          D.YB[g] = yB;
          const double inv = swale::recip(D.J2[g]);
          D.Eb[g] = yE * inv;
          D.Mb[g] = yM * inv;
          D.Bb[g] = yB * inv;
          if (!PLAIN && K.bot_pieces > 0) {  // bottom of stage 3: projection onto the mesh at t_{n+1/2}
            const double xl = D.x[nb + j], xr = D.x[nb + j + 1];
            D.Bb[g] = bottom_average(K, xl + 0.5 * dt * wl, xr + 0.5 * dt * wr);
            D.xn[nb + j] = xl + dt * wl;  // nodes at t_{n+1} for the projection after the step
            if (j == N - 1) D.xn[nb + N] = xr + dt * wr;
          }
        } else {
          const double J3 = (1.0 / 3.0) * J0 + (2.0 / 3.0) * D.J2[g] + (2.0 / 3.0) * dt * dw;
          if (!swale::gt0(J3)) st |= swale::ST_EMESH;
          const double E0v = D.E0[g], M0v = D.M0[g], B0v = D.B0[g];
          if (D.bE) {  // q^n, J^n, x^n kept for a roll-back by k_commit
            D.bE[g] = E0v;
            D.bM[g] = M0v;
            D.bB[g] = B0v;
            D.bJ[g] = J0;
            D.bx[nb + j] = D.x[nb + j];
            if (j == N - 1) D.bx[nb + N] = D.x[nb + N];
          }
          const double yE = (1.0 / 3.0) * (J0 * E0v) + (2.0 / 3.0) * (D.YE[g] + dt * RE);
          const double yM = (1.0 / 3.0) * (J0 * M0v) + (2.0 / 3.0) * (D.YM[g] + dt * RM);
          const double yB = (1.0 / 3.0) * (J0 * B0v) + (2.0 / 3.0) * (D.YB[g] + dt * RB);
          const double inv = swale::recip(J3);
          const double En = yE * inv, Mn = yM * inv, Bn = yB * inv;
          D.E0[g] = En;
          D.M0[g] = Mn;
          D.B0[g] = Bn;
          D.J0[g] = J3;
          jmaxb = J3;
          jminb = J3;
          if (!PLAIN && K.bot_pieces > 0) {  // bottom after the step: projection onto the mesh at t_{n+1}
            const double xl = D.xn[nb + j], xr = D.xn[nb + j + 1];
            D.B0[g] = bottom_average(K, xl, xr);
            D.x[nb + j] = xl;
            if (j == N - 1) D.x[nb + N] = xr;
          } else {
            D.x[nb + j] += dt * wl;
            if (j == N - 1) D.x[nb + N] += dt * wr;
          }
          if (swale::bad(En) || swale::bad(Mn) || swale::bad(Bn)) st |= swale::ST_NONFINITE;
        }
      }
    }
    if (MODE == 0) {
      block_or_status(STAGE == 3 ? &S->st3 : &S->status, st);
      if (STAGE == 1) {
        block_max_to(&S->Jmax[1], jmaxa);
        block_max_to(&S->Jmax[2], jmaxb);
      } else if (STAGE == 3) {
        block_max_to(&S->JmaxN, jmaxb);
        block_min_to(&S->JminN, jminb);
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// End of a step, one block per instance (grid-stride): a clean step advances the instance's time
// and step count; a step whose stage-3 update raised an error (after committing its cells) is
// rolled back from the backups, and one that failed earlier wrote nothing. The stage-3 bits
// join the status word here.
// ------------------------------------------------------------------------------------
__global__ void k_commit(StepConst K, DevState D) {
  for (int i = blockIdx.x; i < K.B; i += gridDim.x) {
    DevScalars* S = D.S + i;
    const bool skip = S->done;
    const unsigned int before = S->status & kErrBits, bad3 = S->st3 & kErrBits;
    __syncthreads();  // every thread has read the words before thread 0 changes them
    if (skip) continue;
    if (!before && bad3 && D.bE) {
      const InstConst ic = D.IC[i];
      const int64_t cb = ic.coff, nb = ic.coff + i;
      for (int64_t j = threadIdx.x; j < ic.N; j += blockDim.x) {
        D.E0[cb + j] = D.bE[cb + j];
        D.M0[cb + j] = D.bM[cb + j];
        D.B0[cb + j] = D.bB[cb + j];
        D.J0[cb + j] = D.bJ[cb + j];
      }
      for (int64_t k = threadIdx.x; k <= ic.N; k += blockDim.x) D.x[nb + k] = D.bx[nb + k];
    }
    if (threadIdx.x == 0) {
      S->status |= S->st3;
      if (!before && !bad3) {
        S->t = S->clipped ? K.t_end : S->t + S->dt;
        S->steps += 1;
      } else {  // the widths stay those of J^n
        S->JmaxN = S->Jmax[0];
        S->JminN = S->Jmin0;
      }
    }
  }
}

// Detector classes of every instance into a dense array (N_i bytes per instance, in order).
__global__ void k_gather_flags(DevState D, int32_t B, uint8_t* out) {
  for (int i = blockIdx.x; i < B; i += gridDim.x) {
    const InstConst ic = D.IC[i];
    const int64_t eb = ic.coff + 2 * (int64_t)i;
    for (int64_t c = threadIdx.x; c < ic.N; c += blockDim.x) out[ic.coff + c] = D.flags[eb + c + 1];
  }
}

// Max of the widths of one instance into S->Jmax[0] and S->Jmax[1] (used by swale_rhs and
// swale_rhs_noalloc, which evaluate a stage outside a step).
__global__ void k_widths_max(const double* __restrict__ J, int64_t N, DevScalars* S) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, J[i]);
  block_max_to(&S->Jmax[0], m);
}

}  // namespace swale_dev
