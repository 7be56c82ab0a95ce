// Device kernels of the discrete adjoint of one SSP-RK3 step (Eq. RK32D) of the well-balanced
// ALE-WENO hybrid scheme: reverse of the RK combination, and for each stage the reverse of the
// interface fluxes, of the source term and of the reconstruction + limiter. They walk the same
// (instance, tile) work lists as the forward kernels; the adjoints of the stage input are
// accumulated with FP64 atomicAdd (each cell receives the contributions of the stencils, fluxes
// and sources that read it; ghost cells map back to their physical image, with the discharge's
// sign flipped at reflective boundaries).
#pragma once

#include "swale_adjoint.cuh"
#include "swale_kernels.cuh"

namespace swale_dev {

// Adjoint work arrays (concatenated like the state; edge adjoints in the edge layout).
struct AdjState {
  double *lE, *lM, *lB;   // lambda: adjoint of q^{n+1} on entry, of q^n on exit
  double *yE, *yM, *yB;   // adjoint of the running RK combination Y
  double *pE, *pM, *pB;   // accumulated adjoint of q^n through the RK combination
  double *aE, *aM, *aB;   // adjoint of the current stage input (atomically accumulated)
  double *rE, *rM, *rB;   // adjoint of the current stage's right-hand side
  double *ab[8];          // adjoints of the edge state (EL, ER, BL, BR, hL, hR, uL, uR)
  double *sE, *sM, *sB, *sJ;  // q^n and J^n of the step being reversed
};

__device__ __forceinline__ Tile utile_of(const DevState& D, int t, int T) {
  return D.utiles ? D.utiles[t] : Tile{0, t * T};
}

// Reverse of the RK combination, one phase per call. With Y3 = J3 q^{n+1}:
//   PH 3: Y = lambda / J3;  p = J0 Y / 3;  y = 2 Y / 3;  r = 2 dt Y / 3
//   PH 2: y += a / J2;      p += 3 J0 y / 4;  r = dt y / 4;  y = y / 4
//   PH 1: y += a / J1;      p += J0 y;        r = dt y
//   PH 0: lambda = p + a
// a (the stage adjoint of the previous phase) is read and cleared.
template <int PH, int T>
__global__ void __launch_bounds__(T) k_adj_rk(DevState D, AdjState A) {
  for (int t = blockIdx.x; t < D.nu; t += gridDim.x) {
    const Tile tl = utile_of(D, t, T);
    const InstConst ic = D.IC[tl.inst];
    const int64_t j = tl.c0 + threadIdx.x;
    if (j >= ic.N) continue;
    const int64_t g = ic.coff + j;
    const double dt = D.S[tl.inst].dt;
    double* lv[3] = {A.lE, A.lM, A.lB};
    double* yv[3] = {A.yE, A.yM, A.yB};
    double* pv[3] = {A.pE, A.pM, A.pB};
    double* av[3] = {A.aE, A.aM, A.aB};
    double* rv[3] = {A.rE, A.rM, A.rB};
    const double J0 = A.sJ[g];
    // All loads of the phase are issued before its first store (the arrays never alias, but
    // the compiler cannot know), so the memory latencies overlap instead of adding up.
    if (PH == 3) {
      const double iJ3 = swale::recip(D.J0[g]);  // J^{n+1} after the recomputed step
      double l[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) l[v] = lv[v][g];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const double Y = l[v] * iJ3;
        pv[v][g] = (1.0 / 3.0) * J0 * Y;
        yv[v][g] = (2.0 / 3.0) * Y;
        rv[v][g] = (2.0 / 3.0) * dt * Y;
      }
    } else if (PH == 2) {
      const double iJ2 = swale::recip(D.J2[g]);
      double y0[3], a[3], p[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        y0[v] = yv[v][g];
        a[v] = av[v][g];
        p[v] = pv[v][g];
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const double y = y0[v] + a[v] * iJ2;
        av[v][g] = 0.0;
        pv[v][g] = p[v] + 0.75 * J0 * y;
        rv[v][g] = 0.25 * dt * y;
        yv[v][g] = 0.25 * y;
      }
    } else if (PH == 1) {
      const double iJ1 = swale::recip(D.J1[g]);
      double y0[3], a[3], p[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        y0[v] = yv[v][g];
        a[v] = av[v][g];
        p[v] = pv[v][g];
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const double y = y0[v] + a[v] * iJ1;
        av[v][g] = 0.0;
        pv[v][g] = p[v] + J0 * y;
        rv[v][g] = dt * y;
      }
    } else {
      double p[3], a[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        p[v] = pv[v][g];
        a[v] = av[v][g];
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        lv[v][g] = p[v] + a[v];
        av[v][g] = 0.0;
      }
    }
  }
}

// Reverse of the interface fluxes of stage STAGE: interface k of cells k-1 and k gets the
// flux adjoints from the right-hand-side adjoints of its two cells and writes the adjoints of
// the right edge of cell k-1 and of the left edge of cell k (each edge slot has one writer).
template <int STAGE, int T>
__global__ void __launch_bounds__(T) k_adj_flux(StepConst K, DevState D, AdjState A) {
  for (int t = blockIdx.x; t < D.nu; t += gridDim.x) {
    const Tile tl = utile_of(D, t, T);
    const InstConst ic = D.IC[tl.inst];
    const DevScalars* S = D.S + tl.inst;
    const int64_t N = ic.N, cb = ic.coff, nb = ic.coff + tl.inst, eb = ic.coff + 2 * (int64_t)tl.inst;
    double alpha = (STAGE == 1) ? S->alpha1 : bitsd(S->A[STAGE - 1]) + S->Wbar;
    if (STAGE > 1 && K.alpha_mode == 2) alpha = stage_alpha(K, tl.inst, STAGE, alpha, S->step_idx);
    for (int i = threadIdx.x; i <= T; i += T) {
      const int64_t k = tl.c0 + i;
      if (k > N || (i == T && k != N)) continue;
      swale::Flux Fb;
      const double rEr = (k < N) ? A.rE[cb + k] : 0.0, rEl = (k > 0) ? A.rE[cb + k - 1] : 0.0;
      const double rMr = (k < N) ? A.rM[cb + k] : 0.0, rMl = (k > 0) ? A.rM[cb + k - 1] : 0.0;
      const double rBr = (k < N) ? A.rB[cb + k] : 0.0, rBl = (k > 0) ? A.rB[cb + k - 1] : 0.0;
      Fb.FE = rEr - rEl;
      Fb.FMm = -rMl;
      Fb.FMp = rMr;
      Fb.FB = rBl - rBr;
      const double wk = (K.mesh == SWALE_MESH_STATIC) ? 0.0 : D.w[nb + k];
      const int64_t el = eb + k, er = eb + k + 1;
      if (k == 0) {  // the ghost cell -1 has no left interface
        A.ab[0][el] = 0.0;
        A.ab[2][el] = 0.0;
        A.ab[4][el] = 0.0;
        A.ab[6][el] = 0.0;
      }
      if (k == N) {  // the ghost cell N has no right interface
        A.ab[1][er] = 0.0;
        A.ab[3][er] = 0.0;
        A.ab[5][er] = 0.0;
        A.ab[7][er] = 0.0;
      }
      const swale::EdgeAdj a = swale::interface_flux_rev(K.sc.g, alpha, wk, D.eER[el], D.eEL[er], D.eBR[el],
                                                         D.eBL[er], D.ehR[el], D.ehL[er], D.euR[el], D.euL[er], Fb);
      // interface_flux_rev names its inputs as (left state, right state) = (EL, ER, ...).
      A.ab[1][el] = a.EL;  // right edge of cell k-1
      A.ab[3][el] = a.BL;
      A.ab[5][el] = a.hL;
      A.ab[7][el] = a.uL;
      A.ab[0][er] = a.ER;  // left edge of cell k
      A.ab[2][er] = a.BR;
      A.ab[4][er] = a.hR;
      A.ab[6][er] = a.uR;
    }
  }
}

// Reverse of the source term of stage STAGE for cell j: adds to the adjoints of its own
// limited edge depths and bottoms, and (atomically) to the stage-input adjoints of the depth
// and bottom averages of cells j-1, j, j+1.
template <int STAGE, int T>
__global__ void __launch_bounds__(T) k_adj_source(StepConst K, DevState D, AdjState A, const double* __restrict__ Eg,
                                                  const double* __restrict__ Bg, const double* __restrict__ Jsg) {
  for (int t = blockIdx.x; t < D.nu; t += gridDim.x) {
    const Tile tl = utile_of(D, t, T);
    const InstConst ic = D.IC[tl.inst];
    const int64_t N = ic.N, cb = ic.coff, eb = ic.coff + 2 * (int64_t)tl.inst;
    const int64_t j = tl.c0 + threadIdx.x;
    if (j >= N) continue;
    const int64_t jm = ghost(j - 1, N, K.bc), jp = ghost(j + 1, N, K.bc);
    const double* E = Eg + cb;
    const double* B = Bg + cb;
    const double* Js = Jsg + cb;
    const double Jm = Js[jm], Jc = Js[j], Jp = Js[jp];
    const int64_t ie = eb + j + 1;
    // The source form's entries: as the forward recompute's update stored them, else computed.
    swale::SourceForm sf;
    if (D.gK) {
      double* const f = reinterpret_cast<double*>(&sf);
#pragma unroll
      for (int k = 0; k < 6; ++k) f[k] = D.gK[(8 + k) * D.geo_stride + ie];
    } else {
      sf = swale::source_form(Jm, Jc, Jp, swale::recip(Jm), swale::recip(Jc), swale::recip(Jp), D.ipair[eb + j],
                              D.ipair[eb + j + 1], D.itri[eb + j + 1]);
    }
    const double hd[5] = {E[jm] - B[jm], E[j] - B[j], E[jp] - B[jp], D.ehL[ie], D.ehR[ie]};
    const double bd[5] = {B[jm], B[j], B[jp], D.eBL[ie], D.eBR[ie]};
    double hdb[5] = {0, 0, 0, 0, 0}, bdb[5] = {0, 0, 0, 0, 0};
    swale::source_cell_form_rev(K.sc.g, hd, bd, sf, A.rM[cb + j], hdb, bdb);
    A.ab[4][ie] += hdb[3];
    A.ab[5][ie] += hdb[4];
    A.ab[2][ie] += bdb[3];
    A.ab[3][ie] += bdb[4];
    const int64_t cells[3] = {jm, j, jp};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&A.aE[cb + cells[k]], hdb[k]);
      atomicAdd(&A.aB[cb + cells[k]], bdb[k] - hdb[k]);
    }
  }
}

// The reverse of a cell whose class the FP32 test leaves open, out of line (the FP64 detector,
// the WENO-Z weights and their adjoints): its registers do not weigh on the smooth cells' code.
struct AdjOpenIn {
  swale::StencilDD DD;
  swale::EdgeAdj ob;
  double h[5], it[3], v0[3][3], dxmax;
};
struct AdjOpenOut {
  swale::StencilDD DDb;
  double v0b[3][3];
};
__device__ __noinline__ AdjOpenOut adj_open_cell(const SchemeConst P, const AdjOpenIn c) {
  AdjOpenOut r;
  swale::recon_cell_rev(P, c.h, c.it, c.v0, c.DD, c.dxmax, c.ob, r.v0b, r.DDb, false);
  return r;
}

// Reverse of the reconstruction + limiter of stage STAGE for cells -1..N (tiles of T cells
// staged like the forward kernel): each cell's reverse sweep gives the adjoints of its stencil
// averages and divided differences, which map to the 5 stencil cells and are added atomically.
template <int STAGE, int T>
__global__ void __launch_bounds__(T, 512 / T) k_adj_recon(StepConst K, DevState D, AdjState A, const double* __restrict__ Eg,
                                                 const double* __restrict__ Mg, const double* __restrict__ Bg,
                                                 const double* __restrict__ Jg) {
  __shared__ double sJ[T + 4], sV[3][T + 4];
  __shared__ double sIP[T + 3], sD2[3][T + 3];
  __shared__ double sIT[T + 2];
  // FP32 copies for the smooth-class test of the forward: pair differences of hu and of the
  // depth (eta's minus the bottom's), triple reciprocals.
  __shared__ float sD2f[2][T + 3], sITf[T + 2];
  const int tid = threadIdx.x;
  const bool refl = (K.bc == SWALE_BC_REFLECTIVE);
  for (int t = blockIdx.x; t < D.nr; t += gridDim.x) {
    const Tile tl = D.rtiles ? D.rtiles[t] : Tile{0, t * T - 1};
    const DevScalars* S = D.S + tl.inst;
    const InstConst ic = D.IC[tl.inst];
    const int64_t N = ic.N, c0 = tl.c0, cb = ic.coff;
    const double* E = Eg + cb;
    const double* M = Mg + cb;
    const double* B = Bg + cb;
    const double* J = Jg + cb;
    const int64_t eb = ic.coff + 2 * (int64_t)tl.inst;
    __syncthreads();
    for (int i = tid; i < T + 4; i += T) {
      const int64_t c = c0 - 2 + i;
      double jv = 1.0, ev = 0.0, mv = 0.0, bv = 0.0;
      if (c >= -3 && c <= N + 2) {
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
      sV[2][i] = bv;
    }
    __syncthreads();
    for (int i = tid; i < T + 3; i += T) {
      const double ip = swale::pair_recip(sJ[i], sJ[i + 1]);
      sIP[i] = ip;
      double d2[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) sD2[v][i] = d2[v] = swale::pair_dd(sV[v][i], sV[v][i + 1], ip);
      sD2f[0][i] = swale::f32_trunc(d2[1]);
      sD2f[1][i] = swale::f32_trunc(d2[0] - d2[2]);
    }
    __syncthreads();
    for (int i = tid; i < T + 2; i += T) {
      const double it = swale::triple_recip(sJ[i], sJ[i + 1], sJ[i + 2]);
      sIT[i] = it;
      sITf[i] = swale::f32_trunc(it);
    }
    __syncthreads();
    const int64_t c = c0 + tid;
    if (c > N) continue;
    double h[5], v0[3][3];
    swale::StencilDD DD, DDb;
#pragma unroll
    for (int k = 0; k < 5; ++k) h[k] = sJ[tid + k];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
#pragma unroll
      for (int a = 0; a < 3; ++a) v0[v][a] = sV[v][tid + a];
#pragma unroll
      for (int a = 0; a < 4; ++a) DD.D2[v][a] = sD2[v][tid + a];
    }
    const int64_t idx = eb + c + 1;
    const swale::EdgeAdj ob = {A.ab[0][idx], A.ab[1][idx], A.ab[2][idx], A.ab[3][idx],
                               A.ab[4][idx], A.ab[5][idx], A.ab[6][idx], A.ab[7][idx]};
    double v0b[3][3];
    const double it3[3] = {sIT[tid], sIT[tid + 1], sIT[tid + 2]};
    // The forward's FP32 test of the smooth class on the same data: where it holds, the FP64
    // class is 0 as well and the indicators are not formed.
    const double dxmax = bitsd(S->Jmax[STAGE - 1]);
    float F32[3], c4f, c3f, itf[3], d2h[4], d2m[4];
    swale::indicator_factors_f32(h, K.sc.beta_dx_global ? dxmax : h[2], F32, c4f, c3f);
#pragma unroll
    for (int a = 0; a < 3; ++a) itf[a] = sITf[tid + a];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      d2h[a] = sD2f[1][tid + a];
      d2m[a] = sD2f[0][tid + a];
    }
    const bool smooth32 =
        swale::sure_smooth_f32(F32, c4f, c3f, d2h, d2m, itf, swale::f32_trunc(K.sc.eps_weno));
    if (smooth32) {
      if (D.gK) {  // the linear form the forward recompute stored for this stage
        double Kf[2][4];
#pragma unroll
        for (int k = 0; k < 8; ++k) Kf[k >> 2][k & 3] = D.gK[k * D.geo_stride + idx];
        swale::recon_cell_rev_lin(K.sc, Kf, v0, DD, ob, v0b, DDb);
      } else {
        swale::recon_cell_rev(K.sc, h, it3, v0, DD, dxmax, ob, v0b, DDb, true);
      }
    } else {
      // The third differences, only where the class is open (the smooth class needs none).
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int a = 0; a < 3; ++a) DD.D3[v][a] = swale::triple_dd(DD.D2[v][a], DD.D2[v][a + 1], it3[a]);
      AdjOpenIn in;
      in.DD = DD;
      in.ob = ob;
      in.dxmax = dxmax;
#pragma unroll
      for (int k = 0; k < 5; ++k) in.h[k] = h[k];
#pragma unroll
      for (int a = 0; a < 3; ++a) in.it[a] = it3[a];
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int a = 0; a < 3; ++a) in.v0[v][a] = v0[v][a];
      const AdjOpenOut r = adj_open_cell(K.sc, in);
      DDb = r.DDb;
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int a = 0; a < 3; ++a) v0b[v][a] = r.v0b[v][a];
    }
    // Stencil cell adjoints: cv[v][k] for cells c-2+k.
    double cv[3][5];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
#pragma unroll
      for (int k = 0; k < 5; ++k) cv[v][k] = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) cv[v][a] += v0b[v][a];
      double d2b[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) d2b[a] = DDb.D2[v][a];
      if (!smooth32) {  // DDb.D3 is 0 in the smooth class
#pragma unroll
        for (int a = 0; a < 3; ++a) {  // D3[a] = (D2[a+1] - D2[a]) it[a]
          const double x = DDb.D3[v][a] * sIT[tid + a];
          d2b[a + 1] += x;
          d2b[a] -= x;
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {  // D2[a] = (v[a+1] - v[a]) ip[a]
        const double x = d2b[a] * sIP[tid + a];
        cv[v][a + 1] += x;
        cv[v][a] -= x;
      }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int64_t vc = c - 2 + k;
      const int64_t s = ghost(vc, N, K.bc);
      const double sgn = (refl && (vc < 0 || vc >= N)) ? -1.0 : 1.0;
      atomicAdd(&A.aE[cb + s], cv[0][k]);
      atomicAdd(&A.aM[cb + s], sgn * cv[1][k]);
      atomicAdd(&A.aB[cb + s], cv[2][k]);
    }
  }
}

// Gauge misfit of the state after a step: gauge g of instance i sits at x = gx[i * G + g]; its
// depth is the average of the cell that contains x on the current mesh. MODE 0 adds
// dt (h - obs)^2 to Jout[i]; MODE 1 adds its gradient 2 dt (h - obs) to lambda (eta: +, b: -).
// obs points at the row of the observed depths for this step (B x G values).
// gcell[id] caches the gauge's cell between calls (-1: not located yet): from there a short walk
// finds the cell on the new mesh (a node moves by less than a cell per step); the first call
// bisects. Either way the cell is c with x[c] <= xg < x[c+1] (clamped to 0..N-1).
template <int MODE>
__global__ void k_misfit(DevState D, AdjState A, int32_t B, int32_t G, const double* __restrict__ gx,
                         const double* __restrict__ obs, double* Jout, int64_t* gcell) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)B * G) return;
  const int i = (int)(id / G);
  const InstConst ic = D.IC[i];
  const double* x = D.x + ic.coff + i;
  const double xg = gx[id];
  int64_t lo = gcell[id];
  if (lo < 0 || lo >= ic.N) {
    lo = 0;
    int64_t hi = ic.N;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (x[mid] <= xg) lo = mid;
      else hi = mid;
    }
  } else {
    while (lo + 1 < ic.N && x[lo + 1] <= xg) ++lo;
    while (lo > 0 && x[lo] > xg) --lo;
  }
  gcell[id] = lo;
  const int64_t g = ic.coff + lo;
  const double r = (D.E0[g] - D.B0[g]) - obs[id];
  const double dt = D.S[i].dt;
  if (MODE == 0) {
    atomicAdd(&Jout[i], dt * r * r);
  } else {
    atomicAdd(&A.lE[g], 2.0 * dt * r);
    atomicAdd(&A.lB[g], -2.0 * dt * r);
  }
}

}  // namespace swale_dev
