// Per-cell and per-interface arithmetic of one stage of the well-balanced ALE-WENO hybrid
// scheme (Zhang, Xia & Xu, arXiv 2208.06588), written once for the device kernels.
//
// Formulation (same mathematics as the paper's definitions, arranged for few FP64 ops):
//  * Step 1 of Sec. 2.2: each sub-stencil quadratic p_r is the derivative of the cubic
//    interpolating the primitive function, kept in Newton form. Its coefficients are the
//    divided differences D2 (pairs of cells) and D3 (triples of cells) of the cell averages,
//    and the geometry enters only through node offsets. The linear weights d_r at the two
//    edges come from matching the coefficients of the outermost averages of the big-stencil
//    quartic and of p_2 / p_0, also in Newton form.
//  * Step 2: beta_r = Dx int (p_r')^2 + Dx^3 int (p_r'')^2 evaluated in closed form about
//    the cell midpoint.
//  * Sec. 4.1 source term: the quartic interpolants (three cell averages + two edge values)
//    are built as the derivative of a confluent Newton (Hermite) form of their primitive;
//    the Newton basis derivatives at the four Gauss-Legendre points are affine in the ratio
//    of the left neighbour's width, with constant coefficients.
// All lengths are physical; nothing here allocates or branches on data except the
// detector classes, the limiter and the dry-edge test that the scheme itself defines.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define SWALE_HD __host__ __device__ __forceinline__
#else
#define SWALE_HD inline
#endif

namespace swale {

// Scalar type of the per-cell arithmetic: double in the CUDA build. A host-only build can
// define SWALE_REAL to an operation-counting type to count the FP64 work per cell.
#ifdef SWALE_REAL
typedef SWALE_REAL real;
#else
typedef double real;
#endif

// Scheme constants passed by value to every kernel.
struct SchemeConst {
  double g, eps_weno, eps_pp, h_dry;
  int32_t beta_dx_global;
};

// Status bits accumulated on the device.
enum : uint32_t {
  ST_EWEIGHT = 1u,    // a linear weight d_r <= 0
  ST_NEGDEPTH = 2u,   // a cell-average depth below -eps_pp entered a stage (warning)
  ST_NONFINITE = 4u,  // a non-finite value appeared
  ST_EMESH = 8u,      // a cell width <= 0
};

// Limited edge state of one cell (edge L = x_{j-1/2}^+, edge R = x_{j+1/2}^-).
struct EdgeState {
  real EL, ER, BL, BR, hL, hR, uL, uR;
};

SWALE_HD real dmax(real a, real b) { return (b > a) ? b : a; }
SWALE_HD real dmin(real a, real b) { return (b < a) ? b : a; }
SWALE_HD real dabs(real a) { return a < 0.0 ? -a : a; }
#ifdef SWALE_REAL
SWALE_HD real rsqrt_(real a) { return swale_sqrt(a); }
#else
SWALE_HD real rsqrt_(real a) { return sqrt(a); }
#endif

// Value and derivative at x of prod_i (x - y_i), accumulated factor by factor.
struct ProdD {
  real p, dp;
};
SWALE_HD ProdD prod_push(ProdD a, real x, real y) {
  real f = x - y;
  ProdD r;
  r.dp = a.dp * f + a.p;
  r.p = a.p * f;
  return r;
}

// Mesh-only data of one cell from the five widths J_{j-2..j+2}.
struct CellGeom {
  real ip[4];    // 1 / (J_m + J_{m+1}), pairs (j-2,j-1) .. (j+1,j+2)
  real it[3];    // 1 / (J_m + J_{m+1} + J_{m+2}), triples starting at j-2, j-1, j
  real G1[2][3]; // G1[e][a] = (x_e - y_a) + (x_e - y_{a+1})
  real G2[2][3]; // G2[e][a] = sum of the pairwise products of (x_e - y_{a..a+2})
  real F[3];     // F[a] = 1.5 J_j - (y_a + y_{a+1} + y_{a+2})
  real d[2][3];  // linear weights d_r at edge e (r = 0,1,2)
  real c4, c3;   // beta factors: 4 Dx J_j and 3 Dx J_j^3 + 36 Dx^3 J_j
};

SWALE_HD void cell_geom(const real J[5], real dx, CellGeom& G, uint32_t& st) {
  // Node offsets relative to x_{j-1/2}: y0 .. y5 bound cells j-2 .. j+2.
  const real y[6] = {-(J[0] + J[1]), -J[1], 0.0, J[2], J[2] + J[3], J[2] + J[3] + J[4]};
  for (int m = 0; m < 4; ++m) G.ip[m] = 1.0 / (J[m] + J[m + 1]);
  for (int m = 0; m < 3; ++m) G.it[m] = 1.0 / (J[m] + J[m + 1] + J[m + 2]);
  const real xe[2] = {0.0, J[2]};
  for (int e = 0; e < 2; ++e) {
    const real x = xe[e];
    for (int a = 0; a < 3; ++a) {
      const real p = x - y[a], q = x - y[a + 1], r = x - y[a + 2];
      G.G1[e][a] = p + q;
      G.G2[e][a] = q * r + p * r + p * q;
    }
    // Coefficient of ubar_{j-2} in p_2(x) (Newton form from the left end of the stencil)
    // and in the big-stencil quartic; their ratio is d_2.
    ProdD L = {1.0, 0.0};
    L = prod_push(L, x, y[0]);
    L = prod_push(L, x, y[1]);
    const real pi2d = L.dp;
    L = prod_push(L, x, y[2]);
    const real pi3d = L.dp;
    L = prod_push(L, x, y[3]);
    const real pi4d = L.dp;
    L = prod_push(L, x, y[4]);
    const real pi5d = L.dp;
    const real a1 = y[2] - y[0], a2 = a1 * (y[3] - y[0]), a3 = a2 * (y[4] - y[0]), a4 = a3 * (y[5] - y[0]);
    const real c20 = 1.0 - pi2d / a1 + pi3d / a2;
    const real C0 = c20 - pi4d / a3 + pi5d / a4;
    // Coefficient of ubar_{j+2} in p_0(x) and in the quartic (Newton form from the right end).
    ProdD R = {1.0, 0.0};
    R = prod_push(R, x, y[5]);
    R = prod_push(R, x, y[4]);
    const real s2d = R.dp;
    R = prod_push(R, x, y[3]);
    const real s3d = R.dp;
    R = prod_push(R, x, y[2]);
    const real s4d = R.dp;
    R = prod_push(R, x, y[1]);
    const real s5d = R.dp;
    const real b1 = y[5] - y[3], b2 = b1 * (y[5] - y[2]), b3 = b2 * (y[5] - y[1]), b4 = b3 * (y[5] - y[0]);
    const real c02 = 1.0 + s2d / b1 + s3d / b2;
    const real C4 = c02 + s4d / b3 + s5d / b4;
    G.d[e][2] = C0 / c20;
    G.d[e][0] = C4 / c02;
    G.d[e][1] = 1.0 - G.d[e][0] - G.d[e][2];
    if (!(G.d[e][0] > 0.0) || !(G.d[e][1] > 0.0) || !(G.d[e][2] > 0.0)) st |= ST_EWEIGHT;
  }
  for (int a = 0; a < 3; ++a) G.F[a] = 1.5 * J[2] - (y[a] + y[a + 1] + y[a + 2]);
  const real h0 = J[2];
  G.c4 = 4.0 * dx * h0;
  G.c3 = 3.0 * dx * h0 * h0 * h0 + 36.0 * dx * dx * dx * h0;
  for (int k = 0; k < 5; ++k)
    if (!(J[k] > 0.0)) st |= ST_EMESH;
}

// Divided differences of one variable on the big stencil.
struct DivDiff {
  real D2[4], D3[3];
};
SWALE_HD void divdiff(const CellGeom& G, const real v[5], DivDiff& D) {
  for (int m = 0; m < 4; ++m) D.D2[m] = (v[m + 1] - v[m]) * G.ip[m];
  for (int m = 0; m < 3; ++m) D.D3[m] = (D.D2[m + 1] - D.D2[m]) * G.it[m];
}

// Sub-stencil value p_r at edge e; sub-stencil r starts at cell a = 2 - r.
SWALE_HD real sub_value(const CellGeom& G, const DivDiff& D, const real v[5], int e, int a) {
  return v[a] + D.D2[a] * G.G1[e][a] + D.D3[a] * G.G2[e][a];
}

// Reconstruction of one cell (Steps 1-4 of Sec. 2.2 with the shared indicators of
// Eq. alphamodified), bound-preserving limiter (Eq. modifiedhjn in 1D, Gauss-Lobatto
// k = 4) and the bottom re-derivation of the Remark in Sec. 4.3.
// Returns the largest |u| + sqrt(g h) over the two edges in *wave_L / *wave_R.
SWALE_HD void recon_cell(const SchemeConst& P, const real J[5], const real E[5], const real M[5],
                         const real B[5], real dxmax, EdgeState& o, uint8_t& flag, real& waveL,
                         real& waveR, uint32_t& st) {
  const real dx = P.beta_dx_global ? dxmax : J[2];
  CellGeom G;
  cell_geom(J, dx, G, st);
  DivDiff DE, DM, DB;
  divdiff(G, E, DE);
  divdiff(G, M, DM);
  divdiff(G, B, DB);
  // Indicators from the conservative variables h = eta - b and hu, summed (shared weights).
  real beta[3];
  for (int r = 0; r < 3; ++r) {
    const int a = 2 - r;
    const real d2h = DE.D2[a] - DB.D2[a], d3h = DE.D3[a] - DB.D3[a];
    const real qh = d2h + d3h * G.F[a], qm = DM.D2[a] + DM.D3[a] * G.F[a];
    beta[r] = G.c4 * (qh * qh + qm * qm) + G.c3 * (d3h * d3h + DM.D3[a] * DM.D3[a]);
  }
  const real tau = dabs(beta[0] - beta[2]);
  const real betaA = (beta[0] + beta[1] + beta[2]) * (1.0 / 3.0);
  const real gam = tau / (betaA + P.eps_weno);
  flag = gam <= 0.5 ? 0 : (gam >= 1.0 ? 2 : 1);
  real X[3] = {1.0, 1.0, 1.0};
  if (flag != 0) {
    for (int r = 0; r < 3; ++r) {
      const real q = tau / (beta[r] + P.eps_weno);
      X[r] = 1.0 + q * q;
    }
  }
  real ev[2], mv[2], bv[2];
  for (int e = 0; e < 2; ++e) {
    real phi[3];
    if (flag == 0) {
      for (int r = 0; r < 3; ++r) phi[r] = G.d[e][r];
    } else {
      real al[3];
      for (int r = 0; r < 3; ++r) al[r] = G.d[e][r] * X[r];
      const real inv = 1.0 / (al[0] + al[1] + al[2]);
      for (int r = 0; r < 3; ++r) phi[r] = al[r] * inv;
      if (flag == 1) {
        const real Mg = 2.0 * gam - 1.0;
        for (int r = 0; r < 3; ++r) phi[r] = Mg * phi[r] + (1.0 - Mg) * G.d[e][r];
      }
    }
    real se = 0.0, sm = 0.0, sb = 0.0;
    for (int r = 0; r < 3; ++r) {
      const int a = 2 - r;
      se += phi[r] * sub_value(G, DE, E, e, a);
      sm += phi[r] * sub_value(G, DM, M, e, a);
      sb += phi[r] * sub_value(G, DB, B, e, a);
    }
    ev[e] = se;
    mv[e] = sm;
    bv[e] = sb;
  }
  // Limiter on h = eta - b with the Gauss-Lobatto mean delta; hu scaled by the same theta.
  real hbar = E[2] - B[2];
  if (hbar < -P.eps_pp) st |= ST_NEGDEPTH;
  hbar = dmax(hbar, 0.0);
  real hL = ev[0] - bv[0], hR = ev[1] - bv[1];
  const real delta = (12.0 * hbar - hL - hR) * 0.1;
  const real mn = dmin(dmin(hL, hR), delta);
  const real epsv = dmin(P.eps_pp, hbar);
  real mL = mv[0], mR = mv[1];
  if (mn < epsv) {
    const real theta = (hbar - epsv) / (hbar - mn);
    const real mbar = M[2];
    hL = theta * (hL - hbar) + hbar;
    hR = theta * (hR - hbar) + hbar;
    mL = theta * (mL - mbar) + mbar;
    mR = theta * (mR - mbar) + mbar;
  }
  o.EL = ev[0];
  o.ER = ev[1];
  o.hL = hL;
  o.hR = hR;
  o.BL = ev[0] - hL;
  o.BR = ev[1] - hR;
  o.uL = hL > P.h_dry ? mL / hL : 0.0;
  o.uR = hR > P.h_dry ? mR / hR : 0.0;
  waveL = dabs(o.uL) + rsqrt_(P.g * dmax(hL, 0.0));
  waveR = dabs(o.uR) + rsqrt_(P.g * dmax(hR, 0.0));
  // NaN propagates into the comparisons as false: catch it explicitly.
  const real chk = o.EL + o.ER + o.hL + o.hR + mL + mR;
  if (!(chk == chk) || dabs(chk) > 1.0e300) st |= ST_NONFINITE;
}

// Interface fluxes of the hydrostatic-reconstruction ALE-LF scheme (Eq. hydro2D-HH2D and
// the bottom flux of Eq. bottomrk): FE (eta), FMm (momentum seen by the left cell),
// FMp (seen by the right cell), FB (bottom). L is the right edge of the left cell, R the
// left edge of the right cell; w is the node velocity, alpha the global viscosity.
struct Flux {
  real FE, FMm, FMp, FB;
};
SWALE_HD Flux interface_flux(real g, real alpha, real w, real EL, real ER, real BL, real BR, real hL,
                             real hR, real uL, real uR) {
  const real bstar = dmax(BL, BR);
  const real sL = dmax(0.0, EL - bstar), sR = dmax(0.0, ER - bstar);
  const real mL = sL * uL, mR = sR * uR;
  Flux f;
  // Hat-H^(1)(q*) + theta simplifies exactly to this expression.
  f.FE = 0.5 * (mL + mR) - 0.5 * w * (EL + ER) - 0.5 * alpha * (ER - EL);
  const real hg = 0.5 * g;
  const real H2 = 0.5 * ((mL * uL + hg * sL * sL - w * mL) + (mR * uR + hg * sR * sR - w * mR)) -
                    0.5 * alpha * (mR - mL);
  f.FMm = H2 + hg * (hL * hL - sL * sL);
  f.FMp = H2 + hg * (hR * hR - sR * sR);
  f.FB = 0.5 * w * (BL + BR) + 0.5 * alpha * (BR - BL);
  return f;
}

// Four-point Gauss-Legendre rule on [0, 1]: nodes and weights.
#define SWALE_GL4_T0 0.0694318442029737124
#define SWALE_GL4_T1 0.330009478207571868
#define SWALE_GL4_T2 0.669990521792428132
#define SWALE_GL4_T3 0.930568155797026288
#define SWALE_GL4_W0 0.173927422568726929
#define SWALE_GL4_W1 0.326072577431273071

// Source term int_cell -g (eta_h - b_h) b_h' dx of Sec. 4.1, with eta_h - b_h interpolating
// the depth data (averages h_{j-1}, h_j, h_{j+1}, limited edge depths h^L, h^R) and b_h the
// bottom data (averages and limited edge bottoms). In the unit coordinate t of the cell,
// rm = J_{j-1}/J_j and rp = J_{j+1}/J_j; irm = 1/rm, irp = 1/rp, i1m = 1/(1+rm),
// i1p = 1/(1+rp), i1mp = 1/(1+rm+rp).
SWALE_HD real source_cell(real g, const real hd[5], const real bd[5], real rm, real irm, real irp,
                            real i1m, real i1p, real i1mp) {
  // Confluent divided differences of the primitive on nodes (-rm, 0, 0, 1, 1, 1+rp):
  // data order (avg_{j-1}, avg_j, avg_{j+1}, v_L, v_R).
  real ch[6], cb[6];
  const real* dat[2] = {hd, bd};
  real* cf[2] = {ch, cb};
  for (int v = 0; v < 2; ++v) {
    const real* u = dat[v];
    const real o2a = (u[3] - u[0]) * irm;  // [z1, z2, z2]
    const real o2b = u[1] - u[3];          // [z2, z2, z3]
    const real o2c = u[4] - u[1];          // [z2, z3, z3]
    const real o2d = (u[2] - u[4]) * irp;  // [z3, z3, z4]
    const real o3a = (o2b - o2a) * i1m;    // [z1, z2, z2, z3]
    const real o3b = o2c - o2b;            // [z2, z2, z3, z3]
    const real o3c = (o2d - o2c) * i1p;    // [z2, z3, z3, z4]
    const real o4a = (o3b - o3a) * i1m;    // [z1, z2, z2, z3, z3]
    const real o4b = (o3c - o3b) * i1p;    // [z2, z2, z3, z3, z4]
    const real o5 = (o4b - o4a) * i1mp;    // [z1 .. z4]
    real* c = cf[v];
    c[1] = u[0];
    c[2] = o2a;
    c[3] = o3a;
    c[4] = o4a;
    c[5] = o5;
  }
  // Basis n_k = (t + rm) m_k(t), m_2 = t, m_3 = t^2, m_4 = t^3 - t^2, m_5 = t^4 - 2 t^3 + t^2.
  // n_k' = (m_k + t m_k') + rm m_k', n_k'' = (2 m_k' + t m_k'') + rm m_k''.
  const real tq[4] = {SWALE_GL4_T0, SWALE_GL4_T1, SWALE_GL4_T2, SWALE_GL4_T3};
  const real wq[4] = {SWALE_GL4_W0, SWALE_GL4_W1, SWALE_GL4_W1, SWALE_GL4_W0};
  real S = 0.0;
  for (int q = 0; q < 4; ++q) {
    const real t = tq[q], t2 = t * t, t3 = t2 * t, t4 = t3 * t;
    const real m[6] = {0, 0, t, t2, t3 - t2, t4 - 2.0 * t3 + t2};
    const real md[6] = {0, 0, 1.0, 2.0 * t, 3.0 * t2 - 2.0 * t, 4.0 * t3 - 6.0 * t2 + 2.0 * t};
    const real mdd[6] = {0, 0, 0.0, 2.0, 6.0 * t - 2.0, 12.0 * t2 - 12.0 * t + 2.0};
    real hv = ch[1], bdv = 0.0;
    for (int k = 2; k <= 5; ++k) {
      const real n1 = (m[k] + t * md[k]) + rm * md[k];
      const real n2 = (2.0 * md[k] + t * mdd[k]) + rm * mdd[k];
      hv += ch[k] * n1;
      bdv += cb[k] * n2;
    }
    S += wq[q] * hv * bdv;
  }
  return -g * S;
}

// Right-hand side of cell j for one stage (Eq. hydro2D with Eq. bottomrk in 1D): fluxes at
// its two interfaces, the source term on its stage width, and the flux differences.
// Edge inputs: the right edge of cell j-1 (l*), both edges of cell j (c*), the left edge of
// cell j+1 (r*). Averages and widths of cells j-1, j, j+1: (Em, Ec, Ep), (Bm, Bc, Bp),
// (Jm, Jc, Jp). wl, wr: velocities of nodes j-1/2 and j+1/2.
struct CellRhs {
  real RE, RM, RB;
};
SWALE_HD CellRhs rhs_cell(real g, real alpha, real wl, real wr, real lE, real lB, real lh, real lu, real cEL,
                          real cER, real cBL, real cBR, real chL, real chR, real cuL, real cuR, real rE, real rB,
                          real rh, real ru, real Em, real Ec, real Ep, real Bm, real Bc, real Bp, real Jm,
                          real Jc, real Jp) {
  const Flux Fl = interface_flux(g, alpha, wl, lE, cEL, lB, cBL, lh, chL, lu, cuL);
  const Flux Fr = interface_flux(g, alpha, wr, cER, rE, cBR, rB, chR, rh, cuR, ru);
  const real ic0 = 1.0 / Jc;
  const real rm = Jm * ic0;
  const real irm = Jc / Jm, irp = Jc / Jp;
  const real i1m = Jc / (Jm + Jc), i1p = Jc / (Jc + Jp), i1mp = Jc / (Jm + Jc + Jp);
  const real hd[5] = {Em - Bm, Ec - Bc, Ep - Bp, chL, chR};
  const real bd[5] = {Bm, Bc, Bp, cBL, cBR};
  const real Sj = source_cell(g, hd, bd, rm, irm, irp, i1m, i1p, i1mp);
  CellRhs o;
  o.RE = -(Fr.FE - Fl.FE);
  o.RM = -(Fr.FMm - Fl.FMp) + Sj;
  o.RB = Fr.FB - Fl.FB;
  return o;
}

}  // namespace swale
