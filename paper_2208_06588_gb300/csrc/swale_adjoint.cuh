// Discrete adjoint of one SSP-RK3 step of the well-balanced ALE-WENO hybrid scheme (Zhang,
// Xia & Xu, arXiv 2208.06588): hand-written reverse mode of the per-cell arithmetic of
// swale_cell.cuh and the kernels that apply it to a whole stage.
//
// Replay convention: dt and the stage viscosities alpha_s are constants (recorded by the
// forward run); the detector classes, the limiter branch, the dry-edge tests and every max/min
// selection are those of the forward state, a tie selecting the first argument; |x| has slope
// sign(x), with slope 0 at x = 0. The mesh (widths, node velocities) is prescribed and carries
// no adjoint.
//
// Each function first recomputes the forward intermediates it needs from the same inputs as
// its forward counterpart, then runs the reverse sweep.
#pragma once

#include "swale_cell.cuh"

namespace swale {

// Adjoints of the eight edge quantities of one cell edge pair or interface.
struct EdgeAdj {
  real EL, ER, BL, BR, hL, hR, uL, uR;
};

// Adjoint of interface_flux: adjoints of the eight edge inputs from those of the four fluxes.
SWALE_HD EdgeAdj interface_flux_rev(real g, real alpha, real w, real EL, real ER, real BL, real BR, real hL,
                                    real hR, real uL, real uR, const Flux& Fb) {
  const bool selR = dlt(BL, BR);
  const real bstar = selR ? BR : BL;
  const real aL = EL - bstar, aR = ER - bstar;
  const bool pL = gt0(aL), pR = gt0(aR);
  const real sL = pL ? aL : real(0.0), sR = pR ? aR : real(0.0);
  const real mL = sL * uL, mR = sR * uR;
  const real hg = 0.5 * g;
  EdgeAdj a = {0, 0, 0, 0, 0, 0, 0, 0};
  real sLb = 0.0, sRb = 0.0, mLb = 0.0, mRb = 0.0;
  const real H2b = Fb.FMm + Fb.FMp;
  // FMm = H2 + hg (hL^2 - sL^2), FMp = H2 + hg (hR^2 - sR^2)
  a.hL = 2.0 * hg * hL * Fb.FMm;
  sLb = sLb - 2.0 * hg * sL * Fb.FMm;
  a.hR = 2.0 * hg * hR * Fb.FMp;
  sRb = sRb - 2.0 * hg * sR * Fb.FMp;
  // FE = (mL + mR)/2 - w (EL + ER)/2 - alpha (ER - EL)/2
  mLb = mLb + 0.5 * Fb.FE;
  mRb = mRb + 0.5 * Fb.FE;
  a.EL = (0.5 * alpha - 0.5 * w) * Fb.FE;
  a.ER = (-0.5 * alpha - 0.5 * w) * Fb.FE;
  // H2 = ((mL uL + hg sL^2 - w mL) + (mR uR + hg sR^2 - w mR))/2 - alpha (mR - mL)/2
  mLb = mLb + H2b * (0.5 * (uL - w) + 0.5 * alpha);
  mRb = mRb + H2b * (0.5 * (uR - w) - 0.5 * alpha);
  a.uL = 0.5 * H2b * mL;
  a.uR = 0.5 * H2b * mR;
  sLb = sLb + H2b * hg * sL;
  sRb = sRb + H2b * hg * sR;
  // FB = w (BL + BR)/2 + alpha (BR - BL)/2
  a.BL = (0.5 * w - 0.5 * alpha) * Fb.FB;
  a.BR = (0.5 * w + 0.5 * alpha) * Fb.FB;
  // m = s u
  sLb = sLb + mLb * uL;
  a.uL = a.uL + mLb * sL;
  sRb = sRb + mRb * uR;
  a.uR = a.uR + mRb * sR;
  // s = max(0, E - b*), b* = max(BL, BR)
  real bsb = 0.0;
  if (pL) {
    a.EL = a.EL + sLb;
    bsb = bsb - sLb;
  }
  if (pR) {
    a.ER = a.ER + sRb;
    bsb = bsb - sRb;
  }
  if (selR) a.BR = a.BR + bsb;
  else a.BL = a.BL + bsb;
  return a;
}

// Adjoint of source_cell_form: accumulates into hdb[5], bdb[5] the adjoints of the depth and
// bottom data for the adjoint Sb of the source value. With acc = h_j (db_R - db_L) + sum_k dh_k u_k
// and u = A db (+ the diagonal part), the adjoint of dh_k is u_k and that of db_l is
// v_l = sum_k dh_k A_kl (+ the diagonal part and +-h_j for R, L); h_j and b_j enter the
// differences with the sign -1.
SWALE_HD void source_cell_form_rev(real g, const real hd[5], const real bd[5], const SourceForm& A, real Sb,
                                   real hdb[5], real bdb[5]) {
  const real hc = hd[1], bc = bd[1];
  const real db0 = bd[0] - bc, db2 = bd[2] - bc, db3 = bd[3] - bc, db4 = bd[4] - bc;
  const real dh0 = hd[0] - hc, dh2 = hd[2] - hc, dh3 = hd[3] - hc, dh4 = hd[4] - hc;
  real u[4];
  source_form_rows(A, db0, db2, db3, db4, u);
  real v[4];
  v[0] = -(A.a02 * dh2) - A.a03 * dh3 - A.a04 * dh4;
  v[1] = A.a02 * dh0 - A.a23 * dh3 - A.a24 * dh4;
  v[2] = (A.a03 * dh0 + A.a23 * dh2) - A.a34 * dh4 - (hc + 0.5 * dh3);
  v[3] = (A.a04 * dh0 + A.a24 * dh2) + A.a34 * dh3 + (hc + 0.5 * dh4);
  const real ab = -g * Sb;  // adjoint of acc
  hdb[0] = hdb[0] + ab * u[0];
  hdb[2] = hdb[2] + ab * u[1];
  hdb[3] = hdb[3] + ab * u[2];
  hdb[4] = hdb[4] + ab * u[3];
  hdb[1] = hdb[1] + ab * ((db4 - db3) - ((u[0] + u[1]) + (u[2] + u[3])));
  bdb[0] = bdb[0] + ab * v[0];
  bdb[2] = bdb[2] + ab * v[1];
  bdb[3] = bdb[3] + ab * v[2];
  bdb[4] = bdb[4] + ab * v[3];
  bdb[1] = bdb[1] - ab * ((v[0] + v[1]) + (v[2] + v[3]));
}

// The limiter of recon_cell (Eq. modifiedhjn, xd in 1D), forward and reverse, for the edge values
// ev[v][e] of (eta, hu, h) and the cell averages v0[v][2]: from the adjoints ob of the limited
// edge state, the adjoints evb of the edge values, and the adjoints of the cell's own averages of
// eta, hu and h added to v0b[v][2]. Shared by recon_cell_rev and recon_cell_rev_lin.
SWALE_HD void limit_cell_rev(const SchemeConst& P, const real ev[3][2], const real v0[3][3], const EdgeAdj& ob,
                             real evb[3][2], real v0b[3][3]) {
  const real hb0 = v0[0][2] - v0[2][2];
  const real hbar = pos0(hb0);
  const real hL0 = ev[0][0] - ev[2][0], hR0 = ev[0][1] - ev[2][1];
  const real delta = (12.0 * hbar - hL0 - hR0) * 0.1;
  const bool selR1 = dlt(hR0, hL0);
  const real m1 = selR1 ? hR0 : hL0;
  const bool selD = dlt(delta, m1);
  const real mn = selD ? delta : m1;
  const bool epsSel = dlt(hbar, P.eps_pp);  // epsv = min(eps_pp, hbar) selects hbar
  const real epsv = epsSel ? hbar : real(P.eps_pp);
  const real mL0 = ev[1][0], mR0 = ev[1][1], mbar = v0[1][2];
  const bool active = dlt(mn, epsv);
  real theta = 1.0, iD = 0.0;
  real hL = hL0, hR = hR0, mL = mL0, mR = mR0;
  if (active) {
    iD = recip(hbar - mn);
    theta = (hbar - epsv) * iD;
    hL = theta * (hL0 - hbar) + hbar;
    hR = theta * (hR0 - hbar) + hbar;
    if (P.limit_hu) {
      mL = theta * (mL0 - mbar) + mbar;
      mR = theta * (mR0 - mbar) + mbar;
    }
  }
  const bool wetL = dlt(P.h_dry, hL), wetR = dlt(P.h_dry, hR);
  for (int v = 0; v < 3; ++v)
    for (int e = 0; e < 2; ++e) evb[v][e] = 0.0;
  real hLb = ob.hL, hRb = ob.hR, mLb = 0.0, mRb = 0.0;
  // EL = ev[0][0], BL = EL - hL (same on the right)
  evb[0][0] = ob.EL + ob.BL;
  hLb = hLb - ob.BL;
  evb[0][1] = ob.ER + ob.BR;
  hRb = hRb - ob.BR;
  // u = m / h on wet edges
  if (wetL) {
    const real iL = recip(hL);
    mLb = mLb + ob.uL * iL;
    hLb = hLb - ob.uL * mL * iL * iL;
  }
  if (wetR) {
    const real iR = recip(hR);
    mRb = mRb + ob.uR * iR;
    hRb = hRb - ob.uR * mR * iR * iR;
  }
  real hbarb = 0.0, mbarb = 0.0, hL0b, hR0b, mL0b, mR0b;
  if (active) {
    real thetab = hLb * (hL0 - hbar) + hRb * (hR0 - hbar);
    hL0b = theta * hLb;
    hR0b = theta * hRb;
    hbarb = (1.0 - theta) * (hLb + hRb);
    if (P.limit_hu) {
      thetab = thetab + mLb * (mL0 - mbar) + mRb * (mR0 - mbar);
      mL0b = theta * mLb;
      mR0b = theta * mRb;
      mbarb = (1.0 - theta) * (mLb + mRb);
    } else {
      mL0b = mLb;
      mR0b = mRb;
    }
    // theta = (hbar - epsv) / (hbar - mn)
    hbarb = hbarb + thetab * (1.0 - theta) * iD;
    const real epsvb = -thetab * iD;
    const real mnb = thetab * theta * iD;
    if (epsSel) hbarb = hbarb + epsvb;
    real deltab = 0.0;
    if (selD) deltab = mnb;
    else if (selR1) hR0b = hR0b + mnb;
    else hL0b = hL0b + mnb;
    hbarb = hbarb + 1.2 * deltab;
    hL0b = hL0b - 0.1 * deltab;
    hR0b = hR0b - 0.1 * deltab;
  } else {
    hL0b = hLb;
    hR0b = hRb;
    mL0b = mLb;
    mR0b = mRb;
  }
  evb[0][0] = evb[0][0] + hL0b;
  evb[2][0] = evb[2][0] - hL0b;
  evb[1][0] = evb[1][0] + mL0b;
  evb[0][1] = evb[0][1] + hR0b;
  evb[2][1] = evb[2][1] - hR0b;
  evb[1][1] = evb[1][1] + mR0b;
  if (!(hb0 < 0.0)) {
    v0b[0][2] = v0b[0][2] + hbarb;
    v0b[2][2] = v0b[2][2] - hbarb;
  }
  v0b[1][2] = v0b[1][2] + mbarb;
}

// Adjoint of recon_cell: from the adjoints ob of the limited edge state of cell j, the adjoints
// of the data it read: v0b[v][a] (averages of cells j-2+a) and DDb (divided differences).
//   it[3]: reciprocal sums of the triples starting at cells j-2, j-1, j (smooth-class form).
// known_smooth: the caller has established the smooth class (the FP32 test of the forward,
// which implies gamma <= 1/2 for the FP64 indicators), so they are not formed; DDb.D3 stays 0.
SWALE_HD void recon_cell_rev(const SchemeConst& P, const real h[5], const real it[3], const real v0[3][3],
                             const StencilDD& DD, real dxmax, const EdgeAdj& ob, real v0b[3][3], StencilDD& DDb,
                             bool known_smooth = false) {
  // ---------------- forward recompute (as recon_cell) ----------------
  const real h0 = h[0], h1 = h[1], h2 = h[2], h3 = h[3], h4 = h[4];
  const real dx = P.beta_dx_global ? dxmax : h2;
  const real s01 = h0 + h1, s12 = h1 + h2, s23 = h2 + h3;
  const real s012 = s01 + h2;
  real G1[2][3], G2[2][3];
  G1[0][0] = s01 + h1;
  G2[0][0] = s01 * h1;
  G1[0][1] = h1;
  G2[0][1] = -(h1 * h2);
  G1[0][2] = -h2;
  G2[0][2] = h2 * s23;
  G1[1][0] = s012 + s12;
  G2[1][0] = s12 * h2 + s012 * (h2 + s12);
  G1[1][1] = s12 + h2;
  G2[1][1] = s12 * h2;
  G1[1][2] = h2;
  G2[1][2] = -(h2 * h3);
  const real Sa = s012 + h3, Sb = Sa + h4, Sc = s12 + h3 + h4;
  const real inv = recip(Sa * Sb * Sc);
  const real iab = Sc * inv, icb = Sa * inv;
  real d[2][3];
  d[1][2] = h3 * (h3 + h4) * iab;
  d[1][0] = s12 * s012 * icb;
  d[0][2] = s23 * (s23 + h4) * iab;
  d[0][0] = h1 * s01 * icb;
  d[0][1] = 1.0 - d[0][0] - d[0][2];
  d[1][1] = 1.0 - d[1][0] - d[1][2];
  real beta[3] = {0.0, 0.0, 0.0}, tdiff = 0.0, tau = 0.0, den = 1.0;
  real F[3] = {0.0, 0.0, 0.0}, c4 = 0.0, c3 = 0.0;  // formed with the indicators
  uint8_t flag = 0;
  if (!known_smooth) {
    F[0] = 1.5 * h2 + s01 + h1;
    F[1] = 0.5 * h2 + h1;
    F[2] = -(0.5 * h2 + h3);
    c4 = 4.0 * dx * h2;
    c3 = (3.0 * h2 * h2 + 36.0 * dx * dx) * dx * h2;
    for (int r = 0; r < 3; ++r) {
      const int a = 2 - r;
      const real d2h = DD.D2[0][a] - DD.D2[2][a], d3h = DD.D3[0][a] - DD.D3[2][a];
      const real qh = d2h + d3h * F[a], qm = DD.D2[1][a] + DD.D3[1][a] * F[a];
      beta[r] = c4 * (qh * qh + qm * qm) + c3 * (d3h * d3h + DD.D3[1][a] * DD.D3[1][a]);
    }
    tdiff = beta[0] - beta[2];
    tau = dabs(tdiff);
    den = (beta[0] + beta[1] + beta[2]) * (1.0 / 3.0) + P.eps_weno;
    flag = le_nn(tau, 0.5 * den) ? 0 : (le_nn(den, tau) ? 2 : 1);
  }
  real phi[2][3], phiN[2][3], al[2][3], q[3], e[3], isE[2], Mg = 0.0;
  if (flag == 0) {
    for (int ee = 0; ee < 2; ++ee)
      for (int r = 0; r < 3; ++r) phi[ee][r] = d[ee][r];
  } else {
    e[0] = beta[0] + P.eps_weno;
    e[1] = beta[1] + P.eps_weno;
    e[2] = beta[2] + P.eps_weno;
    const real e01 = e[0] * e[1];
    const real ie = tau * recip(e01 * e[2]);
    q[0] = e[1] * e[2] * ie;
    q[1] = e[0] * e[2] * ie;
    q[2] = e01 * ie;
    real X[3];
    for (int r = 0; r < 3; ++r) X[r] = 1.0 + q[r] * q[r];
    for (int ee = 0; ee < 2; ++ee)
      for (int r = 0; r < 3; ++r) al[ee][r] = d[ee][r] * X[r];
    const real sL = al[0][0] + al[0][1] + al[0][2], sR = al[1][0] + al[1][1] + al[1][2];
    const real is = recip(sL * sR);
    isE[0] = sR * is;
    isE[1] = sL * is;
    for (int r = 0; r < 3; ++r) {
      phiN[0][r] = al[0][r] * isE[0];
      phiN[1][r] = al[1][r] * isE[1];
    }
    if (flag == 1) {
      Mg = 2.0 * (tau * recip(den)) - 1.0;
      for (int ee = 0; ee < 2; ++ee)
        for (int r = 0; r < 3; ++r) phi[ee][r] = Mg * phiN[ee][r] + (1.0 - Mg) * d[ee][r];
    } else {
      for (int ee = 0; ee < 2; ++ee)
        for (int r = 0; r < 3; ++r) phi[ee][r] = phiN[ee][r];
    }
  }
  // Edge values as the forward computes them: the smooth class through the linear form
  // v_j + sum_m K[e][m] D2[m] (linear_edge_form), the others as sum_r phi_r p_r.
  real p[3][2][3], ev[3][2], Kf[2][4];
  if (flag == 0) {
    linear_edge_form(d, G1, G2, h, it, Kf);
    for (int v = 0; v < 3; ++v)
      for (int ee = 0; ee < 2; ++ee)
        ev[v][ee] = v0[v][2] + Kf[ee][0] * DD.D2[v][0] + Kf[ee][1] * DD.D2[v][1] + Kf[ee][2] * DD.D2[v][2] +
                    Kf[ee][3] * DD.D2[v][3];
  } else {
    for (int v = 0; v < 3; ++v)
      for (int ee = 0; ee < 2; ++ee) {
        real s = 0.0;
        for (int r = 0; r < 3; ++r) {
          const int a = 2 - r;
          p[v][ee][r] = v0[v][a] + DD.D2[v][a] * G1[ee][a] + DD.D3[v][a] * G2[ee][a];
          s = s + phi[ee][r] * p[v][ee][r];
        }
        ev[v][ee] = s;
      }
  }
  // ---------------- reverse sweep ----------------
  for (int v = 0; v < 3; ++v)
    for (int a = 0; a < 3; ++a) v0b[v][a] = 0.0;
  for (int v = 0; v < 3; ++v) {
    for (int a = 0; a < 4; ++a) DDb.D2[v][a] = 0.0;
    for (int a = 0; a < 3; ++a) DDb.D3[v][a] = 0.0;
  }
  real evb[3][2];
  limit_cell_rev(P, ev, v0, ob, evb, v0b);
  if (flag == 0) {  // ev[v][e] = v0[v][2] + sum_m K[e][m] D2[v][m]; K depends on the mesh only
    for (int v = 0; v < 3; ++v)
      for (int ee = 0; ee < 2; ++ee) {
        v0b[v][2] = v0b[v][2] + evb[v][ee];
        for (int m = 0; m < 4; ++m) DDb.D2[v][m] = DDb.D2[v][m] + Kf[ee][m] * evb[v][ee];
      }
    return;
  }
  // Edge values: ev[v][e] = sum_r phi[e][r] p[v][e][r]
  real phib[2][3] = {{0, 0, 0}, {0, 0, 0}};
  for (int v = 0; v < 3; ++v)
    for (int ee = 0; ee < 2; ++ee)
      for (int r = 0; r < 3; ++r) {
        const int a = 2 - r;
        phib[ee][r] = phib[ee][r] + evb[v][ee] * p[v][ee][r];
        const real pb = evb[v][ee] * phi[ee][r];
        v0b[v][a] = v0b[v][a] + pb;
        DDb.D2[v][a] = DDb.D2[v][a] + pb * G1[ee][a];
        DDb.D3[v][a] = DDb.D3[v][a] + pb * G2[ee][a];
      }
  // Weights: phi (transition) = Mg phiN + (1 - Mg) d, Mg = 2 tau / den - 1
  real phiNb[2][3];
  real taub = 0.0, denb = 0.0;
  if (flag == 1) {
    real Mgb = 0.0;
    for (int ee = 0; ee < 2; ++ee)
      for (int r = 0; r < 3; ++r) {
        Mgb = Mgb + phib[ee][r] * (phiN[ee][r] - d[ee][r]);
        phiNb[ee][r] = Mg * phib[ee][r];
      }
    taub = taub + 2.0 * Mgb / den;
    denb = denb - 2.0 * Mgb * tau / (den * den);
  } else {
    for (int ee = 0; ee < 2; ++ee)
      for (int r = 0; r < 3; ++r) phiNb[ee][r] = phib[ee][r];
  }
  // phiN[e][r] = al[e][r] / s_e
  real Xb[3] = {0, 0, 0};
  for (int ee = 0; ee < 2; ++ee) {
    real dot = 0.0;
    for (int r = 0; r < 3; ++r) dot = dot + phiNb[ee][r] * phiN[ee][r];
    for (int r = 0; r < 3; ++r) {
      const real alb = (phiNb[ee][r] - dot) * isE[ee];
      Xb[r] = Xb[r] + alb * d[ee][r];  // al = d X
    }
  }
  real betab[3] = {0, 0, 0};
  for (int r = 0; r < 3; ++r) {
    const real qb = 2.0 * q[r] * Xb[r];  // X = 1 + q^2
    const real ier = recip(e[r]);
    taub = taub + qb * ier;              // q = tau / e_r
    betab[r] = betab[r] - qb * q[r] * ier;
  }
  for (int r = 0; r < 3; ++r) betab[r] = betab[r] + denb * (1.0 / 3.0);
  // d|x|/dx = sign(x) with sign(0) = 0, the convention of the tangent-linear model. (The reverse
  // only reaches here in the transition and non-smooth classes, where tau > 0.)
  const real sgn = (tdiff < 0.0) ? real(-1.0) : ((tdiff > 0.0) ? real(1.0) : real(0.0));
  betab[0] = betab[0] + sgn * taub;
  betab[2] = betab[2] - sgn * taub;
  for (int r = 0; r < 3; ++r) {
    const int a = 2 - r;
    const real d2h = DD.D2[0][a] - DD.D2[2][a], d3h = DD.D3[0][a] - DD.D3[2][a];
    const real qh = d2h + d3h * F[a], qm = DD.D2[1][a] + DD.D3[1][a] * F[a];
    const real qhb = 2.0 * c4 * qh * betab[r], qmb = 2.0 * c4 * qm * betab[r];
    const real d3hb = 2.0 * c3 * d3h * betab[r] + F[a] * qhb;
    const real d2hb = qhb;
    DDb.D2[1][a] = DDb.D2[1][a] + qmb;
    DDb.D3[1][a] = DDb.D3[1][a] + 2.0 * c3 * DD.D3[1][a] * betab[r] + F[a] * qmb;
    DDb.D2[0][a] = DDb.D2[0][a] + d2hb;
    DDb.D2[2][a] = DDb.D2[2][a] - d2hb;
    DDb.D3[0][a] = DDb.D3[0][a] + d3hb;
    DDb.D3[2][a] = DDb.D3[2][a] - d3hb;
  }
}

// recon_cell_rev for a cell of the smooth class whose linear form K (smooth_edge_coeffs) the
// forward recompute stored: the edge values v_j + sum_m K[e][m] D2[m] are formed from it, so the
// mesh geometry is not recomputed; the same reverse as recon_cell_rev with known_smooth.
SWALE_HD void recon_cell_rev_lin(const SchemeConst& P, const real Kf[2][4], const real v0[3][3], const StencilDD& DD,
                                 const EdgeAdj& ob, real v0b[3][3], StencilDD& DDb) {
  real ev[3][2];
  for (int v = 0; v < 3; ++v)
    for (int ee = 0; ee < 2; ++ee)
      ev[v][ee] = v0[v][2] + Kf[ee][0] * DD.D2[v][0] + Kf[ee][1] * DD.D2[v][1] + Kf[ee][2] * DD.D2[v][2] +
                  Kf[ee][3] * DD.D2[v][3];
  for (int v = 0; v < 3; ++v)
    for (int a = 0; a < 3; ++a) v0b[v][a] = 0.0;
  for (int v = 0; v < 3; ++v) {
    for (int a = 0; a < 4; ++a) DDb.D2[v][a] = 0.0;
    for (int a = 0; a < 3; ++a) DDb.D3[v][a] = 0.0;
  }
  real evb[3][2];
  limit_cell_rev(P, ev, v0, ob, evb, v0b);
  for (int v = 0; v < 3; ++v)
    for (int ee = 0; ee < 2; ++ee) {
      v0b[v][2] = v0b[v][2] + evb[v][ee];
      for (int m = 0; m < 4; ++m) DDb.D2[v][m] = DDb.D2[v][m] + Kf[ee][m] * evb[v][ee];
    }
}

}  // namespace swale
