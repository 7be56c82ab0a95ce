// Host build of the per-cell arithmetic on a forward-mode dual scalar: tangents of
// recon_cell, interface_flux and source_cell_form for the dot-product checks of their hand-written
// reverse sweeps (swale_adjoint.cuh). Test tooling.
#include <cmath>
#include <cstdint>

namespace dt {
struct D {
  double v, d;
  D(double a = 0.0) : v(a), d(0.0) {}
  D(double a, double b) : v(a), d(b) {}
};
inline D operator+(D a, D b) { return D(a.v + b.v, a.d + b.d); }
inline D operator-(D a, D b) { return D(a.v - b.v, a.d - b.d); }
inline D operator-(D a) { return D(-a.v, -a.d); }
inline D operator*(D a, D b) { return D(a.v * b.v, a.d * b.v + a.v * b.d); }
inline D operator/(D a, D b) {
  const double q = a.v / b.v;
  return D(q, (a.d - q * b.d) / b.v);
}
inline D& operator+=(D& a, D b) { a = a + b; return a; }
inline bool operator<(D a, D b) { return a.v < b.v; }
inline bool operator>(D a, D b) { return a.v > b.v; }
inline bool operator<=(D a, D b) { return a.v <= b.v; }
inline bool operator>=(D a, D b) { return a.v >= b.v; }
inline bool operator==(D a, D b) { return a.v == b.v; }
inline D swale_sqrt(D a) {
  const double s = std::sqrt(a.v);
  return D(s, s > 0 ? a.d / (2.0 * s) : 0.0);
}
}  // namespace dt

#define SWALE_REAL dt::D
#include "swale_cell.cuh"

using dt::D;

extern "C" {

// The two forms of a smooth-class edge value for one variable on widths h[5] and averages v[5]
// (divided differences formed from them): out = {sum over sub-stencils with the linear
// weights at the left / right edge, cell average + linear form at the left / right edge}.
void ct_edge_forms(const double* h, const double* v, double* out) {
  D hh[5], D2[4], D3[3], v0[3];
  for (int k = 0; k < 5; ++k) hh[k] = D(h[k]);
  for (int a = 0; a < 4; ++a) D2[a] = (D(v[a + 1]) - D(v[a])) * (D(1.0) / (hh[a] + hh[a + 1]));
  D it[3];
  for (int a = 0; a < 3; ++a) {
    it[a] = D(1.0) / (hh[a] + hh[a + 1] + hh[a + 2]);
    D3[a] = (D2[a + 1] - D2[a]) * it[a];
    v0[a] = D(v[a]);
  }
  swale::CellGeom G;
  uint32_t st = 0;
  swale::cell_geom(hh, hh[2], G, st);
  swale::smooth_edge_coeffs(hh, it, G);
  for (int e = 0; e < 2; ++e) {
    out[e] = swale::edge_value(G, G.d, v0, D2, D3, e).v;
    out[2 + e] = (v0[2] + G.K[e][0] * D2[0] + G.K[e][1] * D2[1] + G.K[e][2] * D2[2] + G.K[e][3] * D2[3]).v;
  }
}

// in: h[5], v0[9], D2[12], D3[9]; tangents tv0[9], tD2[12], tD3[9];
// prm = {g, eps, eps_pp, h_dry, dxmax, limit_hu}.
// out: edge state values [8] and tangents [8] (EL, ER, BL, BR, hL, hR, uL, uR), flag.
int ct_recon_tangent(const double* h, const double* v0, const double* D2, const double* D3, const double* tv0,
                     const double* tD2, const double* tD3, const double* prm, double* val, double* tan) {
  swale::SchemeConst P{prm[0], prm[1], prm[2], prm[3], 1, (int32_t)prm[5]};
  D hh[5], vv[3][3];
  swale::StencilDD DD;
  for (int k = 0; k < 5; ++k) hh[k] = D(h[k]);
  for (int v = 0; v < 3; ++v) {
    for (int a = 0; a < 3; ++a) vv[v][a] = D(v0[v * 3 + a], tv0[v * 3 + a]);
    for (int a = 0; a < 4; ++a) DD.D2[v][a] = D(D2[v * 4 + a], tD2[v * 4 + a]);
    for (int a = 0; a < 3; ++a) DD.D3[v][a] = D(D3[v * 3 + a], tD3[v * 3 + a]);
  }
  // recon_cell reconstructs the depth h = eta - b in place of b: map the third variable.
  for (int a = 0; a < 3; ++a) vv[2][a] = vv[0][a] - vv[2][a];
  for (int a = 0; a < 4; ++a) DD.D2[2][a] = DD.D2[0][a] - DD.D2[2][a];
  for (int a = 0; a < 3; ++a) DD.D3[2][a] = DD.D3[0][a] - DD.D3[2][a];
  swale::EdgeState o;
  uint8_t flag;
  uint32_t st = 0;
  const D it3[3] = {D(1.0 / (h[0] + h[1] + h[2])), D(1.0 / (h[1] + h[2] + h[3])), D(1.0 / (h[2] + h[3] + h[4]))};
  swale::recon_cell(P, hh, it3, vv, DD, D(prm[4]), o, flag, st);
  const D outs[8] = {o.EL, o.ER, o.BL, o.BR, o.hL, o.hR, o.uL, o.uR};
  for (int k = 0; k < 8; ++k) {
    val[k] = outs[k].v;
    tan[k] = outs[k].d;
  }
  return flag;
}

// in: e[8] = (EL, ER, BL, BR, hL, hR, uL, uR), te[8]; prm = {g, alpha, w}. out: F[4], tF[4].
void ct_flux_tangent(const double* e, const double* te, const double* prm, double* F, double* tF) {
  D x[8];
  for (int k = 0; k < 8; ++k) x[k] = D(e[k], te[k]);
  const swale::Flux f = swale::interface_flux(D(prm[0]), D(prm[1]), D(prm[2]), x[0], x[1], x[2], x[3], x[4], x[5],
                                              x[6], x[7]);
  const D o[4] = {f.FE, f.FMm, f.FMp, f.FB};
  for (int k = 0; k < 4; ++k) {
    F[k] = o[k].v;
    tF[k] = o[k].d;
  }
}

// The source term as the antisymmetric form (source_form, source_cell_form) from the widths
// w3 = (J_{j-1}, J_j, J_{j+1}). out: S, tS (tangent).
void ct_source_form_tangent(const double* hd, const double* bd, const double* thd, const double* tbd, const double* w3,
                            double g, double* S, double* tS) {
  D a[5], b[5];
  for (int k = 0; k < 5; ++k) {
    a[k] = D(hd[k], thd[k]);
    b[k] = D(bd[k], tbd[k]);
  }
  const double Jm = w3[0], Jc = w3[1], Jp = w3[2];
  const swale::SourceForm f = swale::source_form(D(Jm), D(Jc), D(Jp), D(1.0 / Jm), D(1.0 / Jc), D(1.0 / Jp),
                                                 D(1.0 / (Jm + Jc)), D(1.0 / (Jc + Jp)), D(1.0 / (Jm + Jc + Jp)));
  const D s = swale::source_cell_form(D(g), a, b, f);
  *S = s.v;
  *tS = s.d;
}

}  // extern "C"
