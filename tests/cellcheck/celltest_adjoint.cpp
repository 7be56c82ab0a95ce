// Host build of the hand-written reverse sweeps (swale_adjoint.cuh) for the dot-product checks
// against the dual-number tangents of celltest_tangent.cpp. Test tooling.
#include <cmath>
#include <cstdint>

#include "swale_adjoint.cuh"

extern "C" {

// ob[8] adjoints of (EL, ER, BL, BR, hL, hR, uL, uR) -> v0b[9], D2b[12], D3b[9].
// known: 1 to take the smooth class as known (the FP32 test's shortcut), 0 to let the FP64
// detector decide.
void ct_recon_adjoint_k(const double* h, const double* v0, const double* D2, const double* D3, const double* prm,
                        const double* ob, int known, double* v0b, double* D2b, double* D3b) {
  swale::SchemeConst P{prm[0], prm[1], prm[2], prm[3], 1, (int32_t)prm[5]};
  double vv[3][3];
  swale::StencilDD DD, DDb;
  for (int v = 0; v < 3; ++v) {
    for (int a = 0; a < 3; ++a) vv[v][a] = v0[v * 3 + a];
    for (int a = 0; a < 4; ++a) DD.D2[v][a] = D2[v * 4 + a];
    for (int a = 0; a < 3; ++a) DD.D3[v][a] = D3[v * 3 + a];
  }
  swale::EdgeAdj a{ob[0], ob[1], ob[2], ob[3], ob[4], ob[5], ob[6], ob[7]};
  double vb[3][3];
  const double it3[3] = {1.0 / (h[0] + h[1] + h[2]), 1.0 / (h[1] + h[2] + h[3]), 1.0 / (h[2] + h[3] + h[4])};
  swale::recon_cell_rev(P, h, it3, vv, DD, prm[4], a, vb, DDb, known != 0);
  for (int v = 0; v < 3; ++v) {
    for (int k = 0; k < 3; ++k) v0b[v * 3 + k] = vb[v][k];
    for (int k = 0; k < 4; ++k) D2b[v * 4 + k] = DDb.D2[v][k];
    for (int k = 0; k < 3; ++k) D3b[v * 3 + k] = DDb.D3[v][k];
  }
}

void ct_recon_adjoint(const double* h, const double* v0, const double* D2, const double* D3, const double* prm,
                      const double* ob, double* v0b, double* D2b, double* D3b) {
  ct_recon_adjoint_k(h, v0, D2, D3, prm, ob, 0, v0b, D2b, D3b);
}

// recon_cell_rev_lin with the linear form K that the forward's own geometry gives (cell_geom,
// smooth_edge_coeffs, as the reconstruction kernel stores it): v0b[9], D2b[12], D3b[9].
void ct_recon_adjoint_lin(const double* h, const double* v0, const double* D2, const double* prm, const double* ob,
                          double* v0b, double* D2b, double* D3b) {
  swale::SchemeConst P{prm[0], prm[1], prm[2], prm[3], 1, (int32_t)prm[5]};
  swale::CellGeom G;
  uint32_t st = 0;
  swale::cell_geom(h, prm[4], G, st, false);
  const double it3[3] = {1.0 / (h[0] + h[1] + h[2]), 1.0 / (h[1] + h[2] + h[3]), 1.0 / (h[2] + h[3] + h[4])};
  swale::smooth_edge_coeffs(h, it3, G);
  double vv[3][3];
  swale::StencilDD DD, DDb;
  for (int v = 0; v < 3; ++v) {
    for (int a = 0; a < 3; ++a) vv[v][a] = v0[v * 3 + a];
    for (int a = 0; a < 4; ++a) DD.D2[v][a] = D2[v * 4 + a];
    for (int a = 0; a < 3; ++a) DD.D3[v][a] = 0.0;
  }
  swale::EdgeAdj a{ob[0], ob[1], ob[2], ob[3], ob[4], ob[5], ob[6], ob[7]};
  double vb[3][3];
  swale::recon_cell_rev_lin(P, G.K, vv, DD, a, vb, DDb);
  for (int v = 0; v < 3; ++v) {
    for (int k = 0; k < 3; ++k) v0b[v * 3 + k] = vb[v][k];
    for (int k = 0; k < 4; ++k) D2b[v * 4 + k] = DDb.D2[v][k];
    for (int k = 0; k < 3; ++k) D3b[v * 3 + k] = DDb.D3[v][k];
  }
}

void ct_flux_adjoint(const double* e, const double* prm, const double* Fb, double* eb) {
  swale::Flux f{Fb[0], Fb[1], Fb[2], Fb[3]};
  const swale::EdgeAdj a = swale::interface_flux_rev(prm[0], prm[1], prm[2], e[0], e[1], e[2], e[3], e[4], e[5], e[6],
                                                     e[7], f);
  const double o[8] = {a.EL, a.ER, a.BL, a.BR, a.hL, a.hR, a.uL, a.uR};
  for (int k = 0; k < 8; ++k) eb[k] = o[k];
}

// Reverse of the antisymmetric source form from the widths w3 = (J_{j-1}, J_j, J_{j+1}); out[0] =
// the source value.
void ct_source_form_adjoint(const double* hd, const double* bd, const double* w3, double g, double Sb, double* hdb,
                            double* bdb, double* out) {
  const double Jm = w3[0], Jc = w3[1], Jp = w3[2];
  const swale::SourceForm f = swale::source_form(Jm, Jc, Jp, 1.0 / Jm, 1.0 / Jc, 1.0 / Jp, 1.0 / (Jm + Jc),
                                                 1.0 / (Jc + Jp), 1.0 / (Jm + Jc + Jp));
  for (int k = 0; k < 5; ++k) hdb[k] = bdb[k] = 0.0;
  swale::source_cell_form_rev(g, hd, bd, f, Sb, hdb, bdb);
  out[0] = swale::source_cell_form(g, hd, bd, f);
}

// f32_trunc on the host (the device's double -> float conversion on the integer pipe).
float ct_f32_trunc(double x) { return swale::f32_trunc(x); }

// The device's FP32 smooth-class test and the FP64 class of the same indicators. in: w5[5] (the
// widths J_{j-2..j+2}) and dx (the indicators' length) for the mesh factors, D2h[4], D2m[4] (pair
// differences of h and hu on the pairs starting at cells j-2 .. j+1), it[3] (reciprocal triple
// sums), eps. out[0]: the FP32 test (1: surely smooth),
// out[1]: the FP64 class (second differences, shared_beta, hybrid_phi as the device forms
// them), outb[3]: the FP64 indicators.
void ct_smooth_test(const double* w5, double dx, const double* D2h, const double* D2m, const double* it, double eps,
                    int* out, double* outb) {
  float F32[3], d2h[4], d2m[4], itf[3], c4f, c3f;
  for (int a = 0; a < 4; ++a) {
    d2h[a] = swale::f32_trunc(D2h[a]);
    d2m[a] = swale::f32_trunc(D2m[a]);
  }
  for (int a = 0; a < 3; ++a) itf[a] = swale::f32_trunc(it[a]);
  swale::indicator_factors_f32(w5, dx, F32, c4f, c3f);
  out[0] = swale::sure_smooth_f32(F32, c4f, c3f, d2h, d2m, itf, swale::f32_trunc(eps)) ? 1 : 0;
  swale::CellGeom G{};
  swale::indicator_factors(w5, dx, G);
  for (int e = 0; e < 2; ++e)
    for (int r = 0; r < 3; ++r) G.d[e][r] = 1.0 / 3.0;
  swale::StencilDD DD{};
  for (int a = 0; a < 4; ++a) {
    DD.D2[2][a] = D2h[a];
    DD.D2[1][a] = D2m[a];
  }
  for (int v = 1; v < 3; ++v)
    for (int a = 0; a < 3; ++a) DD.D3[v][a] = swale::triple_dd(DD.D2[v][a], DD.D2[v][a + 1], it[a]);
  double beta[3], phi[2][3];
  swale::shared_beta(G, DD, beta);
  swale::SchemeConst P{9.812, eps, 1e-11, 1e-6, 1, 0};
  out[1] = swale::hybrid_phi(P, beta, G.d, phi);
  for (int r = 0; r < 3; ++r) outb[r] = beta[r];
}

// The non-well-balanced scheme's per-field FP32 smooth tests and the FP64 classes of the same
// fields, formed as the device forms them. in: proj[4] = a11, a12, a21, a22; D2e[4], D2m[4],
// D2h[4] (pair differences of eta, hu, h), it[3], w5[5], dx, eps. out[0..2]: FP32 tests of
// the two characteristic fields and the bottom, out[3..5]: their FP64 classes, gam[3]: their
// FP64 gamma.
void ct_smooth1_test(const double* proj, const double* D2e, const double* D2m, const double* D2h, const double* it,
                     const double* w5, double dx, double eps, int* out, double* gam) {
  float F32[3], itf[3], fd[3][4], fm[3][4], c4f, c3f;
  for (int a = 0; a < 3; ++a) itf[a] = swale::f32_trunc(it[a]);
  swale::indicator_factors_f32(w5, dx, F32, c4f, c3f);
  swale::CellGeom G{};
  swale::indicator_factors(w5, dx, G);
  const double* F = G.F;
  const double c4 = G.c4, c3 = G.c3;
  const float a11 = swale::f32_trunc(proj[0]), a12 = swale::f32_trunc(proj[1]);
  const float a21 = swale::f32_trunc(proj[2]), a22 = swale::f32_trunc(proj[3]);
  for (int a = 0; a < 4; ++a) {
    const float e2 = swale::f32_trunc(D2e[a]), m2 = swale::f32_trunc(D2m[a]), h2 = swale::f32_trunc(D2h[a]);
    fd[0][a] = std::fma(a11, e2, a12 * m2);
    fm[0][a] = std::fma(std::fabs(a11), std::fabs(e2), std::fabs(a12) * std::fabs(m2));
    fd[1][a] = std::fma(a21, e2, a22 * m2);
    fm[1][a] = std::fma(std::fabs(a21), std::fabs(e2), std::fabs(a22) * std::fabs(m2));
    fd[2][a] = e2 - h2;
    fm[2][a] = std::fabs(e2) + std::fabs(h2);
  }
  for (int f = 0; f < 3; ++f)
    out[f] = swale::sure_smooth1_f32(F32, c4f, c3f, fd[f], fm[f], itf, swale::f32_trunc(eps)) ? 1 : 0;
  // FP64 as recon_cell_nonwb_g forms it
  double D2[3][4], D3[3][3], fD2[3][4], fD3[3][3];
  for (int a = 0; a < 4; ++a) {
    D2[0][a] = D2e[a];
    D2[1][a] = D2m[a];
    D2[2][a] = D2h[a];
  }
  for (int v = 0; v < 3; ++v)
    for (int a = 0; a < 3; ++a) D3[v][a] = swale::triple_dd(D2[v][a], D2[v][a + 1], it[a]);
  for (int a = 0; a < 4; ++a) {
    fD2[0][a] = proj[0] * D2[0][a] + proj[1] * D2[1][a];
    fD2[1][a] = proj[2] * D2[0][a] + proj[3] * D2[1][a];
    fD2[2][a] = D2[0][a] - D2[2][a];
  }
  for (int a = 0; a < 3; ++a) {
    fD3[0][a] = proj[0] * D3[0][a] + proj[1] * D3[1][a];
    fD3[1][a] = proj[2] * D3[0][a] + proj[3] * D3[1][a];
    fD3[2][a] = D3[0][a] - D3[2][a];
  }
  swale::SchemeConst P{9.812, eps, 1e-11, 1e-6, 1, 0};
  double d[2][3];
  for (int e = 0; e < 2; ++e)
    for (int r = 0; r < 3; ++r) d[e][r] = 1.0 / 3.0;
  for (int f = 0; f < 3; ++f) {
    double beta[3], phi[2][3];
    for (int r = 0; r < 3; ++r) {
      const int a = 2 - r;
      const double q = fD2[f][a] + fD3[f][a] * F[a];
      beta[r] = c4 * (q * q) + c3 * (fD3[f][a] * fD3[f][a]);
    }
    out[3 + f] = swale::hybrid_phi(P, beta, d, phi);
    gam[f] = std::fabs(beta[0] - beta[2]) / ((beta[0] + beta[1] + beta[2]) / 3.0 + eps);
  }
}

}  // extern "C"
