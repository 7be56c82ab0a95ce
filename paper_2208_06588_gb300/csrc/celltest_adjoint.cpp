// Host build of the hand-written reverse sweeps (swale_adjoint.cuh) for the dot-product checks
// against the dual-number tangents of celltest_tangent.cpp. Test tooling.
#include <cmath>
#include <cstdint>

#include "swale_adjoint.cuh"

extern "C" {

// ob[8] adjoints of (EL, ER, BL, BR, hL, hR, uL, uR) -> v0b[9], D2b[12], D3b[9].
void ct_recon_adjoint(const double* h, const double* v0, const double* D2, const double* D3, const double* prm,
                      const double* ob, double* v0b, double* D2b, double* D3b) {
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
  swale::recon_cell_rev(P, h, it3, vv, DD, prm[4], a, vb, DDb);
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

void ct_source_adjoint(const double* hd, const double* bd, const double* geom, double g, double Sb, double* hdb,
                       double* bdb) {
  swale::SourceGeom sg{geom[0], geom[1], geom[2], geom[3], geom[4], geom[5]};
  for (int k = 0; k < 5; ++k) hdb[k] = bdb[k] = 0.0;
  swale::source_cell_rev(g, hd, bd, sg, Sb, hdb, bdb);
}

// f32_trunc on the host (the device's double -> float conversion on the integer pipe).
float ct_f32_trunc(double x) { return swale::f32_trunc(x); }

// The device's FP32 smooth-class test and the FP64 class of the same indicators. in: F[3], c4,
// c3 (mesh factors), D2h[3], D3h[3], D2m[3], D3m[3] (divided differences of h and hu on the
// sub-stencils starting at cells j-2 .. j), eps. out[0]: the FP32 test (1: surely smooth),
// out[1]: the FP64 class (shared_beta + hybrid_phi), outb[3]: the FP64 indicators.
void ct_smooth_test(const double* F, double c4, double c3, const double* D2h, const double* D3h, const double* D2m,
                    const double* D3m, double eps, int* out, double* outb) {
  float F32[3], d2h[3], d3h[3], d2m[3], d3m[3];
  for (int a = 0; a < 3; ++a) {
    F32[a] = swale::f32_trunc(F[a]);
    d2h[a] = swale::f32_trunc(D2h[a]);
    d3h[a] = swale::f32_trunc(D3h[a]);
    d2m[a] = swale::f32_trunc(D2m[a]);
    d3m[a] = swale::f32_trunc(D3m[a]);
  }
  out[0] = swale::sure_smooth_f32(F32, swale::f32_trunc(c4), swale::f32_trunc(c3), d2h, d3h, d2m, d3m,
                                  swale::f32_trunc(eps)) ? 1 : 0;
  swale::CellGeom G{};
  for (int a = 0; a < 3; ++a) G.F[a] = F[a];
  G.c4 = c4;
  G.c3 = c3;
  for (int e = 0; e < 2; ++e)
    for (int r = 0; r < 3; ++r) G.d[e][r] = 1.0 / 3.0;
  swale::StencilDD DD{};
  for (int a = 0; a < 3; ++a) {
    DD.D2[2][a] = D2h[a];
    DD.D3[2][a] = D3h[a];
    DD.D2[1][a] = D2m[a];
    DD.D3[1][a] = D3m[a];
  }
  double beta[3], phi[2][3];
  swale::shared_beta(G, DD, beta);
  swale::SchemeConst P{9.812, eps, 1e-11, 1e-6, 1, 0};
  out[1] = swale::hybrid_phi(P, beta, G.d, phi);
  for (int r = 0; r < 3; ++r) outb[r] = beta[r];
}

}  // extern "C"
