// Host-only count of the FP64 arithmetic that the stage kernels perform per cell, obtained by
// compiling the same per-cell code (swale_cell.cuh, and the reverse sweeps of swale_adjoint.cuh)
// with an operation-counting scalar type.
// Additions/subtractions, multiplications, divisions and square roots are counted
// separately (a fused multiply-add on the device is one multiplication plus one addition
// here); comparisons, min/max and sign flips are counted apart (they do not use the FP64
// pipe on the target). Used to state the algorithmic FLOPs per cell of the roofline.
#include <cmath>
#include <cstdint>

namespace opc {
struct Counts {
  long long add = 0, mul = 0, div = 0, sqrt = 0, cmp = 0;
};
static Counts C;
struct CD {
  double v;
  CD(double x = 0.0) : v(x) {}
};
inline CD operator+(CD a, CD b) { ++C.add; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { ++C.add; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { ++C.mul; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { ++C.div; return CD(a.v / b.v); }
inline CD operator-(CD a) { return CD(-a.v); }
inline CD& operator+=(CD& a, CD b) { a = a + b; return a; }
inline bool operator<(CD a, CD b) { ++C.cmp; return a.v < b.v; }
inline bool operator>(CD a, CD b) { ++C.cmp; return a.v > b.v; }
inline bool operator<=(CD a, CD b) { ++C.cmp; return a.v <= b.v; }
inline bool operator>=(CD a, CD b) { ++C.cmp; return a.v >= b.v; }
inline bool operator==(CD a, CD b) { ++C.cmp; return a.v == b.v; }
inline CD swale_sqrt(CD a) { ++C.sqrt; return CD(std::sqrt(a.v)); }
}  // namespace opc

#define SWALE_REAL opc::CD
#include "swale_adjoint.cuh"

namespace {
int64_t wrap(int64_t i, int64_t N, int bc) {
  if (bc == 0) return ((i % N) + N) % N;
  if (i < 0) return -1 - i;
  if (i >= N) return 2 * N - 1 - i;
  return i;
}
void take(opc::Counts& into, double* out) {
  out[0] = (double)into.add;
  out[1] = (double)into.mul;
  out[2] = (double)into.div;
  out[3] = (double)into.sqrt;
  out[4] = (double)into.cmp;
}
}  // namespace

extern "C" {

// Counts over cells [c0, c1) of one stage state. out[0..4]: reconstruction per cell summed
// (add, mul, div, sqrt, cmp): the pair and triple terms a cell owns plus recon_cell;
// out[5..9]: update per cell summed: one interface flux, the cell's reciprocal width, the
// source geometry and source, the flux differences (the RK combination is added in Python);
// out[10..14]: one interface flux alone; out[15..17]: smooth / transition / non-smooth cells;
// out[18]: FLOPs of the mesh-only geometry (cell_geom) summed; out[19]: FLOPs of the source
// term's mesh-only values (source_form, or source_geom for the special scheme, and the cell's
// reciprocal width) summed.
void opc_count_stage(int64_t N, const double* E, const double* M, const double* B, const double* J, int32_t bc,
                     double g, double eps_weno, double eps_pp, double h_dry, double alpha, int64_t c0, int64_t c1,
                     double* out, int32_t scheme) {
  using opc::CD;
  swale::SchemeConst P{g, eps_weno, eps_pp, h_dry, 1, 0};
  double dxmax = 0.0;
  for (int64_t j = 0; j < N; ++j) dxmax = J[j] > dxmax ? J[j] : dxmax;
  opc::Counts rec, upd, flux;
  long long cls[3] = {0, 0, 0};
  double geom_flops = 0.0, sgeom_flops = 0.0;
  auto add_to = [](opc::Counts& a) {
    a.add += opc::C.add; a.mul += opc::C.mul; a.div += opc::C.div; a.sqrt += opc::C.sqrt; a.cmp += opc::C.cmp;
  };
  for (int64_t c = c0; c < c1; ++c) {
    CD Jv[7], V[3][7];  // cells c-3 .. c+3
    for (int k = 0; k < 7; ++k) {
      const int64_t i = c - 3 + k, s = wrap(i, N, bc);
      Jv[k] = J[s];
      V[0][k] = E[s];
      V[1][k] = (bc == 2 && (i < 0 || i >= N)) ? -M[s] : M[s];
      V[2][k] = B[s];
    }
    // Divided differences of the stencil (uncounted: each pair / triple is counted once below).
    swale::StencilDD DD;
    CD ip[6], d2[3][6], it[5];
    for (int m = 0; m < 6; ++m) {
      ip[m] = CD(1.0 / (Jv[m].v + Jv[m + 1].v));
      for (int v = 0; v < 3; ++v) d2[v][m] = CD((V[v][m + 1].v - V[v][m].v) * ip[m].v);
    }
    for (int m = 0; m < 5; ++m) it[m] = CD(1.0 / (Jv[m].v + Jv[m + 1].v + Jv[m + 2].v));
    for (int v = 0; v < 3; ++v) {
      for (int a = 0; a < 4; ++a) DD.D2[v][a] = d2[v][a + 1];
      for (int a = 0; a < 3; ++a) DD.D3[v][a] = CD((d2[v][a + 2].v - d2[v][a + 1].v) * it[a + 1].v);
    }
    // The kernels reconstruct the depth h = eta - b in place of b (uncounted input mapping).
    for (int a = 0; a < 4; ++a) DD.D2[2][a] = CD(DD.D2[0][a].v - DD.D2[2][a].v);
    for (int a = 0; a < 3; ++a) DD.D3[2][a] = CD(DD.D3[0][a].v - DD.D3[2][a].v);
    // The work one cell owns: its pair (c, c+1) and its triple, counted with the kernel's code.
    opc::C = opc::Counts();
    const CD ipc = swale::pair_recip(Jv[3], Jv[4]);
    for (int v = 0; v < 3; ++v) (void)swale::pair_dd(V[v][3], V[v][4], ipc);
    const CD itc = swale::triple_recip(Jv[2], Jv[3], Jv[4]);
    for (int v = 0; v < 3; ++v) (void)swale::triple_dd(d2[v][2], d2[v][3], itc);
    CD h5[5], v0[3][3];
    for (int k = 0; k < 5; ++k) h5[k] = Jv[k + 1];
    for (int v = 0; v < 3; ++v)
      for (int a = 0; a < 3; ++a) v0[v][a] = V[v][a + 1];
    for (int a = 0; a < 3; ++a) v0[2][a] = CD(V[0][a + 1].v - V[2][a + 1].v);
    swale::EdgeState o;
    uint8_t flag;
    uint32_t st = 0;
    CD etaG[2];
    const CD it3[3] = {it[1], it[2], it[3]};  // triples starting at cells c-2, c-1, c
    if (scheme == 1) swale::recon_cell_nonwb(P, h5, v0, DD, CD(dxmax), o, flag, st);
    else if (scheme == 2) swale::recon_cell_special(P, h5, v0, DD, CD(dxmax), o, flag, st, etaG);
    else swale::recon_cell(P, h5, it3, v0, DD, CD(dxmax), o, flag, st);
    add_to(rec);
    cls[flag] += 1;
    // The mesh-only part (cell_geom), which a stage on the mesh of the previous stage 2 reuses.
    opc::C = opc::Counts();
    {
      swale::CellGeom Gm;
      uint32_t sg = 0;
      swale::cell_geom(h5, CD(dxmax), Gm, sg);
      if (scheme == 0) swale::smooth_edge_coeffs(h5, it3, Gm);
    }
    geom_flops += (double)(opc::C.add + opc::C.mul + opc::C.div + opc::C.sqrt);
    // Update: one flux (the cell's right interface, with its own edges standing in for the
    // neighbour's), its reciprocal width, the source and the flux differences.
    opc::C = opc::Counts();
    const swale::Flux F =
        scheme != 0 ? swale::interface_flux_plain(CD(g), CD(alpha), CD(0.01), o.ER, o.EL, o.BR, o.BL, o.hR, o.hL,
                                                  o.uR, o.uL)
                    : swale::interface_flux(CD(g), CD(alpha), CD(0.01), o.ER, o.EL, o.BR, o.BL, o.hR, o.hL, o.uR, o.uL);
    const long long f0 = opc::C.add + opc::C.mul + opc::C.div + opc::C.sqrt;
    const CD iJc = CD(1.0) / Jv[3];
    swale::SourceGeom sg;
    swale::SourceForm sf;
    if (scheme == 2)
      sg = swale::source_geom(Jv[2], Jv[3], CD(1.0 / Jv[2].v), iJc, CD(1.0 / Jv[4].v), ip[2], ip[3], it[2]);
    else
      sf = swale::source_form(Jv[2], Jv[3], Jv[4], CD(1.0 / Jv[2].v), iJc, CD(1.0 / Jv[4].v), ip[2], ip[3], it[2]);
    sgeom_flops += (double)(opc::C.add + opc::C.mul + opc::C.div + opc::C.sqrt - f0);
    const CD hd[5] = {V[0][2] - V[2][2], V[0][3] - V[2][3], V[0][4] - V[2][4], o.hL, o.hR};
    const CD bd[5] = {V[2][2], V[2][3], V[2][4], o.BL, o.BR};
    CD Sj;
    if (scheme == 2) {
      const CD eta4[4] = {o.EL, etaG[0], etaG[1], o.ER};
      Sj = swale::source_cell_special(CD(g), V[0][3], eta4, bd, sg, o.BL, o.BR);
    } else {
      Sj = swale::source_cell_form(CD(g), hd, bd, sf);
    }
    (void)swale::cell_rhs(F, F, Sj);
    add_to(upd);
    // The three depth averages above are formed once per cell in the kernel: remove the two
    // extra subtractions counted for the neighbours.
    upd.add -= 2;
    opc::C = opc::Counts();
    (void)swale::interface_flux(CD(g), CD(alpha), CD(0.01), o.ER, o.EL, o.BR, o.BL, o.hR, o.hL, o.uR, o.uL);
    add_to(flux);
  }
  take(rec, out);
  take(upd, out + 5);
  take(flux, out + 10);
  out[15] = (double)cls[0];
  out[16] = (double)cls[1];
  out[17] = (double)cls[2];
  out[18] = geom_flops;
  out[19] = sgeom_flops;
}

// Counts of the reverse sweep of one stage over cells [c0, c1) of one stage state (the same
// stencils as opc_count_stage), with unit adjoint seeds. out[0]: reverse reconstruction per
// cell (recon_cell_rev_lin for a smooth-class cell, from the linear form the forward recompute
// stored, else recon_cell_rev; the cell's own pair and triple terms recomputed, and the scatter of the
// divided-difference adjoints to the five stencil cells); out[1]: reverse source per cell
// (the depth data and source_cell_form_rev on the stored form entries); out[2]:
// reverse flux per interface (interface_flux_rev). FLOPs: add + mul + div + sqrt, summed.
void opc_count_reverse(int64_t N, const double* E, const double* M, const double* B, const double* J, int32_t bc,
                       double g, double eps_weno, double eps_pp, double h_dry, double alpha, int64_t c0, int64_t c1,
                       double* out) {
  using opc::CD;
  swale::SchemeConst P{g, eps_weno, eps_pp, h_dry, 1, 0};
  double dxmax = 0.0;
  for (int64_t j = 0; j < N; ++j) dxmax = J[j] > dxmax ? J[j] : dxmax;
  auto flops = []() { return (double)(opc::C.add + opc::C.mul + opc::C.div + opc::C.sqrt); };
  double rrec = 0.0, rsrc = 0.0, rflux = 0.0;
  for (int64_t c = c0; c < c1; ++c) {
    CD Jv[7], V[3][7];
    for (int k = 0; k < 7; ++k) {
      const int64_t i = c - 3 + k, s = wrap(i, N, bc);
      Jv[k] = J[s];
      V[0][k] = E[s];
      V[1][k] = (bc == 2 && (i < 0 || i >= N)) ? -M[s] : M[s];
      V[2][k] = B[s];
    }
    swale::StencilDD DD;
    CD ip[6], d2[3][6], it[5];
    for (int m = 0; m < 6; ++m) {
      ip[m] = CD(1.0 / (Jv[m].v + Jv[m + 1].v));
      for (int v = 0; v < 3; ++v) d2[v][m] = CD((V[v][m + 1].v - V[v][m].v) * ip[m].v);
    }
    for (int m = 0; m < 5; ++m) it[m] = CD(1.0 / (Jv[m].v + Jv[m + 1].v + Jv[m + 2].v));
    for (int v = 0; v < 3; ++v) {
      for (int a = 0; a < 4; ++a) DD.D2[v][a] = d2[v][a + 1];
      for (int a = 0; a < 3; ++a) DD.D3[v][a] = CD((d2[v][a + 2].v - d2[v][a + 1].v) * it[a + 1].v);
    }
    CD h5[5], v0[3][3];
    for (int k = 0; k < 5; ++k) h5[k] = Jv[k + 1];
    for (int v = 0; v < 3; ++v)
      for (int a = 0; a < 3; ++a) v0[v][a] = V[v][a + 1];
    swale::EdgeState o;
    uint8_t flag;
    uint32_t st = 0;
    const CD it3[3] = {it[1], it[2], it[3]};
    swale::recon_cell(P, h5, it3, v0, DD, CD(dxmax), o, flag, st);
    // The smooth class's linear form as the forward recompute stores it (not counted here).
    swale::CellGeom Gk;
    uint32_t stk = 0;
    swale::cell_geom(h5, CD(dxmax), Gk, stk, false);
    swale::smooth_edge_coeffs(h5, it3, Gk);
    // Reverse reconstruction.
    opc::C = opc::Counts();
    const CD ipc = swale::pair_recip(Jv[3], Jv[4]);
    for (int v = 0; v < 3; ++v) (void)swale::pair_dd(V[v][3], V[v][4], ipc);
    const CD itc = swale::triple_recip(Jv[2], Jv[3], Jv[4]);
    if (flag != 0)  // the third differences only where the class is open
      for (int v = 0; v < 3; ++v) (void)swale::triple_dd(d2[v][2], d2[v][3], itc);
    const swale::EdgeAdj ob = {CD(1.0), CD(1.0), CD(1.0), CD(1.0), CD(1.0), CD(1.0), CD(1.0), CD(1.0)};
    CD v0b[3][3];
    swale::StencilDD DDb;
    // A smooth-class cell reverses from the stored linear form (the kernel's path where its FP32
    // test shows the class), the others recompute the geometry and the weights.
    if (flag == 0) swale::recon_cell_rev_lin(P, Gk.K, v0, DD, ob, v0b, DDb);
    else swale::recon_cell_rev(P, h5, it3, v0, DD, CD(dxmax), ob, v0b, DDb);
    for (int v = 0; v < 3; ++v) {  // the kernel's scatter through D3 = (D2' - D2) it, D2 = (v' - v) ip
      CD cv[5], d2b[4];
      for (int a = 0; a < 4; ++a) d2b[a] = DDb.D2[v][a];
      for (int a = 0; a < 3 && flag != 0; ++a) {  // DDb.D3 is 0 in the smooth class
        const CD x = DDb.D3[v][a] * it[a + 1];
        d2b[a + 1] = d2b[a + 1] + x;
        d2b[a] = d2b[a] - x;
      }
      for (int a = 0; a < 4; ++a) {
        const CD x = d2b[a] * ip[a + 1];
        cv[a + 1] = cv[a + 1] + x;
        cv[a] = cv[a] - x;
      }
    }
    rrec += flops();
    // Reverse source, from the form entries the forward recompute stored (not counted here).
    const swale::SourceForm sf = swale::source_form(Jv[2], Jv[3], Jv[4], CD(1.0 / Jv[2].v), CD(1.0 / Jv[3].v),
                                                    CD(1.0 / Jv[4].v), ip[2], ip[3], it[2]);
    opc::C = opc::Counts();
    const CD hd[5] = {V[0][2].v - V[2][2].v, V[0][3] - V[2][3], V[0][4].v - V[2][4].v, o.hL, o.hR};
    const CD bd[5] = {V[2][2], V[2][3], V[2][4], o.BL, o.BR};
    CD hdb[5] = {}, bdb[5] = {};
    swale::source_cell_form_rev(CD(g), hd, bd, sf, CD(1.0), hdb, bdb);
    rsrc += flops();
    // Reverse flux.
    opc::C = opc::Counts();
    const swale::Flux Fb = {CD(1.0), CD(1.0), CD(1.0), CD(1.0)};
    (void)swale::interface_flux_rev(CD(g), CD(alpha), CD(0.01), o.ER, o.EL, o.BR, o.BL, o.hR, o.hL, o.uR, o.uL, Fb);
    rflux += flops();
  }
  const double n = (double)(c1 - c0);
  out[0] = rrec / n;
  out[1] = rsrc / n;
  out[2] = rflux / n;
}

}  // extern "C"
