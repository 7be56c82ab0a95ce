// Host-only count of the FP64 arithmetic that the stage kernels perform per cell, obtained by
// compiling the same per-cell code (swale_cell.cuh) with an operation-counting scalar type.
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
#include "swale_cell.cuh"

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

// Counts over cells [c0, c1) of one stage state. out[0..4]: reconstruction (add, mul, div,
// sqrt, cmp) summed over the cells; out[5..9]: right-hand side (two interface fluxes, the
// source, the flux differences) summed; out[10..14]: one interface flux (the redundant half
// of the right-hand side); out[15..17]: number of smooth / transition / non-smooth cells.
void opc_count_stage(int64_t N, const double* E, const double* M, const double* B, const double* J, int32_t bc,
                     double g, double eps_weno, double eps_pp, double h_dry, double alpha, int64_t c0, int64_t c1,
                     double* out) {
  using opc::CD;
  swale::SchemeConst P{g, eps_weno, eps_pp, h_dry, 1};
  double dxmax = 0.0;
  for (int64_t j = 0; j < N; ++j) dxmax = J[j] > dxmax ? J[j] : dxmax;
  opc::Counts rec, rhs, flux;
  long long cls[3] = {0, 0, 0};
  for (int64_t c = c0; c < c1; ++c) {
    CD Jv[5], Ev[5], Mv[5], Bv[5];
    for (int k = 0; k < 5; ++k) {
      const int64_t i = c - 2 + k, s = wrap(i, N, bc);
      Jv[k] = J[s];
      Ev[k] = E[s];
      Bv[k] = B[s];
      Mv[k] = (bc == 2 && (i < 0 || i >= N)) ? -M[s] : M[s];
    }
    swale::EdgeState o;
    uint8_t flag;
    CD wl, wr;
    uint32_t st = 0;
    opc::C = opc::Counts();
    swale::recon_cell(P, Jv, Ev, Mv, Bv, CD(dxmax), o, flag, wl, wr, st);
    rec.add += opc::C.add; rec.mul += opc::C.mul; rec.div += opc::C.div; rec.sqrt += opc::C.sqrt;
    rec.cmp += opc::C.cmp;
    cls[flag] += 1;
    // Right-hand side of the cell with its own edges standing in for the neighbours' (the
    // operation count does not depend on the values except through max/min branches).
    opc::C = opc::Counts();
    swale::rhs_cell(CD(g), CD(alpha), CD(0.01), CD(0.02), o.ER, o.BR, o.hR, o.uR, o.EL, o.ER, o.BL, o.BR, o.hL,
                    o.hR, o.uL, o.uR, o.EL, o.BL, o.hL, o.uL, Ev[1], Ev[2], Ev[3], Bv[1], Bv[2], Bv[3], Jv[1],
                    Jv[2], Jv[3]);
    rhs.add += opc::C.add; rhs.mul += opc::C.mul; rhs.div += opc::C.div; rhs.sqrt += opc::C.sqrt;
    rhs.cmp += opc::C.cmp;
    opc::C = opc::Counts();
    swale::interface_flux(CD(g), CD(alpha), CD(0.01), o.ER, o.EL, o.BR, o.BL, o.hR, o.hL, o.uR, o.uL);
    flux.add += opc::C.add; flux.mul += opc::C.mul; flux.div += opc::C.div; flux.sqrt += opc::C.sqrt;
    flux.cmp += opc::C.cmp;
  }
  take(rec, out);
  take(rhs, out + 5);
  take(flux, out + 10);
  out[15] = (double)cls[0];
  out[16] = (double)cls[1];
  out[17] = (double)cls[2];
}

}  // extern "C"
