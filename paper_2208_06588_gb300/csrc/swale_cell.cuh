// Per-cell and per-interface arithmetic of one stage of the well-balanced ALE-WENO hybrid
// scheme (Zhang, Xia & Xu, arXiv 2208.06588), shared by the device kernels and by the host
// operation counter.
//
// Formulation (the paper's definitions, arranged for few FP64 operations; GB300 runs FP64 at
// 1/42 of its FP32 rate and a division costs about nine FMA slots):
//  * Step 1 of Sec. 2.2: each sub-stencil quadratic p_r is the derivative of the cubic that
//    interpolates the primitive function, in Newton form. Its coefficients are the divided
//    differences D2 (pairs of cells) and D3 (triples of cells) of the cell averages; these and
//    their reciprocal widths are computed once per pair / triple and shared by the cells that
//    use them. The linear weights d_r at the two edges have closed forms in the node offsets
//    y0..y5 of the big stencil (obtained by matching the coefficients of the outermost
//    averages of the big-stencil quartic and of p_2 / p_0), e.g. at x_{j+1/2}:
//      d_2 = (y4-y3)(y5-y3) / ((y4-y0)(y5-y0)),  d_0 = (y3-y1)(y3-y0) / ((y5-y1)(y5-y0)).
//  * Step 2: beta_r = Dx int (p_r')^2 + Dx^3 int (p_r'')^2 in closed form about the cell
//    midpoint; the classes come from comparing tau with (beta^A + eps) and (beta^A + eps)/2.
//    On the device the smooth class is first tested in FP32 with an error bound
//    (sure_smooth_f32); the FP64 indicators are formed where that test cannot decide.
//  * Step 3: reciprocals of products stand in for several divisions (one division each).
//  * Sec. 4.1 source: the quartic interpolants (three averages + two edge values) are the
//    derivative of a confluent Newton (Hermite) form of their primitive, brought to monomial
//    form; the integral of the depth times the bottom slope is then taken exactly (the
//    four-point Gauss-Legendre rule of the definition is exact for that degree too).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

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
  int32_t limit_hu;  // 1: the limiter's theta also scales hu about its mean (reading O6b)
};


// Status bits accumulated on the device.
enum : uint32_t {
  ST_EWEIGHT = 1u,    // a linear weight d_r <= 0
  ST_NEGDEPTH = 2u,   // a cell-average depth below -eps_pp entered a stage (warning)
  ST_NONFINITE = 4u,  // a non-finite value appeared
  ST_EMESH = 8u,      // a cell width <= 0
  ST_NODT = 16u,      // no finite time step (zero wave speed, no mesh motion, no end time): dt = 0
  ST_TIMEOUT = 32u,   // a bounded wait for an asynchronous copy gave up (the stage was abandoned)
};

// Limited edge state of one cell (edge L = x_{j-1/2}^+, edge R = x_{j+1/2}^-).
struct EdgeState {
  real EL, ER, BL, BR, hL, hR, uL, uR;
};

// ------------------------------------------------------------------------------------
// Scalar helpers. A GB300 SM retires about two FP64 lanes per clock against 64 INT32 and
// 128 FP32 lanes, and comparisons, min / max and divisions of doubles all occupy the FP64
// pipe. On the device (double, no counting type) these helpers therefore compare IEEE bit
// patterns on the integer pipe (an order-preserving key: the bits, with the magnitude bits
// flipped for negative values) and form reciprocals from the hardware's 20-bit reciprocal
// approximation refined by one third-order step of the Newton-Raphson family for 1/x
// (Householder's order-3 iteration: with e = 1 - x y the exact reciprocal is y / (1 - e) =
// y (1 + e + e^2 + ...), and the step keeps the series to e^2, y <- y (1 + e + e^2), so the
// relative error goes from e to e^3). With e below 2^-20 that leaves the final rounding: within
// one unit in the last place of the correctly rounded 1 / x (swale_check_recip exposes it for
// that test; 3 FMAs instead of a full division). Zero, infinite and
// subnormal arguments give NaN there; no caller passes them on valid data. Elsewhere they are
// the plain operators. Ties of min / max return the first argument.
// ------------------------------------------------------------------------------------
#if defined(__CUDA_ARCH__) && !defined(SWALE_REAL)
#define SWALE_INT_COMPARE 1
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
SWALE_HD double dmax(double a, double b) { return okey(b) > okey(a) ? b : a; }
SWALE_HD double dmin(double a, double b) { return okey(b) < okey(a) ? b : a; }
SWALE_HD bool dlt(double a, double b) { return okey(a) < okey(b); }
// max(a, 0) (a negative zero gives +0).
SWALE_HD double pos0(double a) { return __double_as_longlong(a) < 0 ? 0.0 : a; }
// a > 0.
SWALE_HD bool gt0(double a) { return __double_as_longlong(a) > 0; }
// a <= b for a, b >= +0.
SWALE_HD bool le_nn(double a, double b) {
  return (unsigned long long)__double_as_longlong(a) <= (unsigned long long)__double_as_longlong(b);
}
// NaN, infinite or of magnitude above 1e300.
SWALE_HD bool bad(double a) {
  return ((unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull) > 0x7e37e43c8800759cull;
}
SWALE_HD double dabs(double a) { return fabs(a); }
SWALE_HD double recip(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(fma(e, e, e), y, y);
}
SWALE_HD double dsqrt(double a) { return sqrt(a); }
#else
SWALE_HD real dmax(real a, real b) { return (b > a) ? b : a; }
SWALE_HD real dmin(real a, real b) { return (b < a) ? b : a; }
SWALE_HD bool dlt(real a, real b) { return a < b; }
SWALE_HD real pos0(real a) { return (real(0.0) > a) ? real(0.0) : a; }
SWALE_HD bool gt0(real a) { return a > 0.0; }
SWALE_HD bool le_nn(real a, real b) { return a <= b; }
SWALE_HD real dabs(real a) { return a < 0.0 ? -a : a; }
SWALE_HD bool bad(real a) { return !(a == a) || dabs(a) > 1.0e300; }
SWALE_HD real recip(real x) { return 1.0 / x; }
#ifdef SWALE_REAL
SWALE_HD real dsqrt(real a) { return swale_sqrt(a); }
#else
SWALE_HD real dsqrt(real a) { return sqrt(a); }
#endif
#endif

// Double to float on the integer pipe: the top 23 mantissa bits (rounded toward zero, relative
// error below 2^-23), magnitudes below the normal float range to a signed zero, above it (and
// infinities, NaNs) to a signed infinity. The hardware conversion instruction runs on the FP64
// pipe of GB300 at the DFMA rate (measured), which is the bottleneck of the stage kernels.
SWALE_HD float f32_trunc(double x) {
#if defined(__CUDA_ARCH__)
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
#endif
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // the float's biased exponent (1023 - 127 = 896)
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned mag = e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : (((unsigned)e << 23) | mant));
  const unsigned r = sign | mag;
#if defined(__CUDA_ARCH__)
  return __uint_as_float(r);
#else
  float f;
  memcpy(&f, &r, 4);
  return f;
#endif
}

// The indicator factors of indicator_factors in FP32 from the widths h[5] and the length dx
// (truncated to FP32): every term of F[0], F[1], -F[2], c4 and c3 is positive, so they come out
// within 6 u (F), 8 u (c4) and 12 u (c3) of their values.
SWALE_HD void indicator_factors_f32(const double h[5], double dx, float F[3], float& c4, float& c3) {
  const float h0 = f32_trunc(h[0]), h1 = f32_trunc(h[1]), h2 = f32_trunc(h[2]), h3 = f32_trunc(h[3]);
  const float d = f32_trunc(dx);
  F[0] = fmaf(1.5f, h2, (h0 + h1) + h1);
  F[1] = fmaf(0.5f, h2, h1);
  F[2] = -fmaf(0.5f, h2, h3);
  c4 = (4.0f * d) * h2;
  c3 = (fmaf(3.0f * h2, h2, 36.0f * d * d) * d) * h2;
}

// ------------------------------------------------------------------------------------
// The smooth class decided in FP32 (Step 2 with the shared indicators of Eq. alphamodified).
// GB300 runs FP32 at about 40x its FP64 rate, and in most cells the detector only has to tell
// that gamma is far below 1/2. The indicators beta_r = c4 (qh^2 + qm^2) + c3 (D3h^2 + D3m^2),
// q = D2 + D3 F, are evaluated in FP32 from FP32 copies of the pair differences D2 (top 23 bits,
// f32_trunc), second differences formed from them in FP32, D3 = (D2_right - D2_left) it, and
// FP32 copies of the mesh factors, beside the magnitudes
//   m_r = c4 (Qh^2 + Qm^2) + c3 (Mh^2 + Mm^2),  Q = |D2| + M |F|,  M = (|D2_left| + |D2_right|) it.
// A rounding-error analysis of these few operations (pair differences and triple reciprocals
// within 2^-23 relative, F within 6 u, c4 within 8 u and c3 within 12 u when they are formed in
// FP32 from such widths, FMAs, the second differences within 6 u M, sums of non-negative terms)
// bounds |beta_r(FP32) - beta_r| by 43 u m_r, u = 2^-24; E below takes 96 u (m_0 + m_1 + m_2),
// which also covers the rounding of the FP64 indicators (below 2^-48 m) and of the sum m itself,
// plus a 1e-30 floor for inputs below the FP32 range. If
//   tau32 + E <= (den32 - E) / 2,   tau = |beta_0 - beta_2|, den = mean(beta) + eps,
// (with 8 u of relative slack on tau32 and den32, and eps rounded down) then the FP64 detector
// finds gamma <= 1/2 as well, and the cell is smooth. Overflow or NaN make the test false, as
// does anything closer to the threshold: the FP64 indicators then decide, as before.
//   d2h[4], d2m[4]  pair differences of h and hu on the pairs starting at cells j-2 .. j+1
//   it[3]           reciprocal sums of the triples starting at cells j-2 .. j
// ------------------------------------------------------------------------------------
SWALE_HD bool sure_smooth_f32(const float F[3], float c4, float c3, const float d2h[4], const float d2m[4],
                              const float it[3], float eps) {
  float b[3], msum = 0.0f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int a = 2 - r;
    const float d3h = (d2h[a + 1] - d2h[a]) * it[a], d3m = (d2m[a + 1] - d2m[a]) * it[a];
    const float Mh = (fabsf(d2h[a + 1]) + fabsf(d2h[a])) * it[a], Mm = (fabsf(d2m[a + 1]) + fabsf(d2m[a])) * it[a];
    const float qh = fmaf(d3h, F[a], d2h[a]), qm = fmaf(d3m, F[a], d2m[a]);
    const float Qh = fmaf(Mh, fabsf(F[a]), fabsf(d2h[a])), Qm = fmaf(Mm, fabsf(F[a]), fabsf(d2m[a]));
    b[r] = fmaf(c4, fmaf(qh, qh, qm * qm), c3 * fmaf(d3h, d3h, d3m * d3m));
    msum += fmaf(c4, fmaf(Qh, Qh, Qm * Qm), c3 * fmaf(Mh, Mh, Mm * Mm));
  }
  constexpr float u = 5.9604645e-8f;  // 2^-24
  const float tau = fabsf(b[0] - b[2]);
  const float den = (b[0] + b[1] + b[2]) * (1.0f / 3.0f) + eps;
  const float E = (96.0f * u) * msum + 1e-30f;
  return tau * (1.0f + 8.0f * u) + E <= 0.5f * (den * (1.0f - 8.0f * u) - E);
}

// The same test for one field on its own (the non-well-balanced scheme's characteristic fields
// and bottom, Sec. 2.2 last paragraph): beta_r = c4 q^2 + c3 D3^2 of the field's pair
// differences d2[4], given in FP32 with magnitudes mag[4] that bound them together with their
// error (the fields are combinations of the stencil's differences: |error| <= 6 u mag). The
// analysis of sure_smooth_f32 carries over with Q = mag + M |F|, M = (mag_left + mag_right) it;
// the bound stays within 96 u (m_0 + m_1 + m_2).
SWALE_HD bool sure_smooth1_f32(const float F[3], float c4, float c3, const float d2[4], const float mag[4],
                               const float it[3], float eps) {
  float b[3], msum = 0.0f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int a = 2 - r;
    const float d3 = (d2[a + 1] - d2[a]) * it[a];
    const float M = (mag[a + 1] + mag[a]) * it[a];
    const float q = fmaf(d3, F[a], d2[a]);
    const float Q = fmaf(M, fabsf(F[a]), mag[a]);
    b[r] = fmaf(c4, q * q, c3 * (d3 * d3));
    msum += fmaf(c4, Q * Q, c3 * (M * M));
  }
  constexpr float u = 5.9604645e-8f;  // 2^-24
  const float tau = fabsf(b[0] - b[2]);
  const float den = (b[0] + b[1] + b[2]) * (1.0f / 3.0f) + eps;
  const float E = (96.0f * u) * msum + 1e-30f;
  return tau * (1.0f + 8.0f * u) + E <= 0.5f * (den * (1.0f - 8.0f * u) - E);
}

// Wave speed |u| + sqrt(g max(h, 0)) of one limited edge state (Eq. alpha2D).
SWALE_HD real wave_speed(real g, real h, real u) { return dabs(u) + dsqrt(g * pos0(h)); }

// ------------------------------------------------------------------------------------
// Shared per-pair and per-triple terms (Step 1): reciprocal widths and divided differences.
// ------------------------------------------------------------------------------------
// Pair of cells (m, m+1): 1 / (J_m + J_{m+1}).
SWALE_HD real pair_recip(real Jm, real Jp) { return recip(Jm + Jp); }
// D2 of one variable on the pair.
SWALE_HD real pair_dd(real vm, real vp, real ip) { return (vp - vm) * ip; }
// Triple centred at c: 1 / (J_{c-1} + J_c + J_{c+1}).
SWALE_HD real triple_recip(real Jm, real Jc, real Jp) { return recip(Jm + Jc + Jp); }
// D3 of one variable on the triple from the D2 of its two pairs.
SWALE_HD real triple_dd(real d2l, real d2r, real it) { return (d2r - d2l) * it; }

// Divided differences of the big stencil of cell j for the three variables (eta, hu, h), h =
// eta - b the depth:
// D2[v][a], a = 0..3 the pairs (j-2,j-1)..(j+1,j+2); D3[v][a], a = 0..2 the triples
// starting at j-2, j-1, j.
struct StencilDD {
  real D2[3][4];
  real D3[3][3];
};

// Mesh-only data of cell j (Step 1): Newton-form factors of the sub-stencil quadratics at the
// two edges, the linear weights d_r there, and the factors of the smoothness indicators.
//   h[5]  widths J_{j-2..j+2};  dx  the cell length in the indicators (Step 1)
struct CellGeom {
  real G1[2][3], G2[2][3], d[2][3], F[3], c3, c4;
  real iab, icb;  // 1 / ((y4 - y0)(y5 - y0)), 1 / ((y5 - y1)(y5 - y0))
  // Edge value with the linear weights as the cell average plus a combination of the stencil's
  // first divided differences: v(edge e) = v_j + sum_m K[e][m] D2[m] (smooth_edge_coeffs; the
  // hydrostatic scheme only).
  real K[2][4];
};
#define SWALE_GEOM_BASE 25    // doubles of a CellGeom before K (what every scheme uses)
#define SWALE_GEOM_VALUES 33  // doubles in a CellGeom
// cached per cell: a CellGeom and the source's six mesh-only values (a SourceForm; a SourceGeom
// for the special scheme)
#define SWALE_GEO_ARRAYS (SWALE_GEOM_VALUES + 6)
// Indicator factors of Step 2 (F, c4, c3 of CellGeom) for the widths h[5] and the length dx.
SWALE_HD void indicator_factors(const real h[5], real dx, CellGeom& G) {
  const real h1 = h[1], h2 = h[2], h3 = h[3];
  G.F[0] = 1.5 * h2 + (h[0] + h1) + h1;
  G.F[1] = 0.5 * h2 + h1;
  G.F[2] = -(0.5 * h2 + h3);
  G.c4 = 4.0 * dx * h2;
  G.c3 = (3.0 * h2 * h2 + 36.0 * dx * dx) * dx * h2;
}
// Geometry of the cell; with indicators = false the indicator factors are left out (the device
// forms them in FP32 for its smooth-class test and in FP64 only where that test cannot decide).
SWALE_HD void cell_geom(const real h[5], real dx, CellGeom& G, uint32_t& st, bool indicators = true) {
  const real h0 = h[0], h1 = h[1], h2 = h[2], h3 = h[3], h4 = h[4];
  if (!gt0(h2)) st |= ST_EMESH;
  // Node offsets relative to x_{j-1/2}: y0 = -(h0+h1), y1 = -h1, y2 = 0, y3 = h2,
  // y4 = h2+h3, y5 = h2+h3+h4. Newton-form factors of p_r at the left (x = 0) and right
  // (x = h2) edges: G1 = (x-y_a) + (x-y_{a+1}), G2 = sum of pairwise products of
  // (x-y_a), (x-y_{a+1}), (x-y_{a+2}); sub-stencil r starts at cell a = 2 - r.
  const real s01 = h0 + h1, s12 = h1 + h2, s23 = h2 + h3;
  const real s012 = s01 + h2;
  G.G1[0][0] = s01 + h1;
  G.G2[0][0] = s01 * h1;
  G.G1[0][1] = h1;
  G.G2[0][1] = -(h1 * h2);
  G.G1[0][2] = -h2;
  G.G2[0][2] = h2 * s23;
  G.G1[1][0] = s012 + s12;
  G.G2[1][0] = s12 * h2 + s012 * (h2 + s12);
  G.G1[1][1] = s12 + h2;
  G.G2[1][1] = s12 * h2;
  G.G1[1][2] = h2;
  G.G2[1][2] = -(h2 * h3);
  // Linear weights (closed forms), one division for the four outer weights.
  const real Sa = s012 + h3;         // y4 - y0
  const real Sb = Sa + h4;           // y5 - y0
  const real Sc = s12 + h3 + h4;     // y5 - y1
  const real inv = recip(Sa * Sb * Sc);
  const real iab = Sc * inv, icb = Sa * inv;  // 1/(Sa Sb), 1/(Sc Sb)
  G.iab = iab;
  G.icb = icb;
  G.d[1][2] = h3 * (h3 + h4) * iab;
  G.d[1][0] = s12 * s012 * icb;
  G.d[0][2] = s23 * (s23 + h4) * iab;
  G.d[0][0] = h1 * s01 * icb;
  G.d[0][1] = 1.0 - G.d[0][0] - G.d[0][2];
  G.d[1][1] = 1.0 - G.d[1][0] - G.d[1][2];
  if (!gt0(G.d[0][1]) || !gt0(G.d[1][1])) st |= ST_EWEIGHT;
  // Indicator factors: F[a] = 1.5 h2 - (y_a+y_{a+1}+y_{a+2}); beta = c4 q^2 + c3 D3^2 per variable.
  if (indicators) indicator_factors(h, dx, G);
  for (int e = 0; e < 2; ++e)
    for (int m = 0; m < 4; ++m) G.K[e][m] = real(0.0);
}

// Step 4 with the linear weights d_r (the smooth class) in one linear form. With w_a = d_{2-a}
// the weight of the sub-stencil that starts at cell a and D3[a] = (D2[a+1] - D2[a]) it[a],
//   sum_a w_a (v0[a] + D2[a] G1[a] + D3[a] G2[a]) = sum_a w_a v0[a] + sum_m g_m D2[m],
//   g_m = w_m G1[m] + b_{m-1} - b_m,  b_a = w_a G2[a] it[a]  (terms outside a = 0..2 absent),
// and, as the weights sum to one and v0[2] - v0[1] = D2[1] (h1 + h2),
// v0[2] - v0[0] = D2[1] (h1 + h2) + D2[0] (h0 + h1), sum_a w_a v0[a] = v0[2] - w_0 (h0 + h1) D2[0]
// - (w_0 + w_1) (h1 + h2) D2[1]. So v(edge) = v_j + sum_m K[m] D2[m] with
//   K[0] = g_0 - w_0 (h0 + h1),  K[1] = g_1 - (w_0 + w_1) (h1 + h2),  K[2] = g_2,  K[3] = g_3:
// equal to edge_value with phi = d in exact arithmetic, exact for constant data, and four FMAs
// per variable and edge instead of nine.
//   h[5] the widths, it[3] the reciprocal triple sums of the triples starting at cells j-2..j.
SWALE_HD void linear_edge_form(const real d[2][3], const real G1[2][3], const real G2[2][3], const real h[5],
                               const real it[3], real K[2][4]) {
  const real s01 = h[0] + h[1], s12 = h[1] + h[2];
  for (int e = 0; e < 2; ++e) {
    real w[3], b[3], g[4];
    for (int a = 0; a < 3; ++a) {
      w[a] = d[e][2 - a];
      b[a] = w[a] * G2[e][a] * it[a];
    }
    g[0] = w[0] * G1[e][0] - b[0];
    g[1] = w[1] * G1[e][1] + b[0] - b[1];
    g[2] = w[2] * G1[e][2] + b[1] - b[2];
    g[3] = b[2];
    K[e][0] = g[0] - w[0] * s01;
    K[e][1] = g[1] - (w[0] + w[1]) * s12;
    K[e][2] = g[2];
    K[e][3] = g[3];
  }
}
SWALE_HD void smooth_edge_coeffs(const real h[5], const real it[3], CellGeom& G) {
  linear_edge_form(G.d, G.G1, G.G2, h, it, G.K);
}

// Steps 2-3 from the indicators beta[3]: the class (smooth if gamma <= 1/2, non-smooth if
// gamma >= 1, gamma = tau / (beta^A + eps)) and the hybrid weights phi[e][r] at both edges
// (linear / WENO-Z / blend with M = 2 gamma - 1).
SWALE_HD uint8_t hybrid_phi(const SchemeConst& P, const real beta[3], const real d[2][3], real phi[2][3]) {
  const real tau = dabs(beta[0] - beta[2]);
  const real den = (beta[0] + beta[1] + beta[2]) * (1.0 / 3.0) + P.eps_weno;  // beta^A + eps
  const uint8_t flag = le_nn(tau, 0.5 * den) ? 0 : (le_nn(den, tau) ? 2 : 1);
  if (flag == 0) {
    for (int e = 0; e < 2; ++e)
      for (int r = 0; r < 3; ++r) phi[e][r] = d[e][r];
  } else {
    // WENO-Z: alpha_r = d_r (1 + (tau / (beta_r + eps))^2), normalised per edge.
    const real e0 = beta[0] + P.eps_weno, e1 = beta[1] + P.eps_weno, e2 = beta[2] + P.eps_weno;
    const real e01 = e0 * e1;
    const real ie = tau * recip(e01 * e2);
    const real q[3] = {e1 * e2 * ie, e0 * e2 * ie, e01 * ie};
    real X[3];
    for (int r = 0; r < 3; ++r) X[r] = 1.0 + q[r] * q[r];
    real al[2][3];
    for (int e = 0; e < 2; ++e)
      for (int r = 0; r < 3; ++r) al[e][r] = d[e][r] * X[r];
    const real sL = al[0][0] + al[0][1] + al[0][2], sR = al[1][0] + al[1][1] + al[1][2];
    const real is = recip(sL * sR);
    const real isL = sR * is, isR = sL * is;
    for (int r = 0; r < 3; ++r) {
      phi[0][r] = al[0][r] * isL;
      phi[1][r] = al[1][r] * isR;
    }
    if (flag == 1) {
      const real Mg = 2.0 * (tau * recip(den)) - 1.0;
      for (int e = 0; e < 2; ++e)
        for (int r = 0; r < 3; ++r) phi[e][r] = Mg * phi[e][r] + (1.0 - Mg) * d[e][r];
    }
  }
  return flag;
}

// Step 4 for one variable: sum_r phi_r p_r at edge e, p_r in Newton form from the average v0[a]
// and the divided differences D2[a], D3[a] of its sub-stencil (a = 2 - r).
SWALE_HD real edge_value(const CellGeom& G, const real phi[2][3], const real v0[3], const real D2[4], const real D3[3],
                         int e) {
  real s = 0.0;
  for (int r = 0; r < 3; ++r) {
    const int a = 2 - r;
    s += phi[e][r] * (v0[a] + D2[a] * G.G1[e][a] + D3[a] * G.G2[e][a]);
  }
  return s;
}

// Limiter on h = eta - b with the Gauss-Lobatto mean delta (Eq. modifiedhjn, xd in 1D; hu scaled
// by the same theta only if P.limit_hu), b re-derived as eta - h (Remark in Sec. 4.3), velocities.
//   ev[v][e]  edge values of (eta, hu, h);  hbar0, mbar  the cell's depth and discharge means
SWALE_HD void limit_cell(const SchemeConst& P, const real ev[3][2], real hbar0, real mbar, EdgeState& o,
                         uint32_t& st) {
  real hbar = hbar0;
  if (dlt(hbar, -P.eps_pp)) st |= ST_NEGDEPTH;
  hbar = pos0(hbar);
  real hL = ev[2][0], hR = ev[2][1];
  const real delta = (12.0 * hbar - hL - hR) * 0.1;
  const real mn = dmin(dmin(hL, hR), delta);
  const real epsv = dmin(P.eps_pp, hbar);
  real mL = ev[1][0], mR = ev[1][1];
  if (dlt(mn, epsv)) {
    const real theta = (hbar - epsv) * recip(hbar - mn);
    hL = theta * (hL - hbar) + hbar;
    hR = theta * (hR - hbar) + hbar;
    if (P.limit_hu) {
      mL = theta * (mL - mbar) + mbar;
      mR = theta * (mR - mbar) + mbar;
    }
  }
  o.EL = ev[0][0];
  o.ER = ev[0][1];
  o.hL = hL;
  o.hR = hR;
  o.BL = ev[0][0] - hL;
  o.BR = ev[0][1] - hR;
  // Velocities with one division: u_L = m_L h_R' / (h_L' h_R'), dry edges (h <= h_dry) -> 0.
  const bool wetL = dlt(P.h_dry, hL), wetR = dlt(P.h_dry, hR);
  const real hLs = wetL ? hL : real(1.0), hRs = wetR ? hR : real(1.0);
  const real ihh = recip(hLs * hRs);
  o.uL = wetL ? mL * hRs * ihh : real(0.0);
  o.uR = wetR ? mR * hLs * ihh : real(0.0);
  // NaN propagates into the comparisons as false: catch it explicitly.
  if (bad(o.EL) || bad(o.ER) || bad(hL) || bad(hR) || bad(mL) || bad(mR)) st |= ST_NONFINITE;
}

// Reconstruction of cell j (Steps 1-4 of Sec. 2.2 with the shared indicators of
// Eq. alphamodified), bound-preserving limiter (Eq. modifiedhjn in 1D with the 4-point
// Gauss-Lobatto rule) and the bottom re-derivation of the Remark in Sec. 4.3.
//   h[5]      widths J_{j-2..j+2};   v0[v][a] averages of (eta, hu, h) on cells j-2+a, a = 0..2
//   DD        shared divided differences;   dxmax  the global cell length (Step 1)
// The depth h = eta - b is reconstructed in place of b (the same shared weights, so the edge
// values of b = eta - h are those of reconstructing b; Sec. 4.1 items 1-2).
// Outputs the limited edge state and the class (wave speeds: wave_speed on the edge state).
// Only the cell's own width is checked (every cell checks its own).
// Indicators of h = eta - b and hu, summed (the shared indicators of Eq. alphamodified).
SWALE_HD void shared_beta(const CellGeom& G, const StencilDD& DD, real beta[3]) {
  for (int r = 0; r < 3; ++r) {
    const int a = 2 - r;
    const real d2h = DD.D2[2][a], d3h = DD.D3[2][a];
    const real qh = d2h + d3h * G.F[a], qm = DD.D2[1][a] + DD.D3[1][a] * G.F[a];
    beta[r] = G.c4 * (qh * qh + qm * qm) + G.c3 * (d3h * d3h + DD.D3[1][a] * DD.D3[1][a]);
  }
}

// known_smooth: the caller has established the smooth class already (the device's FP32 test,
// which implies gamma <= 1/2 for the FP64 indicators), so they are not formed.
SWALE_HD void recon_cell_g(const SchemeConst& P, const CellGeom& G, const real v0[3][3], const StencilDD& DD,
                           EdgeState& o, uint8_t& flag, uint32_t& st, bool known_smooth = false) {
  real phi[2][3];
  if (known_smooth) {
    flag = 0;
  } else {
    real beta[3];
    shared_beta(G, DD, beta);
    flag = hybrid_phi(P, beta, G.d, phi);
  }
  // Edge values of eta, hu, h with the shared weights (Step 4); the smooth class through the
  // linear form of smooth_edge_coeffs.
  real ev[3][2];
  if (flag == 0) {
    for (int v = 0; v < 3; ++v)
      for (int e = 0; e < 2; ++e)
        ev[v][e] = v0[v][2] + G.K[e][0] * DD.D2[v][0] + G.K[e][1] * DD.D2[v][1] + G.K[e][2] * DD.D2[v][2] +
                   G.K[e][3] * DD.D2[v][3];
  } else {
    for (int v = 0; v < 3; ++v)
      for (int e = 0; e < 2; ++e) ev[v][e] = edge_value(G, phi, v0[v], DD.D2[v], DD.D3[v], e);
  }
  limit_cell(P, ev, v0[2][2], v0[1][2], o, st);
}
//   it[3]  reciprocal sums of the triples starting at cells j-2, j-1, j
SWALE_HD void recon_cell(const SchemeConst& P, const real h[5], const real it[3], const real v0[3][3],
                         const StencilDD& DD, real dxmax, EdgeState& o, uint8_t& flag, uint32_t& st) {
  CellGeom G;
  cell_geom(h, P.beta_dx_global ? dxmax : h[2], G, st);
  smooth_edge_coeffs(h, it, G);
  recon_cell_g(P, G, v0, DD, o, flag, st);
}

// Reconstruction of cell j for the non-well-balanced scheme (Eq. se2D / s2D; Sec. 2.2, last
// paragraph: local characteristic decomposition). The eigenvectors of d f / d (eta, hu) =
// [[0, 1], [c^2 - u^2, 2u]] at the cell's average state (u = hu / h, c = sqrt(g h)),
// R = [[1, 1], [u - c, u + c]], project the stencil data (averages and, being linear maps of
// them, the divided differences) onto two characteristic fields; each field and the bottom get
// their own indicators, class and weights; the edge values are mapped back with R. A dry cell
// (h <= h_dry) reconstructs eta and hu themselves. The class is the largest of the three.
// Rows of R^-1 = 1/(2c) [[u + c, -1], [-(u - c), 1]] at the cell's average state (identity when
// the cell is dry), with u and c.
struct NonwbProj {
  real a11, a12, a21, a22, u, c;
  bool wet;
};
SWALE_HD NonwbProj nonwb_proj(const SchemeConst& P, const real v0[3][3]) {
  NonwbProj pr{real(1.0), real(0.0), real(0.0), real(1.0), real(0.0), real(0.0), false};
  const real hb = v0[2][2];
  pr.wet = dlt(P.h_dry, hb);
  if (pr.wet) {
    pr.u = v0[1][2] * recip(hb);
    pr.c = dsqrt(P.g * hb);
    const real i2c = 0.5 * recip(pr.c);
    pr.a11 = (pr.u + pr.c) * i2c;
    pr.a12 = -i2c;
    pr.a21 = (pr.c - pr.u) * i2c;
    pr.a22 = i2c;
  }
  return pr;
}

//   known_smooth[3] (may be null): fields whose smooth class the caller has established (the
//   device's FP32 test, which implies it for the FP64 indicators); their indicators are not formed.
SWALE_HD void recon_cell_nonwb_g(const SchemeConst& P, const CellGeom& G, const real v0[3][3], const StencilDD& DD,
                                 EdgeState& o, uint8_t& flag, uint32_t& st, const NonwbProj& pr,
                                 const bool* known_smooth = nullptr) {
  const real hb = v0[2][2];
  const bool wet = pr.wet;
  const real a11 = pr.a11, a12 = pr.a12, a21 = pr.a21, a22 = pr.a22, u = pr.u, c = pr.c;
  real fv0[3][3], fD2[3][4], fD3[3][3];
  // Third field: the bottom b = eta - h.
  for (int a = 0; a < 3; ++a) {
    fv0[0][a] = a11 * v0[0][a] + a12 * v0[1][a];
    fv0[1][a] = a21 * v0[0][a] + a22 * v0[1][a];
    fv0[2][a] = v0[0][a] - v0[2][a];
    fD3[0][a] = a11 * DD.D3[0][a] + a12 * DD.D3[1][a];
    fD3[1][a] = a21 * DD.D3[0][a] + a22 * DD.D3[1][a];
    fD3[2][a] = DD.D3[0][a] - DD.D3[2][a];
  }
  for (int a = 0; a < 4; ++a) {
    fD2[0][a] = a11 * DD.D2[0][a] + a12 * DD.D2[1][a];
    fD2[1][a] = a21 * DD.D2[0][a] + a22 * DD.D2[1][a];
    fD2[2][a] = DD.D2[0][a] - DD.D2[2][a];
  }
  real fe[3][2];
  flag = 0;
  for (int f = 0; f < 3; ++f) {
    real phi[2][3];
    uint8_t fl = 0;
    if (known_smooth && known_smooth[f]) {
      for (int e = 0; e < 2; ++e)
        for (int r = 0; r < 3; ++r) phi[e][r] = G.d[e][r];
    } else {
      real beta[3];
      for (int r = 0; r < 3; ++r) {
        const int a = 2 - r;
        const real q = fD2[f][a] + fD3[f][a] * G.F[a];
        beta[r] = G.c4 * (q * q) + G.c3 * (fD3[f][a] * fD3[f][a]);
      }
      fl = hybrid_phi(P, beta, G.d, phi);
    }
    flag = fl > flag ? fl : flag;
    for (int e = 0; e < 2; ++e) fe[f][e] = edge_value(G, phi, fv0[f], fD2[f], fD3[f], e);
  }
  real ev[3][2];
  for (int e = 0; e < 2; ++e) {
    if (wet) {
      ev[0][e] = fe[0][e] + fe[1][e];
      ev[1][e] = (u - c) * fe[0][e] + (u + c) * fe[1][e];
    } else {
      ev[0][e] = fe[0][e];
      ev[1][e] = fe[1][e];
    }
    ev[2][e] = ev[0][e] - fe[2][e];  // depth = eta - b
  }
  limit_cell(P, ev, hb, v0[1][2], o, st);
}
SWALE_HD void recon_cell_nonwb(const SchemeConst& P, const real h[5], const real v0[3][3], const StencilDD& DD,
                               real dxmax, EdgeState& o, uint8_t& flag, uint32_t& st) {
  CellGeom G;
  cell_geom(h, P.beta_dx_global ? dxmax : h[2], G, st);
  recon_cell_nonwb_g(P, G, v0, DD, o, flag, st, nonwb_proj(P, v0));
}

// Hybrid weights at an interior point (Step 3) with linear weights d(x), which may be
// negative there; then the WENO-Z part uses the split of Shi, Hu & Shu cited in Sec. 2.2:
// d = s+ d+ - s- d- with d~+ = (d + 3|d|) / 2, d~- = d~+ - d, s+- = sum d~+-, d+- = d~+- / s+-,
// each group normalised on its own with the same indicators, phi^N = s+ w+ - s- w-.
SWALE_HD void point_phi(const SchemeConst& P, const real d[3], const real beta[3], uint8_t flag, real phi[3]) {
  if (flag == 0) {
    for (int r = 0; r < 3; ++r) phi[r] = d[r];
    return;
  }
  const real tau = dabs(beta[0] - beta[2]);
  real X[3];
  for (int r = 0; r < 3; ++r) {
    const real q = tau * recip(beta[r] + P.eps_weno);
    X[r] = 1.0 + q * q;
  }
  real pn[3];
  if (gt0(d[0]) && gt0(d[1]) && gt0(d[2])) {
    const real a0 = d[0] * X[0], a1 = d[1] * X[1], a2 = d[2] * X[2];
    const real is = recip(a0 + a1 + a2);
    pn[0] = a0 * is;
    pn[1] = a1 * is;
    pn[2] = a2 * is;
  } else {
    real dp[3], dm[3];
    for (int r = 0; r < 3; ++r) {
      dp[r] = 0.5 * (d[r] + 3.0 * dabs(d[r]));
      dm[r] = dp[r] - d[r];
    }
    const real sp = dp[0] + dp[1] + dp[2], sm = dm[0] + dm[1] + dm[2];
    real ap[3], am[3];
    for (int r = 0; r < 3; ++r) {
      ap[r] = dp[r] * X[r];
      am[r] = dm[r] * X[r];
    }
    // s+ (ap / sum ap) with ap from the unnormalised d~+ (the normalisation cancels).
    const real ip = sp * recip(ap[0] + ap[1] + ap[2]), im = sm * recip(am[0] + am[1] + am[2]);
    for (int r = 0; r < 3; ++r) pn[r] = ap[r] * ip - am[r] * im;
  }
  if (flag == 1) {
    const real den = (beta[0] + beta[1] + beta[2]) * (1.0 / 3.0) + P.eps_weno;
    const real Mg = 2.0 * (tau * recip(den)) - 1.0;
    for (int r = 0; r < 3; ++r) phi[r] = Mg * pn[r] + (1.0 - Mg) * d[r];
  } else {
    for (int r = 0; r < 3; ++r) phi[r] = pn[r];
  }
}

// Interior 4-point Gauss-Lobatto points of the unit cell, (1 -+ 1/sqrt 5) / 2.
#define SWALE_GLO_T1 0.27639320225002103036
#define SWALE_GLO_T2 0.72360679774997896964

// Reconstruction for the special source-term scheme (Sec. 4.2): that of recon_cell plus eta at
// the two interior Gauss-Lobatto points (Eq. gausssij2) with the cell's shared indicators and
// class. At a point at offset x from x_{j-1/2} the Newton factors are G1 = dx_a + dx_{a+1},
// G2 = dx_a dx_{a+1} + (dx_a + dx_{a+1}) dx_{a+2} with dx_k = x - y_k, and the outer linear
// weights follow from the Lagrange bases of the primitive:
//   d_2 = (dx_4 dx_5 + (dx_4 + dx_5) R_0) / ((y4-y0)(y5-y0)), R_0 = dx1 dx2 dx3 / (dx2 dx3 + dx1 dx3 + dx1 dx2),
//   d_0 = (dx_0 dx_1 + (dx_0 + dx_1) R_5) / ((y5-y1)(y5-y0)), R_5 = dx2 dx3 dx4 / (dx3 dx4 + dx2 dx4 + dx2 dx3),
//   d_1 = 1 - d_0 - d_2 (at x = y3 they reduce to the edge weights).
SWALE_HD void recon_cell_special_g(const SchemeConst& P, const CellGeom& G, const real h[5], const real v0[3][3],
                                   const StencilDD& DD, EdgeState& o, uint8_t& flag, uint32_t& st, real etaG[2],
                                   bool known_smooth = false) {
  real beta[3] = {real(0.0), real(0.0), real(0.0)};
  real phi[2][3];
  if (known_smooth) {  // the smooth class established by the caller (see recon_cell_g)
    flag = 0;
    for (int e = 0; e < 2; ++e)
      for (int r = 0; r < 3; ++r) phi[e][r] = G.d[e][r];
  } else {
    shared_beta(G, DD, beta);
    flag = hybrid_phi(P, beta, G.d, phi);
  }
  real ev[3][2];
  for (int v = 0; v < 3; ++v)
    for (int e = 0; e < 2; ++e) ev[v][e] = edge_value(G, phi, v0[v], DD.D2[v], DD.D3[v], e);
  limit_cell(P, ev, v0[2][2], v0[1][2], o, st);
  const real h0 = h[0], h1 = h[1], h2 = h[2], h3 = h[3], h4 = h[4];
  const real y[6] = {-(h0 + h1), -h1, real(0.0), h2, h2 + h3, h2 + h3 + h4};
  for (int q = 0; q < 2; ++q) {
    const real x = (q == 0 ? SWALE_GLO_T1 : SWALE_GLO_T2) * h2;
    real dx[6];
    for (int k = 0; k < 6; ++k) dx[k] = x - y[k];
    const real p123 = dx[1] * dx[2] * dx[3], p234 = dx[2] * dx[3] * dx[4];
    const real R0 = p123 * recip(dx[2] * dx[3] + dx[1] * dx[3] + dx[1] * dx[2]);
    const real R5 = p234 * recip(dx[3] * dx[4] + dx[2] * dx[4] + dx[2] * dx[3]);
    real d[3];
    d[2] = (dx[4] * dx[5] + (dx[4] + dx[5]) * R0) * G.iab;
    d[0] = (dx[0] * dx[1] + (dx[0] + dx[1]) * R5) * G.icb;
    d[1] = 1.0 - d[0] - d[2];
    real pp[3];
    point_phi(P, d, beta, flag, pp);
    real s = 0.0;
    for (int r = 0; r < 3; ++r) {
      const int a = 2 - r;
      const real g1 = dx[a] + dx[a + 1], g2 = dx[a] * dx[a + 1] + g1 * dx[a + 2];
      s += pp[r] * (v0[0][a] + DD.D2[0][a] * g1 + DD.D3[0][a] * g2);
    }
    etaG[q] = s;
  }
}
SWALE_HD void recon_cell_special(const SchemeConst& P, const real h[5], const real v0[3][3], const StencilDD& DD,
                                 real dxmax, EdgeState& o, uint8_t& flag, uint32_t& st, real etaG[2]) {
  CellGeom G;
  cell_geom(h, P.beta_dx_global ? dxmax : h[2], G, st);
  recon_cell_special_g(P, G, h, v0, DD, o, flag, st, etaG);
}

// ------------------------------------------------------------------------------------
// Interface flux (Eq. hydro2D-HH2D and the bottom flux of Eq. bottomrk): FE (eta), FMm
// (momentum seen by the left cell), FMp (seen by the right cell), FB (bottom). L is the right
// edge of the left cell, R the left edge of the right cell; w the node velocity.
// ------------------------------------------------------------------------------------
struct Flux {
  real FE, FMm, FMp, FB;
};
SWALE_HD Flux interface_flux(real g, real alpha, real w, real EL, real ER, real BL, real BR, real hL,
                             real hR, real uL, real uR) {
  const real bstar = dmax(BL, BR);
  const real sL = pos0(EL - bstar), sR = pos0(ER - bstar);
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

// Interface flux of the non-well-balanced scheme: the plain Lax-Friedrichs flux of
// H = F(q) - w q on q = (eta, hu) (Eq. alpha2D) with the limited edge states, discharge h u
// (zero on dry edges); one momentum flux for both cells; the bottom flux of Eq. bottomrk.
SWALE_HD Flux interface_flux_plain(real g, real alpha, real w, real EL, real ER, real BL, real BR, real hL,
                                   real hR, real uL, real uR) {
  const real mL = hL * uL, mR = hR * uR;
  Flux f;
  f.FE = 0.5 * ((mL - w * EL) + (mR - w * ER)) - 0.5 * alpha * (ER - EL);
  const real hg = 0.5 * g;
  const real H2 = 0.5 * ((mL * uL + hg * hL * hL - w * mL) + (mR * uR + hg * hR * hR - w * mR)) -
                  0.5 * alpha * (mR - mL);
  f.FMm = H2;
  f.FMp = H2;
  f.FB = 0.5 * w * (BL + BR) + 0.5 * alpha * (BR - BL);
  return f;
}

// Width ratios of the source interpolant of cell j in its unit coordinate, from the shared
// reciprocals: rm = J_{j-1}/J_j, irm = J_j/J_{j-1}, irp = J_j/J_{j+1}, i1m = J_j/(J_{j-1}+J_j),
// i1p = J_j/(J_j+J_{j+1}), i1mp = J_j/(J_{j-1}+J_j+J_{j+1}).
struct SourceGeom {
  real rm, irm, irp, i1m, i1p, i1mp;
};
SWALE_HD SourceGeom source_geom(real Jm, real Jc, real iJm, real iJc, real iJp, real ipl, real ipr, real itc) {
  SourceGeom s;
  s.rm = Jm * iJc;
  s.irm = Jc * iJm;
  s.irp = Jc * iJp;
  s.i1m = Jc * ipl;
  s.i1p = Jc * ipr;
  s.i1mp = Jc * itc;
  return s;
}

// Source term int_cell -g (eta_h - b_h) b_h' dx of Sec. 4.1, with eta_h - b_h the quartic
// interpolating the depth data (averages h_{j-1}, h_j, h_{j+1}, limited edge depths h^L, h^R;
// the data order of hd) and b_h the quartic of the bottom data bd (averages and limited edge
// bottoms), in the unit coordinate t of the cell, evaluated exactly as an antisymmetric bilinear
// form. With phi_k the quartic cardinal functions of the five data (phi_k reproduces datum k and
// annihilates the others), the integral is h^T K b with K_kl = int_0^1 phi_k phi_l' dt.
// Integrating by parts, K + K^T = e_R e_R^T -
// e_L e_L^T (the data v_L, v_R are the interpolants' values at t = 0, 1), and K 1 = 0 (a constant
// bottom has no slope). So K = A + (e_R e_R^T - e_L e_L^T) / 2 with A antisymmetric and, in the
// differences from the cell's own average (dh_k = h_k - h_j, db_k = b_k - b_j, k in {j-1, j+1,
// L, R}),
//   h^T K b = h_j (db_R - db_L) + dh^T A db + (dh_R db_R - dh_L db_L) / 2,
// which leaves six mesh-only entries of A (indices 0 = j-1, 2 = j+1, 3 = L, 4 = R), rational in
// the width ratios r_m = J_{j-1} / J_j, r_p = J_{j+1} / J_j:
//   A02 = -1 / (35 r_m r_p (1 + r_m)^2 (1 + r_p)^2 (1 + r_m + r_p))
//   A03 = (14 r_p^2 + 21 r_p + 9) / (70 r_m (1 + r_m)^2 (1 + r_p) (1 + r_m + r_p))
//   A04 = (14 r_p^2 + 7 r_p + 2) / (70 r_m r_p (1 + r_m)^2 (1 + r_m + r_p))
//   A23 = -(14 r_m^2 + 7 r_m + 2) / (70 r_m r_p (1 + r_p)^2 (1 + r_m + r_p))
//   A24 = -(14 r_m^2 + 21 r_m + 9) / (70 r_p (1 + r_m) (1 + r_p)^2 (1 + r_m + r_p))
//   A34 = -(r_m^2 (35 r_p^2 + 35 r_p + 14) + r_m (35 r_p^2 + 21 r_p + 7) + 14 r_p^2 + 7 r_p + 2)
//         / (70 r_m r_p (1 + r_m) (1 + r_p))
// (exact integrals of the cardinal functions: about 29 FP64 instructions per cell, against 67
// for the product of the two interpolants in monomial form, and about 41 for the six entries,
// which stage 1 reads from the mesh cache). At rest (h = eta - b, eta constant) the form gives
// -g (eta (b_R - b_L) - (b_R^2 - b_L^2) / 2), the pressure jump, as dh^T A db = -db^T A db = 0.
struct SourceForm {
  real a02, a03, a04, a23, a24, a34;
};
// From the widths J_{j-1}, J_j, J_{j+1}, their reciprocals and the reciprocal pair / triple sums
// 1 / (J_{j-1} + J_j), 1 / (J_j + J_{j+1}), 1 / (J_{j-1} + J_j + J_{j+1}).
SWALE_HD SourceForm source_form(real Jm, real Jc, real Jp, real iJm, real iJc, real iJp, real ipl, real ipr,
                                real itc) {
  const real rm = Jm * iJc, rp = Jp * iJc;
  const real irm = Jc * iJm, irp = Jc * iJp, i1m = Jc * ipl, i1p = Jc * ipr, i1mp = Jc * itc;
  const real irr = irm * irp;
  const real P = irr * i1mp;
  const real Pm2 = P * (i1m * i1m), Pp2 = P * (i1p * i1p);
  // (14 r^2 + 7 r + 2) / 70, (14 r^2 + 21 r + 9) / 70
  const real qp = (0.2 * rp + 0.1) * rp + (1.0 / 35.0), sp = (0.2 * rp + 0.3) * rp + (9.0 / 70.0);
  const real qm = (0.2 * rm + 0.1) * rm + (1.0 / 35.0), sm = (0.2 * rm + 0.3) * rm + (9.0 / 70.0);
  SourceForm f;
  f.a02 = (Pm2 * (i1p * i1p)) * (-1.0 / 35.0);
  f.a03 = sp * ((Pm2 * rp) * i1p);
  f.a04 = qp * Pm2;
  f.a23 = -(qm * Pp2);
  f.a24 = -(sm * ((Pp2 * rm) * i1m));
  const real c2 = (0.5 * rp + 0.5) * rp + 0.2, c1 = (0.5 * rp + 0.3) * rp + 0.1;
  f.a34 = -(((c2 * rm + c1) * rm + qp) * (irr * (i1m * i1p)));
  return f;
}
// The row sums u = A db (with the diagonal part of K) that both source_cell_form and its reverse
// use: acc = h_j (db_R - db_L) + sum_k dh_k u_k.
SWALE_HD void source_form_rows(const SourceForm& A, real db0, real db2, real db3, real db4, real u[4]) {
  u[0] = A.a02 * db2 + A.a03 * db3 + A.a04 * db4;
  u[1] = -(A.a02 * db0) + A.a23 * db3 + A.a24 * db4;
  u[2] = (-(A.a03 * db0) - A.a23 * db2) + A.a34 * db4 - 0.5 * db3;
  u[3] = (-(A.a04 * db0) - A.a24 * db2) - A.a34 * db3 + 0.5 * db4;
}
// The source term from the form A (data hd, bd as above).
SWALE_HD real source_cell_form(real g, const real hd[5], const real bd[5], const SourceForm& A) {
  const real hc = hd[1], bc = bd[1];
  const real db0 = bd[0] - bc, db2 = bd[2] - bc, db3 = bd[3] - bc, db4 = bd[4] - bc;
  real u[4];
  source_form_rows(A, db0, db2, db3, db4, u);
  real acc = hc * (db4 - db3);
  acc += (hd[0] - hc) * u[0];
  acc += (hd[2] - hc) * u[1];
  acc += (hd[3] - hc) * u[2];
  acc += (hd[4] - hc) * u[3];
  return -g * acc;
}

// Source of the special source-term scheme for cell j (Eq. source2 with Eq. bhat2D in 1D, the
// Gauss-Lobatto sum of Eq. gausssij2): (g/2)(b2hat_R - b2hat_L) - g etabar (bhat_R - bhat_L)
// - g sum_q w_q (eta_q - etabar) b_h'(t_q), with b^2hat = ((b-)^2 + (b+)^2) / 2, bhat = (b- + b+) / 2
// at the two edges and b_h' the slope of the cell's bottom interpolant (the quartic of bd) at
// the Gauss-Lobatto points t = 0, (1 -+ 1/sqrt 5)/2, 1 (weights 1/12, 5/12, 5/12, 1/12).
//   eta4: eta at the four points;  bd: bottom data as in source_cell_form;  bLm: right-edge bottom of
//   cell j-1, bRp: left-edge bottom of cell j+1.
SWALE_HD real source_cell_special(real g, real etabar, const real eta4[4], const real bd[5], const SourceGeom& sg,
                                  real bLm, real bRp) {
  const real* u = bd;
  const real o2a = (u[3] - u[0]) * sg.irm;
  const real o2b = u[1] - u[3];
  const real o2c = u[4] - u[1];
  const real o2d = (u[2] - u[4]) * sg.irp;
  const real o3a = (o2b - o2a) * sg.i1m;
  const real o3b = o2c - o2b;
  const real o3c = (o2d - o2c) * sg.i1p;
  const real o4a = (o3b - o3a) * sg.i1m;
  const real o4b = (o3c - o3b) * sg.i1p;
  const real o5 = (o4b - o4a) * sg.i1mp;
  const real cb[6] = {0.0, u[0], o2a, o3a, o4a, o5};
  const double tq[4] = {0.0, SWALE_GLO_T1, SWALE_GLO_T2, 1.0};
  const double wq[4] = {1.0 / 12.0, 5.0 / 12.0, 5.0 / 12.0, 1.0 / 12.0};
  real S2 = 0.0;
  for (int q = 0; q < 4; ++q) {
    const double t = tq[q], t2 = t * t;
    const double md[6] = {0, 0, 1.0, 2.0 * t, 3.0 * t2 - 2.0 * t, 4.0 * t2 * t - 6.0 * t2 + 2.0 * t};
    const double mdd[6] = {0, 0, 0.0, 2.0, 6.0 * t - 2.0, 12.0 * t2 - 12.0 * t + 2.0};
    real bdv = 0.0;
    for (int k = 2; k <= 5; ++k) bdv += cb[k] * ((2.0 * md[k] + t * mdd[k]) + sg.rm * mdd[k]);
    S2 += wq[q] * (eta4[q] - etabar) * bdv;
  }
  const real bL = 0.5 * (bLm + u[3]), bR = 0.5 * (u[4] + bRp);
  const real b2L = 0.5 * (bLm * bLm + u[3] * u[3]), b2R = 0.5 * (u[4] * u[4] + bRp * bRp);
  return (0.5 * g) * (b2R - b2L) - g * etabar * (bR - bL) - g * S2;
}

// Flux differences and source of cell j: R = (R_E, R_M, R_B) of Eq. hydro2D / bottomrk.
struct CellRhs {
  real RE, RM, RB;
};
SWALE_HD CellRhs cell_rhs(const Flux& Fl, const Flux& Fr, real S) {
  CellRhs o;
  o.RE = -(Fr.FE - Fl.FE);
  o.RM = -(Fr.FMm - Fl.FMp) + S;
  o.RB = Fr.FB - Fl.FB;
  return o;
}

}  // namespace swale
