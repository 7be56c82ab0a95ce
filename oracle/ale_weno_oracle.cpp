/*
 * CPU oracle for the one-dimensional well-balanced finite-volume ALE-WENO hybrid
 * scheme with hydrostatic reconstruction (Zhang, Xia & Xu, "Structure-preserving
 * finite volume arbitrary Lagrangian-Eulerian WENO schemes for the shallow water
 * equations", arXiv 2208.06588).
 *
 * TEST INFRASTRUCTURE. This file is the slow, plain reference that the CUDA path is
 * checked against. Only the test suite, __graft_entry__.smoke() and the CPU-baseline /
 * reference arm of bench.py may load it. It shares no code, header, table or helper with
 * the CUDA library, and it never calls into it.
 *
 * Style: every small polynomial is obtained by solving the linear system that defines it
 * (cell-average conditions, point-value conditions) with Gaussian elimination, and the
 * steps follow the order in which the paper states them. FP64 throughout; built with
 * -ffp-contract=off so that the compiler does not fuse multiply-adds.
 *
 * Where the paper leaves a choice open, the reading taken here is stated next to the code
 * that implements it (the same readings are listed with their reasons in the design notes).
 *
 * The state path is templated on the scalar type T so that the same code, instantiated on
 * a forward-mode dual number, gives the tangent-linear model. Mesh quantities (widths,
 * node velocities, dt, alpha) stay double.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

/* ------------------------------------------------------------------------------------ */
/* Parameters (mirrored field by field by oracle/__init__.py).                           */
/* ------------------------------------------------------------------------------------ */
struct OrcParams {
  double g;            // gravitational constant (Sec. 5 uses 9.812)
  double cfl;          // CFL number in dt = cfl * min_j J_j / alpha
  double eps_weno;     // epsilon of the smoothness detector and WENO-Z weights (Step 2, Eq. omegaj)
  double eps_pp;       // positivity floor 1e-11 of the limiter (Eq. modifiedhjn)
  double h_dry;        // an edge depth <= h_dry carries zero velocity
  double mesh_T;       // period T of the prescribed motion x = xi + P sin(2 pi t / T)
  double gauss_sigma;  // Gaussian filter width (cells) of the fluid-driven mesh velocity
  double t_end;        // final time; the last step is clipped to it
  double dt_fixed;     // > 0: every step uses this dt instead of the CFL formula
  int32_t bc;          // 0 periodic, 1 transmissive, 2 reflective
  int32_t mesh;        // 0 static, 1 prescribed profile motion, 2 fluid-driven Gaussian,
                       // 3 constant node velocities x = x0 + v t (Eq. velocity / meshspecial)
  int32_t gauss_half;  // truncation half-width of the Gaussian filter (nodes)
  int32_t beta_dx_global;  // 1: Delta x in the smoothness indicators is max_j J_j (Step 1)
  // Bottom: 0 = cell averages evolved by the ALE scheme of Eq. bottomrk (the paper's default);
  // 1 = L2 projection (Eq. baverage) of a piecewise polynomial b(x) onto every stage mesh.
  int32_t bottom_mode;
  // 0: well-balanced scheme with hydrostatic reconstruction (Sec. 4.1); 1: the non-well-balanced
  // ALE-WENO scheme (Eq. se2D / s2D): local characteristic reconstruction of (eta, hu) and the
  // plain Lax-Friedrichs flux.
  int32_t scheme;
  // 0: alpha as Eq. alpha2D writes it, max |u - w| + sqrt(g h), wherever w is known when the
  // stage runs; 1: the bound max |u| + sqrt(g h) + Wbar (Wbar >= max |w|) in every stage.
  int32_t alpha_bound;
  // 1: the limiter's theta also scales the discharge edge values about their mean (reading O6b);
  // 0: it limits the depth only, as Eq. modifiedhjn is written.
  int32_t limit_hu;
  int32_t bpieces, bdeg;                  // number of pieces, polynomial degree
  const double* bbreaks;                  // bpieces + 1 increasing breakpoints
  const double* bcoef;                    // piece p: sum_k bcoef[p (bdeg+1) + k] (x - bbreaks[p])^k
};

// Piecewise polynomial bottom of the L2-projection mode (set by orc_set_bottom).
std::vector<double> g_bbreaks, g_bcoef;
int32_t g_bdeg = 0;

enum : uint32_t {
  ST_EWEIGHT = 1u,     // a linear weight d_r <= 0 (the split of Shi-Hu-Shu is not applied)
  ST_NEGDEPTH = 2u,    // a cell-average depth below -eps_pp entered a stage (warning)
  ST_NONFINITE = 4u,   // a non-finite value appeared
  ST_EMESH = 8u,       // a cell width became <= 0 (mesh assumption A1 violated)
  ST_NODT = 16u,       // no finite time step: the step used dt = 0 (reading O21)
};

/* ------------------------------------------------------------------------------------ */
/* Scalar helpers; overloaded for the dual type further down.                            */
/* ------------------------------------------------------------------------------------ */
inline double value(double x) { return x; }
inline double vabs(double x) { return std::fabs(x); }
inline double vsqrt(double x) { return std::sqrt(x); }
// max/min returning the first argument on a tie (the tangent follows the first argument).
inline double vmax(double a, double b) { return (b > a) ? b : a; }
inline double vmin(double a, double b) { return (b < a) ? b : a; }

/* Forward-mode dual number for the tangent-linear model. Kinks: |x|' = sign(x) with
 * sign(0) = 0; max/min pass the tangent of the selected argument, the first on a tie. */
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline double value(Dual x) { return x.v; }
inline Dual vabs(Dual x) { return x.v > 0 ? x : (x.v < 0 ? -x : Dual(0.0, 0.0)); }
inline Dual vsqrt(Dual x) {
  double s = std::sqrt(x.v);
  return Dual(s, s > 0 ? x.d / (2.0 * s) : 0.0);
}
inline Dual vmax(Dual a, Dual b) { return (b.v > a.v) ? b : a; }
inline Dual vmin(Dual a, Dual b) { return (b.v < a.v) ? b : a; }

/* Operation-counting scalar: the oracle's own count of the method's floating-point work (the
 * numerator of the roofline of the CUDA path). Every addition, subtraction, multiplication,
 * division and square root on a state-dependent value is counted; sign flips, |x|, max / min and
 * comparisons are not arithmetic, and mesh-only arithmetic (double) is not counted here. */
struct OpCount {
  long long add = 0, mul = 0, div = 0, sqrt = 0;
};
OpCount g_ops;
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double a) : v(a) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops.add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops.add; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops.mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops.div; return Cnt(a.v / b.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline double value(Cnt x) { return x.v; }
inline Cnt vabs(Cnt x) { return Cnt(std::fabs(x.v)); }
inline Cnt vsqrt(Cnt x) { ++g_ops.sqrt; return Cnt(std::sqrt(x.v)); }
inline Cnt vmax(Cnt a, Cnt b) { return (b.v > a.v) ? b : a; }
inline Cnt vmin(Cnt a, Cnt b) { return (b.v < a.v) ? b : a; }

inline double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

/* Gaussian elimination with partial pivoting: solves A X = B in place (A n x n, B n x m,
 * both row-major). The systems here are at most 5 x 5. */
void gauss_solve(int n, double* A, double* B, int m) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
    if (piv != col) {
      for (int c = 0; c < n; ++c) std::swap(A[col * n + c], A[piv * n + c]);
      for (int c = 0; c < m; ++c) std::swap(B[col * m + c], B[piv * m + c]);
    }
    for (int r = col + 1; r < n; ++r) {
      double f = A[r * n + col] / A[col * n + col];
      for (int c = col; c < n; ++c) A[r * n + c] -= f * A[col * n + c];
      for (int c = 0; c < m; ++c) B[r * m + c] -= f * B[col * m + c];
    }
  }
  for (int col = n - 1; col >= 0; --col) {
    for (int c = 0; c < m; ++c) {
      double s = B[col * m + c];
      for (int k = col + 1; k < n; ++k) s -= A[col * n + k] * B[k * m + c];
      B[col * m + c] = s / A[col * n + col];
    }
  }
}

/* Polynomial of degree n-1, p(t) = sum_k a_k t^k, whose averages over the n consecutive
 * intervals [y_i, y_{i+1}] equal given data. Returns the linear map from the data to the
 * coefficients: map[k * n + i] = d a_k / d ubar_i. (The definition of a reconstruction
 * polynomial from cell averages, Step 1 of Sec. 2.2.) */
void average_poly_map(int n, const double* y, double* map) {
  double A[25], X[25];
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k)
      A[i * n + k] = (ipow(y[i + 1], k + 1) - ipow(y[i], k + 1)) / ((k + 1) * (y[i + 1] - y[i]));
  for (int i = 0; i < n * n; ++i) X[i] = 0.0;
  for (int i = 0; i < n; ++i) X[i * n + i] = 1.0;
  gauss_solve(n, A, X, n);
  for (int i = 0; i < n * n; ++i) map[i] = X[i];
}

/* Mesh-only WENO data of one cell j, in the cell's own unit coordinate t = (x - x_{j-1/2}) / J_j
 * (so the cell is [0, 1]). Inputs: the widths J_{j-2..j+2}. */
struct WenoCoeffs {
  double sub[3][9];   // sub[r][k*3+i]: coefficient a_k of p_r per unit of ubar_{j-r+i}
  double c[2][3][3];  // c[e][r][i]: weight of ubar_{j-r+i} in p_r(t_e), e = 0 (t=0), 1 (t=1)
  double big[2][5];   // weight of ubar_{j-2+i} in the quartic of the big stencil at t_e
  double d[2][3];     // linear weights d_r at edge e
};

void weno_coeffs(const double* w5, WenoCoeffs& W) {
  // Node coordinates of the big stencil S_j = {T_{j-2}, ..., T_{j+2}} in units of J_j.
  double y[6];
  y[2] = 0.0;
  y[3] = 1.0;
  y[1] = -w5[1] / w5[2];
  y[0] = y[1] - w5[0] / w5[2];
  y[4] = 1.0 + w5[3] / w5[2];
  y[5] = y[4] + w5[4] / w5[2];
  // Sub-stencil r covers cells j-r .. j-r+2, i.e. nodes y[2-r] .. y[5-r].
  for (int r = 0; r < 3; ++r) average_poly_map(3, y + 2 - r, W.sub[r]);
  double big[25];
  average_poly_map(5, y, big);
  for (int e = 0; e < 2; ++e) {
    const double te = (double)e;
    for (int r = 0; r < 3; ++r)
      for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += W.sub[r][k * 3 + i] * ipow(te, k);
        W.c[e][r][i] = s;
      }
    for (int i = 0; i < 5; ++i) {
      double s = 0.0;
      for (int k = 0; k < 5; ++k) s += big[k * 5 + i] * ipow(te, k);
      W.big[e][i] = s;
    }
    // Linear weights: sum_r d_r p_r(t_e) equals the quartic at t_e. Only p_2 contains
    // ubar_{j-2} and only p_0 contains ubar_{j+2}; matching those two coefficients fixes
    // d_2 and d_0, and consistency (all weights of each polynomial sum to one) gives d_1.
    W.d[e][2] = W.big[e][0] / W.c[e][2][0];
    W.d[e][0] = W.big[e][4] / W.c[e][0][2];
    W.d[e][1] = 1.0 - W.d[e][0] - W.d[e][2];
  }
}

/* Mesh-only WENO data of cell j at an arbitrary point t of its unit coordinate (Step 1 at a
 * point other than an edge, e.g. the Gauss-Lobatto points of the special source term):
 * c[r][i] weights of ubar_{j-r+i} in p_r(t), big[i] weights of ubar_{j-2+i} in the quartic at
 * t, and the linear weights d_r(t) (matching the outermost coefficients as at the edges; at
 * interior points they may be negative). */
struct PointCoeffs {
  double c[3][3];
  double big[5];
  double d[3];
};

void weno_point(const double* w5, double t, PointCoeffs& Q) {
  double y[6];
  y[2] = 0.0;
  y[3] = 1.0;
  y[1] = -w5[1] / w5[2];
  y[0] = y[1] - w5[0] / w5[2];
  y[4] = 1.0 + w5[3] / w5[2];
  y[5] = y[4] + w5[4] / w5[2];
  double sub[3][9], big[25];
  for (int r = 0; r < 3; ++r) average_poly_map(3, y + 2 - r, sub[r]);
  average_poly_map(5, y, big);
  for (int r = 0; r < 3; ++r)
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += sub[r][k * 3 + i] * ipow(t, k);
      Q.c[r][i] = s;
    }
  for (int i = 0; i < 5; ++i) {
    double s = 0.0;
    for (int k = 0; k < 5; ++k) s += big[k * 5 + i] * ipow(t, k);
    Q.big[i] = s;
  }
  Q.d[2] = Q.big[0] / Q.c[2][0];
  Q.d[0] = Q.big[4] / Q.c[0][2];
  Q.d[1] = 1.0 - Q.d[0] - Q.d[2];
}

/* Hybrid weights at a point with linear weights d (Step 3), with the treatment of negative
 * linear weights of Shi, Hu & Shu (2002) cited in Sec. 2.2: when some d_r <= 0 the WENO-Z part
 * splits d = s+ d+ - s- d-, with d~+ = (d + 3|d|) / 2, d~- = d~+ - d, s+- = sum d~+-,
 * d+- = d~+- / s+-; each group gets its own normalised WENO-Z weights w+- (same indicators)
 * and phi^N = s+ w+ - s- w-. Smooth class: phi = d; transition: the blend of Step 3. */
template <class T>
void point_phi(const OrcParams& P, const double d[3], const T beta[3], const T& tau, const T& gam, uint8_t flag,
               T phi[3]) {
  if (flag == 0) {
    for (int r = 0; r < 3; ++r) phi[r] = T(d[r]);
    return;
  }
  T X[3];
  for (int r = 0; r < 3; ++r) {
    T q = tau / (beta[r] + T(P.eps_weno));
    X[r] = T(1.0) + q * q;
  }
  T phiN[3];
  if (d[0] > 0.0 && d[1] > 0.0 && d[2] > 0.0) {
    T al[3], s = T(0.0);
    for (int r = 0; r < 3; ++r) {
      al[r] = T(d[r]) * X[r];
      s += al[r];
    }
    for (int r = 0; r < 3; ++r) phiN[r] = al[r] / s;
  } else {
    double dp[3], dm[3], sp = 0.0, sm = 0.0;
    for (int r = 0; r < 3; ++r) {
      dp[r] = 0.5 * (d[r] + 3.0 * std::fabs(d[r]));
      dm[r] = dp[r] - d[r];
      sp += dp[r];
      sm += dm[r];
    }
    T ap[3], am[3], Sp = T(0.0), Sm = T(0.0);
    for (int r = 0; r < 3; ++r) {
      ap[r] = T(dp[r] / sp) * X[r];
      am[r] = T(dm[r] / sm) * X[r];
      Sp += ap[r];
      Sm += am[r];
    }
    for (int r = 0; r < 3; ++r) phiN[r] = T(sp) * ap[r] / Sp - T(sm) * am[r] / Sm;
  }
  if (flag == 1) {
    T Mg = T(2.0) * gam - T(1.0);
    for (int r = 0; r < 3; ++r) phi[r] = Mg * phiN[r] + (T(1.0) - Mg) * T(d[r]);
  } else {
    for (int r = 0; r < 3; ++r) phi[r] = phiN[r];
  }
}

/* Interior 4-point Gauss-Lobatto points of the unit cell (the special source term). */
const double kGLoT[2] = {0.5 - 0.5 / 2.2360679774997896964, 0.5 + 0.5 / 2.2360679774997896964};

/* Smoothness indicator of Step 2 for the sub-stencil polynomial p_r of data v5, with the
 * factor lam = Delta x / J_j carrying the global cell length into unit coordinates:
 *   beta_r = sum_{l=1,2} (Delta x)^{2l-1} int_cell (d^l p_r / dx^l)^2 dx
 *          = lam * int_0^1 (p_r')^2 dt + lam^3 * int_0^1 (p_r'')^2 dt. */
template <class T>
T beta_of(const WenoCoeffs& W, int r, const T* v5, double lam) {
  T a1 = T(0.0), a2 = T(0.0);
  for (int i = 0; i < 3; ++i) {
    a1 += T(W.sub[r][1 * 3 + i]) * v5[2 - r + i];
    a2 += T(W.sub[r][2 * 3 + i]) * v5[2 - r + i];
  }
  // p' = a1 + 2 a2 t on [0,1]: int (p')^2 = a1^2 + 2 a1 a2 + (4/3) a2^2 ; p'' = 2 a2.
  T i1 = a1 * a1 + T(2.0) * a1 * a2 + T(4.0 / 3.0) * a2 * a2;
  T i2 = T(4.0) * a2 * a2;
  return T(lam) * i1 + T(lam * lam * lam) * i2;
}

/* Steps 2-3 for one scalar field v5 on its own (no shared indicators): class and the hybrid
 * weights phi[e][r] at both edges. Returns gamma. */
template <class T>
double hybrid_weights(const OrcParams& P, const WenoCoeffs& W, double lam, const T* v5, T phi[2][3], uint8_t& flag) {
  T beta[3];
  for (int r = 0; r < 3; ++r) beta[r] = beta_of(W, r, v5, lam);
  const T tau = vabs(beta[0] - beta[2]);
  const T gam = tau / ((beta[0] + beta[1] + beta[2]) / T(3.0) + T(P.eps_weno));
  flag = value(gam) <= 0.5 ? 0 : (value(gam) >= 1.0 ? 2 : 1);
  for (int e = 0; e < 2; ++e) {
    if (flag == 0) {
      for (int r = 0; r < 3; ++r) phi[e][r] = T(W.d[e][r]);
      continue;
    }
    T al[3], sum = T(0.0);
    for (int r = 0; r < 3; ++r) {
      T q = tau / (beta[r] + T(P.eps_weno));
      al[r] = T(W.d[e][r]) * (T(1.0) + q * q);
      sum += al[r];
    }
    for (int r = 0; r < 3; ++r) phi[e][r] = al[r] / sum;
    if (flag == 1) {
      T Mg = T(2.0) * gam - T(1.0);
      for (int r = 0; r < 3; ++r) phi[e][r] = Mg * phi[e][r] + (T(1.0) - Mg) * T(W.d[e][r]);
    }
  }
  return value(gam);
}

/* Step 4 for one field: sum_r phi_r p_r at edge e. */
template <class T>
T edge_value(const WenoCoeffs& W, const T phi[2][3], const T* v5, int e) {
  T v = T(0.0);
  for (int r = 0; r < 3; ++r) {
    T p = T(0.0);
    for (int i = 0; i < 3; ++i) p += T(W.c[e][r][i]) * v5[2 - r + i];
    v += phi[e][r] * p;
  }
  return v;
}

template <class T>
struct EdgeVals;

/* Edge values of the non-well-balanced scheme (Sec. 2.2, last paragraph: local characteristic
 * decomposition for systems). Reading: the eigenvectors of the flux Jacobian d f / d (eta, hu)
 * = [[0, 1], [c^2 - u^2, 2u]] are taken at cell j's average state (u = hu/h, c = sqrt(g h)),
 * R = [[1, 1], [u - c, u + c]]; the five stencil averages are projected with R^-1, each
 * characteristic field is reconstructed with its own indicators, class and weights, and the
 * edge values are mapped back with R. Where the cell is dry (h <= h_dry) the fields are eta and
 * hu themselves. The bottom is reconstructed on its own. The reported class is the largest of
 * the three fields'. */
template <class T>
void nonwb_edges(const OrcParams& P, const WenoCoeffs& W, double lam, const T* e5, const T* m5, const T* b5,
                 EdgeVals<T>& o);

/* Per-cell result of the reconstruction + limiter (cells -1 .. N). Edge e = 0 is the left
 * edge x_{j-1/2}^+ of the cell, e = 1 the right edge x_{j+1/2}^-. */
template <class T>
struct EdgeVals {
  T E[2], M[2], B[2];  // surface level, discharge, bottom (bottom re-derived after limiting)
  T h[2], u[2];        // limited depth and velocity
  T Eg[2];             // special source scheme: eta at the two interior Gauss-Lobatto points
  uint8_t flag;        // 0 smooth, 1 transition, 2 non-smooth (Step 2)
  double gamma;        // detector value
};

template <class T>
void nonwb_edges(const OrcParams& P, const WenoCoeffs& W, double lam, const T* e5, const T* m5, const T* b5,
                 EdgeVals<T>& o) {
  const double hb = value(e5[2]) - value(b5[2]);
  double u = 0.0, c = 0.0;
  const bool wet = hb > P.h_dry;
  if (wet) {
    u = value(m5[2]) / hb;
    c = std::sqrt(P.g * hb);
  }
  T w1[5], w2[5];
  for (int k = 0; k < 5; ++k) {
    if (wet) {  // R^-1 = 1/(2c) [[u + c, -1], [-(u - c), 1]]
      w1[k] = (T(u + c) * e5[k] - m5[k]) / T(2.0 * c);
      w2[k] = (m5[k] - T(u - c) * e5[k]) / T(2.0 * c);
    } else {
      w1[k] = e5[k];
      w2[k] = m5[k];
    }
  }
  T p1[2][3], p2[2][3], pb[2][3];
  uint8_t f1, f2, fb;
  const double g1 = hybrid_weights(P, W, lam, w1, p1, f1);
  const double g2 = hybrid_weights(P, W, lam, w2, p2, f2);
  const double gb = hybrid_weights(P, W, lam, b5, pb, fb);
  o.flag = std::max(f1, std::max(f2, fb));
  o.gamma = std::max(g1, std::max(g2, gb));
  for (int e = 0; e < 2; ++e) {
    const T a = edge_value(W, p1, w1, e), b = edge_value(W, p2, w2, e);
    if (wet) {
      o.E[e] = a + b;
      o.M[e] = T(u - c) * a + T(u + c) * b;
    } else {
      o.E[e] = a;
      o.M[e] = b;
    }
    o.B[e] = edge_value(W, pb, b5, e);
  }
}

/* Ghost index map for the three ghost cells on each side. */
int64_t ghost_src(int64_t i, int64_t N, int bc) {
  if (bc == 0) return ((i % N) + N) % N;
  if (i < 0) return -1 - i;
  if (i >= N) return 2 * N - 1 - i;
  return i;
}

/* Reconstruction (Steps 1-4 of Sec. 2.2 with the shared weights of Eq. alphamodified),
 * then the bound-preserving limiter (Eq. modifiedhjn / xd in one dimension) and the
 * bottom re-derivation of the Remark in Sec. 4.3. Returns the largest |u - w| + sqrt(g h)
 * over the edges that touch interfaces 0..N (Eq. alpha2D; an edge of cell j at node j + e
 * moves with w[j + e]), or the largest |u| + sqrt(g h) when w is null. */
template <class T>
double reconstruct(const OrcParams& P, int64_t N, const T* E, const T* M, const T* B, const double* J,
                   std::vector<EdgeVals<T>>& ed, uint32_t& status, const double* w = nullptr) {
  const int64_t G = 3;
  std::vector<T> Ex(N + 2 * G), Mx(N + 2 * G), Bx(N + 2 * G);
  std::vector<double> Jx(N + 2 * G);
  for (int64_t i = -G; i < N + G; ++i) {
    int64_t s = ghost_src(i, N, P.bc);
    Ex[i + G] = E[s];
    Bx[i + G] = B[s];
    Mx[i + G] = (P.bc == 2 && (i < 0 || i >= N)) ? -M[s] : M[s];
    Jx[i + G] = J[s];
  }
  // Global cell length at this stage's mesh (Step 1: Delta x = max_j Delta_j).
  double dxmax = 0.0;
  for (int64_t j = 0; j < N; ++j) dxmax = std::max(dxmax, J[j]);

  ed.assign(N + 2, EdgeVals<T>());
  double A = 0.0;
  for (int64_t j = -1; j <= N; ++j) {
    const int64_t c = j + G;
    double w5[5];
    for (int k = 0; k < 5; ++k) w5[k] = Jx[c - 2 + k];
    for (int k = 0; k < 5; ++k)
      if (!(w5[k] > 0.0)) status |= ST_EMESH;
    WenoCoeffs W;
    weno_coeffs(w5, W);
    for (int e = 0; e < 2; ++e)
      for (int r = 0; r < 3; ++r)
        if (!(W.d[e][r] > 0.0)) status |= ST_EWEIGHT;

    T e5[5], m5[5], b5[5], h5[5];
    for (int k = 0; k < 5; ++k) {
      e5[k] = Ex[c - 2 + k];
      m5[k] = Mx[c - 2 + k];
      b5[k] = Bx[c - 2 + k];
      h5[k] = e5[k] - b5[k];  // conservative variable h = eta - b (Eq. urec)
    }
    const double lam = P.beta_dx_global ? dxmax / w5[2] : 1.0;
    // Step 2 with shared indicators: beta_r summed over the conservative variables (h, hu).
    T beta[3];
    for (int r = 0; r < 3; ++r) beta[r] = beta_of(W, r, h5, lam) + beta_of(W, r, m5, lam);
    const T tau = vabs(beta[0] - beta[2]);
    const T betaA = (beta[0] + beta[1] + beta[2]) / T(3.0);
    const T gam = tau / (betaA + T(P.eps_weno));
    // Reading of the overlapping ranges: smooth if gamma <= 1/2, non-smooth if gamma >= 1.
    uint8_t flag = value(gam) <= 0.5 ? 0 : (value(gam) >= 1.0 ? 2 : 1);

    EdgeVals<T>& o = ed[j + 1];
    o.flag = flag;
    o.gamma = value(gam);
    if (P.scheme == 1) {
      nonwb_edges(P, W, lam, e5, m5, b5, o);
    } else
    for (int e = 0; e < 2; ++e) {
      // Step 3: phi^L = d, phi^N = WENO-Z, phi^T = M(gamma) phi^N + (1 - M(gamma)) phi^L.
      T phi[3];
      if (flag == 0) {
        for (int r = 0; r < 3; ++r) phi[r] = T(W.d[e][r]);
      } else {
        T al[3], s = T(0.0);
        for (int r = 0; r < 3; ++r) {
          T q = tau / (beta[r] + T(P.eps_weno));
          al[r] = T(W.d[e][r]) * (T(1.0) + q * q);
          s += al[r];
        }
        for (int r = 0; r < 3; ++r) phi[r] = al[r] / s;
        if (flag == 1) {
          T Mg = T(2.0) * gam - T(1.0);
          for (int r = 0; r < 3; ++r) phi[r] = Mg * phi[r] + (T(1.0) - Mg) * T(W.d[e][r]);
        }
      }
      // Step 4 with the same weights for eta, hu and b (Sec. 4.1 items 1-2).
      T ve = T(0.0), vm = T(0.0), vb = T(0.0);
      for (int r = 0; r < 3; ++r) {
        T pe = T(0.0), pm = T(0.0), pb = T(0.0);
        for (int i = 0; i < 3; ++i) {
          pe += T(W.c[e][r][i]) * e5[2 - r + i];
          pm += T(W.c[e][r][i]) * m5[2 - r + i];
          pb += T(W.c[e][r][i]) * b5[2 - r + i];
        }
        ve += phi[r] * pe;
        vm += phi[r] * pm;
        vb += phi[r] * pb;
      }
      o.E[e] = ve;
      o.M[e] = vm;
      o.B[e] = vb;
    }

    if (P.scheme == 2) {
      // Special source scheme: eta at the interior Gauss-Lobatto points by the same hybrid
      // reconstruction (shared indicators and class of this cell), linear weights at the point.
      for (int q = 0; q < 2; ++q) {
        PointCoeffs Q;
        weno_point(w5, kGLoT[q], Q);
        T phi[3];
        point_phi(P, Q.d, beta, tau, gam, flag, phi);
        T v = T(0.0);
        for (int r = 0; r < 3; ++r) {
          T pe = T(0.0);
          for (int i = 0; i < 3; ++i) pe += T(Q.c[r][i]) * e5[2 - r + i];
          v += phi[r] * pe;
        }
        o.Eg[q] = v;
      }
    }
    // Bound-preserving limiter in 1D: 4-point Gauss-Lobatto rule (k >= (p+2)/2 with p = 5),
    // end weights sigma_1 = sigma_4 = 1/12. The interior mean delta follows from
    // hbar = (1 - 2/12) delta + (h^L + h^R)/12.
    T hbar = e5[2] - b5[2];
    if (value(hbar) < -P.eps_pp) status |= ST_NEGDEPTH;
    // Reading: a rounding-level negative mean in a dry cell is treated as zero.
    if (value(hbar) < 0.0) hbar = T(0.0);
    T hL = o.E[0] - o.B[0], hR = o.E[1] - o.B[1];
    T delta = (T(12.0) * hbar - hL - hR) / T(10.0);
    T mn = vmin(vmin(hL, hR), delta);
    T epsv = vmin(T(P.eps_pp), hbar);
    T theta = T(1.0);
    if (value(mn) < value(epsv)) theta = (hbar - epsv) / (hbar - mn);
    hL = theta * (hL - hbar) + hbar;
    hR = theta * (hR - hbar) + hbar;
    o.h[0] = hL;
    o.h[1] = hR;
    // Reading: the discharge edge values are scaled about their mean with the same theta
    // (the positivity limiter of the cited Xing-Zhang-Shu scheme acts on (h, hu) together),
    // so that u = hu / h stays bounded where h is pulled towards the floor.
    const T mbar = m5[2];
    if (P.limit_hu) {
      o.M[0] = theta * (o.M[0] - mbar) + mbar;
      o.M[1] = theta * (o.M[1] - mbar) + mbar;
    }
    // Remark of Sec. 4.3: b^new = eta - h^new; eta itself is left untouched.
    o.B[0] = o.E[0] - hL;
    o.B[1] = o.E[1] - hR;
    for (int e = 0; e < 2; ++e) {
      o.u[e] = (value(o.h[e]) > P.h_dry) ? o.M[e] / o.h[e] : T(0.0);
      if (!std::isfinite(value(o.E[e])) || !std::isfinite(value(o.M[e])) || !std::isfinite(value(o.h[e])))
        status |= ST_NONFINITE;
    }
    // Wave speed over the edges that touch interfaces 0..N.
    for (int e = 0; e < 2; ++e) {
      if ((j == -1 && e == 0) || (j == N && e == 1)) continue;
      double hpos = std::max(value(o.h[e]), 0.0);
      const double rel = w ? value(o.u[e]) - w[j + e] : value(o.u[e]);
      double s = std::fabs(rel) + std::sqrt(P.g * hpos);
      A = std::max(A, s);
    }
  }
  return A;
}

/* Four-point Gauss-Legendre rule on [0, 1] (exact to degree 7). */
void gauss_legendre4(double* t, double* wq) {
  const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
  t[0] = 0.5 * (1.0 - b); wq[0] = 0.5 * wb;
  t[1] = 0.5 * (1.0 - a); wq[1] = 0.5 * wa;
  t[2] = 0.5 * (1.0 + a); wq[2] = 0.5 * wa;
  t[3] = 0.5 * (1.0 + b); wq[3] = 0.5 * wb;
}

/* Source interpolant (Sec. 4.1, after Eq. HH2D): the quartic on cell j that matches the
 * averages on cells j-1, j, j+1 and the two edge values of cell j. Reading: "interpolating
 * fourth-order polynomials" = these five conditions, so that at rest eta_h is constant and
 * b_h takes the same edge values as the flux side. Returns the coefficient map
 * map[k*5 + i] for data (avg_{j-1}, avg_j, avg_{j+1}, v^L, v^R), unit coordinate t. */
void source_interp_map(double rm, double rp, double* map) {
  const double y[4] = {-rm, 0.0, 1.0, 1.0 + rp};
  double A[25], X[25];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 5; ++k)
      A[i * 5 + k] = (ipow(y[i + 1], k + 1) - ipow(y[i], k + 1)) / ((k + 1) * (y[i + 1] - y[i]));
  for (int k = 0; k < 5; ++k) {
    A[3 * 5 + k] = ipow(0.0, k);
    A[4 * 5 + k] = ipow(1.0, k);
  }
  for (int i = 0; i < 25; ++i) X[i] = 0.0;
  for (int i = 0; i < 5; ++i) X[i * 5 + i] = 1.0;
  gauss_solve(5, A, X, 5);
  for (int i = 0; i < 25; ++i) map[i] = X[i];
}

/* Right-hand side of the well-balanced semi-discrete scheme (Eq. hydro2D-HH2D and
 * Eq. bottomrk in 1D) for all cells 0..N-1, given the limited edge values, the node
 * velocities w[0..N] and the global viscosity alpha. */
template <class T>
void rhs(const OrcParams& P, int64_t N, const std::vector<EdgeVals<T>>& ed, const T* E, const T* M, const T* B,
         const double* J, const double* w, double alpha, T* RE, T* RM, T* RB) {
  (void)M;
  const double g = P.g;
  // Interface k: L = right edge of cell k-1 (ed[k]), R = left edge of cell k (ed[k+1]).
  std::vector<T> FE(N + 1), FMm(N + 1), FMp(N + 1), FB(N + 1);
  for (int64_t k = 0; k <= N; ++k) {
    const EdgeVals<T>& l = ed[k];
    const EdgeVals<T>& r = ed[k + 1];
    const T EL = l.E[1], ER = r.E[0], BL = l.B[1], BR = r.B[0];
    const T hL = l.h[1], hR = r.h[0], uL = l.u[1], uR = r.u[0];
    const T wk = T(w[k]), al = T(alpha);
    if (P.scheme == 1 || P.scheme == 2) {
      // Non-well-balanced and special source schemes (Eq. alpha2D on q = (eta, hu), Eq. special2D):
      // plain Lax-Friedrichs flux of
      // H = F(q) - w q with the limited edge states; discharge h u (zero on dry edges).
      const T mL = hL * uL, mR = hR * uR;
      const T al2 = T(alpha);
      FE[k] = T(0.5) * ((mL - wk * EL) + (mR - wk * ER)) - T(0.5) * al2 * (ER - EL);
      const T H2 = T(0.5) * ((mL * uL + T(0.5 * g) * hL * hL - wk * mL) + (mR * uR + T(0.5 * g) * hR * hR - wk * mR)) -
                   T(0.5) * al2 * (mR - mL);
      FMm[k] = H2;
      FMp[k] = H2;
      FB[k] = T(0.5) * wk * (BL + BR) + T(0.5) * al2 * (BR - BL);
      continue;
    }
    // Hydrostatic reconstruction (Eq. HH2D): h*,+- = max(0, eta+- - max(b+, b-)).
    const T bstar = vmax(BL, BR);
    const T sL = vmax(T(0.0), EL - bstar), sR = vmax(T(0.0), ER - bstar);
    // Reading: the starred discharge is h* u (hydrostatic reconstruction of the cited
    // well-balanced scheme); the literal hu+- is singular where h* = 0.
    const T mL = sL * uL, mR = sR * uR;
    const T etasL = sL + BL, etasR = sR + BR;  // eta*,+- = h*,+- + b+-
    // First component: LF flux of H = F(q*) - w q* plus the correction theta (Eq. HH2D).
    const T H1 = T(0.5) * ((mL - wk * etasL) + (mR - wk * etasR)) - T(0.5) * al * (etasR - etasL);
    const T theta = T(0.5) * (wk + al) * (etasR - ER) + T(0.5) * (wk - al) * (etasL - EL);
    FE[k] = H1 + theta;
    // Second component: LF flux of q*, plus the cell-sided pressure correction.
    const T H2 = T(0.5) * ((mL * uL + T(0.5 * g) * sL * sL - wk * mL) + (mR * uR + T(0.5 * g) * sR * sR - wk * mR)) -
                 T(0.5) * al * (mR - mL);
    FMm[k] = H2 + T(0.5 * g) * (hL * hL - sL * sL);  // seen by cell k-1 (outward normal +1)
    FMp[k] = H2 + T(0.5 * g) * (hR * hR - sR * sR);  // seen by cell k (outward normal -1)
    // Bottom flux of Eq. bottomrk: B = 1/2 w.n (b- + b+) + 1/2 alpha (b+ - b-), taken for
    // cell k-1 (n = +1); cell k sees its negative.
    FB[k] = T(0.5) * wk * (BL + BR) + T(0.5) * al * (BR - BL);
  }
  double tq[4], wq[4];
  gauss_legendre4(tq, wq);
  const int64_t G = 3;
  (void)G;
  for (int64_t j = 0; j < N; ++j) {
    // Source term: int_cell -g (eta_h - b_h) b_h' dx, 4-point Gauss-Legendre in the unit
    // coordinate (dx = J dt and d/dx = (1/J) d/dt cancel).
    const int64_t jm = ghost_src(j - 1, N, P.bc), jp = ghost_src(j + 1, N, P.bc);
    const double rm = J[jm] / J[j], rp = J[jp] / J[j];
    double map[25];
    source_interp_map(rm, rp, map);
    const EdgeVals<T>& c = ed[j + 1];
    const T edat[5] = {E[jm], E[j], E[jp], c.E[0], c.E[1]};
    const T bdat[5] = {B[jm], B[j], B[jp], c.B[0], c.B[1]};
    T ea[5], ba[5];
    for (int k = 0; k < 5; ++k) {
      ea[k] = T(0.0);
      ba[k] = T(0.0);
      for (int i = 0; i < 5; ++i) {
        ea[k] += T(map[k * 5 + i]) * edat[i];
        ba[k] += T(map[k * 5 + i]) * bdat[i];
      }
    }
    if (P.scheme == 2) {
      // Special source term (Eq. source2 in 1D with Eq. bhat2D): (g/2) [b^2 hat] - g etabar
      // [b hat] over the two edges (outward normals +-1), plus the 4-point Gauss-Lobatto sum
      // of -g (eta - etabar) b_x (Eq. gausssij2). eta at the points: the edge values and the
      // interior hybrid reconstructions; b_x: the derivative of the cell's bottom interpolant
      // (reading: a fifth-order value needs a fourth-order slope, which the sub-stencil
      // quadratics with the value weights do not give).
      const EdgeVals<T>& lft = ed[j];
      const EdgeVals<T>& rgt = ed[j + 2];
      const T bR = T(0.5) * (c.B[1] + rgt.B[0]), bL = T(0.5) * (lft.B[1] + c.B[0]);
      const T b2R = T(0.5) * (c.B[1] * c.B[1] + rgt.B[0] * rgt.B[0]);
      const T b2L = T(0.5) * (lft.B[1] * lft.B[1] + c.B[0] * c.B[0]);
      const double tgl[4] = {0.0, kGLoT[0], kGLoT[1], 1.0};
      const double wgl[4] = {1.0 / 12.0, 5.0 / 12.0, 5.0 / 12.0, 1.0 / 12.0};
      const T eta[4] = {c.E[0], c.Eg[0], c.Eg[1], c.E[1]};
      T S2 = T(0.0);
      for (int q = 0; q < 4; ++q) {
        T dbh = T(0.0);
        for (int k = 1; k < 5; ++k) dbh += T((double)k * ipow(tgl[q], k - 1)) * ba[k];
        S2 += T(wgl[q]) * (eta[q] - E[j]) * dbh;
      }
      const T Ssp = T(0.5 * g) * (b2R - b2L) - T(g) * E[j] * (bR - bL) - T(g) * S2;
      RE[j] = -(FE[j + 1] - FE[j]);
      RM[j] = -(FMm[j + 1] - FMp[j]) + Ssp;
      RB[j] = FB[j + 1] - FB[j];
      continue;
    }
    T S = T(0.0);
    for (int q = 0; q < 4; ++q) {
      T eh = T(0.0), bh = T(0.0), dbh = T(0.0);
      for (int k = 0; k < 5; ++k) {
        eh += ea[k] * T(ipow(tq[q], k));
        bh += ba[k] * T(ipow(tq[q], k));
        if (k > 0) dbh += T((double)k * ipow(tq[q], k - 1)) * ba[k];
      }
      S += T(wq[q]) * (eh - bh) * dbh;
    }
    S = T(-g) * S;
    RE[j] = -(FE[j + 1] - FE[j]);
    RM[j] = -(FMm[j + 1] - FMp[j]) + S;
    RB[j] = FB[j + 1] - FB[j];
  }
}

/* Fluid-driven node velocity: raw node velocity = mean of the adjacent cell velocities
 * (dry cells carry zero), smoothed by a truncated, renormalised Gaussian; end nodes fixed. */
template <class T>
void fluid_gauss_velocity(const OrcParams& P, int64_t N, const T* E, const T* M, const T* B, std::vector<double>& w) {
  std::vector<double> u(N), raw(N + 1, 0.0);
  for (int64_t j = 0; j < N; ++j) {
    double h = value(E[j]) - value(B[j]);
    u[j] = (h > P.h_dry) ? value(M[j]) / h : 0.0;
  }
  for (int64_t k = 1; k < N; ++k) raw[k] = 0.5 * (u[k - 1] + u[k]);
  w.assign(N + 1, 0.0);
  const int K = P.gauss_half;
  std::vector<double> gw(2 * K + 1);
  for (int m = -K; m <= K; ++m) gw[m + K] = std::exp(-(double)(m * m) / (2.0 * P.gauss_sigma * P.gauss_sigma));
  for (int64_t k = 1; k < N; ++k) {
    double s = 0.0, sw = 0.0;
    for (int m = -K; m <= K; ++m) {
      int64_t q = k + m;
      if (q < 1 || q > N - 1) continue;
      s += gw[m + K] * raw[q];
      sw += gw[m + K];
    }
    w[k] = s / sw;
  }
}

/* One step of the modified third-order SSP-RK method (Eq. RK32D) with the width recursion
 * (Eq. Jacobi2D). State: E = eta bar, M = hu bar, B = b bar, J = cell widths, x = nodes.
 * prof[0..N] is the node profile of the prescribed motion. When alpha_io / dt_io are given
 * with replay = 1, the recorded dt and alpha are used (tangent-linear replay). */
/* L2 projection of the bottom on one cell (Eq. baverage; "a sufficiently accurate quadrature
 * rule"): on every piece the cell overlaps, the 5-point Gauss-Legendre rule (exact for the
 * degree <= 8 pieces) gives the piece's mean over the overlap, normalised by the sum of the
 * weights so that a constant piece averages to its value exactly; the cell average is the
 * length-weighted sum of these means. Quadrature, not differences of antiderivatives: those
 * cancel badly on short cells far from the breakpoint. */
double bottom_average(const OrcParams& P, double a, double c) {
  const double r1 = std::sqrt(5.0 - 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
  const double r2 = std::sqrt(5.0 + 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
  const double xi[5] = {-r2, -r1, 0.0, r1, r2};
  const double w1 = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0, w2 = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
  const double wq[5] = {w2, w1, 128.0 / 225.0, w1, w2};
  double s = 0.0;
  for (int p = 0; p < P.bpieces; ++p) {
    const double x0 = P.bbreaks[p], lo = std::max(a, x0), hi = std::min(c, P.bbreaks[p + 1]);
    if (!(hi > lo)) continue;
    double num = 0.0, den = 0.0;
    for (int q = 0; q < 5; ++q) {
      const double xq = 0.5 * (lo + hi) + 0.5 * (hi - lo) * xi[q];
      double v = 0.0;
      for (int k = 0; k <= P.bdeg; ++k) v += P.bcoef[p * (P.bdeg + 1) + k] * ipow(xq - x0, k);
      num += wq[q] * v;
      den += wq[q];
    }
    s += (hi - lo) * (num / den);
  }
  return s / (c - a);
}

template <class T>
uint32_t ssprk3_step(const OrcParams& P, int64_t N, T* E, T* M, T* B, double* J, double* x, const double* prof,
                     double* t, double* dt_out, uint8_t* flags, double* alpha_rec, int replay) {
  uint32_t st = 0;
  std::vector<EdgeVals<T>> ed;
  std::vector<double> w(N + 1, 0.0);
  double Wbar = 0.0;
  if (P.mesh == 2) {
    fluid_gauss_velocity(P, N, E, M, B, w);
    for (int64_t k = 0; k <= N; ++k) Wbar = std::max(Wbar, std::fabs(w[k]));
  } else if (P.mesh == 1) {
    double pm = 0.0;
    for (int64_t k = 0; k <= N; ++k) pm = std::max(pm, std::fabs(prof[k]));
    // Secant speeds of x = xi + P sin(2 pi t / T) are bounded by (2 pi / T) max |P|.
    Wbar = 2.0 * M_PI / P.mesh_T * pm;
  } else if (P.mesh == 3) {
    // Constant node velocities (Eq. velocity): the mesh of Eq. meshspecial moves on straight rays.
    for (int64_t k = 0; k <= N; ++k) {
      w[k] = prof[k];
      Wbar = std::max(Wbar, std::fabs(w[k]));
    }
  }
  // Eq. alpha2D takes the wave speeds relative to the mesh velocity. Stage 1 of the profile
  // motion cannot: its secant w depends on dt, which depends on alpha_1; there (and on request,
  // alpha_bound = 1) alpha is the bound max |u| + sqrt(g h) + Wbar (reading O4).
  const bool rel1 = !P.alpha_bound && P.mesh != 1, rel = !P.alpha_bound;

  // Stage 1 on the mesh at t_n.
  double A1 = reconstruct(P, N, E, M, B, J, ed, st, rel1 ? w.data() : nullptr);
  if (flags)
    for (int64_t j = 0; j < N; ++j) flags[j] = ed[j + 1].flag;
  double alpha1 = rel1 ? A1 : A1 + Wbar;
  double dt;
  if (replay) {
    dt = *dt_out;
    alpha1 = alpha_rec[0];
  } else if (P.dt_fixed > 0.0) {
    dt = P.dt_fixed;
  } else {
    double jmin = J[0];
    for (int64_t j = 1; j < N; ++j) jmin = std::min(jmin, J[j]);
    dt = P.cfl * jmin / alpha1;
    if (P.mesh == 2) {
      double dwmax = 0.0;
      for (int64_t j = 0; j < N; ++j) dwmax = std::max(dwmax, std::fabs(w[j + 1] - w[j]));
      if (dwmax > 0.0) dt = std::min(dt, 0.5 * jmin / dwmax);
    }
  }
  // The last step is clipped to t_end and then lands on it exactly.
  const bool clipped = P.t_end > 0.0 && P.t_end - *t <= dt;
  if (clipped && !replay) dt = P.t_end - *t;
  // alpha = 0 (a dry state at rest on a mesh that does not move) leaves the CFL condition with
  // no bound; without an end time to clip to there is no step to take (reading O21).
  if (!(dt < INFINITY)) {
    dt = 0.0;
    st |= ST_NODT;
  }
  if (P.mesh == 1 && dt > 0.0) {
    // Node speed (Eq. w1D): secant of the prescribed trajectory over [t_n, t_n + dt].
    const double s0 = std::sin(2.0 * M_PI * (*t) / P.mesh_T);
    const double s1 = std::sin(2.0 * M_PI * (*t + dt) / P.mesh_T);
    for (int64_t k = 0; k <= N; ++k) w[k] = prof[k] * (s1 - s0) / dt;
  }
  // Widths along the linear rays (Eq. Jacobi2D with div w J = w_{j+1/2} - w_{j-1/2}).
  std::vector<double> dw(N), J1(N), J2(N), J3(N);
  for (int64_t j = 0; j < N; ++j) {
    dw[j] = w[j + 1] - w[j];
    J1[j] = J[j] + dt * dw[j];
    J2[j] = 0.75 * J[j] + 0.25 * J1[j] + 0.25 * dt * dw[j];
    J3[j] = (1.0 / 3.0) * J[j] + (2.0 / 3.0) * J2[j] + (2.0 / 3.0) * dt * dw[j];
    if (!(J1[j] > 0.0) || !(J2[j] > 0.0) || !(J3[j] > 0.0)) st |= ST_EMESH;
  }
  std::vector<T> R_E(N), R_M(N), R_B(N), Y1E(N), Y1M(N), Y1B(N), Y2E(N), Y2M(N), Y2B(N);
  std::vector<T> qE(N), qM(N), qB(N);
  rhs(P, N, ed, E, M, B, J, w.data(), alpha1, R_E.data(), R_M.data(), R_B.data());
  for (int64_t j = 0; j < N; ++j) {
    Y1E[j] = T(J[j]) * E[j] + T(dt) * R_E[j];
    Y1M[j] = T(J[j]) * M[j] + T(dt) * R_M[j];
    Y1B[j] = T(J[j]) * B[j] + T(dt) * R_B[j];
    qE[j] = Y1E[j] / T(J1[j]);
    qM[j] = Y1M[j] / T(J1[j]);
    qB[j] = Y1B[j] / T(J1[j]);
  }
  // L2-projection mode: the bottom of stage 2 is the projection onto the mesh at t_{n+1}.
  if (P.bottom_mode == 1)
    for (int64_t j = 0; j < N; ++j) qB[j] = T(bottom_average(P, x[j] + dt * w[j], x[j + 1] + dt * w[j + 1]));
  // Stage 2 on the mesh at t_{n,1} = t_{n+1}.
  double A2 = reconstruct(P, N, qE.data(), qM.data(), qB.data(), J1.data(), ed, st, rel ? w.data() : nullptr);
  double alpha2 = replay ? alpha_rec[1] : (rel ? A2 : A2 + Wbar);
  rhs(P, N, ed, qE.data(), qM.data(), qB.data(), J1.data(), w.data(), alpha2, R_E.data(), R_M.data(), R_B.data());
  for (int64_t j = 0; j < N; ++j) {
    Y2E[j] = T(0.75) * (T(J[j]) * E[j]) + T(0.25) * (Y1E[j] + T(dt) * R_E[j]);
    Y2M[j] = T(0.75) * (T(J[j]) * M[j]) + T(0.25) * (Y1M[j] + T(dt) * R_M[j]);
    Y2B[j] = T(0.75) * (T(J[j]) * B[j]) + T(0.25) * (Y1B[j] + T(dt) * R_B[j]);
    qE[j] = Y2E[j] / T(J2[j]);
    qM[j] = Y2M[j] / T(J2[j]);
    qB[j] = Y2B[j] / T(J2[j]);
  }
  // ... and of stage 3 the projection onto the mesh at t_{n+1/2}.
  if (P.bottom_mode == 1)
    for (int64_t j = 0; j < N; ++j)
      qB[j] = T(bottom_average(P, x[j] + 0.5 * dt * w[j], x[j + 1] + 0.5 * dt * w[j + 1]));
  // Stage 3 on the mesh at t_{n,2} = (t_n + t_{n+1}) / 2.
  double A3 = reconstruct(P, N, qE.data(), qM.data(), qB.data(), J2.data(), ed, st, rel ? w.data() : nullptr);
  double alpha3 = replay ? alpha_rec[2] : (rel ? A3 : A3 + Wbar);
  rhs(P, N, ed, qE.data(), qM.data(), qB.data(), J2.data(), w.data(), alpha3, R_E.data(), R_M.data(), R_B.data());
  for (int64_t j = 0; j < N; ++j) {
    T Y3E = T(1.0 / 3.0) * (T(J[j]) * E[j]) + T(2.0 / 3.0) * (Y2E[j] + T(dt) * R_E[j]);
    T Y3M = T(1.0 / 3.0) * (T(J[j]) * M[j]) + T(2.0 / 3.0) * (Y2M[j] + T(dt) * R_M[j]);
    T Y3B = T(1.0 / 3.0) * (T(J[j]) * B[j]) + T(2.0 / 3.0) * (Y2B[j] + T(dt) * R_B[j]);
    E[j] = Y3E / T(J3[j]);
    M[j] = Y3M / T(J3[j]);
    B[j] = Y3B / T(J3[j]);
    J[j] = J3[j];
  }
  for (int64_t k = 0; k <= N; ++k) x[k] = x[k] + dt * w[k];
  // ... and after the step the projection onto the mesh at t_{n+1}.
  if (P.bottom_mode == 1)
    for (int64_t j = 0; j < N; ++j) B[j] = T(bottom_average(P, x[j], x[j + 1]));
  *t = clipped ? P.t_end : *t + dt;
  *dt_out = dt;
  if (alpha_rec && !replay) {
    alpha_rec[0] = alpha1;
    alpha_rec[1] = alpha2;
    alpha_rec[2] = alpha3;
  }
  return st;
}

OrcParams to_params(const double* p, const int32_t* ip) {
  OrcParams P;
  P.g = p[0]; P.cfl = p[1]; P.eps_weno = p[2]; P.eps_pp = p[3]; P.h_dry = p[4];
  P.mesh_T = p[5]; P.gauss_sigma = p[6]; P.t_end = p[7]; P.dt_fixed = p[8];
  P.bc = ip[0]; P.mesh = ip[1]; P.gauss_half = ip[2]; P.beta_dx_global = ip[3];
  P.bottom_mode = ip[4];
  P.scheme = ip[5];
  P.alpha_bound = ip[6];
  P.limit_hu = ip[7];
  P.bpieces = (int32_t)g_bbreaks.size() - 1;
  P.bdeg = g_bdeg;
  P.bbreaks = g_bbreaks.data();
  P.bcoef = g_bcoef.data();
  if (P.bottom_mode == 1 && P.bpieces < 1) P.bottom_mode = 0;
  return P;
}

}  // namespace

/* ------------------------------------------------------------------------------------ */
/* C entry points used by oracle/__init__.py (ctypes). Parameters are passed as a double  */
/* array p[9] = {g, cfl, eps_weno, eps_pp, h_dry, mesh_T, gauss_sigma, t_end, dt_fixed}   */
/* and an int array ip[8] = {bc, mesh, gauss_half, beta_dx_global, bottom_mode, scheme,    */
/* alpha_bound, limit_hu}.                                                                */
/* ------------------------------------------------------------------------------------ */
extern "C" {

/* Piecewise polynomial bottom b(x) of the L2-projection mode (ip[4] = 1): npieces pieces on
 * breaks[npieces + 1], piece p = sum_k coef[p (deg + 1) + k] (x - breaks[p])^k. */
void orc_set_bottom(int32_t npieces, int32_t deg, const double* breaks, const double* coef) {
  g_bbreaks.assign(breaks, breaks + npieces + 1);
  g_bcoef.assign(coef, coef + (size_t)npieces * (deg + 1));
  g_bdeg = deg;
}

/* Point data of one cell (weno_point): c[9], big[5], d[3] at unit coordinate t. */
void orc_weno_point(const double* w5, double t, double* c, double* big, double* d) {
  PointCoeffs Q;
  weno_point(w5, t, Q);
  std::memcpy(c, Q.c, sizeof(Q.c));
  std::memcpy(big, Q.big, sizeof(Q.big));
  std::memcpy(d, Q.d, sizeof(Q.d));
}

/* Hybrid weights at a point (point_phi) for linear weights d[3], indicators beta[3] and class
 * flag (gamma from beta as in Step 2). */
void orc_point_phi(const double* p, const int32_t* ip, const double* d, const double* beta, int32_t flag,
                   double* phi) {
  OrcParams P = to_params(p, ip);
  const double tau = std::fabs(beta[0] - beta[2]);
  const double gam = tau / ((beta[0] + beta[1] + beta[2]) / 3.0 + P.eps_weno);
  point_phi(P, d, beta, tau, gam, (uint8_t)flag, phi);
}

/* Average of the bottom over [a, c] (the projection of one cell). */
double orc_bottom_average(const double* p, const int32_t* ip, double a, double c) {
  OrcParams P = to_params(p, ip);
  return bottom_average(P, a, c);
}

/* Mesh-only WENO data of one cell from the five widths J_{j-2..j+2}: c[2][3][3], d[2][3],
 * big[2][5] (weights of the quartic at the two edges), sub[3][9] (coefficient maps). */
void orc_weno_coeffs(const double* w5, double* c, double* d, double* big, double* sub) {
  WenoCoeffs W;
  weno_coeffs(w5, W);
  std::memcpy(c, W.c, sizeof(W.c));
  std::memcpy(d, W.d, sizeof(W.d));
  std::memcpy(big, W.big, sizeof(W.big));
  std::memcpy(sub, W.sub, sizeof(W.sub));
}

/* Smoothness indicators beta_r (r = 0,1,2) of data v5 on widths w5 with lam = Dx / J_j. */
void orc_beta(const double* w5, const double* v5, double lam, double* beta) {
  WenoCoeffs W;
  weno_coeffs(w5, W);
  for (int r = 0; r < 3; ++r) beta[r] = beta_of(W, r, v5, lam);
}

/* Source-interpolant coefficient map (5 x 5) for neighbour width ratios rm, rp. */
void orc_source_map(double rm, double rp, double* map) { source_interp_map(rm, rp, map); }

/* Reconstruction + limiter of one stage. edges: 10 arrays of N+2 (cells -1..N):
 * E_L, E_R, M_L, M_R, B_L, B_R, h_L, h_R, u_L, u_R. flags[N+2], gamma[N+2].
 * Returns the largest edge wave speed |u| + sqrt(g h); status in *st. */
double orc_reconstruct(const double* p, const int32_t* ip, int64_t N, const double* E, const double* M,
                       const double* B, const double* J, double* edges, uint8_t* flags, double* gamma,
                       uint32_t* st) {
  OrcParams P = to_params(p, ip);
  std::vector<EdgeVals<double>> ed;
  uint32_t s = 0;
  double A = reconstruct(P, N, E, M, B, J, ed, s);
  const int64_t n2 = N + 2;
  for (int64_t i = 0; i < n2; ++i) {
    const EdgeVals<double>& o = ed[i];
    edges[0 * n2 + i] = o.E[0]; edges[1 * n2 + i] = o.E[1];
    edges[2 * n2 + i] = o.M[0]; edges[3 * n2 + i] = o.M[1];
    edges[4 * n2 + i] = o.B[0]; edges[5 * n2 + i] = o.B[1];
    edges[6 * n2 + i] = o.h[0]; edges[7 * n2 + i] = o.h[1];
    edges[8 * n2 + i] = o.u[0]; edges[9 * n2 + i] = o.u[1];
    if (flags) flags[i] = o.flag;
    if (gamma) gamma[i] = o.gamma;
  }
  if (st) *st = s;
  return A;
}

/* Semi-discrete right-hand side of one stage for given node velocities w[0..N] and alpha
 * (alpha <= 0: alpha of Eq. alpha2D, the largest |u - w| + sqrt(g h) over the edges; with
 * alpha_bound, the largest |u| + sqrt(g h) plus max |w|). *alpha_used: the alpha applied. */
uint32_t orc_rhs(const double* p, const int32_t* ip, int64_t N, const double* E, const double* M, const double* B,
                 const double* J, const double* w, double alpha, double* RE, double* RM, double* RB,
                 double* alpha_used) {
  OrcParams P = to_params(p, ip);
  std::vector<EdgeVals<double>> ed;
  uint32_t s = 0;
  double A = reconstruct(P, N, E, M, B, J, ed, s, P.alpha_bound ? nullptr : w);
  if (!(alpha > 0.0)) {
    double wb = 0.0;
    if (P.alpha_bound)
      for (int64_t k = 0; k <= N; ++k) wb = std::max(wb, std::fabs(w[k]));
    alpha = A + wb;
  }
  rhs(P, N, ed, E, M, B, J, w, alpha, RE, RM, RB);
  if (alpha_used) *alpha_used = alpha;
  return s;
}

/* nsteps steps (or until t reaches t_end > 0) of the fully discrete scheme, in place.
 * flags[N]: stage-1 flags of the last step (may be null). dts[nsteps], alphas[3*nsteps]:
 * recorded dt and stage alphas (may be null). Returns the OR of all status bits. */
uint32_t orc_run(const double* p, const int32_t* ip, int64_t N, double* E, double* M, double* B, double* J,
                 double* x, const double* prof, double* t, int64_t nsteps, int64_t* steps_done, uint8_t* flags,
                 double* dts, double* alphas) {
  OrcParams P = to_params(p, ip);
  uint32_t st = 0;
  int64_t n = 0;
  for (; n < nsteps; ++n) {
    if (P.t_end > 0.0 && *t >= P.t_end) break;
    double dt = 0.0, al[3] = {0, 0, 0};
    st |= ssprk3_step<double>(P, N, E, M, B, J, x, prof, t, &dt, flags, al, 0);
    if (dts) dts[n] = dt;
    if (alphas) { alphas[3 * n] = al[0]; alphas[3 * n + 1] = al[1]; alphas[3 * n + 2] = al[2]; }
    if (st & (ST_NONFINITE | ST_EMESH)) { ++n; break; }
  }
  if (steps_done) *steps_done = n;
  return st;
}

/* Node velocities of the fluid-driven motion (fluid_gauss_velocity) for the state (E, M, B):
 * w[N+1]. */
void orc_fluid_velocity(const double* p, const int32_t* ip, int64_t N, const double* E, const double* M,
                        const double* B, double* w) {
  OrcParams P = to_params(p, ip);
  std::vector<double> wv;
  fluid_gauss_velocity(P, N, E, M, B, wv);
  for (int64_t k = 0; k <= N; ++k) w[k] = wv[k];
}

/* nsteps steps of the fully discrete scheme in replay mode, in place: step n uses dts[n] and
 * the stage viscosities alphas[3n..3n+2] (as recorded by orc_run) instead of computing them.
 * The forward map that orc_tangent differentiates; finite differences of it check the tangent.
 * Returns the OR of all status bits. */
uint32_t orc_run_replay(const double* p, const int32_t* ip, int64_t N, double* E, double* M, double* B, double* J,
                        double* x, const double* prof, double* t, int64_t nsteps, const double* dts,
                        const double* alphas) {
  OrcParams P = to_params(p, ip);
  uint32_t st = 0;
  for (int64_t n = 0; n < nsteps; ++n) {
    double dt = dts[n];
    double al[3] = {alphas[3 * n], alphas[3 * n + 1], alphas[3 * n + 2]};
    st |= ssprk3_step<double>(P, N, E, M, B, J, x, prof, t, &dt, nullptr, al, 1);
  }
  return st;
}

/* The oracle's operation count (Cnt) of one stage's reconstruction + limiter on the state
 * (E, M, B, J) and of one whole SSP-RK3 step from it, summed over the N cells:
 * counts[0..3] = reconstruction (add, mul, div, sqrt), counts[4..7] = step. The state is not
 * changed. */
void orc_count_step(const double* p, const int32_t* ip, int64_t N, const double* E, const double* M,
                    const double* B, const double* J, const double* x, const double* prof, double* counts) {
  OrcParams P = to_params(p, ip);
  std::vector<Cnt> e(E, E + N), m(M, M + N), b(B, B + N);
  std::vector<double> Jc(J, J + N), xc(x, x + N + 1);
  std::vector<EdgeVals<Cnt>> ed;
  uint32_t st = 0;
  g_ops = OpCount();
  reconstruct(P, N, e.data(), m.data(), b.data(), Jc.data(), ed, st);
  const OpCount rec = g_ops;
  g_ops = OpCount();
  double t = 0.0, dt = 0.0, al[3];
  ssprk3_step<Cnt>(P, N, e.data(), m.data(), b.data(), Jc.data(), xc.data(), prof, &t, &dt, nullptr, al, 0);
  const OpCount stp = g_ops;
  const OpCount* c[2] = {&rec, &stp};
  for (int k = 0; k < 2; ++k) {
    counts[4 * k + 0] = (double)c[k]->add;
    counts[4 * k + 1] = (double)c[k]->mul;
    counts[4 * k + 2] = (double)c[k]->div;
    counts[4 * k + 3] = (double)c[k]->sqrt;
  }
}

/* Tangent-linear model of nsteps steps in replay mode: dt and the stage alphas are the
 * recorded ones (dts, alphas from orc_run), flags and limiter branches follow the base
 * trajectory. (dE, dM, dB) is the perturbation on entry and its image on exit. The mesh
 * is prescribed (static or profile motion), so widths and nodes carry no tangent. */
uint32_t orc_tangent(const double* p, const int32_t* ip, int64_t N, double* E, double* M, double* B, double* J,
                     double* x, const double* prof, double* t, int64_t nsteps, const double* dts,
                     const double* alphas, double* dE, double* dM, double* dB) {
  OrcParams P = to_params(p, ip);
  if (P.mesh == 2) return 0xffffffffu;  // fluid-driven motion would need tangent widths
  std::vector<Dual> e(N), m(N), b(N);
  for (int64_t j = 0; j < N; ++j) {
    e[j] = Dual(E[j], dE[j]);
    m[j] = Dual(M[j], dM[j]);
    b[j] = Dual(B[j], dB[j]);
  }
  uint32_t st = 0;
  for (int64_t n = 0; n < nsteps; ++n) {
    double dt = dts[n];
    double al[3] = {alphas[3 * n], alphas[3 * n + 1], alphas[3 * n + 2]};
    st |= ssprk3_step<Dual>(P, N, e.data(), m.data(), b.data(), J, x, prof, t, &dt, nullptr, al, 1);
  }
  for (int64_t j = 0; j < N; ++j) {
    E[j] = e[j].v; M[j] = m[j].v; B[j] = b[j].v;
    dE[j] = e[j].d; dM[j] = m[j].d; dB[j] = b[j].d;
  }
  return st;
}

}  // extern "C"
