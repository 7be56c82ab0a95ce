"""Pins of the oracle's reconstruction pieces against mathematics the paper relies on.

* Step 1 of Sec. 2.2 on a uniform mesh reduces to the textbook fifth-order WENO coefficients
  and linear weights (Jiang & Shu 1996).
* On any nonuniform mesh each sub-stencil polynomial reproduces quadratics and the linear
  weights reproduce quartics (exact cell averages computed here from antiderivatives).
* Step 2's smoothness indicators equal the textbook closed form on a uniform mesh and the
  defining integral (computed here via Shu's primitive-function construction + quadrature)
  on nonuniform meshes.
* The source interpolant (Sec. 4.1) reproduces quartics and makes the source balance the
  pressure jump at rest exactly (the lemma of Sec. 4.3).
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(20220812)


def _nodes(w5):
    w5 = np.asarray(w5, float)
    y = np.concatenate([[0.0], np.cumsum(w5)])
    return y - y[2]  # x_{j-1/2} at 0


def _avgs(coef, y):
    """Exact cell averages of the polynomial sum_k coef[k] x^k over [y_i, y_{i+1}]."""
    P = np.polynomial.polynomial.polyint(coef)
    V = np.polynomial.polynomial.polyval(y, P)
    return np.diff(V) / np.diff(y)


def test_uniform_coefficients_are_textbook_weno5():
    c = oracle.weno_coeffs([1, 1, 1, 1, 1])
    right = np.array([[1 / 3, 5 / 6, -1 / 6], [-1 / 6, 5 / 6, 1 / 3], [1 / 3, -7 / 6, 11 / 6]])
    left = np.array([[11 / 6, -7 / 6, 1 / 3], [1 / 3, 5 / 6, -1 / 6], [-1 / 6, 5 / 6, 1 / 3]])
    np.testing.assert_allclose(c["c"][1], right, atol=1e-14)
    np.testing.assert_allclose(c["c"][0], left, atol=1e-14)
    np.testing.assert_allclose(c["d"][1], [3 / 10, 3 / 5, 1 / 10], atol=1e-14)
    np.testing.assert_allclose(c["d"][0], [1 / 10, 3 / 5, 3 / 10], atol=1e-14)


def test_coefficients_scale_invariant():
    w5 = RNG.uniform(0.5, 2.0, 5)
    a, b = oracle.weno_coeffs(w5), oracle.weno_coeffs(7.3e-5 * w5)
    np.testing.assert_allclose(a["c"], b["c"], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(a["d"], b["d"], rtol=1e-11)


@pytest.mark.parametrize("trial", range(20))
def test_polynomial_reproduction_nonuniform(trial):
    w5 = RNG.uniform(0.4, 2.5, 5)
    y = _nodes(w5)
    h0 = w5[2]
    co = oracle.weno_coeffs(w5)
    # Quadratics: every sub-stencil polynomial is exact at both edges.
    q = RNG.normal(size=3)
    ub = _avgs(q, y)
    for e, xe in ((0, 0.0), (1, h0)):
        exact = np.polynomial.polynomial.polyval(xe, q)
        for r in range(3):
            val = co["c"][e][r] @ ub[2 - r:5 - r]
            assert abs(val - exact) < 1e-11 * (1 + abs(exact))
    # Quartics: the linear weights combine the three quadratics into the quartic's value.
    q4 = RNG.normal(size=5)
    ub = _avgs(q4, y)
    for e, xe in ((0, 0.0), (1, h0)):
        exact = np.polynomial.polynomial.polyval(xe, q4)
        comb = sum(co["d"][e][r] * (co["c"][e][r] @ ub[2 - r:5 - r]) for r in range(3))
        assert abs(comb - exact) < 1e-10 * (1 + abs(exact))
        assert abs(co["big"][e] @ ub - exact) < 1e-10 * (1 + abs(exact))
    # Linear weights satisfy all five matching equations, not only the two used to fix them.
    for e in range(2):
        tot = np.zeros(5)
        for r in range(3):
            tot[2 - r:5 - r] += co["d"][e][r] * co["c"][e][r]
        np.testing.assert_allclose(tot, co["big"][e], atol=1e-10)


def test_beta_uniform_is_jiang_shu():
    for _ in range(10):
        u = RNG.normal(size=5)
        b = oracle.beta([1, 1, 1, 1, 1], u, 1.0)
        um2, um1, u0, up1, up2 = u
        b0 = 13 / 12 * (u0 - 2 * up1 + up2) ** 2 + 0.25 * (3 * u0 - 4 * up1 + up2) ** 2
        b1 = 13 / 12 * (um1 - 2 * u0 + up1) ** 2 + 0.25 * (um1 - up1) ** 2
        b2 = 13 / 12 * (um2 - 2 * um1 + u0) ** 2 + 0.25 * (um2 - 4 * um1 + 3 * u0) ** 2
        np.testing.assert_allclose(b, [b0, b1, b2], rtol=1e-12, atol=1e-14)


def test_beta_nonuniform_matches_defining_integral():
    from scipy.integrate import quad
    for _ in range(8):
        w5 = RNG.uniform(0.5, 2.0, 5) * 0.01
        dx = 0.03  # global cell length (>= every width here)
        y = _nodes(w5)
        u = RNG.normal(size=5)
        b = oracle.beta(w5, u, dx / w5[2])
        for r in range(3):
            # Primitive-function construction: cubic through V(y_m) on the sub-stencil nodes.
            ys = y[2 - r:6 - r]
            V = np.concatenate([[0.0], np.cumsum(u[2 - r:5 - r] * np.diff(ys))])
            cub = np.polynomial.polynomial.polyfit(ys, V, 3)
            p = np.polynomial.polynomial.polyder(cub)
            d1, d2 = np.polynomial.polynomial.polyder(p), np.polynomial.polynomial.polyder(p, 2)
            i1 = quad(lambda s: np.polynomial.polynomial.polyval(s, d1) ** 2, 0, w5[2])[0]
            i2 = quad(lambda s: np.polynomial.polynomial.polyval(s, d2) ** 2, 0, w5[2])[0]
            ref = dx * i1 + dx ** 3 * i2
            assert abs(b[r] - ref) <= 1e-8 * abs(ref) + 1e-14


def test_source_interpolant_reproduces_quartics():
    for _ in range(10):
        rm, rp = RNG.uniform(0.3, 3.0, 2)
        m = oracle.source_map(rm, rp)
        q = RNG.normal(size=5)
        y = np.array([-rm, 0.0, 1.0, 1.0 + rp])
        data = np.concatenate([_avgs(q, y), [np.polynomial.polynomial.polyval(0.0, q),
                                              np.polynomial.polynomial.polyval(1.0, q)]])
        np.testing.assert_allclose(m @ data, q, atol=1e-10)


def test_source_balances_pressure_jump_at_rest():
    """Lemma of Sec. 4.3: at rest (eta = c, hu = 0) the momentum residual vanishes cell by
    cell on a random moving-mesh-like grid with a rough bottom."""
    N = 40
    x = np.concatenate([[0.0], np.cumsum(RNG.uniform(0.5, 1.5, N))])
    J = np.diff(x)
    B = RNG.uniform(0.0, 3.0, N)
    E = np.full(N, 5.0)
    M = np.zeros(N)
    w = RNG.normal(size=N + 1) * 0.1
    for bc in ("periodic", "transmissive", "reflective"):
        P = oracle.Params(bc=bc)
        RE, RM, RB, alpha, st = oracle.rhs(P, E, M, B, J, w, alpha=20.0)
        assert np.abs(RM).max() < 1e-11 * 5.0 ** 2 * 9.812
        # eta-flux at rest is -w c, so R_E = c (w_{j+1} - w_j) (D-GCL for eta).
        assert np.abs(RE - 5.0 * np.diff(w)).max() < 1e-12


def test_limiter_keeps_mean_and_clears_floor():
    """Bound-preserving limiter (Eq. modifiedhjn in 1D): after limiting, the Gauss-Lobatto
    mean (h_L + h_R)/12 + 10/12 delta reproduces the cell mean and all three values are
    >= min(1e-11, hbar); untouched where already positive."""
    N = 30
    x = np.linspace(0, 1, N + 1)
    h = np.where(np.arange(N) < 15, 2.0, 0.0)
    h[15] = 1e-3
    B = 0.1 * np.sin(3 * x[:-1])
    E = h + B
    M = np.where(np.arange(N) < 15, 0.5, 0.0)
    ed, flags, gam, A, st = oracle.reconstruct(oracle.Params(bc="transmissive"), E, M, B, np.diff(x))
    hL, hR = ed["h_L"][1:-1], ed["h_R"][1:-1]
    delta = (12 * h - hL - hR) / 10
    assert np.all(hL >= -1e-15) and np.all(hR >= -1e-15) and np.all(delta >= -1e-14)
    # Remark of Sec. 4.3: bottom edge values are re-derived as eta - h.
    np.testing.assert_allclose(ed["B_L"][1:-1], ed["E_L"][1:-1] - hL, atol=1e-14)
    np.testing.assert_allclose((hL + hR) / 12 + 10 / 12 * delta, h, atol=1e-13)
    assert st == 0
