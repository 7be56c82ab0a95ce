"""Oracle pins for the L2-projection bottom (Sec. 3.3, Eq. baverage) and the bump-aligned
mesh of the dam break over a rectangular bump (Sec. 5.1, Eq. bdam / wangge3)."""
import numpy as np
import pytest

import oracle
from paper_2208_06588_gb300 import workloads as W

RNG = np.random.default_rng(20220812 + 41)


def params_of(pr, **kw):
    d = dict(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, t_end=pr.t_end, dt_fixed=pr.dt_fixed,
             bc=pr.bc, mesh=pr.mesh, bottom=pr.meta.get("bottom"))
    d.update(kw)
    return oracle.Params(**d)


def test_projection_is_the_exact_average_of_a_piecewise_quartic():
    # Exact antiderivatives from numpy's polynomial class, not the oracle's own formula.
    breaks = np.sort(np.concatenate([[0.0, 10.0], RNG.uniform(0.5, 9.5, 5)]))
    coef = RNG.normal(size=(6, 5))
    P = oracle.Params(bottom=(breaks, coef))
    polys = [np.polynomial.Polynomial(c) for c in coef]
    for _ in range(200):
        a, c = np.sort(RNG.uniform(0.0, 10.0, 2))
        exact = 0.0
        for p, poly in enumerate(polys):
            lo, hi = max(a, breaks[p]), min(c, breaks[p + 1])
            if hi > lo:
                F = poly.integ()
                exact += F(hi - breaks[p]) - F(lo - breaks[p])
        got = oracle.bottom_average(P, a, c)
        assert got == pytest.approx(exact / (c - a), rel=1e-11, abs=1e-11)


def test_aligned_bump_stays_exact_and_mass_of_eta_is_conserved():
    pr = W.bump_dam_break(N=96, t_end=60.0)
    P = params_of(pr)
    st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    mass0 = float(np.sum(pr.J * pr.E))
    r = oracle.run(P, st, pr.profile, nsteps=30)
    assert r["steps"] == 30 and r["status"] == 0
    # the bump edges are nodes that never move, so every projected cell average is 0 or 8
    np.testing.assert_array_equal(st.B, pr.b)
    assert st.x[36] == 562.5 and st.x[60] == 937.5
    assert np.all(st.E - st.B > 0.0)
    # the waves have not reached the transmissive ends (sqrt(g 20) t < 750)
    assert 14.1 * st.t < 750.0
    assert abs(np.sum(st.J * st.E) - mass0) <= 1e-12 * mass0
    # the dam has started to break
    assert np.abs(st.M).max() > 1.0


def test_lake_at_rest_with_projected_polynomial_bottom_on_moving_mesh():
    N = 120
    x = np.linspace(0.0, 10.0, N + 1)
    coef = np.array([[0.0, 0.0, 4.0 * 100 / 625, -4.0 * 20 / 625, 4.0 / 625]])  # 4 x^2 (10 - x)^2 / 625
    P = oracle.Params(bc="transmissive", mesh="profile", mesh_T=0.5, cfl=0.6, bottom=(np.array([0.0, 10.0]), coef))
    b = np.array([oracle.bottom_average(P, x[j], x[j + 1]) for j in range(N)])
    E = np.full(N, 10.0)
    prof = (x - 10.0) * x / (3.0 * 100.0)
    st = oracle.State(E, np.zeros(N), b, np.diff(x), x)
    r = oracle.run(P, st, prof, nsteps=40)
    assert r["steps"] == 40 and r["status"] == 0
    assert np.abs(st.E - 10.0).max() < 1e-12
    assert np.abs(st.M).max() < 1e-11
    # the bottom follows the mesh: projection of b on the final nodes
    bn = np.array([oracle.bottom_average(P, st.x[j], st.x[j + 1]) for j in range(N)])
    np.testing.assert_array_equal(st.B, bn)
    assert np.abs(st.x - x).max() > 1e-3  # the mesh did move
