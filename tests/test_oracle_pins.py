"""Pins of three oracle parts that the whole-scheme tests cannot tell apart from plausible
mistakes (no GPU):

* the smoothness detector and the hybrid weights of Sec. 2.2 (Step 2: Eq. alphamodified with
  shared indicators of h and hu; Step 3: Eq. omegaj / omegajjj, the WENO-Z weights with the
  squared ratio tau / (beta + eps), the transition blend M(gamma) = 2 gamma - 1), checked cell
  by cell against an independent numpy construction from the Jiang-Shu closed-form indicators
  and the textbook fifth-order sub-stencil edge values on a uniform mesh;
* the fluid-driven node velocity (a Gaussian-smoothed copy of the fluid velocity, sigma = 8
  cells, truncated at +-24 nodes and renormalised; end nodes fixed), checked against a numpy
  convolution of the raw node velocities and of the window mask;
* the tangent-linear model (the oracle's dual-number instantiation), checked against central
  differences of the oracle's own replayed forward run (dt and the stage viscosities held at
  their recorded values) on a smooth and a wet/dry problem.
"""
import numpy as np
import pytest

import oracle
from paper_2208_06588_gb300 import workloads as W

EPS = 1e-6  # epsilon of Step 2 (the paper's value)


# ------------------------------------------------------------------------------------------
# Detector and hybrid weights on a uniform mesh
# ------------------------------------------------------------------------------------------
def _js_betas(v):
    """Jiang-Shu indicators of the three sub-stencils of a 5-cell stencil v[0..4] (cell j is
    v[2]); index r as in the oracle: sub-stencil r holds cells j-r .. j-r+2."""
    a, b, c, d, e = v
    b0 = 13 / 12 * (c - 2 * d + e) ** 2 + 0.25 * (3 * c - 4 * d + e) ** 2  # cells j .. j+2
    b1 = 13 / 12 * (b - 2 * c + d) ** 2 + 0.25 * (b - d) ** 2              # cells j-1 .. j+1
    b2 = 13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2  # cells j-2 .. j
    return np.array([b0, b1, b2])


def _textbook_edges(v):
    """Sub-stencil values p_r at the left edge x_{j-1/2} and the right edge x_{j+1/2} (uniform)."""
    a, b, c, d, e = v
    right = np.array([(2 * c + 5 * d - e) / 6, (-b + 5 * c + 2 * d) / 6, (2 * a - 7 * b + 11 * c) / 6])
    left = np.array([(11 * c - 7 * d + 2 * e) / 6, (2 * b + 5 * c - d) / 6, (-a + 5 * b + 2 * c) / 6])
    return left, right


D_LEFT = np.array([0.1, 0.6, 0.3])
D_RIGHT = np.array([0.3, 0.6, 0.1])


def _reference(E, M, B, bc="periodic"):
    """gamma, class and the edge values of eta and hu for cells -1..N, built here from the
    closed forms (Step 2 shared over h = eta - b and hu; Step 3 weights; Step 4 edge values)."""
    N = E.size
    out = {"gamma": [], "flag": [], "E_L": [], "E_R": [], "M_L": [], "M_R": []}
    for j in range(-1, N + 1):
        idx = [(j + k) % N for k in range(-2, 3)]
        e5, m5, b5 = E[idx], M[idx], B[idx]
        beta = _js_betas(e5 - b5) + _js_betas(m5)
        tau = abs(beta[0] - beta[2])
        gam = tau / (beta.mean() + EPS)
        flag = 0 if gam <= 0.5 else (2 if gam >= 1.0 else 1)
        out["gamma"].append(gam)
        out["flag"].append(flag)
        for side, d in (("L", D_LEFT), ("R", D_RIGHT)):
            if flag == 0:
                phi = d
            else:
                a = d * (1.0 + (tau / (beta + EPS)) ** 2)
                phi = a / a.sum()
                if flag == 1:
                    Mg = 2.0 * gam - 1.0
                    phi = Mg * phi + (1.0 - Mg) * d
            le, re = _textbook_edges(e5)
            lm, rm = _textbook_edges(m5)
            out["E_" + side].append(phi @ (le if side == "L" else re))
            out["M_" + side].append(phi @ (lm if side == "L" else rm))
    return {k: np.array(v) for k, v in out.items()}


def _recon(E, M, B, bc="periodic"):
    N = E.size
    J = np.full(N, 1.0 / N)
    return oracle.reconstruct(oracle.Params(eps_weno=EPS, bc=bc), E, M, B, J)


def test_detector_zero_on_constant_data():
    N = 16
    E, M, B = np.full(N, 3.0), np.full(N, 0.7), np.full(N, 1.25)
    edges, flags, gam, A, st = _recon(E, M, B)
    assert st == 0
    # zero up to the rounding of the Gaussian elimination that builds the coefficient maps
    assert np.all(np.abs(gam) < 1e-20) and np.all(flags == 0)
    np.testing.assert_allclose(edges["E_L"], 3.0, rtol=1e-15)
    np.testing.assert_allclose(edges["M_R"], 0.7, rtol=1e-15)


def test_detector_zero_on_linear_data():
    """All three Jiang-Shu indicators of linear data equal the squared slope, so tau = 0 and
    gamma = 0 in every cell whose stencil lies inside the domain."""
    N = 24
    i = np.arange(N, dtype=float)
    E = 4.0 + 0.05 * i            # h = eta - b linear as well
    B = 0.5 + 0.01 * i
    M = -0.3 + 0.02 * i
    edges, flags, gam, A, st = _recon(E, M, B, bc="transmissive")
    inner = slice(3, N - 1)  # cells 2 .. N-3 in the edge layout (cell -1 at index 0)
    assert np.all(np.abs(gam[inner]) < 1e-9)
    assert np.all(flags[inner] == 0)
    # exact reconstruction of linear data at the edges (x_{j-1/2}: the mean of the two cells)
    np.testing.assert_allclose(edges["E_L"][inner], 4.0 + 0.05 * (np.arange(2, N - 2) - 0.5), rtol=1e-13)


def test_detector_nonsmooth_across_a_jump():
    N = 32
    E = np.where(np.arange(N) < N // 2, 3.0, 1.5)
    B = np.zeros(N)
    M = np.zeros(N)
    edges, flags, gam, A, st = _recon(E, M, B, bc="transmissive")
    c = N // 2 + 1  # edge layout index of cell N/2
    # the two cells next to the jump see it in the middle of their stencil
    assert flags[c - 1] == 2 and flags[c] == 2
    assert gam[c - 1] > 1.0 and gam[c] > 1.0
    # far from the jump the data are constant
    assert flags[3] == 0 and flags[N - 3] == 0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_hybrid_weights_match_closed_forms(seed):
    """Random data on a uniform periodic mesh put cells in all three classes, including gamma
    in (1/3, 1/2) and (1/2, 1); gamma, the class and the edge values of eta and hu must equal
    the numpy construction cell by cell."""
    rng = np.random.default_rng(20220812 + seed)
    N = 96
    x = np.arange(N) / N
    B = 0.3 + 0.2 * np.sin(2 * np.pi * x)
    h = 2.0 + 0.6 * np.sin(4 * np.pi * x) + rng.uniform(-0.35, 0.35, N) * (rng.random(N) < 0.5)
    E = h + B
    M = 0.5 * np.cos(2 * np.pi * x) + rng.uniform(-0.2, 0.2, N)
    edges, flags, gam, A, st = _recon(E, M, B)
    ref = _reference(E, M, B)
    assert st == 0
    # the limiter is inactive (all edge depths well positive), so the edge values are Step 4's
    assert min(edges["h_L"].min(), edges["h_R"].min()) > 0.5
    g = ref["gamma"]
    # the data reach every class and both sides of the 1/2 threshold
    assert np.sum((g > 1 / 3) & (g < 0.5)) >= 3
    assert np.sum((g > 0.5) & (g < 1.0)) >= 5
    assert np.sum(g >= 1.0) >= 5 and np.sum(g <= 0.5) >= 5
    # no cell within 1e-9 of a threshold (else the class may legitimately differ by rounding)
    assert np.min(np.abs(g - 0.5)) > 1e-9 and np.min(np.abs(g - 1.0)) > 1e-9
    np.testing.assert_array_equal(flags, ref["flag"])
    np.testing.assert_allclose(gam, g, rtol=1e-13, atol=1e-15)
    for k in ("E_L", "E_R", "M_L", "M_R"):
        np.testing.assert_allclose(edges[k], ref[k], rtol=1e-13, atol=1e-13, err_msg=k)


def test_transition_blend_direction():
    """In the transition class the blend leans to the WENO-Z weights as gamma -> 1 and to the
    linear weights as gamma -> 1/2: a cell with gamma close to 1/2 keeps its edge value close to
    the linear-weight value."""
    N = 96
    rng = np.random.default_rng(7)
    x = np.arange(N) / N
    B = np.zeros(N)
    E = 2.0 + 0.6 * np.sin(4 * np.pi * x) + rng.uniform(-0.35, 0.35, N) * (rng.random(N) < 0.5)
    M = rng.uniform(-0.2, 0.2, N)
    edges, flags, gam, A, st = _recon(E, M, B)
    ref = _reference(E, M, B)
    tr = np.where(flags == 1)[0]
    assert tr.size > 0
    for c in tr:
        j = c - 1
        idx = [(j + k) % N for k in range(-2, 3)]
        le, re = _textbook_edges(E[idx])
        lin = D_RIGHT @ re
        gm = gam[c]
        # |edge - linear| = (2 gamma - 1) |phiN . p - d . p| <= (2 gamma - 1) max_r |p_r - lin|
        assert abs(edges["E_R"][c] - lin) <= (2 * gm - 1) * np.max(np.abs(re - lin)) + 1e-13
    np.testing.assert_allclose(edges["E_R"], ref["E_R"], rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------------------------------
# Fluid-driven node velocity
# ------------------------------------------------------------------------------------------
def _gauss_reference(u, sigma=8.0, half=24):
    """w_k for k = 1..N-1: the truncated Gaussian average of raw_k = (u_{k-1} + u_k) / 2 over
    the nodes 1..N-1 of the window, renormalised by the weights that fall inside; w_0 = w_N = 0."""
    N = u.size
    raw = np.zeros(N + 1)
    raw[1:N] = 0.5 * (u[:-1] + u[1:])
    mask = np.zeros(N + 1)
    mask[1:N] = 1.0
    m = np.arange(-half, half + 1)
    g = np.exp(-m.astype(float) ** 2 / (2 * sigma ** 2))
    num = np.convolve(raw * mask, g, mode="same")
    den = np.convolve(mask, g, mode="same")
    w = np.where(mask > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return w


def _fluid(E, M, B, **kw):
    return oracle.fluid_velocity(oracle.Params(mesh="fluid_gauss", bc="transmissive", **kw), E, M, B)


def test_fluid_velocity_of_a_uniform_flow():
    """A uniform velocity u = 0.37 over a varying depth gives w = u at every interior node,
    including those whose window is truncated by the ends, and w = 0 at the two end nodes."""
    N = 120
    x = np.arange(N) / N
    B = 0.2 * np.sin(3 * x)
    h = 1.0 + 0.5 * np.cos(5 * x)
    E, M = h + B, 0.37 * h
    w = _fluid(E, M, B)
    assert w[0] == 0.0 and w[N] == 0.0
    np.testing.assert_allclose(w[1:N], 0.37, rtol=1e-14)


def test_fluid_velocity_matches_truncated_gaussian():
    """Random velocities: every node, near the ends (renormalised window) and inside, equals
    the numpy convolution."""
    rng = np.random.default_rng(11)
    N = 150
    B = rng.uniform(0.0, 0.3, N)
    h = rng.uniform(0.5, 2.0, N)
    u = rng.normal(size=N)
    w = _fluid(h + B, u * h, B)
    np.testing.assert_allclose(w, _gauss_reference(u), rtol=1e-13, atol=1e-15)
    # a linear velocity field is kept exactly where the window is whole and symmetric
    u2 = 0.01 * np.arange(N)
    w2 = _fluid(h + B, u2 * h, B)
    k = np.arange(25, N - 24)
    np.testing.assert_allclose(w2[k], 0.01 * (k - 0.5), rtol=1e-12)
    # ... and not near a wall, where the window is one-sided
    assert abs(w2[3] - 0.01 * 2.5) > 1e-3


def test_fluid_velocity_other_widths():
    rng = np.random.default_rng(12)
    N = 90
    B = np.zeros(N)
    h = rng.uniform(0.5, 2.0, N)
    u = rng.normal(size=N)
    w = _fluid(h, u * h, B, gauss_sigma=3.0, gauss_half=9)
    np.testing.assert_allclose(w, _gauss_reference(u, 3.0, 9), rtol=1e-13, atol=1e-15)


def test_fluid_velocity_dry_cells_carry_no_velocity():
    """Cells whose mean depth is at most h_dry contribute u = 0 (not hu / h)."""
    rng = np.random.default_rng(13)
    N = 100
    B = np.zeros(N)
    h = rng.uniform(0.5, 2.0, N)
    h[40:55] = 5e-7  # below h_dry = 1e-6
    M = rng.normal(size=N) * h
    M[40:55] = 3e-7  # would give u = 0.6 if divided
    u = np.where(h > 1e-6, M / h, 0.0)
    w = _fluid(h, M, B)
    np.testing.assert_allclose(w, _gauss_reference(u), rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------------------------------
# Tangent-linear model against central differences of the replayed forward run
# ------------------------------------------------------------------------------------------
def _params_of(pr, **kw):
    d = dict(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, bc=pr.bc, mesh=pr.mesh, mesh_T=pr.mesh_T, t_end=0.0)
    d.update(kw)
    return oracle.Params(**d)


def _tangent_vs_fd(pr, nsteps, direction, eps, **kw):
    P = _params_of(pr, **kw)
    base = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    rec = oracle.run(P, base.copy(), pr.profile, nsteps=nsteps, record=True)
    assert rec["steps"] == nsteps
    dE, dM, dB = direction
    tE, tM, tB, st = oracle.tangent(P, base.copy(), pr.profile, rec["dts"], rec["alphas"], dE, dM, dB)
    assert st == 0 or st == oracle.ST_NEGDEPTH

    def fwd(s):
        y = oracle.State(pr.E + s * dE, pr.hu + s * dM, pr.b + s * dB, pr.J, pr.x)
        oracle.run_replay(P, y, pr.profile, rec["dts"], rec["alphas"])
        return y

    p, m = fwd(eps), fwd(-eps)
    fd = [(p.E - m.E) / (2 * eps), (p.M - m.M) / (2 * eps), (p.B - m.B) / (2 * eps)]
    return [tE, tM, tB], fd


def _smooth_dir(N, rng, scale=1.0):
    x = (np.arange(N) + 0.5) / N
    return [scale * np.sin(2 * np.pi * (x + rng.random())) + 0.3 * scale * np.cos(6 * np.pi * x),
            scale * np.cos(2 * np.pi * (x + rng.random())),
            0.2 * scale * np.sin(4 * np.pi * (x + rng.random()))]


def test_tangent_matches_central_differences_smooth():
    """Accuracy test of Sec. 5.1 (periodic, moving mesh), 6 replayed steps."""
    pr = W.accuracy_test(48)
    rng = np.random.default_rng(5)
    tan, fd = _tangent_vs_fd(pr, 6, _smooth_dir(pr.N, rng), 1e-6)
    for a, b, name in zip(tan, fd, "EMB"):
        scale = np.abs(a).max()
        assert scale > 0.1
        assert np.abs(a - b).max() <= 1e-7 * scale, name


def test_tangent_matches_central_differences_wet_dry():
    """Moses's second problem (a dry region between two water columns, moving mesh): the
    limiter acts at the wet/dry fronts. The perturbation is confined to the wet cells, so
    no dry edge becomes wet within +-eps and the frozen branches of the replay hold."""
    pr = W.moses_second(N=80, moving=True)
    rng = np.random.default_rng(6)
    d = _smooth_dir(pr.N, rng, scale=0.5)
    wet = pr.h > 1e-3
    d = [v * wet for v in d]
    d[2] = np.zeros(pr.N)  # flat bottom: keep it flat
    tan, fd = _tangent_vs_fd(pr, 8, d, 1e-6)
    for a, b, name in zip(tan[:2], fd[:2], "EM"):
        scale = np.abs(a).max()
        assert scale > 0.1
        assert np.abs(a - b).max() <= 1e-7 * scale, name
    # the limiter was active in these steps: the front cells carry the tangent too
    front = np.where(~wet)[0]
    assert np.abs(tan[0][front]).max() > 1e-6 * np.abs(tan[0]).max()


def test_tangent_is_linear_in_the_direction():
    """T(a u + b v) = a T(u) + b T(v) (the model is linear; a sign error in one branch of a
    kink would break the finite-difference tests above, this one pins superposition)."""
    pr = W.accuracy_test(32)
    rng = np.random.default_rng(8)
    P = _params_of(pr)
    base = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    rec = oracle.run(P, base.copy(), pr.profile, nsteps=3, record=True)
    u, v = _smooth_dir(pr.N, rng), _smooth_dir(pr.N, rng)
    Tu = oracle.tangent(P, base.copy(), pr.profile, rec["dts"], rec["alphas"], *u)[:3]
    Tv = oracle.tangent(P, base.copy(), pr.profile, rec["dts"], rec["alphas"], *v)[:3]
    w = [2.0 * a - 0.5 * b for a, b in zip(u, v)]
    Tw = oracle.tangent(P, base.copy(), pr.profile, rec["dts"], rec["alphas"], *w)[:3]
    for a, b, c in zip(Tu, Tv, Tw):
        np.testing.assert_allclose(c, 2.0 * a - 0.5 * b, rtol=1e-12, atol=1e-12 * np.abs(c).max())
