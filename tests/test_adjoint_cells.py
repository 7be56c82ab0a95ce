"""Dot-product checks of the hand-written reverse sweeps of the per-cell arithmetic (no GPU):
for random directions u and adjoint seeds ob, <ob, T u> from a forward-mode dual-number build
of the same per-cell code must equal <T^T ob, u> from the reverse sweep, in every branch the
scheme has (smooth / transition / non-smooth classes, limiter on / off, wet / dry edges)."""
import numpy as np
import pytest

from tests import cellcheck as C

RNG = np.random.default_rng(424242)
PRM = np.array([9.812, 1e-6, 1e-11, 1e-6, 0.0, 0.0])  # g, eps, eps_pp, h_dry, dxmax, limit_hu


def stencil(E, M, B, h):
    """v0 (averages of cells j-2..j) and the divided differences of the big stencil."""
    v = np.stack([E, M, B])
    ip = 1.0 / (h[:-1] + h[1:])
    D2 = (v[:, 1:] - v[:, :-1]) * ip
    it = 1.0 / (h[:-2] + h[1:-1] + h[2:])
    D3 = (D2[:, 1:] - D2[:, :-1]) * it
    return v[:, :3].ravel(), D2.ravel(), D3.ravel()


def cases():
    out = []
    for k in range(60):
        h = RNG.uniform(0.5, 1.5, 5) * 0.01
        x = np.cumsum(h) - h[0]
        kind = k % 6
        if kind == 0:    # smooth, deep
            B = 0.3 * np.sin(x * 30); E = 2.0 + 0.01 * np.cos(x * 40) + B * 0; M = 0.4 + 0.1 * x
        elif kind == 1:  # jump in the surface
            B = 0.2 * x; E = np.where(np.arange(5) < 2 + (k % 3), 2.0, 1.0) + B; M = 0.3 * np.ones(5)
        elif kind == 2:  # mild kink (transition)
            B = 0.1 * np.ones(5); E = 1.5 + 0.02 * np.abs(np.arange(5) - 2.0 + 0.3 * RNG.normal()); M = 0.1 * x
        elif kind == 3:  # wet / dry front (limiter active)
            B = np.zeros(5); E = np.array([1.0, 0.6, 1e-4, 0.0, 0.0])[::(1 if k % 2 else -1)]; M = 0.2 * E
        elif kind == 4:  # near-dry cell with steep neighbours
            B = np.array([0.0, 0.1, 0.5, 0.9, 1.2]); E = B + np.array([1.0, 0.5, 2e-3, 0.0, 0.0]); M = 0.05 * (E - B)
        else:            # random rough data
            B = RNG.uniform(0, 0.5, 5); E = B + RNG.uniform(0.0, 1.0, 5); M = RNG.normal(size=5) * 0.3
        E = E + 1e-3 * RNG.normal(size=5) * (kind not in (3, 4))
        out.append((h, E, M, B))
    return out


@pytest.mark.parametrize("limit_hu", [0, 1])
@pytest.mark.parametrize("case", range(60))
def test_recon_reverse_matches_tangent(case, limit_hu):
    h, E, M, B = cases()[case]
    v0, D2, D3 = stencil(E, M, B, h)
    prm = PRM.copy()
    prm[4] = 0.015
    prm[5] = limit_hu
    tv0, tD2, tD3 = RNG.normal(size=9), RNG.normal(size=12), RNG.normal(size=9)
    ob = RNG.normal(size=8)
    val, tan, flag = C.recon_tangent(h, v0, D2, D3, tv0, tD2, tD3, prm)
    v0b, D2b, D3b = C.recon_adjoint(h, v0, D2, D3, prm, ob)
    lhs = ob @ tan
    rhs = v0b @ tv0 + D2b @ tD2 + D3b @ tD3
    scale = np.abs(ob * tan).sum() + np.abs(v0b * tv0).sum() + np.abs(D2b * tD2).sum() + np.abs(D3b * tD3).sum()
    assert abs(lhs - rhs) <= 1e-12 * scale + 1e-300, (flag, lhs, rhs)


@pytest.mark.parametrize("limit_hu", [0, 1])
def test_recon_reverse_known_smooth_is_the_same_sweep(limit_hu):
    """The device skips the FP64 indicators of the reverse where the forward's FP32 test shows
    the smooth class: in every class-0 case the sweep with the class given is bit for bit the
    sweep that forms the indicators (and leaves the third-difference adjoints at 0)."""
    n0 = 0
    for case in range(60):
        h, E, M, B = cases()[case]
        v0, D2, D3 = stencil(E, M, B, h)
        prm = PRM.copy()
        prm[4] = 0.015
        prm[5] = limit_hu
        flag = C.recon_tangent(h, v0, D2, D3, np.zeros(9), np.zeros(12), np.zeros(9), prm)[2]
        if flag != 0:
            continue
        n0 += 1
        ob = RNG.normal(size=8)
        full = C.recon_adjoint(h, v0, D2, D3, prm, ob)
        known = C.recon_adjoint(h, v0, D2, D3, prm, ob, known_smooth=True)
        for a, b in zip(full, known):
            assert np.array_equal(a, b)
        assert not known[2].any()
    assert n0 >= 10


@pytest.mark.parametrize("limit_hu", [0, 1])
def test_recon_reverse_from_the_stored_linear_form(limit_hu):
    """The reverse reconstruction of a smooth-class cell from the linear form that the forward's
    own geometry gives (the form the forward recompute of the adjoint stores) is the reverse sweep
    that recomputes the geometry, to rounding, and so the transpose of the forward's tangent."""
    n0 = 0
    for case in range(60):
        h, E, M, B = cases()[case]
        v0, D2, D3 = stencil(E, M, B, h)
        prm = PRM.copy()
        prm[4] = 0.015
        prm[5] = limit_hu
        tv0, tD2 = RNG.normal(size=9), RNG.normal(size=12)
        val, tan, flag = C.recon_tangent(h, v0, D2, D3, tv0, tD2, np.zeros(9), prm)
        if flag != 0:
            continue
        n0 += 1
        ob = RNG.normal(size=8)
        known = C.recon_adjoint(h, v0, D2, D3, prm, ob, known_smooth=True)
        lin = C.recon_adjoint_lin(h, v0, D2, prm, ob)
        for a, b in zip(known, lin):
            assert np.allclose(a, b, rtol=1e-13, atol=1e-13 * (np.abs(a).max() + 1e-300)), (case, a, b)
        assert not lin[2].any()
        v0b, D2b, _ = lin
        lhs, rhs = ob @ tan, v0b @ tv0 + D2b @ tD2
        assert abs(lhs - rhs) <= 1e-12 * (np.abs(ob * tan).sum() + np.abs(v0b * tv0).sum() + np.abs(D2b * tD2).sum())
    assert n0 >= 10


def test_recon_cases_cover_every_class():
    flags = set()
    for h, E, M, B in cases():
        v0, D2, D3 = stencil(E, M, B, h)
        prm = PRM.copy()
        prm[4] = 0.015
        flags.add(C.recon_tangent(h, v0, D2, D3, np.zeros(9), np.zeros(12), np.zeros(9), prm)[2])
    assert flags == {0, 1, 2}


@pytest.mark.parametrize("trial", range(40))
def test_flux_reverse_matches_tangent(trial):
    rng = np.random.default_rng(trial)
    BL, BR = rng.uniform(0, 1, 2)
    if trial % 4 == 0:
        BR = BL  # tie in b* = max(BL, BR)
    EL, ER = max(BL, BR) + rng.uniform(-0.2, 1.0, 2)
    hL, hR = EL - BL, ER - BR
    e = np.array([EL, ER, BL, BR, hL, hR, rng.normal(), rng.normal()])
    prm = np.array([9.812, rng.uniform(5, 20), rng.normal()])
    te, Fb = rng.normal(size=8), rng.normal(size=4)
    F, tF = C.flux_tangent(e, te, prm)
    eb = C.flux_adjoint(e, prm, Fb)
    scale = np.abs(Fb * tF).sum() + np.abs(eb * te).sum()
    assert abs(Fb @ tF - eb @ te) <= 1e-12 * scale


def test_smooth_class_linear_form_equals_the_sub_stencil_sum():
    """The smooth class's edge values as the cell average plus the mesh-only linear form of the
    first divided differences (linear_edge_form) equal the sum over the three sub-stencil
    quadratics with the linear weights (Step 4 with phi = d) to rounding, on random nonuniform
    widths, and are exact (bitwise the average) for constant data."""
    import ctypes
    L = C.lib()
    out = np.zeros(4)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for k in range(400):
        h = np.exp(RNG.uniform(-1.0, 1.0, 5)) * 10.0 ** RNG.uniform(-3, 1)
        v = RNG.normal(size=5) * 10.0 ** RNG.uniform(-2, 2) + RNG.uniform(-5, 5)
        h, v = np.ascontiguousarray(h), np.ascontiguousarray(v)
        L.ct_edge_forms(ptr(h), ptr(v), ptr(out))
        scale = np.abs(v).max()
        assert np.abs(out[:2] - out[2:]).max() <= 1e-13 * scale, (h, v, out)
        c = np.full(5, v[2])
        L.ct_edge_forms(ptr(h), ptr(c), ptr(out))
        assert out[2] == v[2] and out[3] == v[2]


def _exact_source(hd, bd, w3, g):
    """-g int_0^1 p q' dt in exact rational arithmetic: p, q the quartics of the cell's unit
    coordinate whose averages over the three cells (widths w3 relative to the middle one) and
    values at t = 0, 1 are the data hd, bd (solved by fraction-exact elimination)."""
    from fractions import Fraction as Fr
    rm, rp = Fr(w3[0]) / Fr(w3[1]), Fr(w3[2]) / Fr(w3[1])

    def avg(a, b, i):
        return (Fr(b) ** (i + 1) - Fr(a) ** (i + 1)) / (i + 1) / (Fr(b) - Fr(a))

    rows = [[avg(-rm, 0, i) for i in range(5)], [avg(0, 1, i) for i in range(5)],
            [avg(1, 1 + rp, i) for i in range(5)], [Fr(int(i == 0)) for i in range(5)], [Fr(1)] * 5]

    def solve(data):
        M = [r[:] + [Fr(d)] for r, d in zip(rows, data)]
        for c in range(5):
            p = next(r for r in range(c, 5) if M[r][c] != 0)
            M[c], M[p] = M[p], M[c]
            for r in range(5):
                if r != c and M[r][c] != 0:
                    f = M[r][c] / M[c][c]
                    M[r] = [a - f * b for a, b in zip(M[r], M[c])]
        return [M[i][5] / M[i][i] for i in range(5)]

    a, b = solve(hd), solve(bd)
    return -Fr(g) * sum(a[i] * b[m] * Fr(m, i + m) for i in range(5) for m in range(1, 5))


@pytest.mark.parametrize("spread", [0.3, 1.5, 3.0])
def test_source_form_is_the_exact_integral(spread):
    """The antisymmetric bilinear form of the source (source_form, source_cell_form) against the
    exact integral of the interpolant product, on random widths (ratios up to e^(2 spread)) and
    random or smooth data."""
    rng = np.random.default_rng(int(spread * 10))
    for t in range(40):
        w3 = np.exp(rng.uniform(-spread, spread, 3))
        if t % 2:
            xs = np.array([-w3[0] / 2, w3[1] / 2, w3[1] + w3[2] / 2, 0.0, w3[1]]) / w3[1]
            hd, bd = 1.0 + 0.1 * np.sin(xs), 0.5 + 0.05 * np.cos(2 * xs)
        else:
            hd, bd = rng.uniform(0.1, 2.0, 5), rng.uniform(0.0, 1.0, 5)
        ex = float(_exact_source(hd, bd, w3, 9.812))
        _, _, Sf = C.source_form_adjoint(hd, bd, w3, 9.812, 1.0)
        scale = 9.812 * np.abs(hd).max() * np.abs(bd - bd[1]).max()
        assert abs(Sf - ex) <= 1e-13 * scale, (t, Sf, ex)


@pytest.mark.parametrize("trial", range(20))
def test_source_form_reverse_matches_tangent(trial):
    rng = np.random.default_rng(300 + trial)
    w3 = np.exp(rng.uniform(-1.5, 1.5, 3))
    hd, bd = rng.uniform(0.1, 2, 5), rng.uniform(0, 1, 5)
    thd, tbd, Sb = rng.normal(size=5), rng.normal(size=5), rng.normal()
    S, tS = C.source_form_tangent(hd, bd, thd, tbd, w3, 9.812)
    hdb, bdb, Sf = C.source_form_adjoint(hd, bd, w3, 9.812, Sb)
    assert S == Sf
    lhs, rhs = Sb * tS, hdb @ thd + bdb @ tbd
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(hdb * thd).sum() + np.abs(bdb * tbd).sum())


def test_source_form_at_rest_is_the_pressure_jump():
    """Depth data h = eta - b with eta constant: the form gives -g (eta (b_R - b_L) - (b_R^2 -
    b_L^2) / 2) to rounding (the antisymmetric part vanishes on dh = -db), the identity behind the
    well-balanced property (Sec. 4.3)."""
    rng = np.random.default_rng(77)
    for t in range(200):
        w3 = np.exp(rng.uniform(-2.0, 2.0, 3))
        bd = rng.uniform(0.0, 1.0, 5)
        eta = 1.0 + rng.uniform(0.0, 2.0)
        hd = eta - bd
        _, _, Sf = C.source_form_adjoint(hd, bd, w3, 9.812, 1.0)
        jump = -9.812 * (eta * (bd[4] - bd[3]) - 0.5 * (bd[4] ** 2 - bd[3] ** 2))
        assert abs(Sf - jump) <= 1e-14 * 9.812 * eta, (t, Sf, jump)
