"""Whole-scheme pins of the oracle (no GPU): the paper's printed numbers and the properties
its theorems fix (Sec. 2.3 GCL, Sec. 3.4 positivity, Sec. 4.3 well-balance, Sec. 5.1 tests)."""
import os

import numpy as np
import pytest

import oracle
from paper_2208_06588_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
G = 9.812



def _within_paper(N, got, paper):
    """|q_N - q_2N| against the paper's L1 error at N. Resolved meshes (N = 100, 200): within
    5 % (the literal alpha of Eq. alpha2D lands within 3 % of every printed value there; the
    bound alpha + max |w| is about 10 % off at N = 200). N = 50: within 1.5x. N = 25 is
    under-resolved: the self-difference of the two coarsest meshes is a rough proxy of the L1
    error (for the non-well-balanced scheme it falls outside the bracket e_25 -+ e_50 that the
    printed errors allow, under either reading of alpha), so within 2x."""
    f = 1.05 if N >= 100 else (1.5 if N == 50 else 2.0)
    assert paper / f < got < paper * f, (N, got, paper)

def _params(pr, **kw):
    d = dict(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, bc=pr.bc, mesh=pr.mesh, mesh_T=pr.mesh_T, t_end=pr.t_end,
             gauss_sigma=pr.gauss_sigma, gauss_half=pr.gauss_half, dt_fixed=pr.dt_fixed)
    d.update(kw)
    return oracle.Params(**d)


def _run(pr, nsteps=10 ** 7, **kw):
    st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    r = oracle.run(_params(pr, **kw), st, pr.profile, nsteps=nsteps)
    return st, r


def _table(name):
    rows = [l.split() for l in open(os.path.join(GOLD, name)) if l.strip() and not l.startswith("#")]
    return rows


def test_accuracy_matches_paper_table():
    """Sec. 5.1 accuracy test on the paper's moving mesh: |q_N - q_2N| (the mesh is uniform
    again at t_end, so coarse cells are unions of two fine cells) tracks the paper's L1
    errors of Table WENO5h1D (within 5 % on the resolved meshes N = 100, 200, 1.5x at N = 50, 2x at
    N = 25), and the rate from 100 to 200 is ~4."""
    tab = {int(r[0]): (float(r[1]), float(r[2])) for r in _table("paper_accuracy_table.txt")}
    res = {}
    for N in (25, 50, 100, 200, 400):
        pr = W.accuracy_test(N)
        st, r = _run(pr)
        assert r["status"] == 0 and abs(st.t - 0.1) < 1e-14
        # the paper's mesh returns to the initial uniform mesh at t_end
        assert np.abs(st.x - pr.x).max() < 1e-12
        res[N] = st
    diffs = {}
    for N in (25, 50, 100, 200):
        a, b = res[N], res[2 * N]
        dE = np.mean(np.abs(a.E - 0.5 * (b.E[0::2] + b.E[1::2])))
        dM = np.mean(np.abs(a.M - 0.5 * (b.M[0::2] + b.M[1::2])))
        diffs[N] = (dE, dM)
        for got, paper in zip((dE, dM), tab[N]):
            _within_paper(N, got, paper)
    order = np.log2(diffs[100][0] / diffs[200][0])
    assert 3.5 < order < 4.5  # paper: 3.94 at N = 200


@pytest.mark.slow
def test_accuracy_in_the_fifth_order_regime():
    """The next row of Table WENO5h1D: |q_400 - q_800| on the paper's moving mesh lands within 3 %
    of the printed L1 errors at N = 400 (6.81e-7 and 5.82e-6; measured 6.76e-7 and 5.77e-6), and
    the rate from 200 to 400 is the printed 4.66 to within 0.2 (about 50 s of oracle time). The
    N = 800 row needs a 1600-cell run (several minutes): measured once, 2.217e-8 and 1.895e-7
    against the printed 2.24e-8 and 1.91e-7."""
    tab = {int(r[0]): (float(r[1]), float(r[2])) for r in _table("paper_accuracy_table.txt")}
    res = {}
    for N in (200, 400, 800):
        pr = W.accuracy_test(N)
        st, r = _run(pr)
        assert r["status"] == 0 and abs(st.t - 0.1) < 1e-14
        res[N] = st
    diffs = {}
    for N in (200, 400):
        a, b = res[N], res[2 * N]
        diffs[N] = (np.mean(np.abs(a.E - 0.5 * (b.E[0::2] + b.E[1::2]))),
                    np.mean(np.abs(a.M - 0.5 * (b.M[0::2] + b.M[1::2]))))
    for got, paper in zip(diffs[400], tab[400]):
        assert paper / 1.03 < got < paper * 1.03, (got, paper)
    assert abs(np.log2(diffs[200][0] / diffs[400][0]) - 4.66) < 0.2


def test_lake_at_rest_smooth_bottom_is_round_off():
    """Sec. 5.1 well-balance test, smooth bottom (Eq. smo1D), moving mesh, t = 0.5: errors at
    the paper's round-off level (Table smoothh1D: 8.7e-13 L1, 1.1e-13 / 2.4e-13 Linf)."""
    pr = W.lake_at_rest(200, "smooth")
    st, r = _run(pr)
    assert r["status"] == 0
    L = 10.0
    l1E = np.sum(st.J * np.abs(st.E - 10.0)) / L
    l1M = np.sum(st.J * np.abs(st.M)) / L
    assert l1E < 1e-11 and l1M < 1e-11
    assert np.abs(st.E - 10.0).max() < 1e-11 and np.abs(st.M).max() < 1e-11


def test_lake_at_rest_step_bottom_one_step():
    """Discontinuous bottom (Eq. dis1D): the well-balance identity holds to round-off per step."""
    pr = W.lake_at_rest(200, "step")
    st, r = _run(pr, nsteps=1)
    assert np.abs(st.E - 10.0).max() < 1e-12 and np.abs(st.M).max() < 1e-12


def test_lake_at_rest_periodic_sine_motion():
    pr = W.smooth_periodic(200, lake=True)
    st, r = _run(pr)
    assert r["steps"] > 200
    assert np.abs(st.E - 6.0).max() < 1e-12 and np.abs(st.M).max() < 1e-12


def test_gcl_constant_state_kept():
    """Sec. 2.3: a constant state on a flat bottom stays constant under mesh motion (D-GCL)."""
    pr = W.smooth_periodic(200)
    N = pr.N
    st = oracle.State(np.full(N, 3.0), np.full(N, 1.5), np.zeros(N), pr.J, pr.x)
    r = oracle.run(_params(pr, t_end=0.3), st, pr.profile, nsteps=10 ** 6)
    assert r["steps"] > 500
    assert np.abs(st.E - 3.0).max() < 1e-13 and np.abs(st.M - 1.5).max() < 1e-12


def test_mass_conserved_periodic():
    """The eta and b updates are in conservation form: sum J (eta - b) is constant."""
    pr = W.smooth_periodic(200)
    st, r = _run(pr)
    m0 = np.sum(pr.J * pr.h)
    assert abs(np.sum(st.J * (st.E - st.B)) - m0) < 1e-13 * m0
    # widths still tile the periodic domain
    assert abs(st.J.sum() - 1.0) < 1e-13


def _exact_moses1(x, t, hl=5.0, ul=0.0, hr=10.0, ur=40.0):
    """Exact solution of the vacuum-forming Riemann problem: two rarefactions from the
    Riemann invariants u + 2c (left) and u - 2c (right) with a dry gap between them."""
    cl, cr = np.sqrt(G * hl), np.sqrt(G * hr)
    s = x / t
    h = np.zeros_like(x)
    u = np.zeros_like(x)
    L = s <= ul - cl
    h[L], u[L] = hl, ul
    F = (s > ul - cl) & (s < ul + 2 * cl)
    c = (ul + 2 * cl - s[F]) / 3
    h[F], u[F] = c * c / G, (ul + 2 * cl + 2 * s[F]) / 3
    R = s >= ur + cr
    h[R], u[R] = hr, ur
    F2 = (s > ur - 2 * cr) & (s < ur + cr)
    c = (s[F2] - ur + 2 * cr) / 3
    h[F2], u[F2] = c * c / G, (ur - 2 * cr + 2 * s[F2]) / 3
    return h, u


def test_moses_first_converges_to_exact_vacuum_solution():
    """Sec. 5.1 Moses's first problem: L1 error against the exact solution halves with N
    (first order near the vacuum fronts), depth stays non-negative."""
    errs = []
    for N in (100, 200, 400):
        pr = W.moses_first(N, t_end=2.0)
        st, r = _run(pr)
        assert abs(st.t - 2.0) < 1e-12
        h = st.E - st.B
        assert h.min() >= 0.0
        ex = W.cell_averages(lambda s: _exact_moses1(s, st.t)[0], st.x)
        errs.append(np.sum(st.J * np.abs(h - ex)) / 600.0)
    assert errs[0] < 0.1
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8


def test_moses_second_positivity_and_mass():
    """Sec. 5.1 Moses's second problem to t = 1: the dry gap stays non-negative up to the
    stage-alpha overshoot of the CFL bound (Table minwater prints min h = 1e-11), mass is
    conserved."""
    pr = W.moses_second(200, t_end=1.0)
    st, r = _run(pr)
    assert abs(st.t - 1.0) < 1e-12
    h = st.E - st.B
    assert h.min() > -1e-8
    assert abs(np.sum(st.J * h) - np.sum(pr.J * pr.h)) < 1e-12 * np.sum(pr.J * pr.h)
    assert not (r["status"] & (oracle.ST_NONFINITE | oracle.ST_EMESH))


def test_dam_break_dry_small_stays_positive():
    """The large dam-break workload shape at small N: fluid-driven Gaussian mesh velocity,
    dry region; depth non-negative, mass conserved, mesh valid."""
    pr = W.dam_break_dry(N=2000)
    st, r = _run(pr, nsteps=60)
    h = st.E - st.B
    assert r["steps"] == 60
    assert h.min() > -1e-10
    assert abs(np.sum(st.J * h) - np.sum(pr.J * pr.h)) < 1e-12 * np.sum(pr.J * pr.h)
    assert st.J.min() > 0 and abs(st.J.sum() - 10.0) < 1e-11
    assert not (r["status"] & (oracle.ST_NONFINITE | oracle.ST_EMESH))


def test_dry_bed_at_rest():
    """A dry bed at rest stays at rest: with h = 0 every flux and the source vanish. With an end
    time the CFL dt (unbounded, zero wave speed) is clipped to it and one step lands on t_end;
    without one there is no finite dt, and the step takes dt = 0 and reports the status bit 16
    (reading O21)."""
    def at_rest(st, pr):  # to round-off: the RK combination divides J q by J
        assert np.abs(st.E - pr.E).max() <= 4e-16 and np.abs(st.B - pr.b).max() <= 4e-16
        assert not st.M.any() and np.array_equal(st.x, pr.x)

    pr = W.dry_bed(t_end=0.3)
    st, r = _run(pr, nsteps=5)
    assert r["steps"] == 1 and r["status"] == 0 and st.t == 0.3
    at_rest(st, pr)
    for mesh in ("static", "fluid_gauss"):
        pr = W.dry_bed(t_end=0.0, mesh=mesh)
        st, r = _run(pr, nsteps=3)
        assert r["steps"] == 3 and r["status"] == 16 and st.t == 0.0
        at_rest(st, pr)
