"""Pins of the oracle's non-well-balanced ALE-WENO scheme (Eq. se2D / s2D, local characteristic
reconstruction, plain Lax-Friedrichs flux): the paper's Table WENO5n1D, linearity in smooth
regions, the properties it keeps (GCL, mass) and the one it lacks (lake at rest)."""
import os

import numpy as np

import oracle
from paper_2208_06588_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")



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
             scheme="nonwb")
    d.update(kw)
    return oracle.Params(**d)


def _run(pr, nsteps=10 ** 7, **kw):
    st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    r = oracle.run(_params(pr, **kw), st, pr.profile, nsteps=nsteps)
    return st, r


def test_accuracy_matches_paper_table_nonwb():
    """|q_N - q_2N| of the accuracy test (the mesh is uniform again at t_end) tracks the paper's
    Table WENO5n1D (5 % at N = 100, 200; 1.5x at N = 50; 2x at N = 25); rate ~4 from 100 to 200
    (paper: 3.95)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "paper_accuracy_table_nonwb.txt"))
            if l.strip() and not l.startswith("#")]
    tab = {int(r[0]): (float(r[1]), float(r[2])) for r in rows}
    res = {}
    for N in (25, 50, 100, 200, 400):
        pr = W.accuracy_test(N)
        st, r = _run(pr)
        assert r["status"] == 0 and abs(st.t - 0.1) < 1e-14
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
    assert 3.5 < order < 4.5


def test_smooth_cells_reconstruct_like_the_big_stencil_quartic():
    """Where every field is in the smooth class the weights are the linear ones, the projection
    is linear, so the characteristic edge values equal the quartic's edge values of eta and hu
    computed componentwise from the mesh weights (Step 1)."""
    rng = np.random.default_rng(3)
    N = 40
    J = 0.02 * (1.0 + 0.3 * rng.uniform(size=N))
    x = np.concatenate([[0.0], np.cumsum(J)])
    xc = 0.5 * (x[1:] + x[:-1])
    E = 2.0 + 0.1 * np.sin(2 * np.pi * xc / x[-1])
    M = 0.3 + 0.05 * np.cos(2 * np.pi * xc / x[-1])
    B = 0.2 * np.sin(2 * np.pi * xc / x[-1]) ** 2
    P = oracle.Params(bc="periodic", scheme="nonwb")
    edges, flags, gam, A, st = oracle.reconstruct(P, E, M, B, J)
    assert st == 0
    checked = 0
    for j in range(2, N - 2):
        if flags[j + 1] != 0:
            continue
        big = oracle.weno_coeffs(J[j - 2:j + 3])["big"]
        for e, (nE, nM) in enumerate((("E_L", "M_L"), ("E_R", "M_R"))):
            qE = big[e] @ E[j - 2:j + 3]
            qM = big[e] @ M[j - 2:j + 3]
            assert abs(edges[nE][j + 1] - qE) < 1e-12
            assert abs(edges[nM][j + 1] - qM) < 1e-12
        checked += 1
    assert checked > N // 2


def test_gcl_and_mass_but_not_well_balanced():
    # constant state under mesh motion stays constant (GCL), flat bottom
    pr = W.accuracy_test(64)
    N = pr.N
    st = oracle.State(np.full(N, 3.0), np.full(N, 0.7), np.zeros(N), pr.J, pr.x)
    r = oracle.run(_params(pr), st, pr.profile, nsteps=30)
    assert r["status"] == 0
    assert np.abs(st.E - 3.0).max() < 1e-13 and np.abs(st.M - 0.7).max() < 1e-13
    # mass of eta is conserved (periodic)
    pr = W.accuracy_test(64)
    m0 = np.sum(pr.J * pr.E)
    st, r = _run(pr, nsteps=40)
    assert abs(np.sum(st.J * st.E) - m0) < 1e-13 * m0
    # lake at rest over a smooth bottom is NOT kept to round-off (the flux's pressure term and
    # the source quadrature do not cancel), unlike the hydrostatic scheme
    pr = W.lake_at_rest(100, "smooth")
    st, r = _run(pr, nsteps=40)
    err_nonwb = np.abs(st.E - 10.0).max()
    st2 = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    oracle.run(_params(pr, scheme="hydrostatic"), st2, pr.profile, nsteps=40)
    err_wb = np.abs(st2.E - 10.0).max()
    assert err_wb < 1e-12 and err_nonwb > 1e-8
