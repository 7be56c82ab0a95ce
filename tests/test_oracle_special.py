"""Pins of the oracle's special source-term scheme (Sec. 4.2, Eq. special2D / source2 / bhat2D /
gausssij2): point reconstruction at the interior Gauss-Lobatto points, the treatment of negative
linear weights (Shi, Hu & Shu), the paper's Table WENO5h1D (special columns), lake at rest."""
import os

import numpy as np

import oracle
from paper_2208_06588_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(20220812 + 77)
T_GLO = (0.5 - 0.5 / np.sqrt(5.0), 0.5 + 0.5 / np.sqrt(5.0))



def _within_paper(N, got, paper):
    """|q_N - q_2N| against the paper's L1 error at N. Resolved meshes (N = 100, 200): within
    5 % (the literal alpha of Eq. alpha2D lands within 3 % of every printed value there; the
    bound alpha + max |w| is about 10 % off at N = 200). N = 50: within 1.5x. N = 25 is
    under-resolved: the self-difference of the two coarsest meshes is a rough proxy of the L1
    error (for the non-well-balanced scheme it falls outside the bracket e_25 -+ e_50 that the
    printed errors allow, under either reading of alpha), so within 2x."""
    f = 1.05 if N >= 100 else (1.5 if N == 50 else 2.0)
    assert paper / f < got < paper * f, (N, got, paper)

def _avg_matrix(nodes, deg):
    """A[i, k]: average of x^k over [nodes[i], nodes[i+1]] (numpy, exact antiderivatives)."""
    a, b = nodes[:-1], nodes[1:]
    return np.stack([(b ** (k + 1) - a ** (k + 1)) / ((k + 1) * (b - a)) for k in range(deg + 1)], axis=1)


def _weights_numpy(w5, t):
    """Linear weights at unit coordinate t from numpy least squares: sum_r d_r p_r(t) = q(t)
    as maps of the five averages (an independent construction of Step 1 at a point)."""
    y = np.concatenate([[0.0], np.cumsum(w5)]) - (w5[0] + w5[1])
    y = y / w5[2]
    tp = t ** np.arange(5)
    C = tp @ np.linalg.inv(_avg_matrix(y, 4))        # quartic weights of the 5 averages
    cols = []
    for r in range(3):
        a = 2 - r
        c = tp[:3] @ np.linalg.inv(_avg_matrix(y[a:a + 4], 2))
        full = np.zeros(5)
        full[a:a + 3] = c
        cols.append(full)
    d, *_ = np.linalg.lstsq(np.stack(cols, axis=1), C, rcond=None)
    return d


def test_point_linear_weights_match_an_independent_construction():
    for w5 in (np.ones(5), np.exp(RNG.uniform(-1, 1, 5)), np.exp(RNG.uniform(-1.5, 1.5, 5))):
        for t in (*T_GLO, 0.5, 0.0, 1.0):
            got = oracle.weno_point(w5, t)["d"]
            ref = _weights_numpy(w5, t)
            assert np.allclose(got, ref, rtol=1e-10, atol=1e-12), (w5, t, got, ref)
    # uniform mesh: positive at the Gauss-Lobatto points, negative at the midpoint
    d = oracle.weno_point(np.ones(5), T_GLO[0])["d"]
    assert np.all(d > 0)
    assert np.allclose(oracle.weno_point(np.ones(5), 0.5)["d"], [-9 / 80, 49 / 40, -9 / 80], atol=1e-13)


def test_point_reconstruction_reproduces_quartics():
    for _ in range(10):
        J = np.exp(RNG.uniform(-0.7, 0.7, 5))
        x = np.concatenate([[0.0], np.cumsum(J)])
        coef = RNG.normal(size=5)
        ubar = _avg_matrix(x, 4) @ coef
        Q = None
        for t in T_GLO:
            Q = oracle.weno_point(J, t)
            val = sum(Q["d"][r] * (Q["c"][r] @ ubar[2 - r:5 - r]) for r in range(3))
            xt = x[2] + t * J[2]
            assert abs(val - np.polyval(coef[::-1], xt)) < 1e-10 * max(1.0, abs(val))


def test_negative_weight_split():
    P = oracle.Params()
    d = np.array([-9 / 80, 49 / 40, -9 / 80])
    # equal indicators (tau = 0): the split returns the linear weights in every class
    for flag in (1, 2):
        phi = oracle.point_phi(P, d, np.full(3, 0.3), flag)
        assert np.allclose(phi, d, atol=1e-14)
    # different indicators: still a partition of unity, and a positive linear weight case
    # reduces to plain WENO-Z
    beta = np.array([1e-3, 5e-1, 2.0])
    phi = oracle.point_phi(P, d, beta, 2)
    assert abs(phi.sum() - 1.0) < 1e-14
    dpos = np.array([0.2, 0.5, 0.3])
    tau = abs(beta[0] - beta[2])
    al = dpos * (1 + (tau / (beta + 1e-6)) ** 2)
    assert np.allclose(oracle.point_phi(P, dpos, beta, 2), al / al.sum(), rtol=1e-13)


def _run(pr, nsteps=10 ** 7):
    P = oracle.Params(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, bc=pr.bc, mesh=pr.mesh, mesh_T=pr.mesh_T,
                      t_end=pr.t_end, scheme="special")
    st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    r = oracle.run(P, st, pr.profile, nsteps=nsteps)
    return st, r


def test_accuracy_matches_paper_table_special():
    rows = [l.split() for l in open(os.path.join(GOLD, "paper_accuracy_table_special.txt"))
            if l.strip() and not l.startswith("#")]
    tab = {int(r[0]): (float(r[1]), float(r[2])) for r in rows}
    res = {}
    for N in (25, 50, 100, 200, 400):
        st, r = _run(W.accuracy_test(N))
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
    assert 3.5 < np.log2(diffs[100][0] / diffs[200][0]) < 4.5


def test_lake_at_rest_is_round_off_and_mass_is_conserved():
    for bottom in ("smooth", "step"):
        pr = W.lake_at_rest(200, bottom)
        st, r = _run(pr, nsteps=60)
        assert r["status"] == 0
        assert np.abs(st.E - 10.0).max() < 1e-11, bottom
        assert np.abs(st.M).max() < 1e-10, bottom
    pr = W.accuracy_test(64)
    m0 = np.sum(pr.J * pr.E)
    st, r = _run(pr, nsteps=40)
    assert abs(np.sum(st.J * st.E) - m0) < 1e-13 * m0
