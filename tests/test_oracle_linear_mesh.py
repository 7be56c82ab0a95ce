"""Pins of the oracle's constant-node-velocity motion (mesh "linear": the graded moving mesh of
the big-pulse example, Sec. 5.1, Eq. 0.2inis, 0.2ends, velocity, meshspecial), no GPU:

* the nodes move as x(t) = x(0) + w t and land on the end grid of Eq. 0.2ends at t_end, and the
  widths of the GCL recursion (Eq. Jacobi2D) equal the node differences at every step's end;
* the lake at rest stays at rest to round-off on that moving mesh (Sec. 4.3), with eta's mass;
* a constant flow over a flat bottom stays constant (GCL), and its stage viscosities are Eq.
  alpha2D as written, max over the edges of |u - w| + sqrt(g h) with w the velocity of the
  edge's node (reading O4: w is known in every stage of this motion), or with alpha_bound the
  bound |u| + sqrt(g h) + max |w|; every dt is CFL min_j J_j^n / alpha_1 (reading O5) on the
  mesh x(0) + w t_n.
"""
import numpy as np

import oracle
from paper_2208_06588_gb300 import workloads as W


def _params(pr, **kw):
    d = dict(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, bc=pr.bc, mesh=pr.mesh, mesh_T=pr.mesh_T, t_end=pr.t_end)
    d.update(kw)
    return oracle.Params(**d)


def test_nodes_reach_the_end_grid_and_widths_follow_the_nodes():
    pr = W.big_pulse(refine=1, eps=0.2)
    assert pr.mesh == "linear"
    st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    r = oracle.run(_params(pr), st, pr.profile, nsteps=10 ** 6, record=True)
    assert r["status"] == 0 and st.t == pr.t_end
    assert np.abs(st.x - pr.meta["x_end"]).max() < 1e-13
    assert np.abs(st.J - np.diff(st.x)).max() < 1e-13
    # the step sizes add up to t_end; the motion is the straight line between the two grids
    t = np.cumsum(r["dts"])
    assert abs(t[-1] - pr.t_end) < 1e-15
    # a run stopped after k steps sits on x(0) + w t_k
    k = 17
    st2 = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    oracle.run(_params(pr), st2, pr.profile, nsteps=k)
    assert np.abs(st2.x - (pr.x + pr.profile * t[k - 1])).max() < 1e-13
    assert np.abs(st2.J - np.diff(st2.x)).max() < 1e-13


def test_lake_at_rest_on_the_graded_moving_mesh():
    pr = W.big_pulse(refine=1, eps=0.0)
    st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    r = oracle.run(_params(pr), st, pr.profile, nsteps=10 ** 6)
    assert r["status"] == 0 and st.t == pr.t_end and r["steps"] > 200
    assert np.abs(st.E - 1.0).max() < 1e-12
    assert np.abs(st.M).max() < 1e-12
    assert abs(np.sum(st.J * st.E) - np.sum(pr.J * pr.E)) < 1e-13


def test_constant_flow_alpha_reads_the_node_velocities():
    pr = W.big_pulse(refine=1, eps=0.2)
    N, w, g = pr.N, pr.profile, pr.g
    u = -0.5  # against the larger positive node velocities: the literal and bound forms differ
    literal = np.abs(u - w).max() + np.sqrt(g)
    bound = abs(u) + np.sqrt(g) + np.abs(w).max()
    assert bound - literal > 0.1
    for alpha_bound, expect in ((0, literal), (1, bound)):
        st = oracle.State(np.full(N, 1.0), np.full(N, u), np.zeros(N), pr.J.copy(), pr.x.copy())
        steps = 12
        r = oracle.run(_params(pr, alpha_bound=alpha_bound, t_end=0.0), st, pr.profile, nsteps=steps, record=True)
        assert r["status"] == 0 and r["steps"] == steps
        # GCL: the constant state is kept on the moving mesh
        assert np.abs(st.E - 1.0).max() < 1e-13 and np.abs(st.M - u).max() < 1e-13
        assert np.allclose(r["alphas"], expect, rtol=1e-14, atol=0.0), (alpha_bound, r["alphas"][:3], expect)
        # dt_n = CFL min_j J_j^n / alpha_1 on the mesh x(0) + w t_n
        t = 0.0
        for n, dt in enumerate(r["dts"]):
            xn = pr.x + w * t
            assert abs(dt - pr.cfl * np.diff(xn).min() / expect) <= 1e-12 * dt, n  # J^n of the recursion: rounding
            t += dt


def test_alpha_pairs_each_edge_with_its_own_node():
    """Eq. alpha2D on a varying state: the left edge of cell j sits at node j and the right edge
    at node j + 1, each with that node's velocity. The stage viscosity of the right-hand side
    equals the maximum formed in numpy from the reconstruction's own limited edge states (cells
    -1..N, the two outermost edges excluded), and differs from the maximum with the nodes swapped."""
    rng = np.random.default_rng(20220812 + 71)
    N, g = 64, 9.812
    x = np.cumsum(np.concatenate([[0.0], rng.uniform(0.5, 1.5, N)]))
    x /= x[-1]
    J = np.diff(x)
    xc = 0.5 * (x[1:] + x[:-1])
    b = 0.2 * np.sin(2 * np.pi * xc) ** 2
    E = 1.0 + 0.1 * np.cos(6 * np.pi * xc) + 0.05 * (xc > 0.5)
    M = 0.8 * np.sin(10 * np.pi * xc) + rng.uniform(-0.3, 0.3, N)
    w = rng.uniform(-2.0, 2.0, N + 1)
    p = oracle.Params(g=g, bc="transmissive", mesh="linear")
    ed, _, _, _, st = oracle.reconstruct(p, E, M, b, J)
    assert st == 0
    _, _, _, a_used, st = oracle.rhs(p, E, M, b, J, w, alpha=0.0)
    assert st == 0
    c = lambda h: np.sqrt(g * np.maximum(h, 0.0))
    # cell k = 0..N+1 in the arrays is cell k - 1: its left edge at node k - 1, right at node k
    uL, uR, hL, hR = ed["u_L"], ed["u_R"], ed["h_L"], ed["h_R"]
    own = max(np.max(np.abs(uL[1:] - w) + c(hL[1:])), np.max(np.abs(uR[:-1] - w) + c(hR[:-1])))
    swapped = max(np.max(np.abs(uL[1:-1] - w[1:]) + c(hL[1:-1])), np.max(np.abs(uR[1:-1] - w[:-1]) + c(hR[1:-1])))
    assert abs(a_used - own) <= 1e-14 * own, (a_used, own)
    assert abs(swapped - own) > 1e-3 * own
