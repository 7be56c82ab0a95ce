"""Non-well-balanced ALE-WENO scheme (Eq. se2D / s2D, local characteristic reconstruction, plain
Lax-Friedrichs flux) on the GPU against the oracle: smooth runs, shocks and dry fronts, step-1
classes, a batch, and the adjoint refusing it."""
import numpy as np
import pytest

import oracle
from paper_2208_06588_gb300 import binding as B
from paper_2208_06588_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_06588_gb300 import build
    build.build()
    B.lib()


def cfg_of(pr):
    return B.make_config(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, gauss_sigma=pr.gauss_sigma,
                         t_end=pr.t_end, dt_fixed=pr.dt_fixed, bc=pr.bc, mesh=pr.mesh, gauss_half=pr.gauss_half,
                         scheme="nonwb")


def params_of(pr):
    return oracle.Params(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, gauss_sigma=pr.gauss_sigma,
                         t_end=pr.t_end, dt_fixed=pr.dt_fixed, bc=pr.bc, mesh=pr.mesh, gauss_half=pr.gauss_half,
                         scheme="nonwb")


def run_both(pr, nsteps):
    s = B.Solver(cfg_of(pr))
    s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
    done = s.advance(nsteps)
    g = s.state()
    g["flags"] = s.flags()
    g["bits"] = s.status()[0]
    s.close()
    st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    r = oracle.run(params_of(pr), st, pr.profile, nsteps=nsteps)
    assert done == r["steps"]
    return g, st, r


def max_rel(a, r):
    return np.abs(a - r).max() / max(np.abs(r).max(), 1e-300)


def l1_rel(a, r, J):
    return float(np.sum(J * np.abs(a - r)) / max(np.sum(J * np.abs(r)), 1e-300))


@pytest.mark.parametrize("N", [200, 203])
def test_smooth_accuracy_problem(N):
    pr = W.accuracy_test(N)
    g, st, r = run_both(pr, 10 ** 6)
    assert r["status"] == 0 and g["bits"] == 0
    assert abs(g["t"] - 0.1) < 1e-14
    for a, ref in ((g["eta"], st.E), (g["hu"], st.M), (g["b"], st.B)):
        assert max_rel(a, ref) <= 1e-11


@pytest.mark.parametrize("which", ["first", "second"])
def test_wet_dry_riemann_problems(which):
    pr = W.moses_first(200) if which == "first" else W.moses_second(200)
    g, st, r = run_both(pr, 150)
    assert g["bits"] & ~B.BIT_NEGDEPTH == 0
    assert l1_rel(g["eta"], st.E, st.J) <= 1e-9
    assert l1_rel(g["hu"], st.M, st.J) <= 1e-9


def test_step1_flags_and_shock_run():
    pr = W.dam_break_dry(N=4096)
    g, st, r = run_both(pr, 1)
    edges, flags, gam, A, s_ = oracle.reconstruct(params_of(pr), pr.E, pr.hu, pr.b, pr.J)
    f_or = flags[1:-1]
    assert (g["flags"] == f_or).mean() > 0.999
    g, st, r = run_both(pr, 40)
    for a, ref in ((g["eta"], st.E), (g["hu"], st.M)):
        assert l1_rel(a, ref, st.J) <= 1e-9


def test_batch_equals_single_instances_and_adjoint_refuses():
    bt = W.many_basins(B=6, n_min=64, n_max=300, seed=9)
    cfg = B.make_config(eps_weno=bt.eps_weno, mesh_T=bt.mesh_T, bc=bt.bc, mesh=bt.mesh, scheme="nonwb")
    s = B.Solver(cfg)
    s.set_batch(bt)
    s.advance(15)
    out = s.batch_state()
    with pytest.raises(B.SwaleError):
        B.swale_adjoint(s.ctx, 1, 1, 1, np.full(6, 0.5), np.zeros(6), np.zeros(6), np.zeros(s.N), np.zeros(s.N),
                        np.zeros(s.N))
    s.close()
    for i in range(bt.B):
        pr = bt.instance(i)
        c = B.make_config(eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, bc=pr.bc, mesh=pr.mesh, cfl=pr.cfl, scheme="nonwb")
        si = B.Solver(c)
        si.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
        si.advance(15)
        gi = si.state()
        si.close()
        a, b_ = int(bt.off[i]), int(bt.off[i + 1])
        np.testing.assert_array_equal(out["eta"][a:b_], gi["eta"])
        np.testing.assert_array_equal(out["hu"][a:b_], gi["hu"])
