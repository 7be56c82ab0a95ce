"""Discrete adjoint of a gauge misfit (swale_adjoint) on the GPU.

* Dot-product test against the CPU oracle's tangent-linear model: <dJ/dq0, dq> from the GPU
  adjoint equals dJ along dq from the oracle's dual-number instantiation stepped with its own
  recorded dt and alphas (the replay convention of the adjoint).
* Central finite differences of the GPU forward with the stage viscosities replayed.
* Independence from the checkpoint interval (also at a size where the recomputes overlap the
  reverse sweep); a batch equals its instances.
"""
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
    return B.make_config(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, bc=pr.bc, mesh=pr.mesh,
                         dt_fixed=pr.dt_fixed)


def params_of(pr):
    return oracle.Params(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, bc=pr.bc, mesh=pr.mesh,
                         dt_fixed=pr.dt_fixed)


def gauge_cells(x, gx):
    return np.clip(np.searchsorted(x, gx, side="right") - 1, 0, x.size - 2)


def gpu_adjoint(pr, gx, obs, nsteps, ckpt=8, tape=0):
    s = B.Solver(cfg_of(pr))
    s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
    B.swale_set_adjoint_tape(s.ctx, tape)
    N = pr.N
    J, gE, gM, gB = np.zeros(1), np.zeros(N), np.zeros(N), np.zeros(N)
    B.swale_adjoint(s.ctx, nsteps, ckpt, gx.size, np.ascontiguousarray(gx), np.ascontiguousarray(obs), J, gE, gM, gB)
    s.close()
    return J[0], gE, gM, gB


def oracle_tangent_derivative(pr, gx, obs, nsteps, dE, dM, dB):
    """J and dJ along (dE, dM, dB) from the oracle: forward with recorded dt / alphas, then the
    tangent-linear model one step at a time with the misfit's tangent at every step."""
    P = params_of(pr)
    st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
    rec = oracle.run(P, st.copy(), pr.profile, nsteps=nsteps, record=True)
    s = st.copy()
    J = dJ = 0.0
    for n in range(nsteps):
        dt = rec["dts"][n]
        dE, dM, dB, _ = oracle.tangent(P, s, pr.profile, rec["dts"][n:n + 1], rec["alphas"][3 * n:3 * n + 3], dE, dM,
                                       dB)
        c = gauge_cells(s.x, gx)
        r = (s.E[c] - s.B[c]) - obs[n]
        J += dt * np.sum(r * r)
        dJ += 2.0 * dt * np.sum(r * (dE[c] - dB[c]))
    return J, dJ


def basin(N=256, seed=7):
    pr = W.gaussian_basin(N=N, seed=seed)
    rng = np.random.default_rng(seed)
    gx = np.array([0.13, 0.41, 0.62, 0.88])
    return pr, gx, rng


@pytest.mark.parametrize("seed", [7, 8])
def test_dot_product_against_oracle_tangent_linear(seed):
    pr, gx, rng = basin(N=256, seed=seed)
    nsteps = 20
    obs = 0.6 + 0.05 * rng.normal(size=(nsteps, gx.size))
    J, gE, gM, gB = gpu_adjoint(pr, gx, obs, nsteps)
    xc = 0.5 * (pr.x[1:] + pr.x[:-1])
    dE = np.sin(7 * xc) + 0.3 * rng.normal(size=pr.N)
    dM = np.cos(5 * xc) + 0.3 * rng.normal(size=pr.N)
    dB = 0.5 * np.sin(3 * xc) + 0.3 * rng.normal(size=pr.N)
    Jo, dJ_tl = oracle_tangent_derivative(pr, gx, obs, nsteps, dE, dM, dB)
    dJ_adj = gE @ dE + gM @ dM + gB @ dB
    assert abs(J - Jo) <= 1e-11 * Jo
    scale = abs(gE) @ abs(dE) + abs(gM) @ abs(dM) + abs(gB) @ abs(dB)
    assert abs(dJ_adj - dJ_tl) <= 1e-12 * scale, (dJ_adj, dJ_tl, scale)


def gpu_misfit_replay(pr, gx, obs, nsteps, E0, M0, B0, alog):
    s = B.Solver(cfg_of(pr))
    s.set_problem(pr.x, E0, M0, B0, pr.profile, q0_is_eta=True)
    B.swale_alpha_log(s.ctx, 2, nsteps, alog)
    J = 0.0
    for n in range(nsteps):
        dt = s.step()
        st = s.state()
        c = gauge_cells(st["x"], gx)
        r = (st["eta"][c] - st["b"][c]) - obs[n]
        J += dt * np.sum(r * r)
    s.close()
    return J


def test_central_finite_differences():
    pr, gx, rng = basin(N=512, seed=11)
    nsteps = 30
    obs = 0.6 + 0.05 * rng.normal(size=(nsteps, gx.size))
    J, gE, gM, gB = gpu_adjoint(pr, gx, obs, nsteps)
    s = B.Solver(cfg_of(pr))
    s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
    B.swale_alpha_log(s.ctx, 1, nsteps)
    s.advance(nsteps)
    alog = np.zeros(3 * nsteps)
    B.swale_get_alpha_log(s.ctx, alog)
    s.close()
    xc = 0.5 * (pr.x[1:] + pr.x[:-1])
    for dE, dB in ((np.exp(-((xc - 0.4) / 0.1) ** 2), 0 * xc), (0 * xc, 0.5 * np.exp(-((xc - 0.6) / 0.08) ** 2))):
        eps = 1e-5
        Jp = gpu_misfit_replay(pr, gx, obs, nsteps, pr.E + eps * dE, pr.hu, pr.b + eps * dB, alog)
        Jm = gpu_misfit_replay(pr, gx, obs, nsteps, pr.E - eps * dE, pr.hu, pr.b - eps * dB, alog)
        fd = (Jp - Jm) / (2 * eps)
        ad = gE @ dE + gB @ dB
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_checkpoint_interval_does_not_change_the_gradient():
    pr, gx, rng = basin(N=300, seed=12)
    nsteps = 21
    obs = 0.6 + 0.05 * rng.normal(size=(nsteps, gx.size))
    ref = gpu_adjoint(pr, gx, obs, nsteps, ckpt=nsteps)
    for ck in (1, 5, 8):
        got = gpu_adjoint(pr, gx, obs, nsteps, ckpt=ck)
        assert abs(got[0] - ref[0]) <= 1e-14 * ref[0]
        for a, b in zip(got[1:], ref[1:]):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_overlapped_recomputes_do_not_change_the_gradient():
    """At 65536 cells the segment recomputes, the step recomputes and the reverse sweep overlap
    on three streams with buffers handed over by events; the gradient must not depend on how the
    steps are cut into segments (one segment, one-step segments, ragged ones) nor change when
    the same call is repeated."""
    K = 40
    gp = W.gauge_problem(N=65536, nsteps=K, G=16)
    pr = gp.problem
    ref = gpu_adjoint(pr, gp.gauges, gp.h_obs, K, ckpt=K)
    for ck in (1, 3, 16, 16):
        got = gpu_adjoint(pr, gp.gauges, gp.h_obs, K, ckpt=ck)
        assert abs(got[0] - ref[0]) <= 1e-14 * ref[0]
        for a, b in zip(got[1:], ref[1:]):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_tape_gives_the_recomputed_gradient():
    """swale_set_adjoint_tape(1): the reverse sweep reads the stage data that the segment
    recompute kept instead of recomputing each step; the gradient must be the same (to the order
    of atomic additions) for one segment, one-step segments and ragged ones, at a small size and
    at 65536 cells, where the segment recomputes overlap the reverse sweep."""
    pr, gx, rng = basin(N=300, seed=12)
    nsteps = 21
    obs = 0.6 + 0.05 * rng.normal(size=(nsteps, gx.size))
    ref = gpu_adjoint(pr, gx, obs, nsteps, ckpt=5)
    for ck in (1, 5, 8, nsteps):
        got = gpu_adjoint(pr, gx, obs, nsteps, ckpt=ck, tape=1)
        assert abs(got[0] - ref[0]) <= 1e-14 * ref[0]
        for a, b in zip(got[1:], ref[1:]):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    K = 40
    gp = W.gauge_problem(N=65536, nsteps=K, G=16)
    ref = gpu_adjoint(gp.problem, gp.gauges, gp.h_obs, K, ckpt=16)
    for ck in (3, 16):
        got = gpu_adjoint(gp.problem, gp.gauges, gp.h_obs, K, ckpt=ck, tape=1)
        assert abs(got[0] - ref[0]) <= 1e-14 * ref[0]
        for a, b in zip(got[1:], ref[1:]):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("tape", [0, 1])
def test_batched_adjoint_equals_single_instances(tape):
    prs = [W.gaussian_basin(N=n, seed=20 + i) for i, n in enumerate((200, 333, 256))]
    dt = min(p.dt_fixed for p in prs)
    for p in prs:
        p.dt_fixed = dt
    nsteps, G = 12, 3
    rng = np.random.default_rng(5)
    gxs = [np.sort(rng.uniform(0.05, 0.95, G)) for _ in prs]
    obs = [0.6 + 0.05 * rng.normal(size=(nsteps, G)) for _ in prs]
    off = np.concatenate([[0], np.cumsum([p.N for p in prs])]).astype(np.int64)
    bt = W.Batch(name="b", off=off, x=np.concatenate([p.x for p in prs]), h=np.concatenate([p.h for p in prs]),
                 hu=np.concatenate([p.hu for p in prs]), b=np.concatenate([p.b for p in prs]),
                 E=np.concatenate([p.E for p in prs]), profile=np.concatenate([p.profile for p in prs]),
                 cfl=np.array([p.cfl for p in prs]))
    s = B.Solver(cfg_of(prs[0]))
    s.set_batch(bt)
    B.swale_set_adjoint_tape(s.ctx, tape)
    Ntot = int(off[-1])
    J, gE, gM, gB = np.zeros(3), np.zeros(Ntot), np.zeros(Ntot), np.zeros(Ntot)
    obs_b = np.stack([np.stack([o[n] for o in obs]) for n in range(nsteps)])  # nsteps x B x G
    B.swale_adjoint(s.ctx, nsteps, 5, G, np.concatenate(gxs), np.ascontiguousarray(obs_b), J, gE, gM, gB)
    s.close()
    for i, p in enumerate(prs):
        Ji, gEi, gMi, gBi = gpu_adjoint(p, gxs[i], obs[i], nsteps, ckpt=5)
        assert abs(J[i] - Ji) <= 1e-14 * Ji
        sl = slice(int(off[i]), int(off[i + 1]))
        for a, b in ((gE[sl], gEi), (gM[sl], gMi), (gB[sl], gBi)):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_autograd_function_matches_the_adjoint():
    import torch

    from paper_2208_06588_gb300.autograd import gauge_misfit
    pr, gx, rng = basin(N=256, seed=9)
    nsteps = 10
    obs = 0.6 + 0.05 * rng.normal(size=(nsteps, gx.size))
    J, gE, gM, gB = gpu_adjoint(pr, gx, obs, nsteps, ckpt=4)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    E, M, Bt = (t(a).requires_grad_() for a in (pr.E, pr.hu, pr.b))
    Jt = gauge_misfit(E, M, Bt, t(pr.x), t(pr.profile), t(gx), t(obs), cfg_of(pr), nsteps, ckpt_every=4)
    assert Jt.shape == (1,)
    assert abs(Jt.item() - J) <= 1e-14 * J
    (3.0 * Jt.sum()).backward()
    for g, r in ((E.grad, gE), (M.grad, gM), (Bt.grad, gB)):
        assert np.abs(g.cpu().numpy() - 3.0 * r).max() <= 1e-12 * np.abs(3.0 * r).max()
    # the same through the tape
    E2 = t(pr.E).requires_grad_()
    Jt2 = gauge_misfit(E2, t(pr.hu), t(pr.b), t(pr.x), t(pr.profile), t(gx), t(obs), cfg_of(pr), nsteps,
                       ckpt_every=4, tape=True)
    assert abs(Jt2.item() - J) <= 1e-14 * J
    Jt2.sum().backward()
    assert np.abs(E2.grad.cpu().numpy() - gE).max() <= 1e-12 * np.abs(gE).max()


def test_autograd_batched_weights_each_instance():
    import torch

    from paper_2208_06588_gb300.autograd import gauge_misfit
    prs = [W.gaussian_basin(N=n, seed=30 + i) for i, n in enumerate((160, 240))]
    dt = min(p.dt_fixed for p in prs)
    for p in prs:
        p.dt_fixed = dt
    nsteps, G = 6, 2
    rng = np.random.default_rng(6)
    gxs = np.concatenate([np.sort(rng.uniform(0.05, 0.95, G)) for _ in prs])
    obs = 0.6 + 0.05 * rng.normal(size=(nsteps, 2, G))
    off = np.array([0, prs[0].N, prs[0].N + prs[1].N], dtype=np.int64)
    dev = torch.device("cuda:0")
    cat = lambda f: torch.tensor(np.concatenate([f(p) for p in prs]), dtype=torch.float64, device=dev)
    E, M, Bt = cat(lambda p: p.E).requires_grad_(), cat(lambda p: p.hu).requires_grad_(), \
        cat(lambda p: p.b).requires_grad_()
    Jt = gauge_misfit(E, M, Bt, cat(lambda p: p.x), cat(lambda p: p.profile), gxs, obs, cfg_of(prs[0]), nsteps,
                      ckpt_every=3, offsets=off)
    (2.0 * Jt[0] - 5.0 * Jt[1]).backward()
    for i, (p, wgt) in enumerate(zip(prs, (2.0, -5.0))):
        Ji, gEi, _, gBi = gpu_adjoint(p, gxs[i * G:(i + 1) * G], obs[:, i, :], nsteps, ckpt=3)
        assert abs(Jt[i].item() - Ji) <= 1e-14 * Ji
        sl = slice(int(off[i]), int(off[i + 1]))
        for g, r in ((E.grad[sl], gEi), (Bt.grad[sl], gBi)):
            assert np.abs(g.cpu().numpy() - wgt * r).max() <= 1e-12 * np.abs(wgt * r).max()


def test_full_size_gradient_against_finite_differences():
    """The adjoint benchmark case at its full size (N = 65536, 4000 steps, checkpoints every 64
    steps, 16 gauges): the gradient along smooth perturbations of eta0 and of b matches central
    differences of the GPU forward with the stage viscosities replayed."""
    gp = W.gauge_problem(N=65536, nsteps=4000, G=16)
    pr, K = gp.problem, gp.nsteps
    J, gE, gM, gB = gpu_adjoint(pr, gp.gauges, gp.h_obs, K, ckpt=64)
    s = B.Solver(cfg_of(pr))
    s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
    B.swale_alpha_log(s.ctx, 1, K)
    s.advance(K)
    alog = np.zeros(3 * K)
    B.swale_get_alpha_log(s.ctx, alog)
    s.close()

    def misfit(E0, B0):
        s = B.Solver(cfg_of(pr))
        s.set_problem(pr.x, E0, pr.hu, B0, pr.profile, q0_is_eta=True)
        B.swale_alpha_log(s.ctx, 2, K, alog)
        Jm = np.zeros(1)
        # the misfit of a replayed forward: the adjoint call's J (its reverse sweep is unused)
        B.swale_adjoint(s.ctx, K, 64, gp.gauges.size, gp.gauges, np.ascontiguousarray(gp.h_obs), Jm, None, None,
                        None)
        s.close()
        return Jm[0]

    xc = 0.5 * (pr.x[1:] + pr.x[:-1])
    for dE, dB in ((np.exp(-((xc - 0.3) / 0.05) ** 2), 0 * xc), (0 * xc, np.exp(-((xc - 0.55) / 0.05) ** 2))):
        eps = 1e-5
        fd = (misfit(pr.E + eps * dE, pr.b + eps * dB) - misfit(pr.E - eps * dE, pr.b - eps * dB)) / (2 * eps)
        ad = gE @ dE + gB @ dB
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)


def test_adjoint_replays_an_active_alpha_log():
    """With a replay log active, the forward inside swale_adjoint replays it: J equals the
    misfit of a plain replayed forward, and a log that does not cover the steps is refused."""
    pr, gx, rng = basin(N=256, seed=4)
    nsteps = 12
    obs = 0.6 + 0.05 * rng.normal(size=(nsteps, gx.size))
    s = B.Solver(cfg_of(pr))
    s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
    B.swale_alpha_log(s.ctx, 1, nsteps)
    s.advance(nsteps)
    alog = np.zeros(3 * nsteps)
    B.swale_get_alpha_log(s.ctx, alog)
    s.close()
    alog_scaled = 1.1 * alog  # a different, fixed viscosity history
    J_ref = gpu_misfit_replay(pr, gx, obs, nsteps, pr.E, pr.hu, pr.b, alog_scaled)
    s = B.Solver(cfg_of(pr))
    s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
    B.swale_alpha_log(s.ctx, 2, nsteps, alog_scaled)
    J = np.zeros(1)
    B.swale_adjoint(s.ctx, nsteps, 4, gx.size, gx, obs, J, None, None, None)
    assert abs(J[0] - J_ref) <= 1e-13 * J_ref
    with pytest.raises(B.SwaleError):  # the log's rows are used up
        B.swale_adjoint(s.ctx, nsteps, 4, gx.size, gx, obs, J, None, None, None)
    s.close()
