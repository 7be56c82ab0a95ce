"""The error contract of swale_advance on the GPU: a step in which an error appears is not
committed. The instance keeps the state, nodes, time and step count of its last good step,
later steps (also inside captured 8-step graphs) are no-ops for it, and in a batch the other
instances go on. Every failure is made on the host side of the contract: a prescribed mesh
motion that inverts a cell (SWALE_EMESH), the bounded-wait test hook (SWALE_ETIMEOUT) and a dry
bed at rest without an end time (no finite dt). Nothing faults or hangs a GPU.
"""
import numpy as np
import pytest

import oracle
from paper_2208_06588_gb300 import binding as B

pytestmark = pytest.mark.gpu

KEYS = ("eta", "hu", "b", "x")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_06588_gb300 import build
    build.build()
    B.lib()


def inverting(N=300, a=0.005, k=None):
    """Smooth water over a bump on [0, 1]; the profile moves nodes k and k+1 towards each other
    (x = xi + P sin(2 pi t)), so that with a fixed dt the cell between them inverts after a few
    dozen steps."""
    x = np.linspace(0.0, 1.0, N + 1)
    xc = 0.5 * (x[1:] + x[:-1])
    b = 0.2 * np.exp(-((xc - 0.5) / 0.1) ** 2)
    E = 1.0 + 0.01 * np.sin(2 * np.pi * xc)
    hu = 0.05 * np.cos(2 * np.pi * xc)
    P = np.zeros(N + 1)
    k = N // 3 if k is None else k
    P[k], P[k + 1] = a, -a
    return x, E, hu, b, P


CFG = dict(bc="transmissive", mesh="profile", mesh_T=1.0, dt_fixed=1e-3)


def _solver(x, E, hu, b, P):
    s = B.Solver(B.make_config(**CFG))
    s.set_problem(x, E, hu, b, P, q0_is_eta=True)
    return s


def _good_run(x, E, hu, b, P, k):
    s = _solver(x, E, hu, b, P)
    assert s.advance(k) == k
    g = s.state()
    assert s.status()[0] == 0
    s.close()
    return g


def test_inverting_mesh_keeps_the_last_good_step():
    x, E, hu, b, P = inverting()
    # the oracle fails in the same step (it stops after the failing step)
    st = oracle.State(E, hu, b, np.diff(x), x)
    r = oracle.run(oracle.Params(**CFG), st, P, nsteps=200)
    assert r["status"] & oracle.ST_EMESH
    k = r["steps"] - 1  # good steps
    s = _solver(x, E, hu, b, P)
    with pytest.raises(B.SwaleError) as err:
        s.advance(200)  # 25 graphs of 8 steps: the failure happens inside one
    assert err.value.code == -4
    bits, steps, _ = s.status()
    assert bits & B.BIT_EMESH and steps == k
    g = s.state()
    # later steps are no-ops for the failed instance
    with pytest.raises(B.SwaleError):
        s.advance(16)
    g2 = s.state()
    assert s.status()[1] == k
    s.close()
    ref = _good_run(x, E, hu, b, P, k)
    for key in KEYS:
        assert np.array_equal(g[key], ref[key]), key
        assert np.array_equal(g2[key], ref[key]), key
    assert g["t"] == ref["t"] == g2["t"]
    assert np.diff(g["x"]).min() > 0.0


def test_single_steps_follow_the_contract():
    """swale_step one at a time: the failing step and every later one leave the state alone."""
    x, E, hu, b, P = inverting(a=0.01)
    s = _solver(x, E, hu, b, P)
    for _ in range(40):
        s.step()
    bits, steps, _ = s.status()
    g = s.state()
    s.close()
    assert bits & B.BIT_EMESH and 10 < steps < 40
    ref = _good_run(x, E, hu, b, P, steps)
    for key in KEYS:
        assert np.array_equal(g[key], ref[key]), key


def test_batch_instance_failure_leaves_the_others_running():
    """Three instances of different sizes in one batch; the middle one inverts a cell. It keeps
    its last good step, the other two run every step, each equal bitwise to its own run."""
    insts = [inverting(N=200, a=0.0), inverting(N=257, a=0.005, k=100), inverting(N=130, a=0.0)]
    off = np.cumsum([0] + [len(i[1]) for i in insts]).astype(np.int64)
    cat = lambda j: np.concatenate([i[j] for i in insts])
    s = B.Solver(B.make_config(**CFG))
    s.N, s.B = int(off[-1]), 3
    B.swale_batch_set_problem(s.ctx, 3, off, cat(0), cat(1), cat(2), cat(3), cat(4), None, 1)
    with pytest.raises(B.SwaleError) as err:
        s.advance(80)
    assert err.value.code == -4
    out = s.batch_state()
    s.close()
    for i, inst in enumerate(insts):
        one = _solver(*inst)
        n = one.advance(80) if i != 1 else None
        if i == 1:
            with pytest.raises(B.SwaleError):
                one.advance(80)
            n = one.status()[1]
            one.close()
            ref = _good_run(*inst, n)
            assert 10 < n < 80
        else:
            assert n == 80
            ref = one.state()
            one.close()
        a, c = int(off[i]), int(off[i + 1])
        assert np.array_equal(out["eta"][a:c], ref["eta"]), i
        assert np.array_equal(out["hu"][a:c], ref["hu"]), i
        assert np.array_equal(out["x"][a + i:c + i + 1], ref["x"]), i
        assert out["t"][i] == ref["t"], i


def test_timeout_keeps_the_last_good_step():
    """Five good steps, then the bounded-wait hook makes every later step time out: the state is
    bitwise that of the five steps and the step count stays 5."""
    x, E, hu, b, P = inverting(a=0.0)
    s = _solver(x, E, hu, b, P)
    assert s.advance(5) == 5
    B.swale_set_wait_test(s.ctx, 16, 16)
    with pytest.raises(B.SwaleError) as err:
        s.advance(11)
    assert err.value.code == -7
    B.swale_set_wait_test(s.ctx, 0, 0)
    bits, steps, _ = s.status()
    g = s.state()
    s.close()
    assert bits & B.BIT_TIMEOUT and steps == 5
    ref = _good_run(x, E, hu, b, P, 5)
    for key in KEYS:
        assert np.array_equal(g[key], ref[key]), key


def test_adjoint_larger_than_the_device_is_refused_and_the_context_goes_on():
    """A gradient whose checkpoints cannot fit in device memory: swale_adjoint returns
    SWALE_ENOMEM (its one scratch allocation fails; nothing runs), and the context then steps and
    differentiates like a fresh one."""
    import torch
    N, G = 20000, 2
    x, E, hu, b, P = inverting(N=N, a=0.0)
    cfg = dict(CFG, dt_fixed=1e-5)  # CFL about 0.6 on 20000 cells
    total = torch.cuda.mem_get_info()[1]
    nsteps = int(2 * total // (5 * 8 * N)) + 1
    need = B.swale_adjoint_bytes(1, N, nsteps, 1, G)
    assert need > 1.5 * total
    gx = np.array([0.25, 0.75])
    obs = np.full((nsteps, G), 0.9)  # the full observation array, although it is never read

    def solver():
        s = B.Solver(B.make_config(**cfg))
        s.set_problem(x, E, hu, b, P, q0_is_eta=True)
        return s

    s = solver()
    with pytest.raises(B.SwaleError) as err:
        B.swale_adjoint(s.ctx, nsteps, 1, G, gx, obs, np.zeros(1), np.zeros(N))
    assert err.value.code == -2
    assert s.status()[0] == 0
    assert s.advance(3) == 3
    g = s.state()
    J = np.zeros(1)
    B.swale_adjoint(s.ctx, 4, 2, G, gx, obs[:4], J, np.zeros(N))
    s.close()
    r = solver()
    assert r.advance(3) == 3
    ref = r.state()
    assert r.status()[0] == 0
    r.close()
    for key in KEYS:
        assert np.array_equal(g[key], ref[key]), key
    assert np.isfinite(J[0]) and J[0] > 0
