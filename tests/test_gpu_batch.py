"""Batched solver: many independent instances of uneven size advanced by the same launches.

* A batch equals its instances run one at a time, bitwise (the per-cell arithmetic does not
  depend on which block computes a cell, and every reduction is a max).
* The launch shape (tile size, persistent grid) does not change results (bitwise).
* Sampled instances agree with the CPU oracle (max-rel 1e-11 on wet instances, L1-rel 1e-9 on
  instances with dry cells).
* The autotuner restores the state it times from and reuses its cache.
"""
import os

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


def cfg_of(bt):
    return B.make_config(g=bt.g, eps_weno=bt.eps_weno, mesh_T=bt.mesh_T, bc=bt.bc, mesh=bt.mesh, cfl=0.6)


def run_batch(bt, nsteps, tiles=None):
    s = B.Solver(cfg_of(bt))
    s.set_batch(bt)
    if tiles:
        B.swale_set_tiles(s.ctx, *tiles)
    s.advance(nsteps)
    out = s.batch_state()
    out["bits"] = s.status()[0]
    s.close()
    return out


def split(bt, arr, nodes=False, i=0):
    a, c = int(bt.off[i]), int(bt.off[i + 1])
    return arr[a + i:c + i + 1] if nodes else arr[a:c]


def test_batch_equals_single_instances_bitwise():
    bt = W.many_basins(B=12, n_min=200, n_max=3000, seed=101)
    got = run_batch(bt, 12)
    for i in range(bt.B):
        pr = bt.instance(i)
        s = B.Solver(B.make_config(g=pr.g, eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, bc=pr.bc, mesh=pr.mesh,
                                   cfl=pr.cfl))
        s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
        s.advance(12)
        g = s.state()
        s.close()
        assert np.array_equal(split(bt, got["eta"], i=i), g["eta"])
        assert np.array_equal(split(bt, got["hu"], i=i), g["hu"])
        assert np.array_equal(split(bt, got["b"], i=i), g["b"])
        assert np.array_equal(split(bt, got["x"], nodes=True, i=i), g["x"])
        assert got["t"][i] == g["t"]


@pytest.mark.parametrize("tiles", [(64, 64, 0, 0), (256, 256, 0, 0), (128, 64, 300, 600), (64, 256, 152, 152)])
def test_launch_shape_does_not_change_results(tiles):
    bt = W.many_basins(B=20, n_min=100, n_max=2000, seed=102)
    ref = run_batch(bt, 10)
    got = run_batch(bt, 10, tiles)
    for k in ("eta", "hu", "b", "x", "t", "dt"):
        assert np.array_equal(ref[k], got[k]), k


def test_batch_parity_against_oracle_sampled():
    bt = W.many_basins(B=48, n_min=256, n_max=2048, seed=103)
    nsteps = 15
    got = run_batch(bt, nsteps)
    rng = np.random.default_rng(7)
    for i in sorted(rng.choice(bt.B, 10, replace=False)):
        pr = bt.instance(i)
        st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
        P = oracle.Params(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, bc=pr.bc, mesh=pr.mesh)
        oracle.run(P, st, pr.profile, nsteps=nsteps)
        dry = pr.cfl < 0.5
        for name, ref in (("eta", st.E), ("hu", st.M), ("b", st.B)):
            g = split(bt, got[name], i=i)
            if dry:
                err = np.sum(st.J * np.abs(g - ref)) / max(np.sum(st.J * np.abs(ref)), 1e-12)
                assert err < 1e-9, (i, name, err)
            else:
                err = np.abs(g - ref).max() / max(np.abs(ref).max(), 1e-3)
                assert err < 1e-11, (i, name, err)
        assert abs(got["t"][i] - st.t) <= 1e-13 * st.t


def test_full_size_batch_runs_and_samples_match(tmp_path):
    """4096 instances, 256..16384 cells each (3.4e7 cells): two steps, then sampled instances
    against the oracle."""
    bt = W.many_basins(B=4096)
    got = run_batch(bt, 2)
    assert not (got["bits"] & (B.BIT_NONFINITE | B.BIT_EMESH))
    for i in (0, 1234, 4095):
        pr = bt.instance(i)
        st = oracle.State(pr.E, pr.hu, pr.b, pr.J, pr.x)
        P = oracle.Params(g=pr.g, cfl=pr.cfl, eps_weno=pr.eps_weno, mesh_T=pr.mesh_T, bc=pr.bc, mesh=pr.mesh)
        oracle.run(P, st, pr.profile, nsteps=2)
        for name, ref in (("eta", st.E), ("hu", st.M), ("b", st.B)):
            g = split(bt, got[name], i=i)
            err = np.sum(st.J * np.abs(g - ref)) / max(np.sum(st.J * np.abs(ref)), 1e-12)
            assert err < 1e-9, (i, name, err)


def test_autotune_restores_state_and_uses_cache(tmp_path):
    bt = W.many_basins(B=16, n_min=200, n_max=3000, seed=104)
    cache = str(tmp_path / "tune.jsonl")
    s = B.Solver(cfg_of(bt))
    s.set_batch(bt)
    s.advance(3)
    before = s.batch_state()
    tiles = B.swale_autotune(s.ctx, 2, cache)
    after = s.batch_state()
    for k in ("eta", "hu", "b", "x", "t"):
        assert np.array_equal(before[k], after[k]), k
    assert tiles[0] in (64, 128, 256) and tiles[1] in (64, 128, 256)
    assert os.path.exists(cache) and open(cache).read().count("\n") == 1
    assert B.swale_autotune(s.ctx, 2, cache) == tiles  # from the cache, no new line
    assert open(cache).read().count("\n") == 1
    s.close()


def test_steps_after_autotune_match_an_untuned_run(tmp_path):
    """The candidates that the autotuner times overwrite the mesh geometry cache; the steps after
    the restore must not take it for the restored state. The first step after the restore
    recomputes the geometry from J^{n+1} where the untuned run reuses the one from J^(1) (equal
    in exact arithmetic), so the two agree to rounding."""
    bt = W.many_basins(B=12, n_min=200, n_max=3000, seed=105)
    s = B.Solver(cfg_of(bt))
    s.set_batch(bt)
    s.advance(3)
    B.swale_autotune(s.ctx, 2, str(tmp_path / "tune.jsonl"))
    s.advance(6)
    got = s.batch_state()
    s.close()
    ref = run_batch(bt, 9)
    for k in ("eta", "hu", "b", "x", "t", "dt"):
        assert np.abs(ref[k] - got[k]).max() <= 1e-13 * max(np.abs(ref[k]).max(), 1.0), k


@pytest.mark.parametrize("scheme", ["nonwb", "special"])
@pytest.mark.parametrize("tiles", [(64, 64, 0, 0), (256, 128, 0, 0), (128, 128, 304, 608)])
def test_variant_launch_shape_does_not_change_results(scheme, tiles):
    """Agreement to rounding: the compiler may fuse the geometry arithmetic into the variant's
    reconstruction differently in each tile-size instantiation of the kernel (last-bit
    differences once stage 1 reads the geometry stored by stage 2)."""
    bt = W.many_basins(B=10, n_min=100, n_max=1500, seed=106)
    cfg = B.make_config(g=bt.g, eps_weno=bt.eps_weno, mesh_T=bt.mesh_T, bc=bt.bc, mesh=bt.mesh, cfl=0.6,
                        scheme=scheme)
    outs = []
    for t in (None, tiles):
        s = B.Solver(cfg)
        s.set_batch(bt)
        if t:
            B.swale_set_tiles(s.ctx, *t)
        s.advance(8)
        outs.append(s.batch_state())
        s.close()
    for k in ("eta", "hu", "b", "x", "t"):
        assert np.abs(outs[0][k] - outs[1][k]).max() <= 1e-13 * max(np.abs(outs[0][k]).max(), 1.0), k


def test_save_and_resume(tmp_path):
    """swale_save / swale_load: a run resumed from a file continues like the uninterrupted run
    (to rounding: the first resumed step recomputes the mesh geometry), with the same time and
    step count; a context of another configuration refuses the file."""
    bt = W.many_basins(B=6, n_min=200, n_max=1500, seed=107)
    path = str(tmp_path / "state.bin")
    s = B.Solver(cfg_of(bt))
    s.set_batch(bt)
    s.advance(7)
    B.swale_save(s.ctx, path)
    s.advance(5)
    ref = s.batch_state()
    ref_status = s.status()
    s.close()
    r = B.Solver(cfg_of(bt))
    B.swale_load(r.ctx, path)
    r.N, r.B = int(bt.off[-1]), bt.B
    r.advance(5)
    got = r.batch_state()
    assert r.status()[1] == ref_status[1] == 12
    r.close()
    np.testing.assert_allclose(got["t"], ref["t"], rtol=1e-14, atol=0)
    for k in ("eta", "hu", "b", "x"):
        assert np.abs(got[k] - ref[k]).max() <= 1e-13 * max(np.abs(ref[k]).max(), 1.0), k
    other = B.Solver(B.make_config(g=bt.g, eps_weno=bt.eps_weno, mesh_T=bt.mesh_T, bc=bt.bc, mesh=bt.mesh, cfl=0.5))
    with pytest.raises(B.SwaleError):
        B.swale_load(other.ctx, path)
    other.close()


def test_save_and_resume_with_projected_bottom(tmp_path):
    pr = W.bump_dam_break(N=512)
    cfg = B.make_config(cfl=pr.cfl, mesh_T=pr.mesh_T, bc=pr.bc, mesh=pr.mesh)
    path = str(tmp_path / "bump.bin")
    s = B.Solver(cfg)
    s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
    B.swale_set_bottom_function(s.ctx, *pr.meta["bottom"])
    s.advance(10)
    B.swale_save(s.ctx, path)
    s.advance(10)
    ref = s.state()
    s.close()
    r = B.Solver(cfg)
    B.swale_load(r.ctx, path)
    r.N = pr.N
    r.advance(10)
    got = r.state()
    r.close()
    assert abs(got["t"] - ref["t"]) <= 1e-14 * ref["t"]
    np.testing.assert_allclose(got["b"], ref["b"], rtol=1e-13, atol=1e-13)
    for k in ("eta", "hu"):
        assert np.abs(got[k] - ref[k]).max() <= 1e-12 * np.abs(ref[k]).max(), k
