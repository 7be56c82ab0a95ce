"""bench.py's host side without a GPU: the reference arm's JSON line (the oracle timed on a
bounded sample of the workload) and the FLOP models behind the rooflines."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_flop_models():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2208_06588_gb300 import opcount
    from paper_2208_06588_gb300 import workloads as W
    pr = W.gauge_problem(N=4096, nsteps=4, G=16).problem
    c = opcount.count_stage(pr.E, pr.hu, pr.b, pr.J, bc=pr.bc)
    r = opcount.count_reverse(pr.E, pr.hu, pr.b, pr.J, bc=pr.bc)
    fwd = opcount.forward_step_flops(c)
    # three reconstructions (stage 1 without the mesh geometry) and three updates
    assert fwd == 3 * c["recon_flops"] - c["geom_flops"] + 3 * c["update_flops"] - c["source_geom_flops"]
    # the six entries of the antisymmetric source form from the width ratios (and 1 / J_j)
    assert 40 <= c["source_geom_flops"] <= 70
    assert bench.METHOD_SOURCE_GEOM_FLOPS == 7.0
    assert 1000 < fwd < 1500 and 40 < c["geom_flops"] < 120
    adj = opcount.adjoint_step_flops(c, r)
    assert adj == 3 * (fwd + c["geom_flops"] + c["source_geom_flops"]) + 3 * r["stage_rev_flops"] + opcount.RK_REV_OPS
    assert r["recon_rev"] > r["source_rev"] > r["flux_rev"] > 0
    roof = bench.fp64_roofline(1000.0, 1e9, "test")
    assert roof["bound"] == "alu" and abs(roof["achieved"] - 1.0) < 1e-12
    assert abs(roof["frac"] - 1.0 / bench.FP64_PEAK_TFLOPS) < 1e-12


def test_method_flop_counts_are_the_oracles():
    """The roofline numerators bench.py states (ORACLE_*_FLOPS) are the CPU oracle's own count of
    the method's arithmetic on the benchmark workloads (operation-counting scalar type)."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2208_06588_gb300 import workloads as W
    pr = W.dam_break_dry(1 << 18)  # the 2^20 workload's initial state, same shape (count per cell)
    P = oracle.Params(g=pr.g, cfl=pr.cfl, bc=pr.bc, mesh=pr.mesh, gauss_sigma=pr.gauss_sigma, gauss_half=pr.gauss_half)
    c = oracle.count_step(P, pr.E, pr.hu, pr.b, pr.J, pr.x)
    assert abs(c["recon"]["flops"] / bench.ORACLE_RECON_FLOPS - 1) < 5e-4
    assert abs(c["step"]["flops"] / bench.ORACLE_STEP_FLOPS - 1) < 5e-4
    # a whole step is three reconstructions and three updates, and costs more than the kernels'
    # own count (which builds the mesh geometry in closed form and reuses it across stages)
    assert 3 * c["recon"]["flops"] < c["step"]["flops"] < 8 * c["recon"]["flops"]
    bt = W.many_basins(B=4096)
    tot = cells = 0.0
    for i in range(16):
        p = bt.instance(i)
        Pi = oracle.Params(g=p.g, cfl=p.cfl, eps_weno=p.eps_weno, bc=p.bc, mesh=p.mesh, mesh_T=p.mesh_T)
        tot += oracle.count_step(Pi, p.E, p.hu, p.b, p.J, p.x, p.profile)["step"]["flops"] * p.N
        cells += p.N
    assert abs(tot / cells / bench.ORACLE_BATCH_STEP_FLOPS - 1) < 5e-4

    for scheme, (rec, stp) in bench.ORACLE_VARIANT_FLOPS.items():
        Ps = oracle.Params(g=pr.g, cfl=pr.cfl, bc=pr.bc, mesh=pr.mesh, gauss_sigma=pr.gauss_sigma,
                           gauss_half=pr.gauss_half, scheme=scheme)
        cs = oracle.count_step(Ps, pr.E, pr.hu, pr.b, pr.J, pr.x)
        assert abs(cs["recon"]["flops"] / rec - 1) < 5e-4 and abs(cs["step"]["flops"] / stp - 1) < 5e-4, scheme
