"""Seeded synthetic inputs for the 1D ALE-WENO shallow-water solver.

This module only builds input data: node coordinates, cell averages of analytic initial
conditions (5-point Gauss-Legendre per cell, split at discontinuities), prescribed mesh
motion profiles and scheme constants. It contains none of the scheme's arithmetic and is
the one module that both the CUDA path's callers and the CPU oracle's callers share.

Every problem returns a ``Problem``: cell averages (h, hu, b), the surface level
E = h + b, nodes x[0..N], widths J = diff(x), the node profile P of the prescribed motion
x_k(t) = xi_k + P_k sin(2 pi t / T) (zeros when the mesh is static or fluid-driven) and the
constants (g, CFL, boundary condition, mesh kind, T, t_end).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

G_PAPER = 9.812  # Sec. 5
MASTER_SEED = 20220812

_GL5_X = np.array([-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831, 0.9061798459386640])
_GL5_W = np.array([0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                   0.2369268850561891])


def cell_averages(f, x, breaks=()):
    """Cell averages of f over [x_j, x_{j+1}] by 5-point Gauss-Legendre, splitting each cell
    at the given discontinuity points so that piecewise-smooth data is integrated exactly
    enough."""
    x = np.asarray(x, dtype=np.float64)
    return cell_averages_between(f, x[:-1], x[1:], breaks)


def cell_averages_between(f, a, b, breaks=()):
    """Averages of f over the intervals [a_i, b_i] (5-point Gauss-Legendre, split at breaks)."""
    pts = [a] + [np.clip(np.full_like(a, c), a, b) for c in sorted(breaks)] + [b]
    total = np.zeros_like(a)
    for lo, hi in zip(pts[:-1], pts[1:]):
        half, mid = 0.5 * (hi - lo), 0.5 * (hi + lo)
        for xq, wq in zip(_GL5_X, _GL5_W):
            total += wq * half * f(mid + half * xq)
    return total / (b - a)


@dataclass
class Problem:
    name: str
    x: np.ndarray
    h: np.ndarray
    hu: np.ndarray
    b: np.ndarray
    E: np.ndarray
    profile: np.ndarray
    bc: str
    mesh: str
    mesh_T: float = 1.0
    t_end: float = 0.0
    cfl: float = 0.6
    g: float = G_PAPER
    eps_weno: float = 1e-6
    gauss_sigma: float = 8.0
    gauss_half: int = 24
    dt_fixed: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.h.size

    @property
    def J(self):
        return np.diff(self.x)


def _uniform(a, b, N):
    return a + (b - a) * np.arange(N + 1, dtype=np.float64) / N


def _paper_motion_profile(xi, xmin, xmax):
    """Node profile of the paper's default 1D motion (Sec. 5, Eq. wangge1):
    x(t) = xi + sin(2 pi t / t_end) (xi - xmax)(xi - xmin) / (3 (xmax - xmin)^2)."""
    return (xi - xmax) * (xi - xmin) / (3.0 * (xmax - xmin) ** 2)


def _sine_profile(xi, xmin, xmax, A):
    """x(t) = xi + A sin(2 pi (xi - xmin) / L) sin(2 pi t / T)."""
    p = A * np.sin(2.0 * np.pi * (xi - xmin) / (xmax - xmin))
    p[0] = 0.0
    p[-1] = 0.0
    return p


def _make(name, x, hf, huf, bf, breaks=(), lake_level=None, **kw):
    b = cell_averages(bf, x, breaks)
    hu = cell_averages(huf, x, breaks)
    if lake_level is not None:
        E = np.full_like(b, float(lake_level))
        h = E - b
    else:
        h = cell_averages(hf, x, breaks)
        E = h + b
    return Problem(name=name, x=x, h=h, hu=hu, b=b, E=E, **kw)


# --------------------------------------------------------------------------------------
# Problems of the paper's Sec. 5.1 (used as oracle pins)
# --------------------------------------------------------------------------------------
def accuracy_test(N, t_end=0.1, moving=True, cfl=0.1):
    """Sec. 5.1 accuracy test (Eq. inismoo): periodic [0,1], b = sin^2(pi x),
    h = 5 + exp(cos 2 pi x), hu = sin(cos 2 pi x), CFL 0.1, paper mesh motion with T = t_end."""
    x = _uniform(0.0, 1.0, N)
    prof = _paper_motion_profile(x, 0.0, 1.0) if moving else np.zeros(N + 1)
    return _make("accuracy", x, lambda s: 5.0 + np.exp(np.cos(2 * np.pi * s)), lambda s: np.sin(np.cos(2 * np.pi * s)),
                 lambda s: np.sin(np.pi * s) ** 2, profile=prof, bc="periodic",
                 mesh="profile" if moving else "static", mesh_T=t_end, t_end=t_end, cfl=cfl)


def lake_at_rest(N=200, bottom="smooth", t_end=0.5, moving=True):
    """Sec. 5.1 well-balance test: [0,10], eta = 10, hu = 0, b smooth 5 exp(-0.4 (x-5)^2)
    (Eq. smo1D) or the step 4 on [4,8] (Eq. dis1D); paper mesh motion with T = t_end."""
    x = _uniform(0.0, 10.0, N)
    if bottom == "smooth":
        bf, br = (lambda s: 5.0 * np.exp(-0.4 * (s - 5.0) ** 2)), ()
    else:
        bf, br = (lambda s: np.where((s >= 4.0) & (s <= 8.0), 4.0, 0.0)), (4.0, 8.0)
    prof = _paper_motion_profile(x, 0.0, 10.0) if moving else np.zeros(N + 1)
    return _make(f"lake_{bottom}", x, None, lambda s: 0.0 * s, bf, breaks=br, lake_level=10.0, profile=prof,
                 bc="transmissive", mesh="profile" if moving else "static", mesh_T=t_end, t_end=t_end)


def dry_bed(N=64, t_end=0.0, mesh="static", seed=21):
    """A dry bed at rest (h = 0, hu = 0 everywhere) over a sloping bottom with a bump, on a
    seeded nonuniform mesh of [0, 1]; transmissive. With a static mesh every wave speed is zero,
    so the CFL condition gives no bound on dt."""
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.5, 1.5, N)
    x = np.concatenate([[0.0], np.cumsum(J)])
    x /= x[-1]
    xc = 0.5 * (x[1:] + x[:-1])
    b = 0.2 * xc + 0.3 * np.exp(-((xc - 0.6) / 0.1) ** 2)
    prof = np.zeros(N + 1)
    return Problem(name="dry_bed", x=x, h=np.zeros(N), hu=np.zeros(N), b=b, E=b.copy(), profile=prof,
                   bc="transmissive", mesh=mesh, t_end=t_end)


def moses_first(N=200, t_end=2.0, moving=True):
    """Sec. 5.1 Moses's first problem (Eq. flat2): [-200,400], flat bottom, h = 5, u = 0 for
    x <= 0 and h = 10, u = 40 otherwise; transmissive; CFL 0.08."""
    x = _uniform(-200.0, 400.0, N)
    prof = _paper_motion_profile(x, -200.0, 400.0) if moving else np.zeros(N + 1)
    return _make("moses1", x, lambda s: np.where(s <= 0.0, 5.0, 10.0), lambda s: np.where(s <= 0.0, 0.0, 400.0),
                 lambda s: 0.0 * s, breaks=(0.0,), profile=prof, bc="transmissive",
                 mesh="profile" if moving else "static", mesh_T=t_end, t_end=t_end, cfl=0.08)


def moses_second(N=200, t_end=1.0, moving=True):
    """Sec. 5.1 Moses's second problem (Eq. flat3): [-300,300], h = 10 outside (-70,70), dry
    inside, u = 0; transmissive; CFL 0.08."""
    x = _uniform(-300.0, 300.0, N)
    prof = _paper_motion_profile(x, -300.0, 300.0) if moving else np.zeros(N + 1)
    return _make("moses2", x, lambda s: np.where((s > -70.0) & (s < 70.0), 0.0, 10.0), lambda s: 0.0 * s,
                 lambda s: 0.0 * s, breaks=(-70.0, 70.0), profile=prof, bc="transmissive",
                 mesh="profile" if moving else "static", mesh_T=t_end, t_end=t_end, cfl=0.08)


def _pulse_nodes_start(i):
    """Nodes of the graded mesh at t = 0 (Eq. 0.2inis), i = 0..100."""
    i = np.asarray(i, dtype=np.float64)
    return np.where(i <= 25, 0.0372 * i, np.where(i <= 75, 0.93 + 0.008 * (i - 25), 1.33 + 0.0268 * (i - 75)))


def _pulse_nodes_end(i):
    """Nodes of the graded mesh at t_end (Eq. 0.2ends), i = 0..100."""
    i = np.asarray(i, dtype=np.float64)
    return np.select([i <= 7, i <= 35, i <= 68, i <= 98],
                     [2.0 * i / 35.0, 0.4 + (i - 7) / 140.0, 0.6 + 53.0 * (i - 35) / 1650.0, 1.66 + (i - 68) / 150.0],
                     1.86 + 0.07 * (i - 98))


def big_pulse(refine=1, eps=0.2, moving=True, t_end=0.2, cfl=0.6):
    """Sec. 5.1 perturbation of a lake at rest (LeVeque's test): [0, 2], b = 0.25 (cos(10 pi
    (x - 1.5)) + 1) on [1.4, 1.6] else 0, h = 1 - b + eps on [1.1, 1.2] else 1 - b, hu = 0,
    transmissive; eps = 0.2 is the big pulse. moving=True: the graded mesh of the big-pulse
    example, 100 cells whose nodes move with constant velocities (Eq. 0.2inis, Eq. 0.2ends,
    Eq. velocity, Eq. meshspecial: x(t) = x(0) + w t, w = (x(t_end) - x(0)) / t_end); refine > 1
    splits every cell into `refine` equal cells at both ends of the motion (same grading, 100 *
    refine cells). moving=False: the uniform static mesh of the same size."""
    N = 100 * refine
    k = np.arange(N + 1) / refine
    i0 = np.minimum(np.floor(k).astype(int), 99)
    fr = k - i0
    x0 = (1 - fr) * _pulse_nodes_start(i0) + fr * _pulse_nodes_start(i0 + 1)
    x1 = (1 - fr) * _pulse_nodes_end(i0) + fr * _pulse_nodes_end(i0 + 1)
    if not moving:
        x0 = _uniform(0.0, 2.0, N)
        x1 = x0
    x0[0], x0[-1], x1[0], x1[-1] = 0.0, 2.0, 0.0, 2.0
    w = (x1 - x0) / t_end

    def bf(s):
        return np.where((s >= 1.4) & (s <= 1.6), 0.25 * (np.cos(10.0 * np.pi * (s - 1.5)) + 1.0), 0.0)

    def hf(s):
        return 1.0 - bf(s) + np.where((s >= 1.1) & (s <= 1.2), eps, 0.0)

    pr = _make("big_pulse", x0, hf, lambda s: 0.0 * s, bf, breaks=(1.1, 1.2, 1.4, 1.6), profile=w,
               bc="transmissive", mesh="linear" if moving else "static", t_end=t_end, cfl=cfl)
    pr.meta["x_end"] = x1
    return pr


# --------------------------------------------------------------------------------------
# Benchmark workloads
# --------------------------------------------------------------------------------------
def smooth_periodic(N=200, lake=False, t_end=0.1):
    """Single small instance: periodic [0,1], N = 200, b = sin^2(pi x), h = 5 + exp(cos 2 pi x),
    hu = sin(cos 2 pi x); motion x = xi + 0.05 sin(2 pi xi) sin(2 pi t); CFL 0.6, t_end = 0.1.
    lake=True: the lake at rest eta = 6, hu = 0 on the same mesh motion."""
    x = _uniform(0.0, 1.0, N)
    prof = _sine_profile(x, 0.0, 1.0, 0.05)
    if lake:
        return _make("smooth_periodic_lake", x, None, lambda s: 0.0 * s, lambda s: np.sin(np.pi * s) ** 2,
                     lake_level=6.0, profile=prof, bc="periodic", mesh="profile", mesh_T=1.0, t_end=t_end)
    return _make("smooth_periodic", x, lambda s: 5.0 + np.exp(np.cos(2 * np.pi * s)),
                 lambda s: np.sin(np.cos(2 * np.pi * s)), lambda s: np.sin(np.pi * s) ** 2, profile=prof,
                 bc="periodic", mesh="profile", mesh_T=1.0, t_end=t_end)


def _aligned_motion_profile(xi, xmin, xmax, fixed):
    """Node profile of the paper's bump-aligned motion (Eq. wangge3): x(t) = xi +
    sin(2 pi t / t_end) (xi - xmax)(xi - xmin) prod_f (xi - f) / (3 (xmax - xmin)^4); nodes
    starting at the points ``fixed`` never move."""
    p = (xi - xmax) * (xi - xmin) / (3.0 * (xmax - xmin) ** 4)
    for f in fixed:
        p = p * (xi - f)
    return p


def bump_dam_break(N=1 << 20, t_end=60.0):
    """Dam break over a rectangular bump (Sec. 5.1, Eq. bdam / inidam): [0,1500], b = 8 on
    [562.5, 937.5] else 0, eta = 20 for x <= 750 and 15 beyond, hu = 0, transmissive; the
    bump-aligned motion (Eq. wangge3) with T = t_end; the bottom is the L2 projection
    (Eq. baverage) of b onto every stage mesh. N must be a multiple of 8 so that the bump edges
    are nodes (the paper's 100 cells do not put them on nodes; see the design notes). CFL 0.6."""
    if N % 8:
        raise ValueError("N must be a multiple of 8 (bump edges on nodes)")
    x = _uniform(0.0, 1500.0, N)
    breaks = np.array([0.0, 562.5, 937.5, 1500.0])
    coef = np.array([[0.0], [8.0], [0.0]])
    xc = 0.5 * (x[1:] + x[:-1])  # every cell lies on one side of 562.5, 750 and 937.5
    b = np.where((xc > 562.5) & (xc < 937.5), 8.0, 0.0)
    E = np.where(xc < 750.0, 20.0, 15.0)
    pr = Problem(name="bump_dam_break", x=x, h=E - b, hu=np.zeros(N), b=b, E=E,
                 profile=_aligned_motion_profile(x, 0.0, 1500.0, (562.5, 937.5)), bc="transmissive",
                 mesh="profile", mesh_T=t_end, cfl=0.6)
    pr.meta["bottom"] = (breaks, coef)
    return pr


def dam_break_dry(N=1 << 20):
    """Large single instance: N cells on [0,10], transmissive; h = 2 for x < 5, 0.5 on [5,8),
    dry (h = 0) on [8,10]; hu = 0; b = 0.8 exp(-5 (x-5)^2); mesh velocity = Gaussian-smoothed
    fluid velocity (sigma 8 cells, +-24 nodes); CFL 0.08 (the paper's wet/dry value)."""
    x = _uniform(0.0, 10.0, N)
    return _make("dam_break_dry", x, lambda s: np.where(s < 5.0, 2.0, np.where(s < 8.0, 0.5, 0.0)),
                 lambda s: 0.0 * s, lambda s: 0.8 * np.exp(-5.0 * (s - 5.0) ** 2), breaks=(5.0, 8.0),
                 profile=np.zeros(N + 1), bc="transmissive", mesh="fluid_gauss", cfl=0.08,
                 gauss_sigma=8.0, gauss_half=24)


# --------------------------------------------------------------------------------------
# Batched workload: thousands of independent instances of uneven size
# --------------------------------------------------------------------------------------
@dataclass
class Batch:
    """Concatenated instances: cell offsets off[B+1], nodes of instance i at
    x[off[i] + i : off[i+1] + i + 1], per-instance CFL."""
    name: str
    off: np.ndarray
    x: np.ndarray
    h: np.ndarray
    hu: np.ndarray
    b: np.ndarray
    E: np.ndarray
    profile: np.ndarray
    cfl: np.ndarray
    bc: str = "reflective"
    mesh: str = "profile"
    mesh_T: float = 1.0
    g: float = G_PAPER
    eps_weno: float = 1e-6
    meta: dict = field(default_factory=dict)

    @property
    def B(self):
        return self.off.size - 1

    def instance(self, i) -> Problem:
        a, c = int(self.off[i]), int(self.off[i + 1])
        xs = self.x[a + i:c + i + 1]
        return Problem(name=f"{self.name}[{i}]", x=xs, h=self.h[a:c], hu=self.hu[a:c], b=self.b[a:c], E=self.E[a:c],
                       profile=self.profile[a + i:c + i + 1], bc=self.bc, mesh=self.mesh, mesh_T=self.mesh_T,
                       cfl=float(self.cfl[i]), g=self.g, eps_weno=self.eps_weno)


def many_basins(B=4096, n_min=256, n_max=16384, seed=MASTER_SEED + 3, n_cells=None):
    """B instances on [0,1], reflective, cell counts ~ U{n_min..n_max} (or all n_cells);
    bottom = sum of 1-6 Gaussians (heights U[0,0.9], centres U[0,1], widths U[0.02,0.2]);
    still water level 1 plus a Gaussian bump of amplitude U[1e-3,1e-1] (centre U[0.2,0.8],
    width 0.05); h = max(0, eta - b); hu = 0; sine motion x = xi + A sin(2 pi xi) sin(2 pi t)
    with A ~ U[0, 0.05]; CFL 0.6, or 0.08 for instances with a dry cell."""
    root = np.random.SeedSequence(seed)
    kids = root.spawn(B)
    sizes = np.empty(B, dtype=np.int64)
    parts = []
    for i, ss in enumerate(kids):
        rng = np.random.Generator(np.random.PCG64(ss))
        n = int(n_cells) if n_cells is not None else int(rng.integers(n_min, n_max + 1))
        ng = int(rng.integers(1, 7))
        amp, cen, wid = rng.uniform(0, 0.9, ng), rng.uniform(0, 1, ng), rng.uniform(0.02, 0.2, ng)
        eps, c0 = rng.uniform(1e-3, 1e-1), rng.uniform(0.2, 0.8)
        A = rng.uniform(0.0, 0.05)

        def bf(s, amp=amp, cen=cen, wid=wid):
            return sum(a * np.exp(-(s - c) ** 2 / (2 * w * w)) for a, c, w in zip(amp, cen, wid))

        def etaf(s, eps=eps, c0=c0):
            return 1.0 + eps * np.exp(-(s - c0) ** 2 / (2 * 0.05 ** 2))

        x = _uniform(0.0, 1.0, n)
        b = cell_averages(bf, x)
        h = cell_averages(lambda s: np.maximum(0.0, etaf(s) - bf(s)), x)
        prof = _sine_profile(x, 0.0, 1.0, A)
        sizes[i] = n
        parts.append((x, h, b, prof, 0.08 if np.any(h <= 0.0) else 0.6))
    off = np.zeros(B + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    x = np.concatenate([p[0] for p in parts])
    h = np.concatenate([p[1] for p in parts])
    b = np.concatenate([p[2] for p in parts])
    prof = np.concatenate([p[3] for p in parts])
    cfl = np.array([p[4] for p in parts])
    return Batch(name="many_basins", off=off, x=x, h=h, hu=np.zeros_like(h), b=b, E=h + b, profile=prof, cfl=cfl)


# --------------------------------------------------------------------------------------
# Adjoint workloads: gauge misfit of a smooth basin
# --------------------------------------------------------------------------------------
@dataclass
class GaugeProblem:
    problem: Problem
    gauges: np.ndarray   # G gauge positions
    h_obs: np.ndarray    # nsteps x G observed depths
    nsteps: int


def _gaussian_basin_fns(seed, n_gauss=4, n_basis=32):
    """Bottom and initial surface functions of gaussian_basin for one seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    amp, cen, wid = rng.uniform(0, 0.5, n_gauss), rng.uniform(0.1, 0.9, n_gauss), rng.uniform(0.05, 0.2, n_gauss)
    coef = rng.uniform(-0.01, 0.01, n_basis)
    sig = 1.0 / (2 * n_basis)
    xs = np.linspace(0.0, 1.0, 4097)
    peak = float(sum(a * np.exp(-(xs - c) ** 2 / (2 * w * w)) for a, c, w in zip(amp, cen, wid)).max())
    amp = amp * min(1.0, 0.5 / peak)

    def bf(s):
        return sum(a * np.exp(-(s - c) ** 2 / (2 * w * w)) for a, c, w in zip(amp, cen, wid))

    def etaf(s):
        # Basis functions more than 12 widths away contribute below exp(-72) and are skipped;
        # s is sorted (quadrature points of increasing cells), so each window is a slice.
        s = np.asarray(s, dtype=np.float64)
        acc = np.zeros_like(s)
        for k, ck in enumerate(coef):
            c = (k + 0.5) / n_basis
            lo, hi = np.searchsorted(s, [c - 12 * sig, c + 12 * sig])
            acc[lo:hi] += ck * np.exp(-(s[lo:hi] - c) ** 2 / (2 * sig * sig))
        return 1.0 + acc

    return bf, etaf, dict(coef=coef, amp=amp, cen=cen, wid=wid)


def gaussian_basin(N=65536, seed=MASTER_SEED + 4, n_gauss=4, n_basis=32, A=0.02, cfl=0.6):
    """[0,1], reflective; b = sum of n_gauss Gaussians (heights U[0,0.5], centres U[0.1,0.9],
    widths U[0.05,0.2]), scaled down to a maximum of 0.5 where the bumps stack higher;
    eta0 = 1 + sum_{k<n_basis} c_k exp(-(x - (k+1/2)/n_basis)^2 / (2 (1/(2 n_basis))^2)) with
    c_k ~ U[-0.01, 0.01]; hu = 0; sine motion x = xi + A sin(2 pi xi) sin(2 pi t), T = 1;
    fixed dt = 0.9 CFL min J / alpha0 with alpha0 = max sqrt(g h) + 2 pi A (the CFL value at t = 0)."""
    bf, etaf, meta = _gaussian_basin_fns(seed, n_gauss, n_basis)
    x = _uniform(0.0, 1.0, N)
    b = cell_averages(bf, x)
    E = cell_averages(etaf, x)
    h = E - b
    prof = _sine_profile(x, 0.0, 1.0, A)
    alpha0 = float(np.sqrt(G_PAPER * h.max())) + 2 * np.pi * A
    dt = 0.9 * cfl * float(np.diff(x).min()) / alpha0
    pr = Problem(name="gaussian_basin", x=x, h=h, hu=np.zeros(N), b=b, E=E, profile=prof, bc="reflective",
                 mesh="profile", mesh_T=1.0, cfl=cfl, dt_fixed=dt)
    pr.meta.update(meta)
    return pr


def _gauge_depths(N, seed, gx):
    """Initial cell-average depth of gaussian_basin(N, seed) in the cells that hold gx."""
    bf, etaf, _ = _gaussian_basin_fns(seed)
    x = _uniform(0.0, 1.0, N)
    idx = np.minimum((gx * N).astype(np.int64), N - 1)
    return cell_averages_between(etaf, x[idx], x[idx + 1]) - cell_averages_between(bf, x[idx], x[idx + 1])


def gauge_problem(N=65536, nsteps=4000, G=16, seed=MASTER_SEED + 4):
    """The basin of gaussian_basin with G gauges at (g + 1/2)/G and observations h_obs from the
    same generator with seed + 1 (different surface coefficients), sampled as the cell averages
    of the observation run's initial depth at the gauges, held for every step (a synthetic
    stand-in for recorded gauge series)."""
    pr = gaussian_basin(N=N, seed=seed)
    gx = (np.arange(G) + 0.5) / G
    h0 = _gauge_depths(N, seed + 1, gx)
    return GaugeProblem(problem=pr, gauges=gx, h_obs=np.tile(h0, (nsteps, 1)), nsteps=nsteps)


@dataclass
class GaugeBatch:
    batch: Batch
    gauges: np.ndarray   # B*G gauge positions (instance-major)
    h_obs: np.ndarray    # nsteps x B x G observed depths
    nsteps: int


def many_gauge_basins(B=512, n_min=1024, n_max=32768, nsteps=2000, G=16, seed=MASTER_SEED + 5):
    """B instances of gaussian_basin, cell counts ~ U{n_min..n_max}, each with its own seed (and
    its own observation seed) drawn from one SeedSequence; gauges and h_obs as gauge_problem.
    Every instance advances with its own CFL dt (CFL 0.6; the fixed dt of gaussian_basin is
    dropped, since a batch shares one configuration)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(n_min, n_max + 1, size=B)
    seeds = rng.integers(0, 2 ** 31, size=B)
    gx = (np.arange(G) + 0.5) / G
    parts, obs = [], []
    for n, sd in zip(sizes, seeds):
        n, sd = int(n), int(sd)
        parts.append(gaussian_basin(N=n, seed=sd))
        obs.append(_gauge_depths(n, sd + 1, gx))
    off = np.zeros(B + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    cat = lambda f: np.concatenate([f(p) for p in parts])
    bt = Batch(name="many_gauge_basins", off=off, x=cat(lambda p: p.x), h=cat(lambda p: p.h), hu=cat(lambda p: p.hu),
               b=cat(lambda p: p.b), E=cat(lambda p: p.E), profile=cat(lambda p: p.profile),
               cfl=np.full(B, 0.6))
    h_obs = np.broadcast_to(np.stack(obs)[None], (nsteps, B, G)).copy()
    return GaugeBatch(batch=bt, gauges=np.tile(gx, B), h_obs=h_obs, nsteps=nsteps)
