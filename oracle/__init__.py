"""CPU oracle of the 1D well-balanced ALE-WENO hybrid scheme (arXiv 2208.06588).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference arm of ``bench.py`` may import this package. The product path (the CUDA library and
its binding) never imports it and shares no code with it.

The arithmetic lives in ``ale_weno_oracle.cpp`` (plain C++, FP64, ``-ffp-contract=off``);
this module only builds it with g++ and marshals numpy arrays through ctypes.

Parity pins (tests/test_oracle_*.py) tie each function to something other than itself:
uniform-mesh textbook WENO5 values, polynomial reproduction on random meshes, exact
integrals, the lake-at-rest identities of Sec. 4.3, mass conservation, the exact vacuum
Riemann solution of Moses's first problem and the convergence rates of Sec. 5.1; the
detector and hybrid weights against the Jiang-Shu closed forms, the fluid-driven node velocity
against a numpy convolution, and the tangent-linear model against central differences of the
replayed forward run (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ale_weno_oracle.cpp")
_LIB = os.path.join(_HERE, "liborc_aleweno.so")

ST_EWEIGHT, ST_NEGDEPTH, ST_NONFINITE, ST_EMESH = 1, 2, 4, 8

BC = {"periodic": 0, "transmissive": 1, "reflective": 2}
MESH = {"static": 0, "profile": 1, "fluid_gauss": 2, "linear": 3}
SCHEME = {"hydrostatic": 0, "nonwb": 1, "special": 2}


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (no -march flags, portable to aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d, i32, i64, u8, u32 = (ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint8, ctypes.c_uint32)
        L.orc_weno_coeffs.argtypes = [P(d)] * 5
        L.orc_weno_coeffs.restype = None
        L.orc_beta.argtypes = [P(d), P(d), d, P(d)]
        L.orc_beta.restype = None
        L.orc_source_map.argtypes = [d, d, P(d)]
        L.orc_source_map.restype = None
        L.orc_reconstruct.argtypes = [P(d), P(i32), i64, P(d), P(d), P(d), P(d), P(d), P(u8), P(d), P(u32)]
        L.orc_reconstruct.restype = d
        L.orc_rhs.argtypes = [P(d), P(i32), i64, P(d), P(d), P(d), P(d), P(d), d, P(d), P(d), P(d), P(d)]
        L.orc_rhs.restype = u32
        L.orc_run.argtypes = [P(d), P(i32), i64, P(d), P(d), P(d), P(d), P(d), P(d), P(d), i64, P(i64), P(u8),
                              P(d), P(d)]
        L.orc_run.restype = u32
        L.orc_tangent.argtypes = [P(d), P(i32), i64, P(d), P(d), P(d), P(d), P(d), P(d), P(d), i64, P(d), P(d),
                                  P(d), P(d), P(d)]
        L.orc_tangent.restype = u32
        L.orc_fluid_velocity.argtypes = [P(d), P(i32), i64, P(d), P(d), P(d), P(d)]
        L.orc_fluid_velocity.restype = None
        L.orc_run_replay.argtypes = [P(d), P(i32), i64, P(d), P(d), P(d), P(d), P(d), P(d), P(d), i64, P(d), P(d)]
        L.orc_run_replay.restype = u32
        L.orc_count_step.argtypes = [P(d), P(i32), i64, P(d), P(d), P(d), P(d), P(d), P(d), P(d)]
        L.orc_count_step.restype = None
        L.orc_weno_point.argtypes = [P(d), d, P(d), P(d), P(d)]
        L.orc_weno_point.restype = None
        L.orc_point_phi.argtypes = [P(d), P(i32), P(d), P(d), i32, P(d)]
        L.orc_point_phi.restype = None
        L.orc_set_bottom.argtypes = [i32, i32, P(d), P(d)]
        L.orc_set_bottom.restype = None
        L.orc_bottom_average.argtypes = [P(d), P(i32), d, d]
        L.orc_bottom_average.restype = d
        _lib = L
    return _lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Scheme constants; defaults are the paper's (Sec. 5: g = 9.812, CFL 0.6, eps = 1e-6)."""
    g: float = 9.812
    cfl: float = 0.6
    eps_weno: float = 1e-6
    eps_pp: float = 1e-11
    h_dry: float = 1e-6
    mesh_T: float = 1.0
    gauss_sigma: float = 8.0
    t_end: float = 0.0
    dt_fixed: float = 0.0
    bc: str = "periodic"
    mesh: str = "static"
    gauss_half: int = 24
    beta_dx_global: int = 1
    # L2-projection bottom (Eq. baverage): (breaks[npieces+1], coef[npieces, deg+1]) of a
    # piecewise polynomial b(x) = sum_k coef[p, k] (x - breaks[p])^k, or None to evolve b by
    # Eq. bottomrk.
    bottom: tuple | None = None
    # "hydrostatic": the well-balanced scheme of Sec. 4.1; "nonwb": the ALE-WENO scheme of
    # Eq. se2D / s2D with local characteristic reconstruction and the plain LF flux; "special":
    # the well-balanced scheme with the special source term of Sec. 4.2 (Eq. special2D).
    scheme: str = "hydrostatic"
    # 0: alpha of Eq. alpha2D as written (|u - w| + sqrt(g h)) wherever w is known; 1: the bound
    # max |u| + sqrt(g h) + Wbar in every stage.
    alpha_bound: int = 0
    # 1: the limiter's theta also scales the discharge edge values (reading O6b); 0: depth only.
    limit_hu: int = 0

    def arrays(self):
        p = np.array([self.g, self.cfl, self.eps_weno, self.eps_pp, self.h_dry, self.mesh_T, self.gauss_sigma,
                      self.t_end, self.dt_fixed], dtype=np.float64)
        mode = 0
        if self.bottom is not None:
            br, cf = _f64(self.bottom[0]), np.atleast_2d(_f64(self.bottom[1]))
            lib().orc_set_bottom(cf.shape[0], cf.shape[1] - 1, _p(br), _p(np.ascontiguousarray(cf)))
            mode = 1
        ip = np.array([BC[self.bc], MESH[self.mesh], self.gauss_half, self.beta_dx_global, mode,
                       SCHEME[self.scheme], self.alpha_bound, self.limit_hu], dtype=np.int32)
        return p, ip


def weno_point(w5, t):
    """Mesh-only data at unit coordinate t of the cell: c[3,3], big[5], linear weights d[3]."""
    c, big, d = np.zeros(9), np.zeros(5), np.zeros(3)
    lib().orc_weno_point(_p(_f64(w5)), float(t), _p(c), _p(big), _p(d))
    return {"c": c.reshape(3, 3), "big": big, "d": d}


def point_phi(params: Params, d, beta, flag):
    """Hybrid weights at a point (with the negative-weight split) for linear weights d."""
    p, ip = params.arrays()
    phi = np.zeros(3)
    lib().orc_point_phi(_p(p), _p(ip, ctypes.c_int32), _p(_f64(d)), _p(_f64(beta)), int(flag), _p(phi))
    return phi


def bottom_average(params: Params, a, c):
    """Average of the projection-mode bottom over [a, c]."""
    p, ip = params.arrays()
    return lib().orc_bottom_average(_p(p), _p(ip, ctypes.c_int32), float(a), float(c))


def weno_coeffs(w5):
    w5 = _f64(w5)
    c = np.zeros((2, 3, 3)); d = np.zeros((2, 3)); big = np.zeros((2, 5)); sub = np.zeros((3, 9))
    lib().orc_weno_coeffs(_p(w5), _p(c), _p(d), _p(big), _p(sub))
    return {"c": c, "d": d, "big": big, "sub": sub.reshape(3, 3, 3)}


def beta(w5, v5, lam=1.0):
    w5, v5 = _f64(w5), _f64(v5)
    out = np.zeros(3)
    lib().orc_beta(_p(w5), _p(v5), float(lam), _p(out))
    return out


def source_map(rm, rp):
    m = np.zeros(25)
    lib().orc_source_map(float(rm), float(rp), _p(m))
    return m.reshape(5, 5)


EDGE_NAMES = ("E_L", "E_R", "M_L", "M_R", "B_L", "B_R", "h_L", "h_R", "u_L", "u_R")


def reconstruct(params: Params, E, M, B, J):
    """Reconstruction + limiter of one stage; returns (edges dict over cells -1..N, flags, gamma, A, status)."""
    p, ip = params.arrays()
    E, M, B, J = map(_f64, (E, M, B, J))
    N = E.size
    edges = np.zeros((10, N + 2))
    flags = np.zeros(N + 2, dtype=np.uint8)
    gam = np.zeros(N + 2)
    st = ctypes.c_uint32(0)
    A = lib().orc_reconstruct(_p(p), _p(ip, ctypes.c_int32), N, _p(E), _p(M), _p(B), _p(J), _p(edges),
                              _p(flags, ctypes.c_uint8), _p(gam), ctypes.byref(st))
    return dict(zip(EDGE_NAMES, edges)), flags, gam, A, st.value


def rhs(params: Params, E, M, B, J, w, alpha=0.0):
    """Semi-discrete right-hand side (R_E, R_M, R_B), alpha used, status."""
    p, ip = params.arrays()
    E, M, B, J, w = map(_f64, (E, M, B, J, w))
    N = E.size
    RE, RM, RB = np.zeros(N), np.zeros(N), np.zeros(N)
    au = ctypes.c_double(0)
    st = lib().orc_rhs(_p(p), _p(ip, ctypes.c_int32), N, _p(E), _p(M), _p(B), _p(J), _p(w), float(alpha), _p(RE),
                       _p(RM), _p(RB), ctypes.byref(au))
    return RE, RM, RB, au.value, st


@dataclass
class State:
    E: np.ndarray
    M: np.ndarray
    B: np.ndarray
    J: np.ndarray
    x: np.ndarray
    t: float = 0.0

    def copy(self):
        return State(self.E.copy(), self.M.copy(), self.B.copy(), self.J.copy(), self.x.copy(), self.t)


def run(params: Params, state: State, profile=None, nsteps=1, record=False):
    """Advance ``state`` in place by up to ``nsteps`` steps (stops at params.t_end when > 0).

    Returns dict(steps, status, flags[, dts, alphas])."""
    p, ip = params.arrays()
    for name in ("E", "M", "B", "J", "x"):
        setattr(state, name, _f64(getattr(state, name)).copy())
    N = state.E.size
    prof = _f64(profile if profile is not None else np.zeros(N + 1))
    t = ctypes.c_double(state.t)
    done = ctypes.c_int64(0)
    flags = np.zeros(N, dtype=np.uint8)
    dts = np.zeros(max(nsteps, 1)) if record else None
    als = np.zeros(3 * max(nsteps, 1)) if record else None
    st = lib().orc_run(_p(p), _p(ip, ctypes.c_int32), N, _p(state.E), _p(state.M), _p(state.B), _p(state.J),
                       _p(state.x), _p(prof), ctypes.byref(t), int(nsteps), ctypes.byref(done),
                       _p(flags, ctypes.c_uint8), _p(dts) if record else None, _p(als) if record else None)
    state.t = t.value
    out = {"steps": done.value, "status": st, "flags": flags}
    if record:
        out["dts"] = dts[:done.value].copy()
        out["alphas"] = als[:3 * done.value].copy()
    return out


def tangent(params: Params, state: State, profile, dts, alphas, dE, dM, dB):
    """Tangent-linear image of (dE, dM, dB) over len(dts) replayed steps; advances ``state`` too."""
    p, ip = params.arrays()
    for name in ("E", "M", "B", "J", "x"):
        setattr(state, name, _f64(getattr(state, name)).copy())
    N = state.E.size
    prof = _f64(profile if profile is not None else np.zeros(N + 1))
    dts, alphas = _f64(dts), _f64(alphas)
    dE, dM, dB = _f64(dE).copy(), _f64(dM).copy(), _f64(dB).copy()
    t = ctypes.c_double(state.t)
    st = lib().orc_tangent(_p(p), _p(ip, ctypes.c_int32), N, _p(state.E), _p(state.M), _p(state.B), _p(state.J),
                           _p(state.x), _p(prof), ctypes.byref(t), int(dts.size), _p(dts), _p(alphas), _p(dE),
                           _p(dM), _p(dB))
    state.t = t.value
    return dE, dM, dB, st


def fluid_velocity(params: Params, E, M, B):
    """Node velocities w[N+1] of the fluid-driven (Gaussian-filtered) mesh motion for a state."""
    p, ip = params.arrays()
    E, M, B = map(_f64, (E, M, B))
    w = np.zeros(E.size + 1)
    lib().orc_fluid_velocity(_p(p), _p(ip, ctypes.c_int32), E.size, _p(E), _p(M), _p(B), _p(w))
    return w


def run_replay(params: Params, state: State, profile, dts, alphas):
    """Advance ``state`` in place by len(dts) steps with the given dt and stage alphas (replay)."""
    p, ip = params.arrays()
    for name in ("E", "M", "B", "J", "x"):
        setattr(state, name, _f64(getattr(state, name)).copy())
    N = state.E.size
    prof = _f64(profile if profile is not None else np.zeros(N + 1))
    dts, alphas = _f64(dts), _f64(alphas)
    t = ctypes.c_double(state.t)
    st = lib().orc_run_replay(_p(p), _p(ip, ctypes.c_int32), N, _p(state.E), _p(state.M), _p(state.B),
                              _p(state.J), _p(state.x), _p(prof), ctypes.byref(t), int(dts.size), _p(dts),
                              _p(alphas))
    state.t = t.value
    return st


def count_step(params: Params, E, M, B, J, x, profile=None):
    """The oracle's own operation counts, per cell, of one stage's reconstruction + limiter and of
    one whole SSP-RK3 step on the given state: {"recon": {...}, "step": {...}} with add, mul,
    div, sqrt and flops (their sum) each. Only arithmetic on state-dependent values is counted
    (the oracle builds the mesh-only coefficients by Gaussian elimination, not counted)."""
    p, ip = params.arrays()
    E, M, B, J, x = map(_f64, (E, M, B, J, x))
    N = E.size
    prof = _f64(profile if profile is not None else np.zeros(N + 1))
    c = np.zeros(8)
    lib().orc_count_step(_p(p), _p(ip, ctypes.c_int32), N, _p(E), _p(M), _p(B), _p(J), _p(x), _p(prof), _p(c))
    out = {}
    for k, name in enumerate(("recon", "step")):
        v = c[4 * k:4 * k + 4] / N
        out[name] = dict(zip(("add", "mul", "div", "sqrt"), map(float, v)))
        out[name]["flops"] = float(v.sum())
    return out
