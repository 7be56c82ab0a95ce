"""FP64 operation counts per cell of the stage kernels (roofline numerator).

Builds csrc/opcount.cpp with g++: the kernels' own per-cell code (swale_cell.cuh) compiled
on the host with an operation-counting scalar type. A fused multiply-add counts as two
operations (one multiplication, one addition); a division or a square root counts as one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "csrc", "opcount.cpp"), os.path.join(_HERE, "csrc", "swale_cell.cuh"),
        os.path.join(_HERE, "csrc", "swale_adjoint.cuh")]
_LIB = os.path.join(_HERE, "libswale_opcount.so")
BC = {"periodic": 0, "transmissive": 1, "reflective": 2}
# RK combination of a stage per cell (stage-2 form): per variable J0*q, 0.75*(.), dt*R, Y+(.),
# 0.25*(.), sum -> 6 operations; one reciprocal of the stage width; three products.
RK_OPS = 3 * 6 + 1 + 3
# Reverse of the RK combination of one step per cell (k_adj_rk's four phases): phase 3 one
# reciprocal and 3 x 6 products; phase 2 one reciprocal and 3 x 8 operations; phase 1 one
# reciprocal and 3 x 5; phase 0 three additions.
RK_REV_OPS = 19 + 25 + 16 + 3

_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(p) for p in _SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC[0]], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.opc_count_stage.restype = None
        _lib.opc_count_reverse.restype = None
    return _lib


def count_stage(E, M, B, J, bc="transmissive", g=9.812, eps_weno=1e-6, eps_pp=1e-11, h_dry=1e-6, alpha=10.0,
                sample=None, scheme="hydrostatic"):
    E, M, B, J = (np.ascontiguousarray(a, dtype=np.float64) for a in (E, M, B, J))
    N = E.size
    n = N if sample is None else min(N, sample)
    c0 = (N - n) // 2
    out = np.zeros(20)
    vp = ctypes.c_void_p
    lib().opc_count_stage(ctypes.c_int64(N), vp(E.ctypes.data), vp(M.ctypes.data), vp(B.ctypes.data),
                          vp(J.ctypes.data), ctypes.c_int32(BC[bc]), ctypes.c_double(g), ctypes.c_double(eps_weno),
                          ctypes.c_double(eps_pp), ctypes.c_double(h_dry), ctypes.c_double(alpha),
                          ctypes.c_int64(c0), ctypes.c_int64(c0 + n), vp(out.ctypes.data),
                          ctypes.c_int32({"hydrostatic": 0, "nonwb": 1, "special": 2}[scheme]))
    rec, upd, flux = out[0:5] / n, out[5:10] / n, out[10:15] / n
    rf = float(rec[:4].sum())
    uf = float(upd[:4].sum() + RK_OPS)
    keys = ("add", "mul", "div", "sqrt", "cmp")
    return {"recon": dict(zip(keys, map(float, rec))),
            "update_without_rk": dict(zip(keys, map(float, upd))),
            "one_flux": dict(zip(keys, map(float, flux))),
            "recon_flops": rf, "update_flops": uf, "stage_flops": rf + uf, "cells_counted": n,
            "geom_flops": float(out[18] / n), "source_geom_flops": float(out[19] / n),
            "classes": [int(v) for v in out[15:18]]}


def count_reverse(E, M, B, J, bc="transmissive", g=9.812, eps_weno=1e-6, eps_pp=1e-11, h_dry=1e-6, alpha=10.0,
                  sample=None):
    """FLOPs per cell of one stage's reverse sweep (reconstruction, source, one interface flux)."""
    E, M, B, J = (np.ascontiguousarray(a, dtype=np.float64) for a in (E, M, B, J))
    N = E.size
    n = N if sample is None else min(N, sample)
    c0 = (N - n) // 2
    out = np.zeros(3)
    vp = ctypes.c_void_p
    lib().opc_count_reverse(ctypes.c_int64(N), vp(E.ctypes.data), vp(M.ctypes.data), vp(B.ctypes.data),
                            vp(J.ctypes.data), ctypes.c_int32(BC[bc]), ctypes.c_double(g), ctypes.c_double(eps_weno),
                            ctypes.c_double(eps_pp), ctypes.c_double(h_dry), ctypes.c_double(alpha),
                            ctypes.c_int64(c0), ctypes.c_int64(c0 + n), vp(out.ctypes.data))
    return {"recon_rev": float(out[0]), "source_rev": float(out[1]), "flux_rev": float(out[2]),
            "stage_rev_flops": float(out.sum()), "cells_counted": n}


def forward_step_flops(c):
    """FP64 FLOPs per cell of one SSP-RK3 step from a count_stage result: three reconstructions
    and three updates, less the mesh-only parts that stage 1 takes from the previous step's
    stage 2 on the same mesh (the reconstruction's geometry and the source term's width ratios).
    The mesh-velocity kernel is not counted."""
    return 3.0 * c["recon_flops"] - c["geom_flops"] + 3.0 * c["update_flops"] - c["source_geom_flops"]


def adjoint_step_flops(c, r, runs=3):
    """FP64 FLOPs per cell of one step of the checkpointed adjoint: `runs` forward steps (the
    forward run, the segment recompute and, unless the tape keeps the stage data, the recompute
    inside the step), each computing the mesh geometry in all three stages, and the reverse
    sweeps of the three stages with the reverse RK combination. Gauge misfit terms are not
    counted."""
    return runs * (forward_step_flops(c) + c["geom_flops"] + c["source_geom_flops"]) + 3.0 * r["stage_rev_flops"] + \
        RK_REV_OPS
