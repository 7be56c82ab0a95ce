"""Host builds of the per-cell arithmetic for checking the hand-written adjoint (test tooling).

celltest_tangent.cpp compiles the library's swale_cell.cuh on a forward-mode dual scalar
(tangents); celltest_adjoint.cpp compiles the reverse sweeps of swale_adjoint.cuh. Both are
linked into libswale_cellcheck.so beside them; tests compare <ob, T u> with <T^T ob, u> per
function, and check the FP32 smooth-class test against the FP64 detector.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_C = os.path.join(os.path.dirname(os.path.dirname(_HERE)), "paper_2208_06588_gb300", "csrc")
_SRC = [os.path.join(_HERE, f) for f in ("celltest_tangent.cpp", "celltest_adjoint.cpp")]
_DEPS = _SRC + [os.path.join(_C, f) for f in ("swale_cell.cuh", "swale_adjoint.cuh")]
_LIB = os.path.join(_HERE, "libswale_cellcheck.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(p) for p in _DEPS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I", _C, "-o", tmp, *_SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.ct_recon_tangent.restype = ctypes.c_int
        _lib.ct_f32_trunc.restype = ctypes.c_float
        _lib.ct_f32_trunc.argtypes = [ctypes.c_double]
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def recon_tangent(h, v0, D2, D3, tv0, tD2, tD3, prm):
    val, tan = np.zeros(8), np.zeros(8)
    args = [f64(x) for x in (h, v0, D2, D3, tv0, tD2, tD3, prm)]
    flag = lib().ct_recon_tangent(*map(_p, args), _p(val), _p(tan))
    return val, tan, flag


def recon_adjoint(h, v0, D2, D3, prm, ob, known_smooth=False):
    """Reverse sweep of one cell; known_smooth takes the smooth class as given (the shortcut the
    device takes where its FP32 test holds) instead of forming the FP64 indicators."""
    v0b, D2b, D3b = np.zeros(9), np.zeros(12), np.zeros(9)
    args = [f64(x) for x in (h, v0, D2, D3, prm, ob)]
    lib().ct_recon_adjoint_k(*map(_p, args), ctypes.c_int(1 if known_smooth else 0), _p(v0b), _p(D2b), _p(D3b))
    return v0b, D2b, D3b


def recon_adjoint_lin(h, v0, D2, prm, ob):
    """Reverse sweep of a smooth-class cell from the forward's stored linear form."""
    v0b, D2b, D3b = np.zeros(9), np.zeros(12), np.zeros(9)
    args = [f64(x) for x in (h, v0, D2, prm, ob)]
    lib().ct_recon_adjoint_lin(*map(_p, args), _p(v0b), _p(D2b), _p(D3b))
    return v0b, D2b, D3b


def flux_tangent(e, te, prm):
    F, tF = np.zeros(4), np.zeros(4)
    lib().ct_flux_tangent(*map(_p, (f64(e), f64(te), f64(prm))), _p(F), _p(tF))
    return F, tF


def flux_adjoint(e, prm, Fb):
    eb = np.zeros(8)
    lib().ct_flux_adjoint(*map(_p, (f64(e), f64(prm), f64(Fb))), _p(eb))
    return eb


def source_form_tangent(hd, bd, thd, tbd, w3, g):
    S, tS = ctypes.c_double(0), ctypes.c_double(0)
    lib().ct_source_form_tangent(*map(_p, (f64(hd), f64(bd), f64(thd), f64(tbd), f64(w3))), ctypes.c_double(g),
                                 ctypes.byref(S), ctypes.byref(tS))
    return S.value, tS.value


def source_form_adjoint(hd, bd, w3, g, Sb):
    """(hdb, bdb, S) of the antisymmetric source form."""
    hdb, bdb, out = np.zeros(5), np.zeros(5), np.zeros(1)
    arrs = [f64(x) for x in (hd, bd, w3)]
    lib().ct_source_form_adjoint(*map(_p, arrs), ctypes.c_double(g), ctypes.c_double(Sb), _p(hdb), _p(bdb), _p(out))
    return hdb, bdb, out[0]


def smooth_test(w5, dx, D2h, D2m, it, eps=1e-6):
    """(FP32 test says surely smooth, FP64 class, FP64 indicators) of one cell's data: the widths
    w5[5] and length dx of its mesh factors, pair differences D2h[4], D2m[4], reciprocal triple
    sums it[3]."""
    out = np.zeros(2, dtype=np.int32)
    b = np.zeros(3)
    f = ctypes.c_double
    arrs = [f64(x) for x in (w5, D2h, D2m, it)]  # kept alive across the call
    lib().ct_smooth_test(_p(arrs[0]), f(dx), *map(_p, arrs[1:]), f(eps), _p(out), _p(b))
    return bool(out[0]), int(out[1]), b


def f32_trunc(x):
    """The device's double -> float conversion (toward zero, on the integer pipe), host build."""
    return lib().ct_f32_trunc(float(x))


def smooth1_test(proj, D2e, D2m, D2h, it, w5, dx, eps=1e-6):
    """Per-field FP32 tests, FP64 classes and FP64 gamma of the non-well-balanced scheme's three
    fields."""
    out = np.zeros(6, dtype=np.int32)
    gam = np.zeros(3)
    f = ctypes.c_double
    arrs = [f64(x) for x in (proj, D2e, D2m, D2h, it, w5)]
    lib().ct_smooth1_test(*map(_p, arrs), f(dx), f(eps), _p(out), _p(gam))
    return [bool(v) for v in out[:3]], [int(v) for v in out[3:]], gam
