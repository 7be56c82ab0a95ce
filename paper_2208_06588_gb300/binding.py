"""ctypes binding of the C ABI in include/swale.h (argument marshalling only).

Every function here has the name of the C entry point it calls. Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); they are passed as raw pointers. Loading
fails loudly if the CUDA library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libswale.so")

SWALE_OK = 0
STATUS_NAMES = {0: "SWALE_OK", -1: "SWALE_EINVAL", -2: "SWALE_ENOMEM", -3: "SWALE_ECUDA", -4: "SWALE_EMESH",
                -5: "SWALE_ENEGDEPTH", -6: "SWALE_ENONFINITE", -7: "SWALE_ETIMEOUT", -8: "SWALE_EWEIGHT"}
BIT_EWEIGHT, BIT_NEGDEPTH, BIT_NONFINITE, BIT_EMESH, BIT_NODT, BIT_TIMEOUT = 1, 2, 4, 8, 16, 32
BC = {"periodic": 0, "transmissive": 1, "reflective": 2}
MESH = {"static": 0, "profile": 1, "fluid_gauss": 2, "linear": 3}
SCHEME = {"hydrostatic": 0, "nonwb": 1, "special": 2}


class SwaleConfig(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("cfl", ctypes.c_double), ("eps_weno", ctypes.c_double),
                ("eps_pp", ctypes.c_double), ("h_dry", ctypes.c_double), ("mesh_T", ctypes.c_double),
                ("gauss_sigma", ctypes.c_double), ("t_end", ctypes.c_double), ("dt_fixed", ctypes.c_double),
                ("bc", ctypes.c_int32), ("mesh", ctypes.c_int32), ("gauss_half", ctypes.c_int32),
                ("beta_dx_global", ctypes.c_int32), ("scheme", ctypes.c_int32), ("alpha_bound", ctypes.c_int32),
                ("limit_hu", ctypes.c_int32)]


def make_config(g=9.812, cfl=0.6, eps_weno=1e-6, eps_pp=1e-11, h_dry=1e-6, mesh_T=1.0, gauss_sigma=8.0,
                t_end=0.0, dt_fixed=0.0, bc="periodic", mesh="static", gauss_half=24, beta_dx_global=1,
                scheme="hydrostatic", alpha_bound=0, limit_hu=0):
    return SwaleConfig(g, cfl, eps_weno, eps_pp, h_dry, mesh_T, gauss_sigma, t_end, dt_fixed,
                       BC[bc] if isinstance(bc, str) else bc, MESH[mesh] if isinstance(mesh, str) else mesh,
                       gauss_half, beta_dx_global, SCHEME[scheme] if isinstance(scheme, str) else scheme,
                       int(alpha_bound), int(limit_hu))


class SwaleError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Loads libswale.so; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        P = ctypes.POINTER
        L.swale_create.argtypes = [P(vp), P(SwaleConfig), vp]
        L.swale_set_problem.argtypes = [vp, i64, vp, vp, vp, vp, vp, i32]
        L.swale_step.argtypes = [vp, vp]
        L.swale_advance.argtypes = [vp, i64, P(i64)]
        L.swale_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.swale_get_flags.argtypes = [vp, vp]
        L.swale_get_status.argtypes = [vp, P(ctypes.c_uint32), P(i64), P(d)]
        L.swale_rhs.argtypes = [vp, i64, vp, vp, vp, vp, vp, d, vp, vp, vp, P(d), vp, P(ctypes.c_uint32)]
        L.swale_enqueue.argtypes = [vp, i64]
        L.swale_batch_set_problem.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, i32]
        L.swale_batch_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.swale_set_tiles.argtypes = [vp, i32, i32, i32, i32]
        L.swale_get_tiles.argtypes = [vp, vp]
        L.swale_autotune.argtypes = [vp, i32, ctypes.c_char_p, vp]
        L.swale_alpha_log.argtypes = [vp, i32, i64, vp]
        L.swale_get_alpha_log.argtypes = [vp, vp]
        L.swale_adjoint.argtypes = [vp, i64, i64, i32, vp, vp, vp, vp, vp, vp]
        L.swale_adjoint_bytes.argtypes = [i64, i64, i64, i64, i32, i32, P(ctypes.c_uint64)]
        L.swale_set_adjoint_tape.argtypes = [vp, i32]
        L.swale_set_wait_test.argtypes = [vp, i32, ctypes.c_uint32]
        L.swale_set_bottom_function.argtypes = [vp, i32, i32, vp, vp]
        L.swale_save.argtypes = [vp, ctypes.c_char_p]
        L.swale_load.argtypes = [vp, ctypes.c_char_p]
        L.swale_rhs_noalloc.argtypes = [P(SwaleConfig), vp, i64, vp, vp, vp, vp, vp, d, vp, vp, vp, P(d), vp]
        L.swale_set_timing.argtypes = [vp, i32]
        L.swale_check_recip.argtypes = [vp, i64, vp, vp]
        L.swale_get_timing.argtypes = [vp, vp, vp]
        for name in ("swale_create", "swale_set_problem", "swale_step", "swale_advance", "swale_get_state",
                     "swale_get_flags", "swale_get_status", "swale_rhs", "swale_enqueue", "swale_set_timing",
                     "swale_get_timing", "swale_rhs_noalloc", "swale_batch_set_problem", "swale_batch_get_state",
                     "swale_set_tiles", "swale_get_tiles", "swale_autotune", "swale_alpha_log",
                     "swale_get_alpha_log", "swale_adjoint", "swale_adjoint_bytes", "swale_set_bottom_function", "swale_save", "swale_load",
                     "swale_check_recip"):
            getattr(L, name).restype = ctypes.c_int
        L.swale_last_error.argtypes = [vp]
        L.swale_last_error.restype = ctypes.c_char_p
        L.swale_destroy.argtypes = [vp]
        L.swale_destroy.restype = None
        _lib = L
    return _lib


def ptr(a):
    """Raw address of a numpy array or torch tensor (None stays None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def _check(ctx, code):
    if code != SWALE_OK:
        msg = lib().swale_last_error(ctx).decode() if ctx else ""
        raise SwaleError(code, msg)


def swale_create(cfg: SwaleConfig, stream=None):
    ctx = ctypes.c_void_p()
    code = lib().swale_create(ctypes.byref(ctx), ctypes.byref(cfg), stream)
    _check(None, code)
    return ctx


def swale_set_problem(ctx, N, x_nodes, q0, hu, b, profile=None, q0_is_eta=0):
    _check(ctx, lib().swale_set_problem(ctx, int(N), ptr(x_nodes), ptr(q0), ptr(hu), ptr(b), ptr(profile),
                                        int(q0_is_eta)))


def swale_step(ctx, dt_out=None):
    _check(ctx, lib().swale_step(ctx, ptr(dt_out)))


def swale_advance(ctx, max_steps):
    done = ctypes.c_int64(0)
    _check(ctx, lib().swale_advance(ctx, int(max_steps), ctypes.byref(done)))
    return done.value


def swale_batch_set_problem(ctx, B, offsets, x_nodes, q0, hu, b, profile=None, cfl=None, q0_is_eta=0):
    _check(ctx, lib().swale_batch_set_problem(ctx, int(B), ptr(offsets), ptr(x_nodes), ptr(q0), ptr(hu), ptr(b),
                                              ptr(profile), ptr(cfl), int(q0_is_eta)))


def swale_batch_get_state(ctx, hu=None, b=None, eta=None, x_nodes=None, t=None, dt=None):
    _check(ctx, lib().swale_batch_get_state(ctx, ptr(hu), ptr(b), ptr(eta), ptr(x_nodes), ptr(t), ptr(dt)))


def swale_set_tiles(ctx, recon_tile=128, update_tile=128, recon_grid=0, update_grid=0):
    _check(ctx, lib().swale_set_tiles(ctx, int(recon_tile), int(update_tile), int(recon_grid), int(update_grid)))


def swale_get_tiles(ctx):
    t = np.zeros(4, dtype=np.int32)
    _check(ctx, lib().swale_get_tiles(ctx, t.ctypes.data))
    return tuple(int(v) for v in t)


def swale_autotune(ctx, steps=3, cache_path=None):
    t = np.zeros(4, dtype=np.int32)
    cp = cache_path.encode() if cache_path else None
    _check(ctx, lib().swale_autotune(ctx, int(steps), cp, t.ctypes.data))
    return tuple(int(v) for v in t)


def swale_set_bottom_function(ctx, breaks=None, coef=None):
    """L2-projection bottom: breaks[npieces+1], coef[npieces, degree+1] (None: evolve b)."""
    if breaks is None:
        _check(ctx, lib().swale_set_bottom_function(ctx, 0, 0, None, None))
        return
    br = np.ascontiguousarray(breaks, dtype=np.float64)
    cf = np.ascontiguousarray(np.atleast_2d(coef), dtype=np.float64)
    _check(ctx, lib().swale_set_bottom_function(ctx, cf.shape[0], cf.shape[1] - 1, ptr(br), ptr(cf)))


def swale_save(ctx, path):
    _check(ctx, lib().swale_save(ctx, os.fsencode(path)))


def swale_load(ctx, path):
    _check(ctx, lib().swale_load(ctx, os.fsencode(path)))


def swale_alpha_log(ctx, mode, nsteps=0, log=None):
    _check(ctx, lib().swale_alpha_log(ctx, int(mode), int(nsteps), ptr(log)))


def swale_get_alpha_log(ctx, log):
    _check(ctx, lib().swale_get_alpha_log(ctx, ptr(log)))


def swale_adjoint(ctx, nsteps, ckpt_every, G, gauges_x, h_obs, J=None, dJ_deta0=None, dJ_dhu0=None, dJ_db0=None):
    _check(ctx, lib().swale_adjoint(ctx, int(nsteps), int(ckpt_every), int(G), ptr(gauges_x), ptr(h_obs), ptr(J),
                                    ptr(dJ_deta0), ptr(dJ_dhu0), ptr(dJ_db0)))


def swale_set_wait_test(ctx, tries, pad_bytes):
    _check(ctx, lib().swale_set_wait_test(ctx, int(tries), int(pad_bytes)))


def swale_set_adjoint_tape(ctx, enable):
    _check(ctx, lib().swale_set_adjoint_tape(ctx, int(enable)))


def swale_adjoint_bytes(B, Ntot, nsteps, ckpt_every, G, tape=0):
    n = ctypes.c_uint64(0)
    code = lib().swale_adjoint_bytes(int(B), int(Ntot), int(nsteps), int(ckpt_every), int(G), int(tape),
                                     ctypes.byref(n))
    if code != SWALE_OK:
        raise SwaleError(code, "swale_adjoint_bytes")
    return n.value


def swale_enqueue(ctx, nsteps):
    _check(ctx, lib().swale_enqueue(ctx, int(nsteps)))


def swale_set_timing(ctx, enable):
    _check(ctx, lib().swale_set_timing(ctx, 1 if enable else 0))


FAMILIES = ("prologue", "mesh_velocity", "reconstruction", "update")


def swale_get_timing(ctx):
    ms = np.zeros(4)
    n = np.zeros(4, dtype=np.int64)
    _check(ctx, lib().swale_get_timing(ctx, ms.ctypes.data, n.ctypes.data))
    return {f: (float(ms[i]), int(n[i])) for i, f in enumerate(FAMILIES)}


def swale_get_state(ctx, h=None, hu=None, b=None, eta=None, x_nodes=None, t=None):
    _check(ctx, lib().swale_get_state(ctx, ptr(h), ptr(hu), ptr(b), ptr(eta), ptr(x_nodes), ptr(t)))


def swale_get_flags(ctx, flags):
    _check(ctx, lib().swale_get_flags(ctx, ptr(flags)))


def swale_get_status(ctx):
    bits, steps, dt = ctypes.c_uint32(0), ctypes.c_int64(0), ctypes.c_double(0)
    _check(ctx, lib().swale_get_status(ctx, ctypes.byref(bits), ctypes.byref(steps), ctypes.byref(dt)))
    return bits.value, steps.value, dt.value


def swale_rhs(ctx, N, E, M, B, J, w, alpha, RE, RM, RB, flags=None):
    A = ctypes.c_double(0)
    bits = ctypes.c_uint32(0)
    _check(ctx, lib().swale_rhs(ctx, int(N), ptr(E), ptr(M), ptr(B), ptr(J), ptr(w), float(alpha), ptr(RE),
                                ptr(RM), ptr(RB), ctypes.byref(A), ptr(flags), ctypes.byref(bits)))
    return A.value, bits.value


NOALLOC_MAX_CELLS = 65536


def swale_rhs_noalloc(cfg: SwaleConfig, stream, N, E, M, B, J, w, alpha, RE, RM, RB, flags=None, want_A=True):
    """Allocation-free right-hand side: device arrays in and out, scratch in a fixed device array."""
    A = ctypes.c_double(0)
    code = lib().swale_rhs_noalloc(ctypes.byref(cfg), stream, int(N), ptr(E), ptr(M), ptr(B), ptr(J), ptr(w),
                                   float(alpha), ptr(RE), ptr(RM), ptr(RB), ctypes.byref(A) if want_A else None,
                                   ptr(flags))
    if code != SWALE_OK:
        raise SwaleError(code, "swale_rhs_noalloc")
    return A.value


def swale_check_recip(stream, n, x, y):
    """y = the kernels' reciprocal of x (device arrays of n doubles), asynchronous on stream."""
    code = lib().swale_check_recip(stream, int(n), ptr(x), ptr(y))
    if code != SWALE_OK:
        raise SwaleError(code, "swale_check_recip")


def swale_last_error(ctx):
    return lib().swale_last_error(ctx).decode()


def swale_destroy(ctx):
    lib().swale_destroy(ctx)


class Solver:
    """One solver instance: owns a context; arrays in and out are numpy (host) unless the
    caller passes torch tensors to the raw functions above."""

    def __init__(self, cfg: SwaleConfig, stream=None):
        self.ctx = swale_create(cfg, stream)
        self.N = 0

    def set_problem(self, x, q0, hu, b, profile=None, q0_is_eta=False):
        x, q0, hu, b = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, q0, hu, b))
        prof = None if profile is None else np.ascontiguousarray(profile, dtype=np.float64)
        self.N = q0.size
        swale_set_problem(self.ctx, self.N, x, q0, hu, b, prof, 1 if q0_is_eta else 0)

    def step(self):
        dt = np.zeros(1)
        swale_step(self.ctx, dt)
        return float(dt[0])

    def advance(self, max_steps):
        return swale_advance(self.ctx, max_steps)

    def state(self):
        N = self.N
        h, hu, b, eta, x, t = (np.zeros(N), np.zeros(N), np.zeros(N), np.zeros(N), np.zeros(N + 1), np.zeros(1))
        swale_get_state(self.ctx, h, hu, b, eta, x, t)
        return {"h": h, "hu": hu, "b": b, "eta": eta, "x": x, "t": float(t[0])}

    def flags(self):
        f = np.zeros(self.N, dtype=np.uint8)
        swale_get_flags(self.ctx, f)
        return f

    def status(self):
        return swale_get_status(self.ctx)

    def set_batch(self, batch, q0_is_eta=True):
        """A workloads.Batch (concatenated instances)."""
        self.N = int(batch.off[-1])
        self.B = batch.B
        arr = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        swale_batch_set_problem(self.ctx, batch.B, np.ascontiguousarray(batch.off, dtype=np.int64), arr(batch.x),
                                arr(batch.E if q0_is_eta else batch.h), arr(batch.hu), arr(batch.b),
                                arr(batch.profile), arr(batch.cfl), 1 if q0_is_eta else 0)

    def batch_state(self):
        N, B = self.N, self.B
        hu, b, eta, x, t, dt = (np.zeros(N), np.zeros(N), np.zeros(N), np.zeros(N + B), np.zeros(B), np.zeros(B))
        swale_batch_get_state(self.ctx, hu, b, eta, x, t, dt)
        return {"hu": hu, "b": b, "eta": eta, "x": x, "t": t, "dt": dt}

    def close(self):
        if self.ctx:
            swale_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
