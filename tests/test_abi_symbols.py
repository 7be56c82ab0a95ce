"""The C ABI library loads and exports every entry point that include/swale.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(swale_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("swale_create", "swale_set_problem", "swale_step", "swale_advance", "swale_get_state",
                 "swale_get_flags", "swale_rhs", "swale_last_error", "swale_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2208_06588_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    L = ctypes.CDLL(binding.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_abi():
    from paper_2208_06588_gb300 import binding
    for n in declared_symbols():
        assert hasattr(binding, n), n


def test_autograd_wrapper_has_no_cpu_path():
    import torch

    from paper_2208_06588_gb300 import binding as B
    from paper_2208_06588_gb300.autograd import gauge_misfit
    z = torch.zeros(8, dtype=torch.float64, requires_grad=True)
    with pytest.raises(ValueError, match="CUDA"):
        gauge_misfit(z, z, z, torch.linspace(0, 1, 9), None, [0.5], [[0.0]], B.make_config(), 1)


def test_adjoint_bytes_formula():
    """swale_adjoint_bytes is host arithmetic: 5 (ceil(K/C) + 2 C + 3) + 201 doubles and two
    bytes per cell, plus per-instance scalars, gauges, observations and the viscosity log, and
    up to 511 bytes per array (each is rounded up to 256 bytes and keeps 256 bytes of slack)."""
    from paper_2208_06588_gb300 import binding as B
    Nt, Bn, K, C, G = 1_000_000, 4, 4000, 64, 16
    n = B.swale_adjoint_bytes(Bn, Nt, K, C, G)
    per_cell = 8 * (5 * (-(-K // C) + 2 * C + 3) + 201) + 2
    assert per_cell * Nt <= n <= per_cell * Nt + 8 * (K * Bn * (G + 3)) + 2_000_000
    assert B.swale_adjoint_bytes(Bn, Nt, K, K, G) > B.swale_adjoint_bytes(Bn, Nt, K, 64, G)
    # with the tape: (ceil(K/C) + 2 C + 1) state copies and 2 C tape slots of 81 doubles per cell
    nt = B.swale_adjoint_bytes(Bn, Nt, K, C, G, tape=1)
    per_cell_t = 8 * (5 * (-(-K // C) + 2 * C + 1) + 50 + 2 * C * 81) + 1
    assert per_cell_t * Nt <= nt <= per_cell_t * Nt + 8 * (K * Bn * (G + 3)) + 4_000_000
    with pytest.raises(B.SwaleError):
        B.swale_adjoint_bytes(0, Nt, K, C, G)
    with pytest.raises(B.SwaleError):
        B.swale_adjoint_bytes(Bn, Nt, K, C, G, tape=2)


C_CLIENT = r"""
#include <stdio.h>
#include "swale.h"

/* A plain C client of the boundary: one instance, a few steps, the state back. */
int run(const double* x, const double* eta, const double* hu, const double* b, int64_t n, double* out_eta) {
  swale_config cfg = {9.812, 0.6, 1e-6, 1e-11, 1e-6, 1.0, 8.0, 0.0, 0.0,
                      SWALE_BC_PERIODIC, SWALE_MESH_STATIC, 24, 1, SWALE_SCHEME_HYDROSTATIC, 0, 0};
  swale_ctx* ctx = NULL;
  swale_status s = swale_create(&ctx, &cfg, NULL);
  if (s != SWALE_OK) return (int)s;
  s = swale_set_problem(ctx, n, x, eta, hu, b, NULL, 1);
  int64_t done = 0;
  if (s == SWALE_OK) s = swale_advance(ctx, 10, &done);
  if (s == SWALE_OK) s = swale_get_state(ctx, NULL, NULL, NULL, out_eta, NULL, NULL);
  if (s != SWALE_OK) fprintf(stderr, "%s\n", swale_last_error(ctx));
  swale_destroy(ctx);
  return (int)s;
}
"""


def test_header_is_plain_c_and_links(tmp_path):
    """include/swale.h compiles as C11 (no C++ in the boundary) and a C client links against the
    library (nothing is run: no GPU here)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2208_06588_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    inc = os.path.join(ROOT, "include")
    obj = tmp_path / "client.o"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-pedantic", "-fPIC", "-I", inc, "-c", str(src), "-o",
                    str(obj)], check=True)
    libdir = os.path.dirname(binding.LIB_PATH)
    subprocess.run([gcc, "-shared", "-o", str(tmp_path / "libclient.so"), str(obj), "-L", libdir, "-lswale",
                    "-Wl,-rpath," + libdir], check=True)
