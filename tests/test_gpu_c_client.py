"""The boundary from a plain C program (no Python in the loop): a C client built against
include/swale.h and libswale.so advances a problem and its result equals the Python binding's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2208_06588_gb300 import binding as B
from paper_2208_06588_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "swale.h"

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  int64_t n = 0;
  if (fread(&n, 8, 1, f) != 1) return 4;
  double* x = malloc((n + 1) * 8);
  double* eta = malloc(n * 8);
  double* hu = malloc(n * 8);
  double* b = malloc(n * 8);
  double* prof = malloc((n + 1) * 8);
  if (fread(x, 8, n + 1, f) != (size_t)(n + 1) || fread(eta, 8, n, f) != (size_t)n || fread(hu, 8, n, f) != (size_t)n ||
      fread(b, 8, n, f) != (size_t)n || fread(prof, 8, n + 1, f) != (size_t)(n + 1))
    return 5;
  fclose(f);
  swale_config cfg = {9.812, 0.6, 1e-6, 1e-11, 1e-6, 1.0, 8.0, 0.1, 0.0,
                      SWALE_BC_PERIODIC, SWALE_MESH_PROFILE, 24, 1, SWALE_SCHEME_HYDROSTATIC, 0, 0};
  swale_ctx* ctx = NULL;
  swale_status s = swale_create(&ctx, &cfg, NULL);
  if (s == SWALE_OK) s = swale_set_problem(ctx, n, x, eta, hu, b, prof, 1);
  int64_t done = 0;
  if (s == SWALE_OK) s = swale_advance(ctx, 1000000, &done);
  if (s == SWALE_OK) s = swale_get_state(ctx, NULL, hu, b, eta, x, NULL);
  if (s != SWALE_OK) {
    fprintf(stderr, "error %d: %s\n", (int)s, swale_last_error(ctx));
    return 6;
  }
  swale_destroy(ctx);
  FILE* o = fopen(argv[2], "wb");
  fwrite(&done, 8, 1, o);
  fwrite(eta, 8, n, o);
  fwrite(hu, 8, n, o);
  fclose(o);
  return 0;
}
"""


def test_c_client_matches_the_binding(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2208_06588_gb300 import build
    build.build()
    pr = W.smooth_periodic(200)
    src = tmp_path / "client.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "client"
    libdir = os.path.dirname(B.LIB_PATH)
    subprocess.run([gcc, "-std=c11", "-O1", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L",
                    libdir, "-lswale", "-Wl,-rpath," + libdir], check=True)
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        np.array([pr.N], dtype=np.int64).tofile(f)
        for a in (pr.x, pr.E, pr.hu, pr.b, pr.profile):
            np.ascontiguousarray(a, dtype=np.float64).tofile(f)
    subprocess.run([str(exe), str(inp), str(out)], check=True, timeout=300)
    raw = np.fromfile(out, dtype=np.float64)
    steps = int(raw[:1].view(np.int64)[0])
    eta_c, hu_c = raw[1:1 + pr.N], raw[1 + pr.N:1 + 2 * pr.N]
    s = B.Solver(B.make_config(cfl=0.6, mesh_T=pr.mesh_T, t_end=0.1, bc="periodic", mesh="profile"))
    s.set_problem(pr.x, pr.E, pr.hu, pr.b, pr.profile, q0_is_eta=True)
    n = s.advance(10 ** 6)
    g = s.state()
    s.close()
    assert steps == n > 0 and abs(g["t"] - 0.1) < 1e-14
    np.testing.assert_array_equal(eta_c, g["eta"])
    np.testing.assert_array_equal(hu_c, g["hu"])
