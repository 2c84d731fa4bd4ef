"""The boundary used from plain C: a program compiled against include/gs.h
alone and linked to the in-tree libgs.so (no Python, no torch in it) shoots
and differentiates host-resident point sets, exact and Barnes-Hut; its
outputs match the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1907_04834_gb300 import inputs, native

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "gs.h"

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  const int64_t N = atoll(argv[1]);
  const char* dir = argv[2];
  const int mode = atoi(argv[3]);
  char path[4096];
  double* q0 = malloc(sizeof(double) * 3 * N);
  double* p0 = malloc(sizeof(double) * 3 * N);
  double* X = malloc(sizeof(double) * 3 * N);
  double* out = malloc(sizeof(double) * (9 * N + 5));
  snprintf(path, sizeof path, "%s/in.bin", dir);
  FILE* f = fopen(path, "rb");
  if (!f || fread(q0, sizeof(double), 3 * N, f) != (size_t)(3 * N) ||
      fread(p0, sizeof(double), 3 * N, f) != (size_t)(3 * N) ||
      fread(X, sizeof(double), 3 * N, f) != (size_t)(3 * N))
    return 3;
  fclose(f);
  gs_ctx* ctx = NULL;
  if (gs_create(0, &ctx) != GS_OK) return 4;
  gs_params prm = {0};
  prm.sigma = 2.0;
  prm.lambda = 1.0;
  prm.thresh_sigmas = 3.0;
  prm.T = 5;
  prm.mode = mode;
  double* q1 = out;
  double* p1 = out + 3 * N;
  double* g = out + 6 * N;
  double* H = out + 9 * N;
  double* E = out + 9 * N + 2;
  gs_status s = gs_shoot(ctx, q0, p0, N, &prm, q1, p1, H, NULL);
  if (s == GS_OK) s = gs_shoot_grad(ctx, q0, p0, X, N, &prm, E, g, NULL, NULL);
  if (s == GS_OK) s = gs_sync(ctx, NULL);
  if (s != GS_OK) {
    fprintf(stderr, "gs error %d: %s\n", (int)s, gs_last_error(ctx));
    return 5;
  }
  gs_destroy(ctx);
  snprintf(path, sizeof path, "%s/out.bin", dir);
  f = fopen(path, "wb");
  if (!f || fwrite(out, sizeof(double), 9 * N + 5, f) != (size_t)(9 * N + 5)) return 6;
  fclose(f);
  return 0;
}
"""


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = native.build()
    d = tmp_path_factory.mktemp("ccaller")
    src, exe = d / "caller.c", d / "caller"
    src.write_text(PROGRAM)
    libdir = os.path.dirname(lib)
    subprocess.run([cc, "-O2", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir],
                   check=True)
    return exe


@pytest.mark.parametrize("mode", [0, 1])
def test_c_caller_matches_oracle(oracle, program, tmp_path, mode):
    w = inputs.make("slab", 2500, 61, T=5, sigma=2.0)
    N = w.N
    np.concatenate([w.q0.ravel(), w.p0.ravel(), w.X.ravel()]).astype(np.float64).tofile(
        tmp_path / "in.bin")
    r = subprocess.run([str(program), str(N), str(tmp_path), str(mode)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(tmp_path / "out.bin", dtype=np.float64)
    q1, p1, g = (out[k * 3 * N:(k + 1) * 3 * N].reshape(N, 3) for k in range(3))
    H, E = out[9 * N:9 * N + 2], out[9 * N + 2:]
    q1o, p1o, Ho = oracle.shoot(w.q0, w.p0, 2.0, 5, mode=mode)
    Eo, go, _ = oracle.shoot_grad(w.q0, w.p0, w.X, 2.0, 5, 1.0, mode=mode)
    assert np.abs(q1 - q1o).max() <= 1e-5 * 2.0
    assert np.abs(H - Ho).max() <= 1e-5 * abs(Ho[0])
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    assert abs(E[0] - Eo[0]) <= 1e-6 * abs(Eo[0])
