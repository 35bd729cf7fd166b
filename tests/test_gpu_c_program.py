"""The boundary as a C program uses it on a GPU: a strict C99 program links
libfj.so and calls fj_create, fj_graph_upload, fj_solve_ex (host pointers),
fj_quantities, fj_solve_batch and fj_destroy on a weighted Erdos-Renyi graph;
its printed z and quantities match the float64 oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle.fj_oracle as fo
from paper_2101_08143_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "fj.h"

/* argv[1]: a file with "n m", then m lines "src dst w", then n lines "s" */
int main(int argc, char** argv) {
  if (argc < 2) return 1;
  FILE* f = fopen(argv[1], "r");
  long long n, m, i;
  if (!f || fscanf(f, "%lld %lld", &n, &m) != 2) return 2;
  int32_t* src = malloc(sizeof(int32_t) * m);
  int32_t* dst = malloc(sizeof(int32_t) * m);
  float* w = malloc(sizeof(float) * m);
  double* s = malloc(sizeof(double) * n);
  double* z = malloc(sizeof(double) * n);
  for (i = 0; i < m; ++i)
    if (fscanf(f, "%d %d %f", &src[i], &dst[i], &w[i]) != 3) return 3;
  for (i = 0; i < n; ++i)
    if (fscanf(f, "%lf", &s[i]) != 1) return 4;
  fclose(f);
  fj_ctx* ctx = NULL;
  fj_graph* g = NULL;
  if (fj_create(0, &ctx) != FJ_OK) return 5;
  if (fj_graph_upload(ctx, n, m, src, dst, w, FJ_HOST_PTRS, &g) != FJ_OK) return 6;
  fj_opts o;
  fj_default_opts(&o);
  fj_quant q, q2, q3;
  fj_info info;
  if (fj_solve_ex(ctx, g, 1, s, z, &q, &o, &info) != FJ_OK) return 7;
  if (fj_quantities(ctx, g, 1, s, &q2, &o, NULL) != FJ_OK) return 8;
  {
    const fj_graph* gs[1];
    int32_t ks[1] = {1};
    const double* ss[1];
    fj_quant* qs[1];
    gs[0] = g;
    ss[0] = s;
    qs[0] = &q3;
    if (fj_solve_batch(ctx, 1, gs, ks, ss, NULL, qs, &o, NULL) != FJ_OK) return 9;
  }
  printf("%.17g %.17g %.17g %.17g %.17g\n", q.C_I, q.D, q.P, q.C, q.I_dc);
  printf("%.17g %.17g %.17g %.17g %.17g\n", q2.C_I, q2.D, q2.P, q2.C, q2.I_dc);
  printf("%.17g %.17g %.17g %.17g %.17g\n", q3.C_I, q3.D, q3.P, q3.C, q3.I_dc);
  printf("%d %.3e\n", info.iterations, info.rel_residual);
  for (i = 0; i < n; ++i) printf("%.17g\n", z[i]);
  fj_graph_free(ctx, g);
  fj_destroy(ctx);
  free(src); free(dst); free(w); free(s); free(z);
  return 0;
}
"""


def test_c_program_solves_through_the_abi(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2101_08143_gb300 import fj
    fj.load()
    libdir = os.path.dirname(fj.library_path())
    exe = tmp_path / "fjc"
    (tmp_path / "fjc.c").write_text(PROGRAM)
    r = subprocess.run([cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(tmp_path / "fjc.c"), "-o", str(exe), "-L", libdir, "-lfj", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    g = synth.erdos_renyi(3000, 15000, seed=131, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 132)[:, 0]
    inp = tmp_path / "graph.txt"
    with open(inp, "w") as f:
        f.write(f"{g.n} {g.m}\n")
        for a, b, w in zip(g.src, g.dst, g.w):
            f.write(f"{int(a)} {int(b)} {float(w)!r}\n")
        for v in s:
            f.write(f"{float(v)!r}\n")
    r = subprocess.run([str(exe), str(inp)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr)
    lines = r.stdout.strip().splitlines()
    q_rows = [list(map(float, lines[j].split())) for j in range(3)]
    z = np.array([float(x) for x in lines[4:]])
    zo = fo.solve(g.n, g.src, g.dst, g.w, s)
    qo = fo.quantities_from_z(g.n, g.src, g.dst, g.w, s, zo)
    for row in q_rows:
        for name, val in zip(fo.QUANTITY_NAMES, row):
            assert fo.relative_error(qo[name], val) <= 1e-6, (name, val, qo[name])
    assert q_rows[0] == q_rows[1]
    np.testing.assert_allclose(z, zo, rtol=0, atol=1e-8)
