"""The boundary as a C program sees it: include/fj.h compiles as strict C99,
a program links against libfj.so, and the host-only calls (defaults,
version, argument checks, last error) behave as declared; the struct sizes
a C compiler gives match the ctypes binding.  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

from paper_2101_08143_gb300 import fj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "fj.h"

int main(void) {
  fj_opts o;
  fj_info info;
  fj_default_opts(&o);
  if (!(o.tol > 0.0) || o.precision != FJ_PREC_MIXED || o.flags != FJ_HOST_PTRS) return 2;
  if (fj_solve_ex(NULL, NULL, 1, NULL, NULL, NULL, NULL, &info) != FJ_ERR_ARG) return 3;
  if (strstr(fj_last_error(), "non-NULL") == NULL) return 4;
  if (fj_set_grid(NULL, 1) != FJ_ERR_ARG || fj_tune(NULL, NULL, 1, NULL, NULL, 1, NULL) != FJ_ERR_ARG) return 5;
  printf("%s|%u|%u|%u|%u\n", fj_version(), (unsigned)sizeof(fj_opts), (unsigned)sizeof(fj_info),
         (unsigned)sizeof(fj_quant), (unsigned)sizeof(fj_tune_result));
  return 0;
}
"""


def test_header_compiles_as_c99_and_links(tmp_path):
    import ctypes
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = fj.load()  # builds libfj.so if needed
    libdir = os.path.dirname(fj.library_path())
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-lfj", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    version, s_opts, s_info, s_quant, s_tune = r.stdout.strip().split("|")
    assert version == lib.fj_version().decode()
    assert int(s_opts) == ctypes.sizeof(fj.Opts)
    assert int(s_info) == ctypes.sizeof(fj.Info)
    assert int(s_quant) == ctypes.sizeof(fj.Quant)
    assert int(s_tune) == ctypes.sizeof(fj.TuneResult)
