"""The boundary from C: include/mpcg.h compiles as strict C99, and a C
program linked against libmpcg.so runs host-only calls (the default options
and the smoothed-aggregation setup of a small matrix, which touch no
device)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "mpcg.h"

int main(void) {
  mpcg_options o;
  mg_amg_options a;
  if (mpcg_default_options(&o) != MPCG_OK || mg_amg_default_options(&a) != MPCG_OK) return 1;
  /* 1D Laplacian tridiag(-1, 2, -1), n = 600 */
  enum { N = 600 };
  static int ptr[N + 1], col[3 * N];
  static double val[3 * N];
  int k = 0;
  for (int i = 0; i < N; ++i) {
    ptr[i] = k;
    if (i > 0) { col[k] = i - 1; val[k++] = -1.0; }
    col[k] = i; val[k++] = 2.0;
    if (i < N - 1) { col[k] = i + 1; val[k++] = -1.0; }
  }
  ptr[N] = k;
  mg_csr A = {N, ptr, col, val};
  mg_amg_host* h = NULL;
  if (mg_amg_setup_host(&A, &a, &h) != MPCG_OK) { printf("%s\n", mpcg_last_error()); return 2; }
  printf("m=%d nu=%d theta=%.2f levels=%d fine=%lld coarse=%lld\n", o.m, o.nu, a.theta, mg_amg_host_levels(h),
         mg_amg_host_size(h, mg_amg_host_levels(h) - 1), mg_amg_host_size(h, 0));
  mg_amg_host_destroy(h);
  /* a refused request sets the message */
  A.n = 0;
  if (mg_amg_setup_host(&A, &a, &h) != MPCG_ERR_ARG) return 3;
  return 0;
}
"""


def test_header_is_c99_and_host_calls_work_from_c(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2402_12833_gb300 import build
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-lmpcg", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    line = out.stdout.strip()
    assert line.startswith("m=5 nu=2 theta=0.40 ")
    fields = dict(t.split("=") for t in line.split())
    assert int(fields["levels"]) >= 2 and int(fields["fine"]) == 600 and int(fields["coarse"]) <= 256
