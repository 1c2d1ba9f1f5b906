"""The boundary is plain C: a C99 program that includes only `include/nsmg.h`
compiles with -Wall -Werror, links against the in-tree library and calls the entry
points that need no GPU (defaults, status strings, workspace sizes, argument checks)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_2008_03885_gb300", "_lib")

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "nsmg.h"

int main(void) {
  mg_options o;
  mg_default_options(&o);
  if (o.nu1 < 1 || o.nu2 < 0 || o.omega <= 0.0) return 10;
  if (strlen(mg_status_string(MG_OK)) == 0) return 11;
  mg_grid g = {4096, 1.0};
  size_t fp64 = mg_workspace_bytes(&g, 4, MG_COARSEN_REDBLACK, MG_OP_GALERKIN, &o);
  o.precision = MG_PREC_MIXED_FP32;
  size_t mixed = mg_workspace_bytes(&g, 4, MG_COARSEN_REDBLACK, MG_OP_GALERKIN, &o);
  if (fp64 == 0 || mixed <= fp64) return 12;
  mg_grid bad = {1000, 1.0};  /* not a power of two */
  if (mg_workspace_bytes(&bad, 4, MG_COARSEN_REDBLACK, MG_OP_GALERKIN, &o) != 0) return 13;
  mg_handle* h = NULL;
  if (mg_setup(&bad, 4, MG_COARSEN_REDBLACK, MG_OP_GALERKIN, &o, &h) != MG_ERR_INVALID || h) return 14;
  mg_batch_options bo = {0, 0};
  mg_batch* b = NULL;
  if (mg_batch_create_ex(NULL, 1, &bo, &b) != MG_ERR_INVALID || b) return 15;
  mg_handle* none[1] = {NULL};
  bo.workers = 65;  /* above the 64 worker streams allowed */
  if (mg_batch_create_ex(none, 1, &bo, &b) != MG_ERR_INVALID || b) return 16;
  if (mg_batch_destroy(NULL) != MG_OK) return 17;
  printf("%zu %zu\n", fp64, mixed);
  return 0;
}
"""


def _lib_present():
    return os.path.exists(os.path.join(LIBDIR, "libnsmg.so"))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c99_client_compiles_links_and_runs(tmp_path):
    if not _lib_present():
        pytest.skip("libnsmg.so not built")
    src = tmp_path / "client.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "client"
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
           "-L", LIBDIR, "-lnsmg", "-Wl,-rpath," + LIBDIR, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stderr)
    fp64, mixed = map(int, run.stdout.split())
    assert mixed > fp64 > 0
