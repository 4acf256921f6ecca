"""The C ABI library builds for sm_103a, loads, and exports every entry point include/gs.h declares;
a C program compiles against the header and links the library (CPU only: no GPU call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    return sorted(set(re.findall(r"GS_API\s+[\w\s\*]*?\b(gs_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("gs_field_init", "gs_add_image", "gs_select_neighbors", "gs_optimize_step", "gs_render",
                     "gs_integrate", "gs_raster_forward", "gs_raster_backward", "gs_adam_step", "gs_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2503_13086_gb300 as gs
    path = gs.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    # the binding declares argument types for exactly the header's entry points
    assert sorted(gs.SYMBOLS) == declared_symbols()


def test_host_only_calls_without_a_gpu():
    import paper_2503_13086_gb300 as gs
    lib = gs.load()
    assert b"sm_103a" in lib.gs_version()
    cfg = gs.FieldConfig()
    lib.gs_field_config_default(ctypes.byref(cfg))
    assert cfg.T_I == 200 and cfg.N_m == 10 and cfg.T_a == 200
    assert abs(cfg.eta0 - 1.6e-4) < 1e-10 and abs(cfg.etaf - 1.6e-6) < 1e-12
    assert abs(cfg.lambda_ssim - 0.2) < 1e-7
    # argument checks fail cleanly with a status and a message, no GPU touched
    assert lib.gs_field_init(None, None, None) == 1
    assert b"NULL" in lib.gs_last_error()
    assert lib.gs_wait_probe(0, None, None) == 1
    assert b"out_error" in lib.gs_last_error()
    assert lib.gs_loss_wait_probe(0, None, None) == 1
    assert b"out_error" in lib.gs_last_error()
    assert lib.gs_field_corrupt_guard(None, 0, None, 0) == 1
    assert cfg.debug_canaries == 0 and cfg.sparse_adam == 0 and cfg.densify_stats == 0


def test_tiling_candidates_on_the_host():
    import paper_2503_13086_gb300 as gs
    cands = gs.tiling_candidates()
    assert cands[0] == (16, 16, 256)  # the 3DGS tile, the default
    assert len(set(cands)) == len(cands) <= gs.MAX_TILINGS
    for tw, th, b in cands:
        # whole 8 x 4 warp blocks, at most 256 pixels (one thread each), whole 32-entry chunks
        assert tw % 8 == 0 and th % 4 == 0 and 32 <= tw * th <= 256 and b % 32 == 0
    cfg = gs.FieldConfig()
    gs.load().gs_field_config_default(ctypes.byref(cfg))
    assert cfg.tiling.astuple() == (0, 0, 0)  # autotuned by default


def test_loading_a_file_that_is_not_a_field_fails_cleanly(tmp_path):
    import paper_2503_13086_gb300 as gs
    lib = gs.load()
    junk = tmp_path / "junk.gsf"
    junk.write_bytes(b"not a field" * 10)
    h = ctypes.c_void_p()
    assert lib.gs_field_load(str(junk).encode(), None, ctypes.byref(h)) == 8  # GS_ERR_IO
    assert b"not a saved field" in lib.gs_last_error()
    assert lib.gs_field_load(str(tmp_path / "missing.gsf").encode(), None, ctypes.byref(h)) == 8
    assert not h.value


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "gs.h"
int main(void) {
  gs_field_config c;
  gs_field_config_default(&c);
  if (c.T_I != 200 || c.N_m != 10) return 1;
  /* three images in a chain 0 - 1 - 2, image 1 arriving */
  float M[9] = {0.f, 0.5f, 0.f, 0.5f, 0.f, 0.25f, 0.f, 0.25f, 0.f};
  int32_t T[3] = {10, 0, 300}, slots[200], keys[10], ns = 0, nk = 0;
  float w[3], lr[3];
  c.N_m = 2;
  if (gs_schedule_plan(&c, M, T, 3, 1, slots, &ns, keys, &nk, w, lr) != GS_OK) return 2;
  if (ns != 200 || nk != 2 || keys[0] != 1 || keys[1] != 0) return 3;
  if (w[1] != 1.f || w[0] != 0.5f || w[2] != 0.25f) return 4;
  int count[3] = {0, 0, 0};
  for (int i = 0; i < ns; ++i) count[slots[i]]++;
  if (count[0] + count[1] != 100 || count[2] != 100) return 5;  /* key half, semi-global half */
  if (gs_schedule_plan(&c, M, T, 3, 7, slots, &ns, keys, &nk, w, lr) != GS_ERR_INVALID_ARG) return 6;
  if (strlen(gs_last_error()) == 0) return 7;
  printf("ok %d %d %d\n", count[0], count[1], count[2]);
  return 0;
}
"""


def test_a_c_program_uses_the_abi(tmp_path):
    """The header is plain C (C99, pedantic) and a C program links the library and runs a host-side
    entry point (the Eq. 3-5 schedule), no GPU needed."""
    import shutil
    import subprocess
    import paper_2503_13086_gb300 as gs
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = gs.library_path()
    if not os.path.exists(lib):
        gs.build()
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(src), lib,
                        "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok")
