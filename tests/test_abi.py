"""The C ABI library builds for sm_103a, loads, and exports every entry point include/gs.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

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
