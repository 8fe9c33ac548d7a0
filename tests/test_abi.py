"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/gsblitz.h declares (no GPU needed: nothing is called that computes)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gsblitz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(gs_[a-z0-9_]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gs_preprocess", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_importance",
                     "gs_adam_step", "gs_photometric_loss", "gs_workspace_create", "gs_workspace_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2605_13794_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_same_exports():
    from paper_2605_13794_gb300 import binding
    assert sorted(binding.EXPORTS) == declared_functions()


def test_host_side_argument_checks_without_gpu():
    # capacity validation and default parameters run on the host only
    from paper_2605_13794_gb300 import binding as B
    L = B.lib()
    p = B.GSRenderParams()
    L.gs_default_params(ctypes.byref(p))
    assert p.tile_w == 16 and p.tile_h == 16 and abs(p.alpha_min - 1 / 255) < 1e-9 and abs(p.T_min - 1e-4) < 1e-9
    bad = B.GSCapacity(10, 10, 1 << 31, 10, 10, 1, 0)
    assert L.gs_workspace_bytes(ctypes.byref(bad)) == -1
    ok = B.GSCapacity(1000, 1000, 10000, 100, 10000, 1, 0)
    assert L.gs_workspace_bytes(ctypes.byref(ok)) > 0
    ws = ctypes.c_void_p()
    assert L.gs_workspace_create(ctypes.byref(bad), ctypes.byref(ws)) == B.GS_ERR_INVALID_ARG
    assert b"2^30" in L.gs_last_error()


def test_graph_entry_points_reject_bad_arguments_without_gpu():
    # the legacy NULL stream cannot be captured; NULL graphs are rejected or ignored
    from paper_2605_13794_gb300 import binding as B
    L = B.lib()
    null = ctypes.c_void_p(0)
    assert L.gs_graph_capture_begin(null) == B.GS_ERR_INVALID_ARG
    assert b"legacy NULL stream" in L.gs_last_error()
    out = ctypes.c_void_p(1)
    assert L.gs_graph_capture_end(null, ctypes.byref(out)) == B.GS_ERR_INVALID_ARG
    assert out.value is None
    assert L.gs_graph_capture_end(null, null) == B.GS_ERR_INVALID_ARG
    assert L.gs_graph_launch(null, null) == B.GS_ERR_INVALID_ARG
    assert L.gs_graph_destroy(null) == B.GS_OK
