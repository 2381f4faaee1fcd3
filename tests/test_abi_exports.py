"""The C-ABI library loads and exports every function include/sdg.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(sdg_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sdg_grid_create", "sdg_grid_activate_depth", "sdg_render_forward", "sdg_render_backward",
                 "sdg_adam_step", "sdg_server_submit", "sdg_train_step_rays", "sdg_last_error"):
        assert must in names
    assert len(names) >= 30


def test_library_loads_and_exports_every_declared_symbol():
    import paper_2305_13220_b300 as sdg
    lib = ctypes.CDLL(sdg._abi.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(sdg._abi.SIGNATURES) <= set(declared_functions())


def test_errors_without_gpu_work_are_reported():
    import paper_2305_13220_b300 as sdg
    A = sdg._abi
    L = A.lib()
    assert L.sdg_grid_create(None, None) == A.ERR_ARG
    assert b"null" in L.sdg_last_error()
    assert L.sdg_grid_destroy(None) == A.OK
    assert L.sdg_ctx_release(None) == A.OK
    assert L.sdg_server_destroy(None) == A.OK
    assert L.sdg_version().startswith(b"sdg")
    assert L.sdg_grid_activate_depth_frames(None, None, 1, 4, 4, None, None, 1, None) == A.ERR_ARG
