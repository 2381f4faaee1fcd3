"""ctypes declarations of libsdg's C ABI (include/sdg.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SDG_LIBRARY selects another build of the library in this directory (libsdg_checked.so: the bounds-checked build)
LIB_PATH = os.path.join(HERE, os.environ.get("SDG_LIBRARY", "libsdg.so"))

OK, ERR_ARG, ERR_OOM, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_IO, ERR_NOT_FOUND = range(9)
F32, BF16 = 0, 1
GROUP_GEO, GROUP_SDF, GROUP_RGB, GROUP_SEM, GROUP_WEIGHT = range(5)
KIND_VALUE, KIND_GRAD, KIND_ADAM_M, KIND_ADAM_V = range(4)
MODE_RECOMPUTE, MODE_STORE = 0, 1
ORDER_AUTO, ORDER_GIVEN, ORDER_SURFACE = 0, 1, 2
OPT_ADAM, OPT_RMSPROP = 0, 1
WALK_PASS, WALK_IN_WARP = 0, 1
TRACE_CELLS = 32

ERROR_NAMES = {OK: "SDG_OK", ERR_ARG: "SDG_ERR_ARG", ERR_OOM: "SDG_ERR_OOM", ERR_CAPACITY: "SDG_ERR_CAPACITY",
               ERR_CUDA: "SDG_ERR_CUDA", ERR_TIMEOUT: "SDG_ERR_TIMEOUT", ERR_BUSY: "SDG_ERR_BUSY",
               ERR_IO: "SDG_ERR_IO", ERR_NOT_FOUND: "SDG_ERR_NOT_FOUND"}


class GridDesc(C.Structure):
    _fields_ = [("voxel_size", C.c_float), ("beta", C.c_float), ("max_blocks", C.c_int64),
                ("rgb_dtype", C.c_int32), ("n_sem", C.c_int32), ("device", C.c_int32), ("reserved", C.c_int32),
                ("stream", C.c_void_p)]


class RenderOpts(C.Structure):
    _fields_ = [("n_samples", C.c_int32), ("seed", C.c_uint32), ("ray_id0", C.c_uint32), ("stratified", C.c_int32),
                ("mode", C.c_int32), ("bg", C.c_float * 3)]


class RenderOut(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("opac", C.c_void_p), ("sem", C.c_void_p)]


class LossOpts(C.Structure):
    _fields_ = [("lambda_depth", C.c_float), ("lambda_sem", C.c_float), ("ray_order", C.c_int32),
                ("learn_beta", C.c_int32), ("norm_rays", C.c_int64), ("prepared", C.c_int32),
                ("reserved", C.c_int32)]


class AdamOpts(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("step", C.c_int32), ("algo", C.c_int32)]


class TraceOut(C.Structure):
    _fields_ = [("n_cells", C.c_void_p), ("S", C.c_void_p), ("t", C.c_void_p), ("cell", C.c_void_p),
                ("block", C.c_void_p), ("valid", C.c_void_p), ("seg", C.c_void_p), ("rgb", C.c_void_p),
                ("depth", C.c_void_p), ("opac", C.c_void_p)]


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32), ("n_streams", C.c_int32),
                ("chunk_rays", C.c_int32), ("max_batch_rays", C.c_int32), ("device", C.c_int32),
                ("reserved", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("scene_id", C.c_int32), ("H", C.c_int32), ("W", C.c_int32), ("K", C.c_float * 4),
                ("Twc", C.c_float * 12), ("n_samples", C.c_int32), ("seed", C.c_uint32), ("stratified", C.c_int32),
                ("tnear", C.c_float), ("tfar", C.c_float)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("H", C.c_int32), ("W", C.c_int32), ("rgb", C.c_void_p),
                ("depth", C.c_void_p), ("opac", C.c_void_p), ("t_submit_ms", C.c_double),
                ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("launches", C.c_int64), ("rays_rendered", C.c_int64), ("bytes_in_use", C.c_int64),
                ("peak_bytes_in_use", C.c_int64), ("in_flight", C.c_int32), ("queued", C.c_int32)]


_p = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_P = C.POINTER

SIGNATURES = {
    "sdg_grid_create": [_P(GridDesc), _P(_p)],
    "sdg_grid_destroy": [_p],
    "sdg_grid_activate_points": [_p, _p, _i64, _i32, _P(_i64)],
    "sdg_grid_activate_depth": [_p, _p, _i32, _i32, _P(C.c_float), _P(C.c_float), _i32, _P(_i64)],
    "sdg_grid_activate_depth_frames": [_p, _p, _i32, _i32, _i32, _P(C.c_float), _P(C.c_float), _i32, _P(_i64)],
    "sdg_grid_activate_keys": [_p, _p, _i64, _P(_i64)],
    "sdg_grid_num_blocks": [_p, _P(_i64)],
    "sdg_grid_keys": [_p, _p],
    "sdg_grid_lookup": [_p, _p, _i64, _p],
    "sdg_grid_channel": [_p, _i32, _i32, _P(_p), _P(_i64)],
    "sdg_grid_zero_grad": [_p],
    "sdg_grid_save": [_p, C.c_char_p],
    "sdg_grid_load": [C.c_char_p, _P(GridDesc), _P(_p)],
    "sdg_grid_get_step": [_p, _P(_i32)],
    "sdg_grid_set_step": [_p, _i32],
    "sdg_grid_sync": [_p],
    "sdg_grid_set_pass_events": [_p, _p, _p],
    "sdg_checked_status": [_i32, _i32, _P(C.c_uint64), _P(_i32)],
    "sdg_render_forward": [_p, _p, _i64, _P(RenderOpts), _P(RenderOut), _P(_p)],
    "sdg_render_backward": [_p, _p, _p, _p, _p],
    "sdg_ctx_release": [_p],
    "sdg_loss_l1": [_p, _i64, _p, _p, _p, _p, _p, _p, _P(LossOpts), _p, _p, _p, _p],
    "sdg_query": [_p, _p, _i64, _p, _p],
    "sdg_eikonal": [_p, _p, _i64, C.c_float, _p, _p],
    "sdg_grid_get_beta": [_p, _p],
    "sdg_grid_set_beta": [_p, C.c_float],
    "sdg_grid_beta_grad": [_p, _p],
    "sdg_loss_depth_ssi": [_p, _i64, _p, _p, C.c_float, _p, _p, _p, _p],
    "sdg_train_step_rays_normal": [_p, _p, _i64, _p, _p, _p, _P(RenderOpts), _P(LossOpts), C.c_float, _p, _p],
    "sdg_lattice_filter": [_p, _i64, C.c_int32, _p, C.c_int32, _p, _p, C.c_int32, _p],
    "sdg_crf_meanfield": [_p, _i64, C.c_int32, _p, C.c_int32, _p, _p, C.c_float, _p],
    "sdg_crf_loss": [_p, C.c_int32, _i64, _p, _p, C.c_float, _p, _p],
    "sdg_fuse_frames": [_p, _i64, C.c_int32, C.c_int32, _p, _p, _p, _p, _p, C.c_float],
    "sdg_fuse_finalize": [_p],
    "sdg_train_step_rays": [_p, _p, _i64, _p, _p, _p, _P(RenderOpts), _P(LossOpts), _p, _p],
    "sdg_train_prepare": [_p, _p, _i64, _p, _P(LossOpts), _i32],
    "sdg_adam_step": [_p, _P(AdamOpts)],
    "sdg_server_create": [_P(ServerOpts), _P(_p)],
    "sdg_server_add_scene": [_p, _p, _P(_i32)],
    "sdg_server_submit": [_p, _P(Request), _P(C.c_uint64)],
    "sdg_server_poll": [_p, C.c_uint64, _P(Result)],
    "sdg_server_wait": [_p, C.c_uint64, _i64, _P(Result)],
    "sdg_server_release": [_p, C.c_uint64],
    "sdg_server_get_stats": [_p, _P(ServerStats)],
    "sdg_server_destroy": [_p],
    "sdg_debug_fail_alloc_after": [_i64],
    "sdg_debug_trace": [_p, _p, _i64, _P(RenderOpts), _i32, _P(TraceOut)],
    "sdg_debug_trace_view": [_p, _i32, _i32, _P(C.c_float), _P(C.c_float), C.c_float, C.c_float, _P(RenderOpts),
                             _p, _P(TraceOut)],
}

_lib = None


class SdgError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib():
    """The loaded libsdg.so.  Raises ImportError when the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsdg.so is not built ({LIB_PATH}); run `python paper_2305_13220_b300/build.py`")
        L = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.sdg_last_error.restype = C.c_char_p
        L.sdg_last_error.argtypes = []
        L.sdg_version.restype = C.c_char_p
        L.sdg_version.argtypes = []
        _lib = L
    return _lib


def check(code: int, where: str):
    if code != OK:
        raise SdgError(code, where, lib().sdg_last_error().decode(errors="replace"))
    return code


def call(name: str, *args) -> int:
    """Calls an ABI function and raises SdgError on a non-OK status."""
    return check(getattr(lib(), name)(*args), name)


def checked_status(device: int = 0, clear: bool = False):
    """(status word, whether the loaded library is the bounds-checked build); see sdg_checked_status."""
    st, ck = C.c_uint64(), C.c_int32()
    call("sdg_checked_status", device, 1 if clear else 0, C.byref(st), C.byref(ck))
    return st.value, bool(ck.value)
