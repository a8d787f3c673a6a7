"""ctypes loader and prototypes for libspr.so (the C ABI of include/spr.h).

Only argument marshalling lives here: every step of the renderer runs in the
library's CUDA kernels.  Importing this module never falls back to anything:
if libspr.so is missing, loading raises."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "libspr.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "spr.h")

SPR_OK = 0
SPR_ERR_INVALID_ARG = -1
SPR_ERR_OUT_OF_MEMORY = -2
SPR_ERR_CACHE_TOO_SMALL = -3
SPR_ERR_CUDA = -4
SPR_ERR_DEVICE_TIMEOUT = -5
SPR_ERR_NOT_CONVERGED = -6
SPR_ERR_NOT_IMPLEMENTED = -7
SPR_ERR_NO_DEVICE = -8
SPR_ERR_DEVICE_ERROR = -9
SPR_SPEC_FIXED = 0
SPR_SPEC_ADAPTIVE = 1
SPR_SPEC_HASHED = 2
SPR_SPEC_LEARNED = 3
SPR_K_LIMIT = 4096
SPR_K_PER_RAY_LIMIT = 64
SPR_CODEC_FRC4 = 1


class SprError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("spr status %d: %s" % (status, message))
        self.status = status


class VolumeDesc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("rate", ctypes.c_int32), ("codec", ctypes.c_int32)]


class PassStats(ctypes.Structure):
    _fields_ = [("pass_", ctypes.c_int32), ("k", ctypes.c_int32), ("k_used", ctypes.c_int32),
                ("retries", ctypes.c_int32), ("n_active", ctypes.c_int64),
                ("n_processed", ctypes.c_int64), ("n_entries", ctypes.c_int64),
                ("n_visible", ctypes.c_int64), ("n_requested", ctypes.c_int64),
                ("n_decoded", ctypes.c_int64), ("n_evicted", ctypes.c_int64),
                ("n_term_hit", ctypes.c_int64), ("n_term_miss", ctypes.c_int64),
                ("n_active_after", ctypes.c_int64), ("utilization", ctypes.c_double),
                ("ms", ctypes.c_float), ("ms_stage", ctypes.c_float * 6),
                ("n_steps", ctypes.c_int64), ("max_steps", ctypes.c_int64)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "ms_stage"}
        d["pass"] = d.pop("pass_")
        d["ms_stage"] = list(self.ms_stage)
        return d


class RenderStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("blocks_decoded", ctypes.c_int64), ("bytes_decoded", ctypes.c_int64),
                ("entries", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("n_rays", ctypes.c_int64), ("n_hits", ctypes.c_int64),
                ("ms_total", ctypes.c_float), ("ms_raygen", ctypes.c_float),
                ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Framebuffer(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("depth", ctypes.c_void_p), ("rgba", ctypes.c_void_p),
                ("block", ctypes.c_void_p), ("cell", ctypes.c_void_p),
                ("final_pass", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("memory_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("spec_mode", ctypes.c_int32),
                ("k", ctypes.c_int32), ("k_max", ctypes.c_int32), ("max_passes", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("eye", ctypes.c_float * 3), ("p00", ctypes.c_float * 3),
                ("du", ctypes.c_float * 3), ("dv", ctypes.c_float * 3), ("iso", ctypes.c_float),
                ("t_arrival", ctypes.c_double), ("depth", ctypes.c_void_p),
                ("rgba", ctypes.c_void_p), ("block", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_first_pass", ctypes.c_double), ("t_done", ctypes.c_double),
                ("blocks_decoded", ctypes.c_int64), ("entries", ctypes.c_int64),
                ("ms_device", ctypes.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class ServerStats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("renderers", ctypes.c_int64), ("memory_used", ctypes.c_size_t),
                ("renders", ctypes.c_int64), ("requests_done", ctypes.c_int64),
                ("renderers_created", ctypes.c_int64), ("renderers_destroyed", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


SPR_POLICY_FEATURES = 12
SPR_POLICY_FLOOR = 1
SPR_POLICY_FLOOR_AFTER_FIRST = 2
SPR_POLICY_PARAMS = 5122


class TrainDesc(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("tau", ctypes.c_float), ("seed", ctypes.c_uint32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_void_p)

_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
PROTOTYPES = {
    "spr_last_error": ([], ctypes.c_char_p),
    "spr_status_string": ([_i32], ctypes.c_char_p),
    "spr_version": ([], _i32),
    "spr_set_allocator": ([ALLOC_FN, FREE_FN, _vp], _i32),
    "spr_encode_f32": ([_vp, _vp, _i32, _vp, _vp], _i32),
    "spr_encode_u8": ([_vp, _vp, _i32, _vp, _vp], _i32),
    "spr_decode_blocks": ([_vp, _i64, _i32, _vp, _i64, _vp, _vp], _i32),
    "spr_volume_decode_blocks": ([_vp, _vp, _i64, _vp, _vp], _i32),
    "spr_create_volume": ([_vp, _vp, _sz, _i32, _vp, _vp], _i32),
    "spr_destroy_volume": ([_vp], _i32),
    "spr_volume_ranges": ([_vp, _vp, _vp, _vp], _i32),
    "spr_count_active_blocks": ([_vp, ctypes.c_float, _vp, _vp, _vp], _i32),
    "spr_volume_shape": ([_vp, _vp, _vp], _i32),
    "spr_create_renderer": ([_vp, _i32, _i32, _vp], _i32),
    "spr_destroy_renderer": ([_vp], _i32),
    "spr_set_camera": ([_vp, _vp, _vp, _vp, _vp], _i32),
    "spr_set_view_count": ([_vp, _i32], _i32),
    "spr_set_view": ([_vp, _i32, _vp, _vp, _vp, _vp, ctypes.c_float], _i32),
    "spr_set_isovalue": ([_vp, ctypes.c_float], _i32),
    "spr_set_cache_budget": ([_vp, _sz], _i32),
    "spr_set_speculation": ([_vp, _i32, _i32, _i32], _i32),
    "spr_set_warp_walk_threshold": ([_vp, _i64], _i32),
    "spr_set_segment_walk": ([_vp, _i64], _i32),
    "spr_set_intersect_staging": ([_vp, _i32], _i32),
    "spr_reset_cache": ([_vp], _i32),
    "spr_set_profiling": ([_vp, _i32], _i32),
    "spr_render_pass": ([_vp, _vp, _vp], _i32),
    "spr_render_to_convergence": ([_vp, _vp, _i32, _vp, _vp], _i32),
    "spr_get_framebuffer": ([_vp, _vp], _i32),
    "spr_read_framebuffer": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "spr_exclusive_scan_u32": ([_vp, _vp, _i64, _vp, _vp], _i32),
    "spr_debug_scan_withhold": ([_vp, _vp, _i64, _i64, _i64, _vp], _i32),
    "spr_exclusive_scan_u32_noalloc": ([_vp, _vp, _i64, _vp, _vp], _i32),
    "spr_render_submit": ([_vp, _vp, _i32], _i32),
    "spr_batch_create": ([_vp, _i32, _vp], _i32),
    "spr_batch_destroy": ([_vp], _i32),
    "spr_batch_render": ([_vp, _vp, _i32, _vp], _i32),
    "spr_render_query": ([_vp, _vp, _vp], _i32),
    "spr_render_collect": ([_vp, _vp, _vp], _i32),
    "spr_renderer_memory": ([_vp, _vp], _i32),
    "spr_renderer_memory_estimate": ([_vp, _i32, _i32, _i32, _sz, _i32, _i32, _vp], _i32),
    "spr_server_create": ([_vp, _vp], _i32),
    "spr_server_destroy": ([_vp], _i32),
    "spr_server_add_volume": ([_vp, _vp, _sz, _vp], _i32),
    "spr_server_clock": ([_vp], ctypes.c_double),
    "spr_server_reserve": ([_vp, _i32, _i32, _i32, _i32], _i32),
    "spr_server_submit": ([_vp, _vp, _vp], _i32),
    "spr_server_poll": ([_vp, _vp, _i32, _vp], _i32),
    "spr_server_info": ([_vp, _vp], _i32),
    "spr_set_policy": ([_vp, _vp, ctypes.c_float, _i32], _i32),
    "spr_set_trace": ([_vp, _vp, _vp, _vp, _i64, ctypes.c_uint32], _i32),
    "spr_trace_labels": ([_vp, _vp, _vp, _vp], _i32),
    "spr_policy_forward": ([_vp, _vp, _i64, _vp, _vp], _i32),
    "spr_policy_grad": ([_vp, _vp, _vp, _i64, ctypes.c_float, _vp, _vp, _vp], _i32),
    "spr_policy_train": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp], _i32),
}

_lock = threading.Lock()
_lib = None


def load():
    """Load libspr.so (raises when it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO_PATH):
                raise RuntimeError("libspr.so is missing: run __graft_entry__.build() or "
                                   "python paper_2309_10212_gb300/build.py")
            lib = ctypes.CDLL(SO_PATH)
            for name, (args, res) in PROTOTYPES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def check(status: int):
    if status != SPR_OK:
        msg = load().spr_last_error().decode(errors="replace")
        raise SprError(status, msg or load().spr_status_string(status).decode())
    return status
