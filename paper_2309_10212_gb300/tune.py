"""Autotuner for the renderer's free parameters.

The image does not depend on the speculation cap k_max (Sec. 4 limits it to
64), on the live-ray count below which a pass walks one ray per warp, or on
the number of views rendered together; only the time to the final image
does.  `autotune` renders a set of camera poses from a cold cache under each
candidate setting, times every render with CUDA events around the library
calls, keeps the fastest setting and applies it to the renderer."""
import ctypes
import itertools
import statistics

from . import _lib, api


def _cam_args(cam):
    f3 = ctypes.c_float * 3
    return tuple(f3(*[float(v) for v in cam[k]]) for k in ("eye", "p00", "du", "dv"))


def time_renders(r, cams, stream, reps=1):
    """Mean ms to the final image over the poses (cold cache each), with the
    renderer's current settings."""
    import torch
    L = _lib.load()
    args = [_cam_args(c) for c in cams]
    times = []
    for rep in range(reps + 1):             # the first round warms up
        for a in args:
            rs = _lib.RenderStats()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _lib.check(L.spr_reset_cache(r.handle))
            _lib.check(L.spr_set_camera(r.handle, *a))
            _lib.check(L.spr_render_to_convergence(r.handle, ctypes.c_void_p(stream.cuda_stream), 4096,
                                                   ctypes.byref(rs), None))
            e1.record(stream)
            e1.synchronize()
            if rep:
                times.append(e0.elapsed_time(e1))
    return statistics.mean(times)


def autotune(r, cams, k_max=(8, 16, 32, 64), warp_walk=(4096, 16384, 65536), reps=1, stream=None):
    """Try every (k_max, warp-walk threshold) pair with adaptive speculation;
    apply and return the fastest: {"k_max", "warp_walk", "ms", "table"}."""
    import torch
    stream = stream or torch.cuda.current_stream()
    table = []
    for k, t in itertools.product(k_max, warp_walk):
        api.spr_set_speculation(r, api.SPR_SPEC_ADAPTIVE, k_max=k)
        api.spr_set_warp_walk_threshold(r, t)
        table.append({"k_max": k, "warp_walk": t, "ms": round(time_renders(r, cams, stream, reps), 4)})
    best = min(table, key=lambda row: row["ms"])
    api.spr_set_speculation(r, api.SPR_SPEC_ADAPTIVE, k_max=best["k_max"])
    api.spr_set_warp_walk_threshold(r, best["warp_walk"])
    return dict(best, table=table)
