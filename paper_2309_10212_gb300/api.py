"""Python binding of the C ABI (include/spr.h), same names as the C calls.

Device buffers are torch CUDA tensors and streams are torch streams; the
binding only marshals pointers and sizes.  Every computation runs in the CUDA
library; without a built libspr.so or a CUDA device the calls raise."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (SPR_CODEC_FRC4, SPR_K_LIMIT, SPR_K_PER_RAY_LIMIT, SPR_SPEC_ADAPTIVE,  # noqa: F401
                   SPR_SPEC_FIXED, SPR_SPEC_HASHED, SPR_SPEC_LEARNED, SprError, check, load)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise SprError(_lib.SPR_ERR_NO_DEVICE, "CUDA is not available")
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_ptr(t, dtype=None):
    torch = _torch()
    assert isinstance(t, torch.Tensor) and t.is_cuda, "expected a CUDA tensor"
    assert t.is_contiguous(), "expected a contiguous tensor"
    if dtype is not None:
        assert t.dtype == dtype, "expected %s, got %s" % (dtype, t.dtype)
    return ctypes.c_void_p(t.data_ptr())


def _f3(v):
    a = (ctypes.c_float * 3)()
    a[:] = [float(x) for x in np.asarray(v, dtype=np.float32)]
    return a


def _i3(v):
    a = (ctypes.c_int32 * 3)()
    a[:] = [int(x) for x in v]
    return a


def nblocks(dims):
    return tuple((int(d) + 3) // 4 for d in dims)


def spr_version() -> int:
    return load().spr_version()


# ------------------------------------------------------------------ codec
def spr_encode_u8(vol, rate: int, out=None, stream=None):
    """Compress a CUDA uint8 volume of shape (Dz, Dy, Dx); returns the block
    stream as a CUDA uint8 tensor."""
    torch = _torch()
    dims = (vol.shape[2], vol.shape[1], vol.shape[0])
    nb = nblocks(dims)
    if out is None:
        out = torch.empty(nb[0] * nb[1] * nb[2] * 8 * rate, dtype=torch.uint8, device=vol.device)
    check(load().spr_encode_u8(_dev_ptr(vol, torch.uint8), _i3(dims), rate, _dev_ptr(out),
                               _stream(stream)))
    return out


def spr_encode_f32(vol, rate: int, out=None, stream=None):
    torch = _torch()
    dims = (vol.shape[2], vol.shape[1], vol.shape[0])
    nb = nblocks(dims)
    if out is None:
        out = torch.empty(nb[0] * nb[1] * nb[2] * 8 * rate, dtype=torch.uint8, device=vol.device)
    check(load().spr_encode_f32(_dev_ptr(vol, torch.float32), _i3(dims), rate, _dev_ptr(out),
                                _stream(stream)))
    return out


def spr_decode_blocks(blocks, n_blocks: int, rate: int, ids=None, n=None, out=None,
                      stream=None):
    """Decompress blocks (all of them, or the CUDA uint32 `ids`) into a CUDA
    float32 tensor of shape (n, 64)."""
    torch = _torch()
    if n is None:
        n = n_blocks if ids is None else ids.numel()
    if out is None:
        out = torch.empty((n, 64), dtype=torch.float32, device=blocks.device)
    idp = None if ids is None else _dev_ptr(ids, torch.int32)
    check(load().spr_decode_blocks(_dev_ptr(blocks), int(n_blocks), rate, idp, int(n),
                                   _dev_ptr(out, torch.float32), _stream(stream)))
    return out


def spr_exclusive_scan_u32(x, out=None, stream=None):
    """Exclusive prefix sum of a CUDA int32 tensor (read as uint32); returns
    (out, total)."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(x)
    total = torch.zeros(1, dtype=torch.int32, device=x.device)
    check(load().spr_exclusive_scan_u32(_dev_ptr(x), _dev_ptr(out), x.numel(), _dev_ptr(total),
                                        _stream(stream)))
    return out, total


def spr_exclusive_scan_u32_noalloc(x, out, total, stream=None):
    """The allocation-free prefix sum: the caller supplies `out` (like x) and
    `total` (one int32 on the device); the library allocates nothing."""
    check(load().spr_exclusive_scan_u32_noalloc(_dev_ptr(x), _dev_ptr(out), x.numel(),
                                                _dev_ptr(total), _stream(stream)))
    return out, total


def spr_debug_scan_withhold(x, withhold_tile: int, spin_limit: int, out=None, stream=None):
    """The bounded-wait test hook; returns the status instead of raising."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(x)
    return load().spr_debug_scan_withhold(_dev_ptr(x), _dev_ptr(out), x.numel(),
                                          int(withhold_tile), int(spin_limit), _stream(stream))


# ----------------------------------------------------------------- volume
class Volume:
    def __init__(self, handle, dims, rate):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)
        self.rate = rate

    @property
    def nblocks(self):
        return nblocks(self.dims)

    def close(self):
        if self.handle:
            spr_destroy_volume(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spr_create_volume(dims, rate: int, blocks, stream=None) -> Volume:
    """blocks: CUDA uint8 tensor (copied on the device) or numpy uint8 array
    (copied from the host)."""
    desc = _lib.VolumeDesc()
    desc.dims[:] = [int(d) for d in dims]
    desc.rate = rate
    desc.codec = SPR_CODEC_FRC4
    h = ctypes.c_void_p()
    L = load()
    if isinstance(blocks, np.ndarray):
        b = np.ascontiguousarray(blocks, dtype=np.uint8)
        _torch()
        check(L.spr_create_volume(ctypes.byref(desc), b.ctypes.data_as(ctypes.c_void_p), b.nbytes,
                                  0, _stream(stream), ctypes.byref(h)))
    else:
        check(L.spr_create_volume(ctypes.byref(desc), _dev_ptr(blocks), blocks.numel(), 1,
                                  _stream(stream), ctypes.byref(h)))
    return Volume(h, dims, rate)


def spr_volume_decode_blocks(vol: Volume, ids=None, n=None, out=None, stream=None):
    """Decompress blocks of a volume (all of them, or the CUDA uint32 `ids`)
    into a CUDA float32 tensor of shape (n, 64), grouped by parse length the
    way the renderer decodes its cache misses; the values equal
    spr_decode_blocks'."""
    torch = _torch()
    if n is None:
        nb = vol.nblocks
        n = nb[0] * nb[1] * nb[2] if ids is None else ids.numel()
    if out is None:
        out = torch.empty((n, 64), dtype=torch.float32, device="cuda" if ids is None else ids.device)
    idp = None if ids is None else _dev_ptr(ids, torch.int32)
    check(load().spr_volume_decode_blocks(vol.handle, idp, int(n), _dev_ptr(out, torch.float32),
                                          _stream(stream)))
    return out


def spr_destroy_volume(vol: Volume):
    if vol.handle:
        check(load().spr_destroy_volume(vol.handle))
        vol.handle = None


def spr_volume_ranges(vol: Volume, stream=None):
    """(fine, coarse) value ranges as float32 arrays of shape (n, 2)."""
    nb = ctypes.c_int64 * 3
    a, c = nb(), nb()
    check(load().spr_volume_shape(vol.handle, a, c))
    fine = np.zeros((a[0] * a[1] * a[2], 2), np.float32)
    coarse = np.zeros((c[0] * c[1] * c[2], 2), np.float32)
    check(load().spr_volume_ranges(vol.handle, fine.ctypes.data_as(ctypes.c_void_p),
                                   coarse.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return fine, coarse


def spr_count_active_blocks(vol: Volume, iso: float, stream=None):
    """(active, needed): blocks whose range holds iso, and those plus their
    +x/+y/+z neighbours (what decoding every active block costs)."""
    a, n = ctypes.c_int64(), ctypes.c_int64()
    check(load().spr_count_active_blocks(vol.handle, float(iso), ctypes.byref(a), ctypes.byref(n),
                                         _stream(stream)))
    return a.value, n.value


# --------------------------------------------------------------- renderer
class Renderer:
    def __init__(self, handle, vol: Volume, W: int, H: int):
        self.handle = handle
        self.vol = vol
        self.W, self.H = W, H
        self._recs = None   # per-pass record buffer, reused across renders

    def records(self, n: int):
        """A ctypes array of at least n pass records (kept between calls)."""
        if self._recs is None or len(self._recs) < n:
            self._recs = (_lib.PassStats * n)()
        return self._recs

    def close(self):
        if self.handle:
            spr_destroy_renderer(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spr_create_renderer(vol: Volume, W: int, H: int) -> Renderer:
    h = ctypes.c_void_p()
    check(load().spr_create_renderer(vol.handle, W, H, ctypes.byref(h)))
    return Renderer(h, vol, W, H)


def spr_destroy_renderer(r: Renderer):
    if r.handle:
        check(load().spr_destroy_renderer(r.handle))
        r.handle = None


def spr_set_camera(r: Renderer, eye, p00=None, du=None, dv=None):
    """eye may be a dict with keys eye, p00, du, dv (as synth.cameras makes)."""
    if isinstance(eye, dict):
        eye, p00, du, dv = eye["eye"], eye["p00"], eye["du"], eye["dv"]
    check(load().spr_set_camera(r.handle, _f3(eye), _f3(p00), _f3(du), _f3(dv)))


def spr_set_view_count(r: Renderer, n_views: int):
    check(load().spr_set_view_count(r.handle, int(n_views)))


def spr_set_view(r: Renderer, view: int, cam: dict, iso: float):
    """cam: a dict with eye, p00, du, dv (as synth.cameras makes)."""
    check(load().spr_set_view(r.handle, int(view), _f3(cam["eye"]), _f3(cam["p00"]), _f3(cam["du"]),
                              _f3(cam["dv"]), float(iso)))


def spr_set_isovalue(r: Renderer, iso: float):
    check(load().spr_set_isovalue(r.handle, float(iso)))


def spr_set_cache_budget(r: Renderer, nbytes: int):
    check(load().spr_set_cache_budget(r.handle, int(nbytes)))


def spr_set_speculation(r: Renderer, mode: int, k: int = 1, k_max: int = 64):
    check(load().spr_set_speculation(r.handle, int(mode), int(k), int(k_max)))


def spr_set_warp_walk_threshold(r: Renderer, n_rays: int):
    check(load().spr_set_warp_walk_threshold(r.handle, int(n_rays)))


def spr_set_segment_walk(r: Renderer, lanes: int):
    check(load().spr_set_segment_walk(r.handle, int(lanes)))


def spr_set_intersect_staging(r: Renderer, on: bool):
    check(load().spr_set_intersect_staging(r.handle, 1 if on else 0))


def spr_reset_cache(r: Renderer):
    check(load().spr_reset_cache(r.handle))


def spr_set_profiling(r: Renderer, on: bool):
    check(load().spr_set_profiling(r.handle, 1 if on else 0))


def spr_render_pass(r: Renderer, stream=None) -> dict:
    st = _lib.PassStats()
    check(load().spr_render_pass(r.handle, _stream(stream), ctypes.byref(st)))
    return st.as_dict()


def spr_render_to_convergence(r: Renderer, max_passes: int = 10000, stream=None,
                              allow_partial: bool = False):
    """Returns (render stats, [pass stats])."""
    rs = _lib.RenderStats()
    per = r.records(min(max_passes, 4096))
    status = load().spr_render_to_convergence(r.handle, _stream(stream), int(max_passes),
                                              ctypes.byref(rs), per)
    if not (allow_partial and status == _lib.SPR_ERR_NOT_CONVERGED):
        check(status)
    return rs.as_dict(), [per[i].as_dict() for i in range(min(rs.passes, max_passes, 4096))]


class Batch:
    """Renderers rendered together by one graph launch (spr_batch_*)."""

    def __init__(self, handle, renderers):
        self.handle = handle
        self.renderers = list(renderers)   # kept alive with the batch

    def close(self):
        if self.handle:
            check(load().spr_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spr_batch_create(renderers) -> Batch:
    arr = (ctypes.c_void_p * len(renderers))(*[r.handle.value if hasattr(r.handle, "value") else r.handle
                                              for r in renderers])
    h = ctypes.c_void_p()
    check(load().spr_batch_create(arr, len(renderers), ctypes.byref(h)))
    return Batch(h, renderers)


def spr_batch_render(b: Batch, max_passes: int = 10000, stream=None):
    """Returns each renderer's render stats."""
    stats = (_lib.RenderStats * len(b.renderers))()
    check(load().spr_batch_render(b.handle, _stream(stream), int(max_passes), stats))
    return [stats[i].as_dict() for i in range(len(b.renderers))]


def spr_get_framebuffer(r: Renderer) -> dict:
    """Zero-copy CUDA tensors viewing the renderer's framebuffer."""
    torch = _torch()
    fb = _lib.Framebuffer()
    check(load().spr_get_framebuffer(r.handle, ctypes.byref(fb)))
    n = fb.width * fb.height

    class _View:
        def __init__(self, ptr, typestr):
            self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                             "data": (ptr, False), "version": 2}
    out = {}
    for name, typestr in (("depth", "<f4"), ("rgba", "<u4"), ("block", "<u4"), ("cell", "<u8"),
                          ("final_pass", "<i4"), ("status", "|u1")):
        out[name] = torch.as_tensor(_View(getattr(fb, name), typestr), device="cuda")
    return out


def spr_read_framebuffer(r: Renderer, stream=None) -> dict:
    """Host copies (numpy) of the framebuffer (all views, stacked)."""
    fb = _lib.Framebuffer()
    check(load().spr_get_framebuffer(r.handle, ctypes.byref(fb)))
    n = fb.width * fb.height
    out = dict(depth=np.empty(n, np.float32), rgba=np.empty(n, np.uint32),
               block=np.empty(n, np.uint32), cell=np.empty(n, np.uint64),
               final_pass=np.empty(n, np.int32), status=np.empty(n, np.uint8))
    p = {k: v.ctypes.data_as(ctypes.c_void_p) for k, v in out.items()}
    check(load().spr_read_framebuffer(r.handle, _stream(stream), p["depth"], p["rgba"],
                                      p["block"], p["cell"], p["final_pass"], p["status"]))
    return out


# ---------------------------------------------------- asynchronous render
def spr_render_submit(r: Renderer, max_passes: int = 10000, stream=None):
    """Enqueue a whole render on `stream` without waiting."""
    check(load().spr_render_submit(r.handle, _stream(stream), int(max_passes)))


def spr_render_query(r: Renderer):
    """(passes completed so far, device finished) of a submitted render."""
    p, d = ctypes.c_int32(), ctypes.c_int32()
    check(load().spr_render_query(r.handle, ctypes.byref(p), ctypes.byref(d)))
    return p.value, bool(d.value)


def spr_render_collect(r: Renderer, allow_partial: bool = False):
    """Wait for the submitted render; returns (render stats, [pass stats])."""
    rs = _lib.RenderStats()
    per = r.records(4096)
    status = load().spr_render_collect(r.handle, ctypes.byref(rs), per)
    if not (allow_partial and status == _lib.SPR_ERR_NOT_CONVERGED):
        check(status)
    return rs.as_dict(), [per[i].as_dict() for i in range(min(rs.passes, 4096))]


def spr_renderer_memory(r: Renderer) -> int:
    n = ctypes.c_size_t()
    check(load().spr_renderer_memory(r.handle, ctypes.byref(n)))
    return n.value


def spr_renderer_memory_estimate(vol: Volume, W: int, H: int, n_views: int, cache_bytes: int,
                                 mode: int = SPR_SPEC_ADAPTIVE, k: int = 1) -> int:
    n = ctypes.c_size_t()
    check(load().spr_renderer_memory_estimate(vol.handle, int(W), int(H), int(n_views),
                                              int(cache_bytes), int(mode), int(k), ctypes.byref(n)))
    return n.value


# ---------------------------------------------------- learned speculation
SPR_POLICY_FEATURES = _lib.SPR_POLICY_FEATURES
SPR_POLICY_PARAMS = _lib.SPR_POLICY_PARAMS


def _params(params):
    p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
    assert p.size == SPR_POLICY_PARAMS, "expected %d parameters" % SPR_POLICY_PARAMS
    return p


SPR_POLICY_FLOOR = _lib.SPR_POLICY_FLOOR
SPR_POLICY_FLOOR_AFTER_FIRST = _lib.SPR_POLICY_FLOOR_AFTER_FIRST


def spr_set_policy(r: Renderer, params, margin: float = 0.0, floor="all"):
    """params: SPR_POLICY_PARAMS floats (W1[64][12], b1, W2[64][64], b2,
    W3[2][64], b3); floor: "all" (counts never below the paper's uniform
    count), "after_first" (from the second pass on) or None/False."""
    p = _params(params)
    if floor is True or floor == "all":
        flags = SPR_POLICY_FLOOR
    elif floor == "after_first":
        flags = SPR_POLICY_FLOOR_AFTER_FIRST
    else:
        flags = 0
    check(load().spr_set_policy(r.handle, p.ctypes.data_as(ctypes.c_void_p), float(margin), flags))


class Trace:
    """Device buffers of a training trace (features, ray ids, blocks taken
    before the sample, labels)."""

    def __init__(self, capacity: int):
        torch = _torch()
        self.capacity = int(capacity)
        self.features = torch.zeros((capacity, SPR_POLICY_FEATURES), dtype=torch.float32, device="cuda")
        self.rays = torch.zeros(capacity, dtype=torch.int32, device="cuda")
        self.consumed = torch.zeros(capacity, dtype=torch.int32, device="cuda")
        self.labels = torch.zeros(capacity, dtype=torch.int32, device="cuda")
        self.n = 0


def spr_set_trace(r: Renderer, trace: "Trace | None", sample_mod: int = 1):
    L = load()
    if trace is None:
        check(L.spr_set_trace(r.handle, None, None, None, 0, 1))
        return
    check(L.spr_set_trace(r.handle, _dev_ptr(trace.features), _dev_ptr(trace.rays),
                          _dev_ptr(trace.consumed), trace.capacity, int(sample_mod)))


def spr_trace_labels(r: Renderer, trace: Trace, stream=None) -> int:
    n = ctypes.c_int64()
    check(load().spr_trace_labels(r.handle, _dev_ptr(trace.labels), ctypes.byref(n), _stream(stream)))
    trace.n = n.value
    return n.value


def spr_policy_forward(params, features, stream=None):
    """features: CUDA float32 (n, 12); returns CUDA float32 (n, 2)."""
    torch = _torch()
    p = _params(params)
    n = features.shape[0]
    out = torch.empty((n, 2), dtype=torch.float32, device=features.device)
    check(load().spr_policy_forward(p.ctypes.data_as(ctypes.c_void_p), _dev_ptr(features, torch.float32), n,
                                    _dev_ptr(out), _stream(stream)))
    return out


def spr_policy_grad(params, features, labels, tau: float = 0.9, stream=None):
    """(gradient as float32 numpy, (loss0, loss1)) of the mean loss."""
    torch = _torch()
    p = _params(params)
    g = np.zeros(SPR_POLICY_PARAMS, np.float32)
    loss = (ctypes.c_double * 2)()
    check(load().spr_policy_grad(p.ctypes.data_as(ctypes.c_void_p), _dev_ptr(features, torch.float32),
                                 _dev_ptr(labels), features.shape[0], float(tau),
                                 g.ctypes.data_as(ctypes.c_void_p), loss, _stream(stream)))
    return g, (loss[0], loss[1])


def spr_policy_train(features, labels, params, epochs: int = 5, batch: int = 8192, lr: float = 2e-3,
                     tau: float = 0.9, seed: int = 1, stream=None):
    """Adam on the policy loss; returns (trained params, mean loss per epoch)."""
    torch = _torch()
    p = _params(params).copy()
    d = _lib.TrainDesc(int(epochs), int(batch), float(lr), 0.9, 0.999, 1e-8, float(tau), int(seed))
    losses = np.zeros(epochs, np.float32)
    check(load().spr_policy_train(_dev_ptr(features, torch.float32), _dev_ptr(labels), features.shape[0],
                                  p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(d),
                                  losses.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return p, losses


# ---------------------------------------------------------------- serving
class Server:
    """A render service (spr_server_*): queued requests admitted by free
    streams and device memory, merged into batched renders, overlapped on
    the device.  `outputs` keeps the caller's result tensors alive until the
    request completes."""

    def __init__(self, handle):
        self.handle = handle
        self.outputs = {}
        self.volumes = []

    def close(self):
        if self.handle:
            check(load().spr_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spr_server_create(memory_bytes: int, max_inflight: int = 4, max_batch: int = 8,
                      mode: int = SPR_SPEC_ADAPTIVE, k: int = 1, k_max: int = 64,
                      max_passes: int = 100000) -> Server:
    d = _lib.ServerDesc(int(memory_bytes), int(max_inflight), int(max_batch), int(mode), int(k),
                        int(k_max), int(max_passes))
    h = ctypes.c_void_p()
    check(load().spr_server_create(ctypes.byref(d), ctypes.byref(h)))
    return Server(h)


def spr_server_destroy(s: Server):
    s.close()


def spr_server_add_volume(s: Server, vol: Volume, cache_bytes_per_view: int) -> int:
    i = ctypes.c_int32()
    check(load().spr_server_add_volume(s.handle, vol.handle, int(cache_bytes_per_view),
                                       ctypes.byref(i)))
    s.volumes.append(vol)
    return i.value


def spr_server_reserve(s: Server, volume: int, W: int, H: int, n_views: int = 1):
    check(load().spr_server_reserve(s.handle, int(volume), int(W), int(H), int(n_views)))


def spr_server_clock(s: Server) -> float:
    return load().spr_server_clock(s.handle)


def spr_server_submit(s: Server, volume: int, cam: dict, iso: float, W: int, H: int,
                      t_arrival: float = -1.0, outputs: dict | None = None) -> int:
    """Queue a request; `outputs` maps depth/rgba/block/status to CUDA tensors
    of W*H entries that receive the image.  Returns the request id."""
    q = _lib.Request()
    q.volume, q.width, q.height = int(volume), int(W), int(H)
    q.eye[:] = [float(x) for x in np.asarray(cam["eye"], np.float32)]
    q.p00[:] = [float(x) for x in np.asarray(cam["p00"], np.float32)]
    q.du[:] = [float(x) for x in np.asarray(cam["du"], np.float32)]
    q.dv[:] = [float(x) for x in np.asarray(cam["dv"], np.float32)]
    q.iso = float(iso)
    q.t_arrival = float(t_arrival)
    outputs = outputs or {}
    for name in ("depth", "rgba", "block", "status"):
        t = outputs.get(name)
        if t is not None:
            assert t.numel() >= W * H
            setattr(q, name, _dev_ptr(t).value)
    i = ctypes.c_int64()
    check(load().spr_server_submit(s.handle, ctypes.byref(q), ctypes.byref(i)))
    if outputs:
        s.outputs[i.value] = outputs
    return i.value


def spr_server_poll(s: Server, max_out: int = 256) -> list:
    """Advance the service; returns the results of requests completed since
    the last poll (dicts)."""
    out = (_lib.Result * max_out)()
    n = ctypes.c_int()
    check(load().spr_server_poll(s.handle, out, int(max_out), ctypes.byref(n)))
    res = [out[i].as_dict() for i in range(n.value)]
    for r in res:
        s.outputs.pop(r["id"], None)
    return res


def spr_server_info(s: Server) -> dict:
    st = _lib.ServerStats()
    check(load().spr_server_info(s.handle, ctypes.byref(st)))
    return st.as_dict()


# -------------------------------------------------------------- allocator
_keep = []


def spr_set_allocator(alloc=None, free=None):
    """Install Python callables alloc(nbytes, stream) -> int pointer (0 on
    failure) and free(ptr, nbytes, stream) as the library's device allocator;
    no arguments restores cudaMalloc."""
    if alloc is None:
        check(load().spr_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None))
        _keep.clear()
        return

    def a(nbytes, stream, ctx):
        try:
            return int(alloc(int(nbytes), stream)) or None
        except Exception:
            return None

    def f(ptr, nbytes, stream, ctx):
        try:
            free(int(ptr), int(nbytes), stream)
        except Exception:
            pass
    cb = (_lib.ALLOC_FN(a), _lib.FREE_FN(f))
    check(load().spr_set_allocator(cb[0], cb[1], None))
    _keep[:] = [cb]


def use_torch_allocator():
    """Route the library's device memory through torch's caching allocator."""
    torch = _torch()

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream or 0)

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)
    spr_set_allocator(alloc, free)
