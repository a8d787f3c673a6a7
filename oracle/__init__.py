"""CPU oracle for speculative progressive isosurface raycasting (arXiv 2309.10212).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
definition that the CUDA path is checked against.  Only the tests, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product
library never does, and the two share no code.

The arithmetic lives in plain C (``orc*.c``, see ``orc.h`` for the full
definitions and paper citations); this module builds it with gcc on first use
and wraps it with ctypes and numpy.

Conventions: ``dims = (Dx, Dy, Dz)``; volumes are numpy arrays of shape
``(Dz, Dy, Dx)`` (x fastest); a camera is a dict or tuple of four float32
triples ``eye, p00, du, dv``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liborc.so")
_SOURCES = ["orc_codec.c", "orc_grid.c", "orc_render.c", "orc_sim.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liborc.so (gcc, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "orc.h")
    if not force and os.path.exists(_SO):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_SO) >= newest:
            return _SO
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas"]
    tmp = _SO + ".tmp%d" % os.getpid()
    for extra in (["-fopenmp"], []):
        cmd = base + extra + srcs + ["-lm", "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _SO)
            return _SO
    raise RuntimeError("oracle build failed:\n" + r.stderr)


class _Pixel(ctypes.Structure):
    _fields_ = [("hit", ctypes.c_int32), ("enters", ctypes.c_int32),
                ("t", ctypes.c_double), ("depth", ctypes.c_double),
                ("cell", ctypes.c_int32 * 3), ("block", ctypes.c_uint32),
                ("grey", ctypes.c_int32), ("amb", ctypes.c_uint32),
                ("n_visible", ctypes.c_int32), ("hit_index", ctypes.c_int32)]


PIXEL_DTYPE = np.dtype([("hit", "<i4"), ("enters", "<i4"), ("t", "<f8"), ("depth", "<f8"),
                        ("cell", "<i4", (3,)), ("block", "<u4"), ("grey", "<i4"),
                        ("amb", "<u4"), ("n_visible", "<i4"), ("hit_index", "<i4")], align=True)

STATS_DTYPE = np.dtype([("pass", "<i4"), ("n_active", "<i8"), ("k", "<i4"), ("k_used", "<i4"),
                        ("n_processed", "<i8"), ("retries", "<i4"), ("n_entries", "<i8"),
                        ("n_visible", "<i8"), ("n_requested", "<i8"), ("n_decoded", "<i8"),
                        ("n_evicted", "<i8"), ("n_term_hit", "<i8"), ("n_term_miss", "<i8")],
                       align=True)

AMB_FACE, AMB_VALUE, AMB_TANGENT, AMB_SHALLOW = 1, 2, 4, 8
AMB_INTERNAL = 0x10000
SPEC_FIXED, SPEC_ADAPTIVE, SPEC_PER_RAY = 0, 1, 2


class _Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("p00", ctypes.c_float * 3),
                ("du", ctypes.c_float * 3), ("dv", ctypes.c_float * 3)]


class _Volume(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("vals", ctypes.c_void_p),
                ("fine", ctypes.c_void_p), ("comp", ctypes.c_void_p), ("rate", ctypes.c_int32),
                ("lazy_fine", ctypes.c_int32), ("decodes", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            for name, args, res in [
                ("orc_encode_block", [vp, i32, vp], i32),
                ("orc_decode_block", [vp, i32, vp], i32),
                ("orc_decode_block_ints", [vp, i32, vp, vp, vp], i32),
                ("orc_coeff_order", [vp], None),
                ("orc_int_to_negabinary", [ctypes.c_int32], ctypes.c_uint32),
                ("orc_negabinary_to_int", [ctypes.c_uint32], ctypes.c_int32),
                ("orc_fwd_lift4", [vp], None),
                ("orc_inv_lift4", [vp], None),
                ("orc_fwd_xform", [vp], None),
                ("orc_inv_xform", [vp], None),
                ("orc_encode_volume_f32", [vp, vp, i32, vp], i32),
                ("orc_encode_volume_u8", [vp, vp, i32, vp], i32),
                ("orc_decode_volume", [vp, vp, i32, vp], i32),
                ("orc_ranges", [vp, vp, vp, vp, vp], i32),
                ("orc_check_camera", [vp, vp], i32),
                ("orc_ray_dir", [vp, i32, i32, i32, i32, vp], None),
                ("orc_render", [vp, vp, i32, i32, ctypes.c_float, vp, i64, i32, vp, vp, vp,
                                i32], i32),
                ("orc_trace_cells", [vp, vp, i32, i32, i32, i32, vp, i64], i64),
                ("orc_entry_block", [vp, vp, i32, i32, i32, i32], ctypes.c_uint32),
                ("orc_march", [vp, vp, i32, i32, ctypes.c_float, vp, i64, vp, i32], i32),
                ("orc_simulate", [i32, i32, vp, vp, vp, vp, vp, vp, i32, i32, i32, i64, i32,
                                  vp, vp, vp], i32),
                ("orc_spec_count", [i64, i64, i32], i32),
                ("orc_sizeof_pixel", [], i32),
                ("orc_sizeof_pass_stats", [], i32),
                ("orc_sizeof_volume", [], i32),
            ]:
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            assert L.orc_sizeof_pixel() == PIXEL_DTYPE.itemsize, "orc_pixel layout"
            assert L.orc_sizeof_pass_stats() == STATS_DTYPE.itemsize, "orc_pass_stats layout"
            assert L.orc_sizeof_volume() == ctypes.sizeof(_Volume), "orc_volume layout"
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def nthreads_default() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------- codec
def encode_block(values, rate: int) -> np.ndarray:
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float32).reshape(64))
    out = np.zeros(8 * rate, dtype=np.uint8)
    rc = lib().orc_encode_block(_ptr(v), rate, _ptr(out))
    if rc:
        raise ValueError("orc_encode_block failed: %d" % rc)
    return out


def decode_block(stream, rate: int) -> np.ndarray:
    s = np.ascontiguousarray(np.asarray(stream, dtype=np.uint8))
    assert s.size >= 8 * rate
    out = np.zeros(64, dtype=np.float32)
    rc = lib().orc_decode_block(_ptr(s), rate, _ptr(out))
    if rc:
        raise ValueError("orc_decode_block failed: %d" % rc)
    return out


def decode_block_ints(stream, rate: int):
    s = np.ascontiguousarray(np.asarray(stream, dtype=np.uint8))
    c = np.zeros(64, dtype=np.int32)
    e = np.zeros(1, dtype=np.int32)
    nz = np.zeros(1, dtype=np.int32)
    lib().orc_decode_block_ints(_ptr(s), rate, _ptr(c), _ptr(e), _ptr(nz))
    return c, int(e[0]), bool(nz[0])


def coeff_order() -> np.ndarray:
    p = np.zeros(64, dtype=np.int32)
    lib().orc_coeff_order(_ptr(p))
    return p


def int_to_negabinary(x: int) -> int:
    return int(lib().orc_int_to_negabinary(int(x)))


def negabinary_to_int(u: int) -> int:
    return int(lib().orc_negabinary_to_int(int(u) & 0xFFFFFFFF))


def fwd_lift4(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32).copy())
    lib().orc_fwd_lift4(_ptr(a))
    return a


def inv_lift4(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32).copy())
    lib().orc_inv_lift4(_ptr(a))
    return a


def fwd_xform(c):
    a = np.ascontiguousarray(np.asarray(c, dtype=np.int32).reshape(64).copy())
    lib().orc_fwd_xform(_ptr(a))
    return a


def inv_xform(c):
    a = np.ascontiguousarray(np.asarray(c, dtype=np.int32).reshape(64).copy())
    lib().orc_inv_xform(_ptr(a))
    return a


def nblocks(dims):
    return tuple((int(d) + 3) // 4 for d in dims)


def encode_volume(vol: np.ndarray, dims, rate: int) -> np.ndarray:
    """Compress a (Dz, Dy, Dx) float32 or uint8 volume; returns the block stream."""
    nb = nblocks(dims)
    out = np.zeros(nb[0] * nb[1] * nb[2] * 8 * rate, dtype=np.uint8)
    v = np.ascontiguousarray(vol)
    assert v.shape == (dims[2], dims[1], dims[0])
    if v.dtype == np.uint8:
        rc = lib().orc_encode_volume_u8(_ptr(v), _ptr(_dims(dims)), rate, _ptr(out))
    else:
        v = np.ascontiguousarray(v, dtype=np.float32)
        rc = lib().orc_encode_volume_f32(_ptr(v), _ptr(_dims(dims)), rate, _ptr(out))
    if rc:
        raise ValueError("orc_encode_volume failed: %d" % rc)
    return out


def decode_volume(comp: np.ndarray, dims, rate: int) -> np.ndarray:
    c = np.ascontiguousarray(comp, dtype=np.uint8)
    out = np.zeros((dims[2], dims[1], dims[0]), dtype=np.float32)
    rc = lib().orc_decode_volume(_ptr(c), _ptr(_dims(dims)), rate, _ptr(out))
    if rc:
        raise ValueError("orc_decode_volume failed: %d" % rc)
    return out


# ---------------------------------------------------------------- ranges
def ranges(decoded: np.ndarray, dims):
    """(raw, fine, coarse) ranges as float32 arrays of shape (n, 2)."""
    nb = nblocks(dims)
    nc = tuple((b + 3) // 4 for b in nb)
    raw = np.zeros((nb[0] * nb[1] * nb[2], 2), dtype=np.float32)
    fine = np.zeros_like(raw)
    coarse = np.zeros((nc[0] * nc[1] * nc[2], 2), dtype=np.float32)
    d = np.ascontiguousarray(decoded, dtype=np.float32)
    rc = lib().orc_ranges(_ptr(d), _ptr(_dims(dims)), _ptr(raw), _ptr(fine), _ptr(coarse))
    if rc:
        raise ValueError("orc_ranges failed: %d" % rc)
    return raw, fine, coarse


# ---------------------------------------------------------------- rays
def _camera(cam) -> _Camera:
    if isinstance(cam, dict):
        parts = [cam["eye"], cam["p00"], cam["du"], cam["dv"]]
    else:
        parts = list(cam)
    c = _Camera()
    for name, v in zip(("eye", "p00", "du", "dv"), parts):
        arr = np.asarray(v, dtype=np.float32)
        getattr(c, name)[:] = [float(x) for x in arr]
    return c


def check_camera(cam, dims) -> int:
    c = _camera(cam)
    return int(lib().orc_check_camera(ctypes.byref(c), _ptr(_dims(dims))))


def ray_dirs(cam, W: int, H: int) -> np.ndarray:
    """float32 directions of all pixels, shape (H*W, 3)."""
    c = _camera(cam)
    out = np.zeros((H * W, 3), dtype=np.float32)
    d = np.zeros(3, dtype=np.float32)
    L = lib()
    for j in range(H):
        for i in range(W):
            L.orc_ray_dir(ctypes.byref(c), W, H, i, j, _ptr(d))
            out[i + W * j] = d
    return out


class Volume:
    """A decoded volume plus its fine ranges, as the oracle renderer wants it;
    or, from `on_demand`, the compressed blocks alone, each decoded the first
    time a ray reaches it (Sec. 3.5) and kept in a bounded per-thread memo
    for the duration of one render call.  Both forms give identical results."""

    def __init__(self, decoded: np.ndarray, dims, fine=None):
        self.dims = tuple(int(d) for d in dims)
        self.fine = None if fine is None else np.ascontiguousarray(fine, dtype=np.float32)
        self.comp = None
        self.rate = 0
        self.last_decodes = 0
        self._decodes = np.zeros(1, dtype=np.int64)
        self._s = _Volume()
        self._s.dims[:] = list(self.dims)
        if decoded is None:
            self.decoded = None
            self._s.vals = None
        else:
            self.decoded = np.ascontiguousarray(decoded, dtype=np.float32)
            assert self.decoded.shape == (dims[2], dims[1], dims[0])
            self._s.vals = self.decoded.ctypes.data
        self._s.fine = None if self.fine is None else self.fine.ctypes.data
        self._s.decodes = self._decodes.ctypes.data

    @classmethod
    def from_compressed(cls, comp, dims, rate):
        dec = decode_volume(comp, dims, rate)
        _, fine, _ = ranges(dec, dims)
        return cls(dec, dims, fine)

    @classmethod
    def on_demand(cls, comp, dims, rate: int, lazy_fine: bool = False):
        """Blocks decoded on demand from `comp` (the volume's FRC4 stream at
        `rate` bits/value).  With lazy_fine, fine ranges are formed on demand
        too, so that render(..., lists=True) works without a decoded grid."""
        v = cls(None, dims)
        nb = nblocks(dims)
        c = np.ascontiguousarray(comp, dtype=np.uint8)
        assert c.size >= nb[0] * nb[1] * nb[2] * 8 * rate
        v.comp = c
        v.rate = int(rate)
        v._s.comp = c.ctypes.data
        v._s.rate = int(rate)
        v._s.lazy_fine = 1 if lazy_fine else 0
        return v

    def _done(self):
        self.last_decodes = int(self._decodes[0])


def render(vol: Volume, cam, W: int, H: int, iso: float, pixels=None, full_lists=False,
           lists=False, nthreads=None):
    """Per-pixel first hits.  Returns a PIXEL_DTYPE array; with lists=True also
    (vis_off, vis) holding every pixel's visible blocks."""
    c = _camera(cam)
    nt = nthreads_default() if nthreads is None else nthreads
    if pixels is None:
        pix_p, n = None, W * H
    else:
        px = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        pix_p, n = _ptr(px), px.size
    out = np.zeros(n, dtype=PIXEL_DTYPE)
    L = lib()
    rc = L.orc_render(ctypes.byref(vol._s), ctypes.byref(c), W, H, float(iso), pix_p, n,
                      1 if (full_lists or lists) else 0, _ptr(out), None, None, nt)
    vol._done()
    if rc:
        raise ValueError("orc_render failed: %d" % rc)
    if not lists:
        return out
    counts = out["n_visible"].astype(np.int64)
    off = np.zeros(n, dtype=np.int64)
    np.cumsum(counts[:-1], out=off[1:])
    vis = np.zeros(max(1, int(counts.sum())), dtype=np.uint32)
    out2 = np.zeros(n, dtype=PIXEL_DTYPE)
    rc = L.orc_render(ctypes.byref(vol._s), ctypes.byref(c), W, H, float(iso), pix_p, n, 1,
                      _ptr(out2), _ptr(off), _ptr(vis), nt)
    vol._done()
    if rc:
        raise ValueError("orc_render failed: %d" % rc)
    return out2, off, vis


def march(vol: Volume, cam, W: int, H: int, iso: float, pixels=None, nthreads=None):
    c = _camera(cam)
    nt = nthreads_default() if nthreads is None else nthreads
    if pixels is None:
        pix_p, n = None, W * H
    else:
        px = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        pix_p, n = _ptr(px), px.size
    out = np.zeros(n, dtype=PIXEL_DTYPE)
    rc = lib().orc_march(ctypes.byref(vol._s), ctypes.byref(c), W, H, float(iso), pix_p, n,
                         _ptr(out), nt)
    vol._done()
    if rc:
        raise ValueError("orc_march failed: %d" % rc)
    return out


def trace_cells(dims, cam, W, H, px, py, cap=1 << 16) -> np.ndarray:
    c = _camera(cam)
    cells = np.zeros((cap, 3), dtype=np.int32)
    n = lib().orc_trace_cells(_ptr(_dims(dims)), ctypes.byref(c), W, H, px, py, _ptr(cells),
                              cap)
    assert n <= cap
    return cells[:n].copy()


def entry_blocks(dims, cam, W, H) -> np.ndarray:
    c = _camera(cam)
    L = lib()
    d = _dims(dims)
    out = np.zeros(W * H, dtype=np.uint32)
    for j in range(H):
        for i in range(W):
            out[i + W * j] = L.orc_entry_block(_ptr(d), ctypes.byref(c), W, H, i, j)
    return out


# ---------------------------------------------------------------- passes
def spec_count(slots: int, n_active: int, k_max: int = 64) -> int:
    return int(lib().orc_spec_count(int(slots), int(n_active), int(k_max)))


def simulate(W, H, dims, pix, vis_off, vis, spec_mode=SPEC_ADAPTIVE, k=1, k_max=64,
             n_slots=None, max_passes=10000, kray=None):
    """Progressive pass simulation from a cold cache.  `pix`, `vis_off`, `vis`
    come from render(..., lists=True) over all pixels in order.  With
    spec_mode SPEC_PER_RAY, kray[P-1, p] is pixel p's own count in pass P
    (capped by k_max, which halves on cache overflow), and at most
    kray.shape[0] passes run.  Returns (stats array, final_pass per pixel)."""
    assert pix.size == W * H
    kr = None
    if spec_mode == SPEC_PER_RAY:
        kr = np.ascontiguousarray(kray, dtype=np.int32)
        assert kr.ndim == 2 and kr.shape[1] == W * H
        max_passes = min(max_passes, kr.shape[0])
    if n_slots is None:
        nb = nblocks(dims)
        n_slots = max(8, nb[0] * nb[1] * nb[2])
    enters = np.ascontiguousarray(pix["enters"], dtype=np.int32)
    hit_index = np.ascontiguousarray(np.where(pix["hit"] != 0, pix["hit_index"], -1),
                                     dtype=np.int32)
    n_vis = np.ascontiguousarray(pix["n_visible"], dtype=np.int32)
    off = np.ascontiguousarray(vis_off, dtype=np.int64)
    v = np.ascontiguousarray(vis, dtype=np.uint32)
    stats = np.zeros(max_passes, dtype=STATS_DTYPE)
    final = np.zeros(W * H, dtype=np.int32)
    n = lib().orc_simulate(W, H, _ptr(_dims(dims)), _ptr(enters), _ptr(hit_index), _ptr(off),
                           _ptr(n_vis), _ptr(v), spec_mode, k, k_max, int(n_slots),
                           max_passes, _ptr(kr) if kr is not None else None, _ptr(stats),
                           _ptr(final))
    if n < 0:
        raise ValueError("orc_simulate failed: %d" % n)
    return stats[:n].copy(), final
