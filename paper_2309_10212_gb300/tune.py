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


# ------------------------------------------------------------ batched renders
# Requests are dicts with "vol" (index into `vols`), "W", "H", "cam", "iso".
# A shape is (vol, W, H); the batched form renders, per round, up to V
# pending requests of every shape as the views of that shape's renderer, and
# all the shapes' renderers with one spr_batch_render.  The knobs it adds to
# the renderer's own: V (views per renderer), how a total cache budget is
# split among the shapes' renderers, and k_max.

def cache_split(shapes, V, policy, total_bytes, per_view_bytes):
    """Cache bytes of each shape's renderer: "per_view" gives each view its
    own share (per_view_bytes[vol] x V), scaled down to fit total_bytes;
    "equal" splits total_bytes evenly; "pixels" in proportion to W*H."""
    if policy == "per_view":
        want = {s: per_view_bytes[s[0]] * V for s in shapes}
    elif policy == "equal":
        want = {s: total_bytes / len(shapes) for s in shapes}
    elif policy == "pixels":
        tot = sum(s[1] * s[2] for s in shapes)
        want = {s: total_bytes * s[1] * s[2] / tot for s in shapes}
    else:
        raise ValueError(policy)
    scale = min(1.0, total_bytes / sum(want.values()))
    return {s: max(8 * 256, int(want[s] * scale) // 256 * 256) for s in shapes}


class BatchRunner:
    """Pooled renderers per (shape, V, cache, k_max) and batches per round
    composition, kept between calls so that timed runs capture nothing."""

    def __init__(self, vols, stream):
        self.vols, self.stream = vols, stream
        self.renderers, self.batches = {}, {}

    def renderer(self, shape, V, cache, k_max):
        key = (shape, V, cache, k_max)
        r = self.renderers.get(key)
        if r is None:
            vol, W, H = shape
            r = api.spr_create_renderer(self.vols[vol], W, H)
            api.spr_set_cache_budget(r, cache)
            api.spr_set_speculation(r, api.SPR_SPEC_ADAPTIVE, k_max=k_max)
            api.spr_set_view_count(r, V)   # capacity V; rounds use up to V views
            self.renderers[key] = r
        return r

    def batch(self, rs):
        key = tuple(id(r) for r in rs)
        b = self.batches.get(key)
        if b is None:
            b = api.spr_batch_create(rs)
            self.batches[key] = b
        return b

    def close(self):
        for b in self.batches.values():
            b.close()
        for r in self.renderers.values():
            r.close()
        self.batches, self.renderers = {}, {}

    def run(self, requests, V, split, total_bytes, per_view_bytes, k_max, keep=None):
        """Render the requests in rounds; returns dict(ms (device time of the
        rounds), wall_ms, rounds, blocks_decoded).  keep(i, fb_view) is called
        with each request's image (device tensors) when given."""
        import time

        import torch
        shapes = sorted({(q["vol"], q["W"], q["H"]) for q in requests})
        caches = cache_split(shapes, V, split, total_bytes, per_view_bytes)
        pending = {s: [i for i, q in enumerate(requests) if (q["vol"], q["W"], q["H"]) == s] for s in shapes}
        rounds = []
        while any(pending.values()):
            rnd = []
            for s in shapes:
                take, pending[s] = pending[s][:V], pending[s][V:]
                if take:
                    rnd.append((s, take))
            rounds.append(rnd)
        ms, dec = 0.0, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for rnd in rounds:
            rs = []
            for s, take in rnd:
                r = self.renderer(s, V, caches[s], k_max)
                api.spr_reset_cache(r)
                api.spr_set_view_count(r, len(take))
                for v, i in enumerate(take):
                    api.spr_set_view(r, v, requests[i]["cam"], requests[i]["iso"])
                rs.append(r)
            b = self.batch(rs)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            stats = api.spr_batch_render(b, 4096, stream=self.stream)
            e1.record(self.stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            dec += sum(st["blocks_decoded"] for st in stats)
            if keep:
                for (s, take), r in zip(rnd, rs):
                    fb = api.spr_get_framebuffer(r)
                    n = s[1] * s[2]
                    for v, i in enumerate(take):
                        keep(i, {k: t[v * n:(v + 1) * n] for k, t in fb.items()})
        wall = 1e3 * (time.perf_counter() - t0)
        return dict(ms=round(ms, 3), wall_ms=round(wall, 3), rounds=len(rounds), blocks_decoded=dec)


def run_requests_plain(vols, requests, per_view_bytes, k_max, stream, pool, keep=None):
    """The plain loop: every request rendered alone, one after another, by a
    pooled one-view renderer of its shape (cold cache each)."""
    import time

    import torch
    ms, dec = 0.0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, q in enumerate(requests):
        key = (q["vol"], q["W"], q["H"])
        r = pool.get(key)
        if r is None:
            r = api.spr_create_renderer(vols[q["vol"]], q["W"], q["H"])
            api.spr_set_cache_budget(r, per_view_bytes[q["vol"]])
            api.spr_set_speculation(r, api.SPR_SPEC_ADAPTIVE, k_max=k_max)
            pool[key] = r
        api.spr_reset_cache(r)
        api.spr_set_camera(r, q["cam"])
        api.spr_set_isovalue(r, q["iso"])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rs, _ = api.spr_render_to_convergence(r, 4096, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        dec += rs["blocks_decoded"]
        if keep:
            keep(i, api.spr_get_framebuffer(r))
    wall = 1e3 * (time.perf_counter() - t0)
    return dict(ms=round(ms, 3), wall_ms=round(wall, 3), rounds=len(requests), blocks_decoded=dec)


def autotune_batch(runner, requests, total_bytes, per_view_bytes, views=(1, 2, 4, 8),
                   splits=("per_view", "equal", "pixels"), k_max=(16, 64)):
    """Time every (views per renderer, cache split, k_max) on `requests`
    (after one untimed run of each, which captures its graphs); return the
    fastest by device time, with the table."""
    table = []
    for V, split, k in itertools.product(views, splits, k_max):
        runner.run(requests, V, split, total_bytes, per_view_bytes, k)   # warm-up, captures
        res = runner.run(requests, V, split, total_bytes, per_view_bytes, k)
        runner.close()   # one configuration's renderers at a time
        table.append(dict(views=V, split=split, k_max=k, **res))
    best = min(table, key=lambda row: row["ms"])
    return dict(best, table=table)
