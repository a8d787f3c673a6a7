"""Batched rendering: several views (camera, isovalue) of one volume in one
wavefront with a shared cache.  Each view's image must equal its single-view
render (the batch only changes which pass a pixel finishes in), and match the
oracle; the shared cache decodes no more blocks than the views rendered one
by one."""
import numpy as np
import pytest

import synth
from test_gpu_render import Scene, check_counters, compare

pytestmark = pytest.mark.gpu

FB_KEYS = ("depth", "rgba", "block", "cell", "status")


@pytest.fixture(scope="module")
def spr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_10212_gb300 as m
    return m


def views_of(orc, dims, seed, n, W, H, isos, lists=False):
    vol = synth.volumes.value_noise(dims, seed=seed, ref=max(dims))
    scenes = []
    for v in range(n):
        iso = float(np.float32(np.quantile(vol, isos[v % len(isos)])))
        cam = synth.cameras.random_pose(dims, seed=seed + 10 * v + 1, W=W, H=H, distance_factor=1.6)
        scenes.append(Scene(orc, dims, vol, 8, iso, cam, W, H, lists=lists))
    return scenes


def stacked(scenes):
    """The views as one image of W x (H * views) pixels for the oracle's pass
    simulator: pixel p of view v is ray v * W * H + p, as in the renderer,
    and with H a multiple of 4 the screen tiles come in the renderer's order
    (view by view)."""
    pix = np.concatenate([s.pix for s in scenes])
    offs, base = [], 0
    for s in scenes:
        offs.append(s.off + base)
        base += s.vis.size
    return pix, np.concatenate(offs), np.concatenate([s.vis for s in scenes])


def render_batch(spr, scenes, slots=None, **spec):
    import torch
    sc0 = scenes[0]
    v = spr.spr_create_volume(sc0.dims, sc0.rate, torch.from_numpy(sc0.comp).cuda())
    r = spr.spr_create_renderer(v, sc0.W, sc0.H)
    nb = sc0.ovol.fine.shape[0]
    spr.spr_set_cache_budget(r, 256 * (slots if slots else max(8, nb)))
    if spec.get("mode") == "fixed":
        spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=spec["k"])
    else:
        spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=spec.get("k_max", 64))
    spr.spr_set_view_count(r, len(scenes))
    for i, sc in enumerate(scenes):
        spr.spr_set_view(r, i, sc.cam, sc.iso)
    rs, passes = spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    n = sc0.W * sc0.H
    return [{k: fb[k][i * n:(i + 1) * n] for k in fb} for i in range(len(scenes))], rs, passes


@pytest.mark.parametrize("spec", [dict(mode="fixed", k=1), dict(mode="fixed", k=3), dict(k_max=64)])
def test_batch_views_equal_single_renders(spr, orc, spec):
    scenes = views_of(orc, (40, 36, 32), 7, 4, 64, 48, (0.4, 0.6))
    batch, rs, _ = render_batch(spr, scenes, **spec)
    decoded_single = 0
    for sc, fb in zip(scenes, batch):
        single, rs1, _ = render_batch(spr, [sc], **spec)
        for key in FB_KEYS:
            assert np.array_equal(fb[key], single[0][key]), key
        compare(sc, fb)
        decoded_single += rs1["blocks_decoded"]
    assert rs["converged"] == 1
    assert rs["blocks_decoded"] <= decoded_single


def test_batch_tight_cache(spr, orc):
    """24 slots for 3 views: the overflow rule halves k and the ray window
    over the combined live list; images are unchanged."""
    scenes = views_of(orc, (48, 40, 44), 21, 3, 48, 40, (0.62,))
    batch, rs, passes = render_batch(spr, scenes, slots=24)
    assert any(p["retries"] for p in passes)
    for sc, fb in zip(scenes, batch):
        single, _, _ = render_batch(spr, [sc])
        for key in FB_KEYS:
            assert np.array_equal(fb[key], single[0][key]), key
        compare(sc, fb)


def test_view_count_limits(spr, orc):
    import torch
    sc = views_of(orc, (16, 16, 16), 2, 1, 16, 16, (0.5,))[0]
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, 16, 16)
    for bad in (0, 65):
        with pytest.raises(spr.SprError):
            spr.spr_set_view_count(r, bad)
    spr.spr_set_view_count(r, 2)
    spr.spr_set_view(r, 0, sc.cam, sc.iso)
    with pytest.raises(spr.SprError):      # view 1 has no camera
        spr.spr_render_to_convergence(r, 100)
    with pytest.raises(spr.SprError):
        spr.spr_set_view(r, 2, sc.cam, sc.iso)
    r.close()
    v.close()


def test_autotune_picks_a_candidate_and_keeps_the_image(spr, orc):
    import torch
    from paper_2309_10212_gb300 import tune
    scenes = views_of(orc, (40, 36, 32), 7, 2, 64, 48, (0.5,))
    sc = scenes[0]
    want, _, _ = render_batch(spr, [sc])
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, sc.W, sc.H)
    spr.spr_set_cache_budget(r, 256 * sc.ovol.fine.shape[0])
    spr.spr_set_isovalue(r, sc.iso)
    spr.spr_set_camera(r, sc.cam)
    res = tune.autotune(r, [s.cam for s in scenes], k_max=(2, 64), warp_walk=(0, 1 << 20))
    assert (res["k_max"], res["warp_walk"]) in [(2, 0), (2, 1 << 20), (64, 0), (64, 1 << 20)]
    assert len(res["table"]) == 4
    spr.spr_set_camera(r, sc.cam)
    spr.spr_render_to_convergence(r, 100000)
    got = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    for key in FB_KEYS:
        assert np.array_equal(got[key], want[0][key]), key


def test_view_count_within_capacity(spr, orc):
    """A renderer sized for 4 views renders 2, then 3, then 4 views without
    reallocating: views past the active count generate no rays, and every
    active view equals its single-view render."""
    import torch
    scenes = views_of(orc, (36, 32, 28), 9, 4, 48, 40, (0.45, 0.6))
    sc0 = scenes[0]
    v = spr.spr_create_volume(sc0.dims, sc0.rate, torch.from_numpy(sc0.comp).cuda())
    r = spr.spr_create_renderer(v, sc0.W, sc0.H)
    spr.spr_set_cache_budget(r, 256 * sc0.ovol.fine.shape[0])
    singles = [render_batch(spr, [sc])[0][0] for sc in scenes]
    spr.spr_set_view_count(r, 4)
    mem = None
    n = sc0.W * sc0.H
    for nv, order in ((4, (0, 1, 2, 3)), (2, (3, 1)), (3, (2, 0, 1)), (1, (1,))):
        spr.spr_set_view_count(r, nv)
        for i, s in enumerate(order):
            spr.spr_set_view(r, i, scenes[s].cam, scenes[s].iso)
        rs, _ = spr.spr_render_to_convergence(r, 100000)
        assert rs["n_rays"] == sum(int((singles[s]["status"] != 2).sum()) +
                                   int(((singles[s]["status"] == 2) & (singles[s]["final_pass"] > 0)).sum())
                                   for s in order)
        fb = spr.spr_read_framebuffer(r)
        assert fb["depth"].size == nv * n
        for i, s in enumerate(order):
            for key in FB_KEYS:
                assert np.array_equal(fb[key][i * n:(i + 1) * n], singles[s][key]), (nv, i, key)
        # entry buffers and scan scratch are sized at the first render
        mem = mem or spr.spr_renderer_memory(r)
        assert spr.spr_renderer_memory(r) == mem
    r.close()
    v.close()


@pytest.mark.parametrize("spec,sim,slots", [(dict(mode="fixed", k=3), dict(spec_mode=0, k=3), None),
                                            (dict(k_max=64), dict(spec_mode=1, k_max=64), None),
                                            (dict(k_max=64), dict(spec_mode=1, k_max=64), 40)])
def test_batch_counters_match_pass_simulator(spr, orc, spec, sim, slots):
    """Three views with two isovalues in one wavefront: every per-pass counter
    and every pixel's final pass equal the oracle's pass simulator run on the
    views stacked into one image (one live list, one speculation budget of
    views x W x H, one cache)."""
    scenes = views_of(orc, (40, 36, 32), 7, 3, 64, 48, (0.4, 0.6), lists=True)
    assert all(np.all(s.pix["amb"] == 0) for s in scenes), "counters are compared on clear scenes"
    batch, rs, passes = render_batch(spr, scenes, slots=slots, **spec)
    pix, off, vis = stacked(scenes)
    W, H = scenes[0].W, scenes[0].H
    if slots:
        sim = dict(sim, n_slots=slots)
    st, final = orc.simulate(W, H * len(scenes), scenes[0].dims, pix, off, vis, **sim)
    check_counters(st, passes)
    assert np.array_equal(np.concatenate([fb["final_pass"] for fb in batch]), final)
    assert rs["blocks_decoded"] == int(st["n_decoded"].sum())
    if slots:
        assert st["retries"].sum() > 0


def _renderer(spr, vols, sc, slots, spec, views=None):
    import torch
    key = (sc.dims, sc.rate, id(sc.comp))
    if key not in vols:
        vols[key] = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(vols[key], sc.W, sc.H)
    spr.spr_set_cache_budget(r, 256 * slots)
    if spec.get("mode") == "fixed":
        spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=spec["k"])
    else:
        spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=spec.get("k_max", 64))
    views = views or [sc]
    spr.spr_set_view_count(r, len(views))
    for i, v in enumerate(views):
        spr.spr_set_view(r, i, v.cam, v.iso)
    return r


def test_multi_volume_batch_equals_lone_renders(spr, orc):
    """Three volumes of different sizes and rates, image sizes, view counts,
    speculation rules and cache budgets rendered by one graph launch: every
    image (and final pass) equals the renderer's own render, matches the
    oracle, and the counters equal the lone renders'.  Rendered twice (the
    captured graph is reused), then again after one renderer's cache budget
    changed (the graph is captured anew); caches are emptied between rounds."""
    a = views_of(orc, (24, 20, 18), 51, 1, 48, 40, (0.6,))
    b = views_of(orc, (40, 36, 30), 52, 2, 64, 48, (0.45, 0.65))
    c = views_of(orc, (64, 64, 64), 53, 1, 96, 64, (0.5,))
    groups = [(a, 60, dict(mode="fixed", k=2)), (b, 400, dict(k_max=64)), (c, 1000, dict(k_max=16))]
    vols = {}
    rs = [_renderer(spr, vols, g[0], slots, spec, views=g) for g, slots, spec in groups]
    batch = spr.spr_batch_create(rs)
    try:
        for rnd in range(3):
            if rnd == 2:
                spr.spr_set_cache_budget(rs[1], 256 * 300)
            if rnd:
                for r, (g, _, _) in zip(rs, groups):   # fresh renders from cold caches
                    spr.spr_reset_cache(r)
                    for i, sc in enumerate(g):
                        spr.spr_set_view(r, i, sc.cam, sc.iso)
            stats = spr.spr_batch_render(batch)
            for r, (g, slots, spec), st in zip(rs, groups, stats):
                assert st["converged"] == 1
                fb = spr.spr_read_framebuffer(r)
                n = g[0].W * g[0].H
                # the renderer alone, same settings
                lone = _renderer(spr, vols, g[0], slots if not (rnd == 2 and r is rs[1]) else 300, spec, views=g)
                rs1, _ = spr.spr_render_to_convergence(lone, 100000)
                want = spr.spr_read_framebuffer(lone)
                lone.close()
                for key in fb:
                    assert np.array_equal(fb[key], want[key]), (rnd, key)
                for k in ("passes", "blocks_decoded", "entries", "evictions", "n_hits"):
                    assert st[k] == rs1[k], (rnd, k, st[k], rs1[k])
                for i, sc in enumerate(g):
                    compare(sc, {k: v[i * n:(i + 1) * n] for k, v in fb.items()})
    finally:
        batch.close()
        for r in rs:
            r.close()
        for v in vols.values():
            v.close()


def test_batch_rejects_continued_and_duplicate(spr, orc):
    a = views_of(orc, (24, 20, 18), 51, 1, 48, 40, (0.6,))
    vols = {}
    r = _renderer(spr, vols, a[0], 60, dict(k_max=64))
    with pytest.raises(spr.SprError):
        spr.spr_batch_create([r, r])
    batch = spr.spr_batch_create([r])
    spr.spr_batch_render(batch)
    with pytest.raises(spr.SprError):   # no new camera: not a fresh render
        spr.spr_batch_render(batch)
    spr.spr_set_camera(r, a[0].cam)
    spr.spr_batch_render(batch)
    batch.close()
    r.close()
    for v in vols.values():
        v.close()
