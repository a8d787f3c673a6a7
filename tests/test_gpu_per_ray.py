"""Per-ray speculation (each live ray takes its own count k_i every pass, the
per-ray speculation count the paper leaves to future work in Sec. 6): the
image is the same as with the paper's uniform rule for any counts, since a
ray's blocks are still visited in order and its earliest hit wins; only the
passes and the blocks decoded change.  SPR_SPEC_HASHED draws k_i from a hash
of (ray, pass), which exercises the per-ray entry layout without a model."""
import numpy as np
import pytest

import synth
from test_gpu_batch import render_batch, views_of
from test_gpu_render import check_counters, compare, value_scene

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


def render(spr, sc, mode, k=1, k_max=64, slots=None, warp_walk=None, seg=0):
    import torch
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, sc.W, sc.H)
    spr.spr_set_camera(r, sc.cam)
    spr.spr_set_isovalue(r, sc.iso)
    nb = sc.ovol.fine.shape[0]
    spr.spr_set_cache_budget(r, 256 * (slots if slots else max(8, nb)))
    if warp_walk is not None:
        spr.spr_set_warp_walk_threshold(r, warp_walk)
    spr.spr_set_segment_walk(r, seg)
    spr.spr_set_speculation(r, mode, k=k, k_max=k_max)
    rs, passes = spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    return fb, rs, passes


@pytest.mark.parametrize("dims,seed", [((24, 20, 18), 41), ((40, 36, 30), 42), ((64, 64, 64), 43)])
@pytest.mark.parametrize("k_max", [2, 7, 32, 64])
def test_hashed_counts_keep_the_image(spr, orc, dims, seed, k_max):
    sc = value_scene(orc, dims, seed, 80, 64)
    want, rs0, _ = render(spr, sc, spr.SPR_SPEC_ADAPTIVE, k_max=64)
    got, rs1, passes = render(spr, sc, spr.SPR_SPEC_HASHED, k_max=k_max)
    for key in FB_KEYS:
        assert np.array_equal(got[key], want[key]), key
    assert rs1["converged"] == 1 and rs1["n_hits"] == rs0["n_hits"]
    assert all(p["k"] == k_max for p in passes)
    compare(sc, got)


@pytest.mark.parametrize("warp_walk,seg", [(0, 0), (1 << 30, 0), (0, 1 << 30), (0, 2 * 96 * 64)])
def test_hashed_counts_both_walks(spr, orc, warp_walk, seg):
    """The thread-per-ray, warp-per-ray and segmented walks take the same
    per-ray counts and give the same image and counters."""
    sc = value_scene(orc, (48, 40, 36), 44, 96, 64)
    a, rsa, pa = render(spr, sc, spr.SPR_SPEC_HASHED, k_max=9, warp_walk=0)
    b, rsb, pb = render(spr, sc, spr.SPR_SPEC_HASHED, k_max=9, warp_walk=warp_walk, seg=seg)
    for key in FB_KEYS:
        assert np.array_equal(a[key], b[key]), key
    keys = ("n_active", "n_entries", "n_visible", "n_requested", "n_decoded", "n_term_hit", "n_term_miss")
    assert [[p[k] for k in keys] for p in pa] == [[p[k] for k in keys] for p in pb]


def hashed_counts(npix, passes, k_max):
    """The counts SPR_SPEC_HASHED draws, written from the definition in
    spr.h (unsigned 32-bit arithmetic): row P-1 holds pass P's count of every
    ray, before the overflow cap."""
    m = np.uint64(0xFFFFFFFF)
    q = np.arange(npix, dtype=np.uint64)
    rows = []
    for P in range(1, passes + 1):
        h = ((q * np.uint64(0x9E3779B1)) & m) ^ np.uint64((P * 0x85EBCA77) & 0xFFFFFFFF)
        h ^= h >> np.uint64(15)
        h = (h * np.uint64(0x2C1B3C6D)) & m
        h ^= h >> np.uint64(12)
        rows.append(1 + (h % np.uint64(k_max)).astype(np.int64))
    return np.stack(rows).astype(np.int32)


@pytest.mark.parametrize("k_max,slots", [(9, None), (64, None), (24, 60), (48, 120)])
def test_hashed_counters_match_pass_simulator(spr, orc, k_max, slots):
    """Every per-pass counter, each pixel's final pass and the blocks decoded
    equal the oracle's pass simulator fed the same per-ray counts, with a
    cache that holds every block and with caches that overflow (the cap
    halves, then the ray window does)."""
    sc = value_scene(orc, (48, 40, 44), 21, 80, 64, rate=4, q=0.62, lists=True)
    assert np.all(sc.pix["amb"] == 0), "counters are compared on a clear scene"
    fb, rs, passes = render(spr, sc, spr.SPR_SPEC_HASHED, k_max=k_max, slots=slots)
    compare(sc, fb)
    sim = dict(spec_mode=orc.SPEC_PER_RAY, k_max=k_max,
               kray=hashed_counts(sc.W * sc.H, 1000, k_max))
    if slots:
        sim["n_slots"] = slots
    st, final = orc.simulate(sc.W, sc.H, sc.dims, sc.pix, sc.off, sc.vis, **sim)
    assert len(st) < 1000
    check_counters(st, passes)
    assert np.array_equal(fb["final_pass"], final)
    assert rs["blocks_decoded"] == int(st["n_decoded"].sum())
    if slots:
        assert st["retries"].sum() > 0


def test_per_ray_k1_equals_fixed_k1(spr, orc):
    """With k_max = 1 every ray takes one block: the passes and their counters
    are those of fixed k = 1 (which the oracle's pass simulator pins)."""
    sc = value_scene(orc, (32, 28, 24), 45, 64, 48)
    a, _, pa = render(spr, sc, spr.SPR_SPEC_FIXED, k=1)
    b, _, pb = render(spr, sc, spr.SPR_SPEC_HASHED, k_max=1)
    for key in FB_KEYS:
        assert np.array_equal(a[key], b[key]), key
    keys = ("n_active", "n_processed", "n_entries", "n_visible", "n_requested", "n_decoded", "n_evicted",
            "n_term_hit", "n_term_miss", "n_active_after")
    assert [[p[k] for k in keys] for p in pa] == [[p[k] for k in keys] for p in pb]


def test_hashed_counts_tight_cache(spr, orc):
    """A cache too small for the counts: the attempt is redone with the cap
    halved (then the ray window), and the image does not change."""
    sc = value_scene(orc, (48, 44, 40), 46, 64, 64)
    want, _, _ = render(spr, sc, spr.SPR_SPEC_ADAPTIVE)
    got, rs, passes = render(spr, sc, spr.SPR_SPEC_HASHED, k_max=48, slots=24)
    assert any(p["retries"] for p in passes)
    for key in FB_KEYS:
        assert np.array_equal(got[key], want[key]), key


def test_hashed_counts_batched_views(spr, orc):
    scenes = views_of(orc, (40, 36, 32), 47, 3, 64, 48, (0.45, 0.6))
    batch, _, _ = render_batch(spr, scenes, k_max=64)
    import torch
    sc0 = scenes[0]
    v = spr.spr_create_volume(sc0.dims, sc0.rate, torch.from_numpy(sc0.comp).cuda())
    r = spr.spr_create_renderer(v, sc0.W, sc0.H)
    spr.spr_set_cache_budget(r, 256 * sc0.ovol.fine.shape[0])
    spr.spr_set_speculation(r, spr.SPR_SPEC_HASHED, k_max=13)
    spr.spr_set_view_count(r, len(scenes))
    for i, sc in enumerate(scenes):
        spr.spr_set_view(r, i, sc.cam, sc.iso)
    spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    n = sc0.W * sc0.H
    for i in range(len(scenes)):
        for key in FB_KEYS:
            assert np.array_equal(fb[key][i * n:(i + 1) * n], batch[i][key]), (i, key)


def test_per_ray_mode_limits(spr, orc):
    import torch
    sc = value_scene(orc, (16, 16, 16), 48, 16, 16)
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, 16, 16)
    for bad in (0, spr.SPR_K_PER_RAY_LIMIT + 1):
        with pytest.raises(spr.SprError):
            spr.spr_set_speculation(r, spr.SPR_SPEC_HASHED, k_max=bad)
    r.close()
    v.close()
