"""The traversal kernels against each other and the oracle.

Passes with few live rays walk one ray per warp (the blocks of an occupied
coarse cell found at once from exactly ranked plane crossings), the others one
ray per thread (step by step); the segmented walk splits each ray's path at
block planes of its dominant axis among a group of lanes.  All implement the
walk of Sec. 3.3 and must visit the same blocks in the same order.  With any
of them forced for every pass the framebuffers and the per-pass counters are
identical, and all match the oracle."""
import numpy as np
import pytest

import synth
from test_gpu_render import Scene, compare, value_scene

pytestmark = pytest.mark.gpu

THREAD, WARP = 0, 1 << 31
PASS_KEYS = ("k", "k_used", "retries", "n_active", "n_processed", "n_entries", "n_visible",
             "n_requested", "n_decoded", "n_evicted", "n_term_hit", "n_term_miss", "n_active_after")


@pytest.fixture(scope="module")
def spr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_10212_gb300 as m
    return m


def render(spr, sc, walk, mode=None, k=1, k_max=64, slots=None, seg=0):
    import torch
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, sc.W, sc.H)
    spr.spr_set_camera(r, sc.cam)
    spr.spr_set_isovalue(r, sc.iso)
    nb = sc.ovol.fine.shape[0]
    spr.spr_set_cache_budget(r, 256 * (slots if slots else max(8, nb)))
    if mode == "fixed":
        spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=k)
    else:
        spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=k_max)
    spr.spr_set_warp_walk_threshold(r, walk)
    spr.spr_set_segment_walk(r, seg)
    rs, passes = spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    return fb, rs, passes


def same(a, b):
    fa, ra, pa = a
    fb, rb, pb = b
    for key in fa:
        assert np.array_equal(fa[key], fb[key]), key
    assert len(pa) == len(pb)
    for x, y in zip(pa, pb):
        for key in PASS_KEYS:
            assert x[key] == y[key], (x["pass"], key, x[key], y[key])
    assert ra["blocks_decoded"] == rb["blocks_decoded"]


@pytest.mark.parametrize("dims,seed,W,H", [((33, 17, 26), 4, 64, 48), ((64, 64, 64), 5, 128, 96),
                                           ((48, 40, 44), 21, 80, 64)])
@pytest.mark.parametrize("spec", [("fixed", 1), ("fixed", 3), ("adaptive", 64)])
def test_warp_walk_equals_thread_walk(spr, orc, dims, seed, W, H, spec):
    sc = value_scene(orc, dims, seed, W, H)
    mode, k = spec
    kw = dict(mode="fixed", k=k) if mode == "fixed" else dict(k_max=k)
    a = render(spr, sc, THREAD, **kw)
    b = render(spr, sc, WARP, **kw)
    same(a, b)
    compare(sc, a[0])


def test_tight_cache_overflow_both_walks(spr, orc):
    """A cache of 24 slots forces k halving and ray windows in most passes."""
    sc = value_scene(orc, (48, 40, 44), 21, 80, 64)
    a = render(spr, sc, THREAD, slots=24)
    b = render(spr, sc, WARP, slots=24)
    same(a, b)
    assert any(p["retries"] for p in a[2])
    compare(sc, a[0])


def test_diagonal_rays_both_walks(spr, orc):
    """Eye on the volume's main diagonal, looking along it: the central rays
    cross x, y and z block planes at the same instants (diagonal steps)."""
    dims = (40, 40, 40)
    vol = synth.volumes.value_noise(dims, seed=31, ref=40)
    iso = float(np.float32(np.quantile(vol, 0.7)))
    cam = synth.cameras.look_at((-12.0, -12.0, -12.0), (39.0, 39.0, 39.0), (0, 0, 1), 30.0, 64, 64)
    sc = Scene(orc, dims, vol, 8, iso, cam, 64, 64)
    for k in (1, 4):
        a = render(spr, sc, THREAD, mode="fixed", k=k)
        b = render(spr, sc, WARP, mode="fixed", k=k)
        same(a, b)
    compare(sc, a[0], max_amb=0.1)


def test_eye_inside_both_walks(spr, orc):
    dims = (32, 32, 32)
    vol = synth.volumes.value_noise(dims, seed=8, ref=32)
    iso = float(np.float32(np.quantile(vol, 0.8)))
    cam = synth.cameras.look_at((15.5, 16.25, 14.0), (31, 31, 31), (0, 0, 1), 70.0, 64, 64)
    sc = Scene(orc, dims, vol, 8, iso, cam, 64, 64)
    a = render(spr, sc, THREAD, mode="fixed", k=2)
    b = render(spr, sc, WARP, mode="fixed", k=2)
    same(a, b)
    compare(sc, a[0])


def test_threshold_rejects_negative(spr, orc):
    sc = value_scene(orc, (16, 16, 16), 2, 16, 16)
    import torch
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, 16, 16)
    with pytest.raises(spr.SprError):
        spr.spr_set_warp_walk_threshold(r, -1)
    r.close()
    v.close()


# lane budgets of the segmented walk: 32 lanes per ray in every pass of these
# small images, and about two lanes per ray in the first pass (more later)
SEG_ALL = 1 << 30


@pytest.mark.parametrize("dims,seed,W,H", [((33, 17, 26), 4, 64, 48), ((64, 64, 64), 5, 128, 96),
                                           ((48, 40, 44), 21, 80, 64)])
@pytest.mark.parametrize("spec", [("fixed", 1), ("fixed", 3), ("adaptive", 64)])
@pytest.mark.parametrize("seg", ["all", "two"])
def test_segment_walk_equals_thread_walk(spr, orc, dims, seed, W, H, spec, seg):
    sc = value_scene(orc, dims, seed, W, H)
    mode, k = spec
    kw = dict(mode="fixed", k=k) if mode == "fixed" else dict(k_max=k)
    a = render(spr, sc, THREAD, **kw)
    b = render(spr, sc, THREAD, seg=SEG_ALL if seg == "all" else 2 * W * H, **kw)
    same(a, b)
    compare(sc, b[0])


def test_segment_walk_many_blocks_per_lane(spr, orc):
    """k = 4096 with two lanes per ray: a lane finds more visible blocks than
    its shared-memory buffer holds and walks its part again, writing
    directly; k = 40 with 32 lanes: most lanes' parts end before the k-th."""
    sc = value_scene(orc, (64, 64, 64), 5, 96, 64)
    for k, seg in ((4096, 2 * 96 * 64), (40, SEG_ALL), (33, 4 * 96 * 64)):
        a = render(spr, sc, THREAD, mode="fixed", k=k)
        b = render(spr, sc, THREAD, mode="fixed", k=k, seg=seg)
        same(a, b)
        compare(sc, b[0])


def test_segment_walk_tight_cache(spr, orc):
    sc = value_scene(orc, (48, 40, 44), 21, 80, 64)
    a = render(spr, sc, THREAD, slots=24)
    for seg in (SEG_ALL, 2 * 80 * 64):
        b = render(spr, sc, THREAD, slots=24, seg=seg)
        same(a, b)
    assert any(p["retries"] for p in a[2])


def test_segment_walk_diagonal_and_inside(spr, orc):
    dims = (40, 40, 40)
    vol = synth.volumes.value_noise(dims, seed=31, ref=40)
    iso = float(np.float32(np.quantile(vol, 0.7)))
    cam = synth.cameras.look_at((-12.0, -12.0, -12.0), (39.0, 39.0, 39.0), (0, 0, 1), 30.0, 64, 64)
    sc = Scene(orc, dims, vol, 8, iso, cam, 64, 64)
    for k in (1, 4, 64):
        same(render(spr, sc, THREAD, mode="fixed", k=k), render(spr, sc, THREAD, mode="fixed", k=k, seg=SEG_ALL))
    dims = (32, 32, 32)
    vol = synth.volumes.value_noise(dims, seed=8, ref=32)
    iso = float(np.float32(np.quantile(vol, 0.8)))
    cam = synth.cameras.look_at((15.5, 16.25, 14.0), (31, 31, 31), (0, 0, 1), 70.0, 64, 64)
    sc = Scene(orc, dims, vol, 8, iso, cam, 64, 64)
    same(render(spr, sc, THREAD, mode="fixed", k=2), render(spr, sc, THREAD, mode="fixed", k=2, seg=SEG_ALL))


def test_segment_walk_rejects_negative(spr, orc):
    sc = value_scene(orc, (16, 16, 16), 2, 16, 16)
    import torch
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, 16, 16)
    with pytest.raises(spr.SprError):
        spr.spr_set_segment_walk(r, -1)
    r.close()
    v.close()


@pytest.mark.parametrize("dims,seed,W,H", [((33, 17, 26), 4, 64, 48), ((64, 64, 64), 5, 128, 96)])
@pytest.mark.parametrize("spec", [("fixed", 1), ("fixed", 5), ("adaptive", 64)])
def test_staged_intersection_same_image(spr, orc, dims, seed, W, H, spec):
    """The intersection reading corners from each block's dual grid staged in
    shared memory gives the same keys, so the same framebuffer and counters,
    as the per-cell loads; both match the oracle."""
    import torch
    sc = value_scene(orc, dims, seed, W, H)
    mode, k = spec
    out = []
    for staged in (False, True):
        v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
        r = spr.spr_create_renderer(v, sc.W, sc.H)
        spr.spr_set_camera(r, sc.cam)
        spr.spr_set_isovalue(r, sc.iso)
        spr.spr_set_cache_budget(r, 256 * max(8, sc.ovol.fine.shape[0]))
        if mode == "fixed":
            spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=k)
        else:
            spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=k)
        spr.spr_set_intersect_staging(r, staged)
        rs, passes = spr.spr_render_to_convergence(r, 100000)
        out.append((spr.spr_read_framebuffer(r), rs, passes))
        r.close()
        v.close()
    same(out[0], out[1])
    compare(sc, out[1][0])


def test_sparse_volume_hyper_cells(spr, orc):
    """A volume several hyper cells (64^3 blocks) wide, nearly empty: six
    Gaussian blobs in 600x300x80 voxels, so whole super and hyper cells hold
    no block of the isovalue and the walks skip them in one step.  The
    one-thread, segmented and warp walks agree and match the oracle on every
    pixel."""
    dims = (600, 300, 80)
    u8 = synth.volumes.gaussian_blobs(dims, seed=12, n=6, noise=0.0)
    cam = synth.cameras.look_at((-100.0, 150.0, 200.0), (300.0, 150.0, 40.0), (0, 0, 1), 40.0, 96, 64)
    sc = Scene(orc, dims, u8, 2, 0.3, cam, 96, 64)
    a = render(spr, sc, THREAD)
    assert int((a[0]["status"] == 1).sum()) > 500
    same(a, render(spr, sc, THREAD, seg=SEG_ALL))
    same(a, render(spr, sc, WARP))
    compare(sc, a[0])



def grid_camera(eye, dx, step, n):
    """n x n rays along (dx, (i + 0.5 - n/2) step, (j + 0.5 - n/2) step): all
    exact in float32, and for odd n the middle column has d_y = 0 and the
    middle row d_z = 0 exactly."""
    f = lambda v: np.asarray(v, dtype=np.float32)
    h = -0.5 * n * step
    return dict(eye=f(eye), p00=f((dx, h, h)), du=f((0.0, step, 0.0)), dv=f((0.0, 0.0, step)))


# a sphere of radius 9 in one corner of a 96 x 80 x 72 volume
BOX_DIMS, BOX_CENTRE = (96, 80, 72), (70.0, 20.0, 50.0)
BOX_CAMS = [
    # along +x through the sphere's centre
    (grid_camera((-30.0, 20.3125, 50.1875), 1.0, 2.0 ** -5, 17), 17, 17),
    # the same directions with the axis-parallel row below the box
    (grid_camera((-30.0, 20.3125, 5.1875), 1.0, 2.0 ** -5, 17), 17, 17),
    # eye inside the volume, outside the box, looking back along -x
    (grid_camera((90.0, 21.3125, 49.1875), -1.0, 2.0 ** -3, 17), 17, 17),
    # eye inside the box, outside the sphere
    (grid_camera((78.5, 27.3125, 57.1875), -1.0, 2.0 ** -2, 17), 17, 17),
    (synth.cameras.look_at((-60.0, -50.0, 120.0), (48.0, 40.0, 36.0), (0, 0, 1), 50.0, 48, 40), 48, 40),
]


def test_occupied_box(spr, orc):
    """The box of blocks that hold the isovalue is small: the walks start
    where each ray enters it and stop where it leaves it.  Rays that enter
    the volume but miss the box stay live in the first pass (the live count,
    k and every counter as without the box).  Rays with a zero direction
    component inside and outside the box's range, an eye inside the volume
    but outside the box and an eye inside the box: the one-thread, segmented
    and warp walks agree and match the oracle, and the first pass holds every
    ray that enters the volume.  An isovalue no block holds ends every ray in
    the first pass with nothing decoded."""
    vol = synth.volumes.sphere(BOX_DIMS, BOX_CENTRE, 9.0)
    hits = 0
    for cam, w, h in BOX_CAMS:
        sc = Scene(orc, BOX_DIMS, vol, 8, 0.5, cam, w, h)
        a = render(spr, sc, THREAD)
        same(a, render(spr, sc, THREAD, seg=SEG_ALL))
        same(a, render(spr, sc, WARP))
        compare(sc, a[0])
        n_enter = int((orc.entry_blocks(BOX_DIMS, cam, w, h) != 0xFFFFFFFF).sum())
        assert a[2][0]["n_active"] == n_enter > 0
        hits += int((a[0]["status"] == 1).sum())
    assert hits > 100
    # no block holds the isovalue: every entering ray ends in pass 1
    cam, w, h = BOX_CAMS[-1]
    sc = Scene(orc, BOX_DIMS, vol, 8, 2.0, cam, w, h)
    fb, rs, passes = render(spr, sc, THREAD)
    assert len(passes) == 1 and rs["blocks_decoded"] == 0 and rs["n_hits"] == 0
    assert passes[0]["n_active"] == int((orc.entry_blocks(BOX_DIMS, cam, w, h) != 0xFFFFFFFF).sum()) > 0
    assert np.all(fb["status"] == 2)
    compare(sc, fb)
