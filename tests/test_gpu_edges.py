"""Degenerate and ragged cases of the pass pipeline against the oracle: an
isovalue outside the volume's range (nothing to decode, every ray leaves in
one pass), a camera that looks away (no ray enters, no pass runs), image
sizes that do not fill the 8x4 ray tiles, volumes only two voxels thick along
an axis, and a constant volume."""
import numpy as np
import pytest

import synth
from test_gpu_render import Scene, compare, gpu_render

pytestmark = pytest.mark.gpu

MODES = [("fixed", 1), ("adaptive", 64), ("hashed", 9)]


@pytest.fixture(scope="module")
def spr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_10212_gb300 as m
    return m


def render_mode(spr, sc, mode, k):
    if mode == "hashed":
        import torch
        v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
        r = spr.spr_create_renderer(v, sc.W, sc.H)
        spr.spr_set_camera(r, sc.cam)
        spr.spr_set_isovalue(r, sc.iso)
        spr.spr_set_cache_budget(r, 256 * max(8, sc.ovol.fine.shape[0]))
        spr.spr_set_speculation(r, spr.SPR_SPEC_HASHED, k_max=k)
        rs, passes = spr.spr_render_to_convergence(r, 100000)
        fb = spr.spr_read_framebuffer(r)
        r.close()
        v.close()
        return fb, rs, passes
    return gpu_render(spr, sc, mode=mode, k=k, k_max=k)


@pytest.mark.parametrize("mode,k", MODES)
def test_isovalue_outside_the_range(spr, orc, mode, k):
    dims = (24, 20, 18)
    vol = synth.volumes.value_noise(dims, seed=61, ref=24)
    cam = synth.cameras.random_pose(dims, seed=62, W=40, H=32, distance_factor=1.6)
    sc = Scene(orc, dims, vol, 8, float(np.float32(vol.max() + 0.25)), cam, 40, 32)
    fb, rs, passes = render_mode(spr, sc, mode, k)
    assert rs["converged"] == 1 and rs["n_hits"] == 0 and rs["blocks_decoded"] == 0
    assert rs["passes"] <= 1
    assert np.all(fb["status"] == 2) and np.all(np.isinf(fb["depth"]))
    compare(sc, fb)


@pytest.mark.parametrize("mode,k", MODES)
def test_camera_looking_away(spr, orc, mode, k):
    dims = (20, 20, 20)
    vol = synth.volumes.value_noise(dims, seed=63, ref=20)
    # eye outside the volume, looking further away from it
    cam = synth.cameras.look_at((40.0, 9.5, 9.5), (80.0, 9.5, 9.5), (0, 0, 1), 30.0, 24, 16)
    sc = Scene(orc, dims, vol, 8, float(np.float32(np.quantile(vol, 0.5))), cam, 24, 16)
    fb, rs, passes = render_mode(spr, sc, mode, k)
    assert rs["n_rays"] == 0 and rs["passes"] == 0 and rs["converged"] == 1
    assert np.all(fb["status"] == 2) and np.all(fb["final_pass"] == 0)
    compare(sc, fb)


@pytest.mark.parametrize("W,H", [(1, 1), (37, 29), (9, 5)])
@pytest.mark.parametrize("mode,k", MODES)
def test_ragged_image_sizes(spr, orc, W, H, mode, k):
    dims = (26, 22, 19)
    vol = synth.volumes.value_noise(dims, seed=64, ref=26)
    cam = synth.cameras.random_pose(dims, seed=65, W=W, H=H, distance_factor=1.2)
    sc = Scene(orc, dims, vol, 8, float(np.float32(np.quantile(vol, 0.55))), cam, W, H)
    fb, rs, _ = render_mode(spr, sc, mode, k)
    assert rs["converged"] == 1 and fb["depth"].size == W * H
    compare(sc, fb, max_amb=1.0 if W * H < 50 else 0.02)


@pytest.mark.parametrize("dims", [(2, 17, 13), (19, 2, 11), (9, 14, 2), (2, 2, 2)])
def test_two_voxel_thin_volumes(spr, orc, dims):
    vol = synth.volumes.value_noise(dims, seed=66, ref=max(dims))
    iso = float(np.float32(np.quantile(vol, 0.5)))
    cam = synth.cameras.random_pose(dims, seed=67 + dims[0], W=48, H=40, distance_factor=1.5)
    sc = Scene(orc, dims, vol, 8, iso, cam, 48, 40)
    for mode, k in MODES:
        fb, rs, _ = render_mode(spr, sc, mode, k)
        assert rs["converged"] == 1
        compare(sc, fb, max_amb=0.1)


def test_constant_volume(spr, orc):
    """A constant field has no isosurface at any other isovalue: no block is
    active, nothing is decoded, every ray leaves."""
    dims = (17, 15, 13)
    vol = np.full((dims[2], dims[1], dims[0]), 0.375, np.float32)
    cam = synth.cameras.random_pose(dims, seed=68, W=32, H=24, distance_factor=1.4)
    for iso in (0.25, 0.5):
        sc = Scene(orc, dims, vol, 8, iso, cam, 32, 24)
        fb, rs, _ = render_mode(spr, sc, "adaptive", 64)
        assert rs["n_hits"] == 0 and rs["blocks_decoded"] == 0
        compare(sc, fb)
