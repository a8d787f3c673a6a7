"""The paper-scale workload's structure at a size the oracle renders whole:
the Richtmyer-Meshkov-like mixing layer (a two-fluid interface perturbed by
seeded sinusoids and fractal noise, 8-bit density) generated at 160x160x150
with its lengths scaled, 2 bits/value, isovalue 0.5, the paper-scale camera
direction (azimuth 30 degrees, elevation 20 degrees) moved in to 0.8
diagonals so that the small volume fills the frame.  Every
pixel against the oracle, and the image bit-identical across speculation
rules and a cache too small for a pass."""
import numpy as np
import pytest

import synth
from test_gpu_render import Scene, compare

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


@pytest.fixture(scope="module")
def scene(orc):
    dims = (160, 160, 150)
    u8 = synth.volumes.mixing_layer(dims)
    vol = synth.volumes.u8_to_f32(u8)
    W, H = 320, 180
    cam = synth.cameras.orbit(dims, 30.0, 20.0, 0.8, W, H, up=(0.0, 0.0, 1.0))
    return Scene(orc, dims, vol, 2, 0.5, cam, W, H), u8


def render(spr, sc, u8, mode, k, slots):
    import torch
    comp = spr.spr_encode_u8(torch.from_numpy(np.ascontiguousarray(u8)).cuda(), 2)
    assert np.array_equal(comp.cpu().numpy(), sc.comp)      # the device encoder equals the oracle's
    v = spr.spr_create_volume(sc.dims, 2, comp)
    r = spr.spr_create_renderer(v, sc.W, sc.H)
    spr.spr_set_camera(r, sc.cam)
    spr.spr_set_isovalue(r, sc.iso)
    spr.spr_set_cache_budget(r, 256 * slots)
    if mode == "fixed":
        spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=k)
    else:
        spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=k)
    rs, passes = spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    return fb, rs, passes


def test_mixing_layer_matches_oracle(spr, orc, scene):
    sc, u8 = scene
    nb = sc.ovol.fine.shape[0]
    want, rs, _ = render(spr, sc, u8, "adaptive", 64, nb)
    n = compare(sc, want)
    assert n > 5000 and rs["converged"] == 1
    # the other rules and a cache of 1/16 of the blocks give the same image
    for mode, k, slots in (("fixed", 1, nb), ("fixed", 16, max(8, nb // 16)), ("adaptive", 16, max(8, nb // 16))):
        got, rs2, passes = render(spr, sc, u8, mode, k, slots)
        for key in FB_KEYS:
            assert np.array_equal(got[key], want[key]), (mode, k, slots, key)
