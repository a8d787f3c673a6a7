"""The paper-scale workload at its full size, in the configuration bench.py
times (2048x2048x1920 mixing layer, 2 bits/value, isovalue 0.5, 1280x720,
adaptive speculation up to 64, 4 GB cache).  The oracle cannot hold this
volume decoded (30 GB), so the checks are properties that hold at any size:
the image is the same under another speculation rule and budget, every hit
lies in the cell and block the framebuffer names, and at sampled hits the
trilinear field of the oracle's decoded corner values equals the isovalue at
the reported depth."""
import numpy as np
import pytest

import synth

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
def paper(spr):
    import torch

    import bench
    wl = dict(bench.WORKLOADS["paper"])
    comp = bench.compressed_on_device(wl, spr, torch)
    vol = spr.spr_create_volume(wl["dims"], wl["rate"], comp)
    yield wl, comp, vol
    vol.close()


def render(spr, vol, wl, cam, mode, k, cache_bytes):
    r = spr.spr_create_renderer(vol, wl["W"], wl["H"])
    spr.spr_set_cache_budget(r, cache_bytes)
    if mode == "fixed":
        spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=k)
    else:
        spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=k)
    spr.spr_set_isovalue(r, wl["iso"])
    spr.spr_set_camera(r, cam)
    rs, _ = spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    return fb, rs


def ray_dir(cam, i, j):
    """The pixel's direction as the renderer forms it (single precision, no
    fused multiply-add: numpy float32 operations round each step)."""
    f32 = np.float32
    p00, du, dv = (np.asarray(cam[k], np.float32) for k in ("p00", "du", "dv"))
    return (p00 + f32(i + 0.5) * du) + f32(j + 0.5) * dv


def test_paper_scale_invariance_and_hit_residuals(spr, orc, paper):
    wl, comp, vol = paper
    dims, W, H, iso = wl["dims"], wl["W"], wl["H"], wl["iso"]
    cam = synth.cameras.paper_pose(dims, W, H)
    a, rs_a = render(spr, vol, wl, cam, "adaptive", wl["k"], wl["cache_bytes"])
    assert rs_a["converged"] == 1 and rs_a["n_hits"] > 20000
    # another rule, and a cache of a quarter: the same image
    b, rs_b = render(spr, vol, wl, cam, "fixed", 16, wl["cache_bytes"] // 4)
    for key in FB_KEYS:
        assert np.array_equal(a[key], b[key]), key
    assert rs_b["passes"] != rs_a["passes"] or rs_b["blocks_decoded"] != rs_a["blocks_decoded"]

    Dx, Dy, Dz = dims
    nb = [(d + 3) // 4 for d in dims]
    hits = np.nonzero(a["status"] == 1)[0]
    rng = np.random.default_rng(7)
    sample = rng.choice(hits, size=300, replace=False)
    rate = wl["rate"]
    blocks = {}

    def voxel(x, y, z):
        bid = (x // 4) + nb[0] * ((y // 4) + nb[1] * (z // 4))
        if bid not in blocks:
            lo = bid * 8 * rate
            blocks[bid] = orc.decode_block(comp[lo:lo + 8 * rate].cpu().numpy(), rate)
        return float(blocks[bid][(x % 4) + 4 * (y % 4) + 16 * (z % 4)])

    eye = np.asarray(cam["eye"], np.float64)
    worst = 0.0
    for p in sample:
        i, j = int(p % W), int(p // W)
        d = ray_dir(cam, i, j).astype(np.float64)
        t = float(a["depth"][p]) / np.linalg.norm(d)
        x = eye + t * d
        c = int(a["cell"][p])
        cx, cy, cz = c % Dx, (c // Dx) % Dy, c // (Dx * Dy)
        # the hit lies in the named cell (depth rounds to ~2.4e-4 voxels here)
        for q, lo in zip(x, (cx, cy, cz)):
            assert lo - 2e-3 <= q <= lo + 1 + 2e-3, (p, x, (cx, cy, cz))
        # the block that owns the cell
        assert int(a["block"][p]) == (cx // 4) + nb[0] * ((cy // 4) + nb[1] * (cz // 4))
        # the trilinear interpolant of the decoded corners is the isovalue there
        u = np.clip(x - np.array([cx, cy, cz], np.float64), 0.0, 1.0)
        f = 0.0
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = (u[0] if dx else 1 - u[0]) * (u[1] if dy else 1 - u[1]) * (u[2] if dz else 1 - u[2])
                    f += w * voxel(cx + dx, cy + dy, cz + dz)
        worst = max(worst, abs(f - iso))
    assert worst < 2e-3, worst
