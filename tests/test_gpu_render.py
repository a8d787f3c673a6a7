"""GPU parity of the whole pass pipeline (Sec. 3, 4) against the oracle.

Per pixel, outside the oracle's ambiguity mask (hits within 1e-5 voxels of a
cell face, |f| < 1e-5 at a face crossing or extremum before the hit, or a
crossing flatter than 1e-3 per voxel): hit/miss, block id and cell id are
bit-exact, depth is within 1e-3 voxels and grey within 1/255.  Across
speculation counts, cache budgets and progressive vs single-pass rendering,
framebuffers are bit-identical; per-pass counters equal the oracle's pass
simulator."""
import numpy as np
import pytest

import synth
from parity import check_counters, resolved_pix

pytestmark = pytest.mark.gpu

DEPTH_TOL = 1e-3


@pytest.fixture(scope="module")
def spr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_10212_gb300 as m
    return m


class Scene:
    def __init__(self, orc, dims, vol, rate, iso, cam, W, H, lists=False):
        self.dims, self.rate, self.iso, self.cam, self.W, self.H = dims, rate, iso, cam, W, H
        self.comp = orc.encode_volume(vol, dims, rate)
        self.ovol = orc.Volume.from_compressed(self.comp, dims, rate)
        if lists:
            self.pix, self.off, self.vis = orc.render(self.ovol, cam, W, H, iso, lists=True)
        else:
            self.pix = orc.render(self.ovol, cam, W, H, iso)


def value_scene(orc, dims, seed, W, H, rate=8, q=0.6, dist=1.6, lists=False):
    vol = synth.volumes.value_noise(dims, seed=seed, ref=max(dims))
    iso = float(np.float32(np.quantile(vol, q)))
    cam = synth.cameras.random_pose(dims, seed=seed + 100, W=W, H=H, distance_factor=dist)
    return Scene(orc, dims, vol, rate, iso, cam, W, H, lists)


def gpu_render(spr, sc, mode=None, k=1, k_max=64, slots=None, max_passes=100000):
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
    rs, passes = spr.spr_render_to_convergence(r, max_passes)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    return fb, rs, passes


def compare(sc, fb, max_amb=0.02):
    want = sc.pix
    dims = sc.dims
    clear = want["amb"] == 0
    assert clear.mean() >= 1 - max_amb, "ambiguous fraction %.4f" % (1 - clear.mean())
    assert not np.any(want["amb"] & 0x10000)
    hit = fb["status"] == 1
    assert np.array_equal(fb["status"] == 0, np.zeros_like(hit)), "live rays left"
    assert np.array_equal(hit[clear], want["hit"][clear] == 1), \
        "hit/miss differs at %s" % np.nonzero(hit[clear] != (want["hit"][clear] == 1))[0][:10]
    both = clear & hit
    assert np.array_equal(fb["block"][both], want["block"][both])
    cell_o = (want["cell"][:, 0].astype(np.uint64) + np.uint64(dims[0]) *
              (want["cell"][:, 1].astype(np.uint64) + np.uint64(dims[1]) * want["cell"][:, 2].astype(np.uint64)))
    assert np.array_equal(fb["cell"][both], cell_o[both])
    dd = np.abs(fb["depth"][both].astype(np.float64) - want["depth"][both])
    assert dd.max(initial=0) < DEPTH_TOL, dd.max()
    grey = fb["rgba"][both] & 255
    assert np.abs(grey.astype(np.int64) - want["grey"][both]).max(initial=0) <= 1
    miss = clear & ~hit
    assert np.all(np.isinf(fb["depth"][miss])) and np.all(fb["block"][miss] == 0xFFFFFFFF)
    return int(both.sum())


@pytest.mark.parametrize("dims,seed", [((8, 8, 8), 1), ((16, 16, 16), 2), ((20, 12, 9), 3),
                                       ((33, 17, 26), 4), ((64, 64, 64), 5)])
def test_tiny_volumes_match_oracle(spr, orc, dims, seed):
    sc = value_scene(orc, dims, seed, 64, 48)
    fb, rs, _ = gpu_render(spr, sc)
    n = compare(sc, fb)
    assert n > 50
    assert rs["converged"] == 1


@pytest.mark.parametrize("rate", [1, 2, 32])
def test_rates(spr, orc, rate):
    sc = value_scene(orc, (24, 24, 24), 7, 48, 48, rate=rate)
    fb, _, _ = gpu_render(spr, sc)
    compare(sc, fb)


def test_eye_inside_volume(spr, orc):
    dims = (32, 32, 32)
    vol = synth.volumes.value_noise(dims, seed=8, ref=32)
    iso = float(np.float32(np.quantile(vol, 0.8)))
    cam = synth.cameras.look_at((15.5, 16.25, 14.0), (31, 31, 31), (0, 0, 1), 70.0, 64, 64)
    sc = Scene(orc, dims, vol, 8, iso, cam, 64, 64)
    fb, _, _ = gpu_render(spr, sc)
    compare(sc, fb)


def test_small_workload_k1_k4_and_cache(spr, orc):
    """64^3 value noise, 8 bits/value, 256x256, cache 25% of the blocks, k in {1, 4}."""
    dims = (64, 64, 64)
    vol = synth.volumes.value_noise(dims, seed=1)
    cam = synth.cameras.small_pose(dims, 256, 256)
    sc = Scene(orc, dims, vol, 8, 0.5, cam, 256, 256, lists=True)
    slots = 4096 // 4
    results = []
    for k in (1, 4):
        fb, rs, passes = gpu_render(spr, sc, mode="fixed", k=k, slots=slots)
        compare(sc, fb)
        results.append(fb)
        st, final = orc.simulate(256, 256, dims, resolved_pix(sc, fb), sc.off, sc.vis,
                                 spec_mode=orc.SPEC_FIXED, k=k, n_slots=slots)
        check_counters(st, passes)
        assert np.array_equal(fb["final_pass"], final)
        assert rs["blocks_decoded"] == int(st["n_decoded"].sum())
    for key in results[0]:
        if key != "final_pass":          # the pass a pixel finishes in depends on k
            assert np.array_equal(results[0][key], results[1][key]), key


def test_invariance_across_k_budget_and_single_pass(spr, orc):
    sc = value_scene(orc, (40, 36, 44), 11, 96, 80, rate=4, q=0.55)
    base, _, _ = gpu_render(spr, sc)
    compare(sc, base)
    variants = [dict(mode="fixed", k=1), dict(mode="fixed", k=2), dict(mode="fixed", k=7),
                dict(mode="fixed", k=64), dict(mode="fixed", k=4096),
                dict(mode="adaptive", k_max=8), dict(slots=8), dict(slots=50),
                dict(mode="fixed", k=16, slots=30)]
    for kw in variants:
        fb, rs, passes = gpu_render(spr, sc, **kw)
        for key in base:
            if key == "final_pass":
                continue
            assert np.array_equal(fb[key], base[key]), (kw, key)
        if kw.get("k") == 4096:
            assert rs["passes"] <= 2


def test_counters_match_pass_simulator(spr, orc):
    sc = value_scene(orc, (48, 40, 44), 21, 80, 64, rate=4, q=0.62, lists=True)
    for kw, sim in [(dict(), dict(spec_mode=1, k_max=64)),
                    (dict(mode="fixed", k=3), dict(spec_mode=0, k=3)),
                    (dict(mode="fixed", k=8, slots=60), dict(spec_mode=0, k=8, n_slots=60)),
                    (dict(slots=24), dict(spec_mode=1, k_max=64, n_slots=24))]:
        fb, rs, passes = gpu_render(spr, sc, **kw)
        compare(sc, fb)
        st, final = orc.simulate(sc.W, sc.H, sc.dims, resolved_pix(sc, fb), sc.off, sc.vis, **sim)
        check_counters(st, passes)
        assert np.array_equal(fb["final_pass"], final)
        assert rs["blocks_decoded"] == int(st["n_decoded"].sum())


def test_medium_workload_sampled_pixels(spr, orc):
    """512^3 u8 Gaussian blobs, 2 bits/value, 1280x720, orbit pose 3, cache
    10% of the decoded size: compared on 4000 sampled pixels plus two rows."""
    import torch
    dims = (512, 512, 512)
    W, H = 1280, 720
    u8 = synth.volumes.gaussian_blobs(dims, seed=2, device="cuda")
    comp = spr.spr_encode_u8(u8, 2)
    comp_o = orc.encode_volume(u8.cpu().numpy(), dims, 2)
    assert np.array_equal(comp.cpu().numpy(), comp_o)
    dec = orc.decode_volume(comp_o, dims, 2)
    _, fine, _ = orc.ranges(dec, dims)
    ovol = orc.Volume(dec, dims, fine)
    cam = synth.cameras.medium_pose(3, dims, W, H)
    rng = np.random.default_rng(0)
    pixels = np.unique(np.concatenate([rng.integers(0, W * H, 4000), np.arange(360 * W, 362 * W)]))
    want = orc.render(ovol, cam, W, H, 0.3, pixels=pixels)
    v = spr.spr_create_volume(dims, 2, comp)
    r = spr.spr_create_renderer(v, W, H)
    spr.spr_set_camera(r, cam)
    spr.spr_set_isovalue(r, 0.3)
    spr.spr_set_cache_budget(r, int(0.1 * 512 ** 3 * 4))
    spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=16)
    rs, _ = spr.spr_render_to_convergence(r, 10000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    sub = {k: v_[pixels] for k, v_ in fb.items()}

    class S:
        pass
    sc = S()
    sc.pix, sc.dims = want, dims
    n = compare(sc, sub, max_amb=0.01)
    assert n > 500
    assert rs["converged"] == 1


def test_errors(spr, orc):
    import torch
    sc = value_scene(orc, (16, 16, 16), 31, 16, 16)
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, 16, 16)
    with pytest.raises(spr.SprError) as e:
        spr.spr_render_pass(r)            # no camera yet
    assert e.value.status == -1
    bad = dict(sc.cam)
    bad["eye"] = sc.cam["eye"] + np.float32(1 / 1024)
    with pytest.raises(spr.SprError) as e:
        spr.spr_set_camera(r, bad)
    assert e.value.status == -1
    with pytest.raises(spr.SprError) as e:
        spr.spr_set_cache_budget(r, 7 * 256)
    assert e.value.status == -3
    with pytest.raises(spr.SprError):
        spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=0)
    spr.spr_set_camera(r, sc.cam)
    spr.spr_set_isovalue(r, sc.iso)
    rs, _ = spr.spr_render_to_convergence(r, 1, allow_partial=True)
    assert rs["passes"] == 1
    r.close()
    v.close()


def test_allocator_cap_gives_out_of_memory(spr, orc):
    import torch
    sc = value_scene(orc, (16, 16, 16), 32, 16, 16)
    blocks = torch.from_numpy(sc.comp).cuda()
    used = {"n": 0}
    live = {}

    def alloc(nbytes, stream):
        if used["n"] + nbytes > 1 << 16:
            return 0
        used["n"] += nbytes
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, nbytes, stream):
        live.pop(ptr, None)
        used["n"] -= nbytes
    spr.spr_set_allocator(alloc, free)
    try:
        v = spr.spr_create_volume(sc.dims, sc.rate, blocks)
        with pytest.raises(spr.SprError) as e:
            spr.spr_create_renderer(v, 512, 512)
        assert e.value.status == -2
        v.close()
    finally:
        spr.spr_set_allocator()
    assert used["n"] == 0


def test_graph_and_host_driven_passes_agree(spr, orc):
    """The whole-render graph (a conditional while node over passes) and the
    host-driven passes used for per-stage timing give identical images and
    per-pass counters."""
    import torch
    sc = value_scene(orc, (40, 36, 44), 41, 96, 80, rate=4, q=0.6)
    out = []
    for prof in (False, True, False):
        v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
        r = spr.spr_create_renderer(v, sc.W, sc.H)
        spr.spr_set_camera(r, sc.cam)
        spr.spr_set_isovalue(r, sc.iso)
        spr.spr_set_cache_budget(r, 256 * 60)
        spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=6)
        spr.spr_set_profiling(r, prof)
        rs, passes = spr.spr_render_to_convergence(r, 10000)
        out.append((spr.spr_read_framebuffer(r), rs, passes))
        r.close()
        v.close()
    compare(sc, out[0][0])
    for fb, rs, passes in out[1:]:
        for key in fb:
            assert np.array_equal(fb[key], out[0][0][key]), key
        assert len(passes) == len(out[0][2])
        for a, b in zip(passes, out[0][2]):
            for name in ("n_active", "k_used", "n_entries", "n_visible", "n_requested",
                         "n_decoded", "n_evicted", "n_term_hit", "n_term_miss", "retries"):
                assert a[name] == b[name], name
    assert out[0][1]["passes"] > 2


def test_progressive_single_passes_then_graph(spr, orc):
    """spr_render_pass twice, then spr_render_to_convergence finishes the same
    render: the image equals a one-call render."""
    import torch
    sc = value_scene(orc, (32, 30, 28), 43, 64, 64, rate=8, q=0.6)
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, sc.W, sc.H)
    spr.spr_set_camera(r, sc.cam)
    spr.spr_set_isovalue(r, sc.iso)
    spr.spr_set_speculation(r, spr.SPR_SPEC_FIXED, k=1)
    p1 = spr.spr_render_pass(r)
    p2 = spr.spr_render_pass(r)
    assert p1["pass"] == 1 and p2["pass"] == 2
    rs, passes = spr.spr_render_to_convergence(r, 10000)
    assert passes[0]["pass"] == 3
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    compare(sc, fb)
