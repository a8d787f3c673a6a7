"""The paper-scale workload at its full size, in the configuration bench.py
times: the 2048x2048x1920 mixing layer at 2 bits/value, isovalue 0.5,
1280x720, adaptive speculation up to 64, a 4 GB cache (the configuration of
the paper's R-M figure, Sec. 5.1).

The input is the oracle's own encoding of the synth volume; the library's
encoder is checked to produce the same 2 GB stream.  The oracle decodes the
blocks its rays reach on demand, so it renders this volume without a decoded
copy (30 GB): every pixel of the image is compared element by element -- hit
or miss, block and cell ids bit-exact outside the oracle's ambiguity mask,
depth within 1e-3 voxels, grey within 1/255.  The image is also the same
under another speculation rule with a quarter of the cache."""
import numpy as np
import pytest

import synth
from parity import check_counters, resolved_pix

pytestmark = pytest.mark.gpu

FB_KEYS = ("depth", "rgba", "block", "cell", "status")
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


@pytest.fixture(scope="module")
def paper(spr, orc):
    import torch

    import bench
    wl = dict(bench.WORKLOADS["paper"])
    lib_comp, comp = bench.compress_volume(wl, spr, torch, library=True, oracle_side=True)
    # the library's encoder gives the oracle's stream, byte for byte
    step = 256 << 20
    for lo in range(0, comp.size, step):
        hi = min(comp.size, lo + step)
        same = torch.equal(lib_comp[lo:hi].cpu(), torch.from_numpy(comp[lo:hi]))
        assert same, "encoder differs from the oracle in bytes %d..%d" % (lo, hi)
    del lib_comp
    vol = spr.spr_create_volume(wl["dims"], wl["rate"], torch.from_numpy(comp).cuda())
    torch.cuda.empty_cache()
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
    rs, passes = spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    return fb, rs, passes


def test_paper_scale_matches_oracle(spr, orc, paper):
    wl, comp, vol = paper
    dims, W, H, iso = wl["dims"], wl["W"], wl["H"], wl["iso"]
    cam = synth.cameras.paper_pose(dims, W, H)
    fb, rs, _ = render(spr, vol, wl, cam, "adaptive", wl["k"], wl["cache_bytes"])
    assert rs["converged"] == 1 and rs["n_hits"] > 20000

    # every pixel of the image against the oracle
    ov = orc.Volume.on_demand(comp, dims, wl["rate"])
    want = orc.render(ov, cam, W, H, iso)
    assert ov.last_decodes > 0
    clear = want["amb"] == 0
    assert clear.mean() >= 0.99, "ambiguous fraction %.4f" % (1 - clear.mean())
    assert not np.any(want["amb"] & 0x10000)

    status = fb["status"]
    assert np.all(status != 0), "live rays left"
    hit = status == 1
    assert np.array_equal(hit[clear], want["hit"][clear] == 1), \
        "hit/miss differs at pixels %s" % np.nonzero(clear & (hit != (want["hit"] == 1)))[0][:10]
    both = clear & hit
    assert both.sum() > 20000 and (clear & ~hit).sum() > 100000   # hits and misses both compared
    assert np.array_equal(fb["block"][both], want["block"][both])
    cell_o = (want["cell"][:, 0].astype(np.uint64) + np.uint64(dims[0]) *
              (want["cell"][:, 1].astype(np.uint64) + np.uint64(dims[1]) * want["cell"][:, 2].astype(np.uint64)))
    assert np.array_equal(fb["cell"][both], cell_o[both])
    dd = np.abs(fb["depth"][both].astype(np.float64) - want["depth"][both])
    assert dd.max() < DEPTH_TOL, dd.max()
    grey = fb["rgba"][both] & 255
    assert np.abs(grey.astype(np.int64) - want["grey"][both]).max() <= 1
    miss = clear & ~hit
    assert np.all(np.isinf(fb["depth"][miss])) and np.all(fb["block"][miss] == 0xFFFFFFFF)
    # ambiguous pixels: the GPU's answer is one the oracle's tolerance allows
    amb = ~clear & hit & (want["hit"] == 1)
    assert np.abs(fb["depth"][amb].astype(np.float64) - want["depth"][amb]).max(initial=0) < DEPTH_TOL

    # another rule, and a cache of a quarter: the same image
    b, rs_b, _ = render(spr, vol, wl, cam, "fixed", 16, wl["cache_bytes"] // 4)
    for key in FB_KEYS:
        assert np.array_equal(fb[key], b[key]), key
    assert rs_b["passes"] != rs["passes"] or rs_b["blocks_decoded"] != rs["blocks_decoded"]


def test_paper_scale_counters_match_pass_simulator(spr, orc, paper):
    """Every per-pass counter of the paper-scale render (live rays, k, entries,
    visible and requested blocks, blocks decoded, evictions, hits, exits) and
    every pixel's final pass equal the oracle's pass simulator run on the
    oracle's visible lists of all 921,600 rays (fine ranges formed on demand
    from decoded neighbours), with the 4 GB cache; and again with a cache of
    600,000 slots, which the second pass overflows (k halves and the pass is
    redone, and blocks are evicted)."""
    wl, comp, vol = paper
    dims, W, H, iso = wl["dims"], wl["W"], wl["H"], wl["iso"]
    cam = synth.cameras.paper_pose(dims, W, H)
    ov = orc.Volume.on_demand(comp, dims, wl["rate"], lazy_fine=True)
    pix, off, vis = orc.render(ov, cam, W, H, iso, lists=True)

    class Scene:
        pass
    sc = Scene()
    sc.pix, sc.off, sc.vis = pix, off, vis
    for slots in (wl["cache_bytes"] // 256, 600000):
        fb, rs, passes = render(spr, vol, wl, cam, "adaptive", wl["k"], slots * 256)
        st, final = orc.simulate(W, H, dims, resolved_pix(sc, fb), off, vis, spec_mode=orc.SPEC_ADAPTIVE,
                                 k_max=wl["k"], n_slots=slots)
        check_counters(st, passes)
        assert np.array_equal(fb["final_pass"], final)
        assert rs["blocks_decoded"] == int(st["n_decoded"].sum())
        if slots == 600000:
            assert st["retries"].sum() > 0 and st["n_evicted"].sum() > 0
