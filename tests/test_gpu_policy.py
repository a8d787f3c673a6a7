"""The learned speculation policy on the GPU against the oracle.

* The tensor-core MLP (tcgen05, bf16 operands, fp32 accumulation) against
  the oracle's network with the same bfloat16 roundings, over several tiles
  and a ragged tail; the counts it implies against the oracle's rule away
  from rounding boundaries.
* The fp32 training gradient against the oracle's double-precision gradient;
  training lowers the loss.
* Training traces: the recorded features against the oracle's geometry at
  the first pass, the labels against the visible-block lists of the oracle's
  raycaster.
* A learned render is bit-identical to the plain render for any policy
  (untrained or trained): the policy only reorders work."""
import numpy as np
import pytest

import synth
from oracle import policy as OP
from test_gpu_render import compare, value_scene

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


def rand_features(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1, 1, size=(n, OP.N_IN)).astype(np.float32)


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 4097, 300001])
def test_tensor_core_forward_matches_oracle(spr, n):
    import torch
    p = OP.init_params(11).astype(np.float32)
    X = rand_features(n, n)
    got = spr.spr_policy_forward(p, torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    want = OP.forward(p, X, bf16_round=True)
    err = np.abs(got - want)
    # fp32 accumulation against double: a hidden activation may round to the
    # neighbouring bfloat16, which moves an output by ~2^-8 of a term
    assert err.max() <= 2e-2 * (1.0 + np.abs(want).max()), err.max()
    assert np.mean(err) < 2e-3
    # the unrounded network is close too (bf16 is the only difference)
    assert np.abs(got - OP.forward(p, X)).max() < 0.1 * (1.0 + np.abs(want).max())


def test_forward_of_scaled_weights_is_exact_on_bf16_grids(spr):
    """Weights and inputs that are exact in bfloat16 with small integer
    products: every sum is exact in fp32, so the tensor cores give the
    oracle's outputs bit for bit."""
    import torch
    rng = np.random.Generator(np.random.PCG64(4))
    p = (rng.integers(-4, 5, size=OP.N_PARAMS) / 8.0).astype(np.float32)
    X = (rng.integers(-8, 9, size=(513, OP.N_IN)) / 4.0).astype(np.float32)
    got = spr.spr_policy_forward(p, torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    want = OP.forward(p, X, bf16_round=True)
    assert np.array_equal(got, want)


def test_counts_follow_the_rule(spr):
    import torch
    p = OP.init_params(12).astype(np.float32)
    p[OP.OFF_B3 + 1] = 2.0                  # counts around 4
    X = rand_features(4096, 5)
    y = spr.spr_policy_forward(p, torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    want = OP.forward(p, X, bf16_round=True)
    k_gpu = OP.policy_k(y[:, 1], 0.25, 32)
    k_orc = OP.policy_k(want[:, 1], 0.25, 32)
    # the count may differ only where 2^(y + margin) lies within the output
    # tolerance of an integer
    z = np.exp2(want[:, 1] + 0.25)
    near = np.abs(z - np.round(z)) < 0.05 * z
    assert np.array_equal(k_gpu[~near], k_orc[~near])


def test_gradient_matches_oracle(spr):
    import torch
    p = OP.init_params(13).astype(np.float32)
    X = rand_features(5000, 6)
    lab = np.random.Generator(np.random.PCG64(8)).integers(1, 70, size=5000).astype(np.int32)
    g, (l0, l1) = spr.spr_policy_grad(p, torch.from_numpy(X).cuda(), torch.from_numpy(lab).cuda(), tau=0.9)
    want = OP.grad(p, X, lab, 0.9)
    wl0, wl1 = OP.loss(p, X, lab, 0.9)
    assert abs(l0 - wl0) <= 1e-4 * wl0 and abs(l1 - wl1) <= 1e-4 * wl1
    assert np.abs(g - want).max() <= 1e-4 * np.abs(want).max()


def test_training_lowers_the_loss(spr):
    import torch
    X = rand_features(60000, 9)
    # a learnable target: needed blocks grow with feature 0 and shrink with 3
    need = np.clip(np.round(np.exp2(2.5 + 1.5 * X[:, 0] - X[:, 3])), 1, 64).astype(np.int32)
    Xd, Ld = torch.from_numpy(X).cuda(), torch.from_numpy(need).cuda()
    p0 = OP.init_params(14).astype(np.float32)
    before = OP.loss(p0, X, need, 0.9)[0]
    p1, losses = spr.spr_policy_train(Xd, Ld, p0, epochs=6, batch=2048, lr=3e-3)
    after = OP.loss(p1, X, need, 0.9)[0]
    assert after < 0.1 * before, (before, after, losses)
    assert losses[-1] < losses[0]


def render(spr, sc, mode, k_max=32, params=None, margin=0.0, trace=None, slots=None, floor=True):
    import torch
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, sc.W, sc.H)
    spr.spr_set_camera(r, sc.cam)
    spr.spr_set_isovalue(r, sc.iso)
    nb = sc.ovol.fine.shape[0]
    spr.spr_set_cache_budget(r, 256 * (slots if slots else max(8, nb)))
    if params is not None:
        spr.spr_set_policy(r, params, margin, floor=floor)
    spr.spr_set_speculation(r, mode, k_max=k_max)
    if trace is not None:
        spr.spr_set_trace(r, trace, 1)
    rs, passes = spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    if trace is not None:
        spr.spr_trace_labels(r, trace)
    r.close()
    v.close()
    return fb, rs, passes


@pytest.mark.parametrize("floor", [True, "after_first", False])
@pytest.mark.parametrize("bias", [-1.0, 1.5, 4.0])
def test_learned_render_keeps_the_image(spr, orc, bias, floor):
    sc = value_scene(orc, (48, 40, 36), 51, 96, 72)
    want, rs0, p0 = render(spr, sc, spr.SPR_SPEC_ADAPTIVE, k_max=32)
    p = OP.init_params(15).astype(np.float32)
    p[OP.OFF_B3 + 1] = bias
    got, rs1, passes = render(spr, sc, spr.SPR_SPEC_LEARNED, k_max=32, params=p, floor=floor)
    for key in FB_KEYS:
        assert np.array_equal(got[key], want[key]), key
    assert rs1["n_hits"] == rs0["n_hits"]
    if floor is True:   # no ray advances less per pass than under the plain rule
        assert rs1["passes"] <= rs0["passes"]
    compare(sc, got)


def test_learned_render_tight_cache(spr, orc):
    sc = value_scene(orc, (48, 44, 40), 52, 64, 64)
    want, _, _ = render(spr, sc, spr.SPR_SPEC_ADAPTIVE)
    p = OP.init_params(16).astype(np.float32)
    p[OP.OFF_B3 + 1] = 5.0                  # counts at the cap: the cache overflows
    got, _, passes = render(spr, sc, spr.SPR_SPEC_LEARNED, k_max=32, params=p, slots=24)
    assert any(pp["retries"] for pp in passes)
    for key in FB_KEYS:
        assert np.array_equal(got[key], want[key]), key


def features_at_entry(orc, sc, pix):
    """The oracle's first-pass features of every ray that enters the volume."""
    dims, W, H = sc.dims, sc.W, sc.H
    nb = np.array([(x + 3) // 4 for x in dims])
    lin = orc.entry_blocks(dims, sc.cam, W, H).astype(np.int64)   # 0xFFFFFFFF where the ray misses
    ent = np.stack([lin % nb[0], (lin // nb[0]) % nb[1], lin // (nb[0] * nb[1])], axis=1)
    ent[lin == 0xFFFFFFFF] = -1
    d = orc.ray_dirs(sc.cam, W, H).astype(np.float64)
    fine = sc.ovol.fine
    tb = np.array([(x - 1 + 3) // 4 for x in dims])
    nc = (nb + 3) // 4
    ns = (nc + 3) // 4
    occ = ((fine[:, 0] <= sc.iso) & (sc.iso <= fine[:, 1])).reshape(nb[2], nb[1], nb[0])
    # occupied blocks per coarse cell, occupied coarse cells per super cell
    cnt = np.zeros((nc[2], nc[1], nc[0]), np.int64)
    for z in range(nb[2]):
        for y in range(nb[1]):
            for x in range(nb[0]):
                cnt[z // 4, y // 4, x // 4] += occ[z, y, x]
    scnt = np.zeros((ns[2], ns[1], ns[0]), np.int64)
    for z in range(nc[2]):
        for y in range(nc[1]):
            for x in range(nc[0]):
                scnt[z // 4, y // 4, x // 4] += cnt[z, y, x] > 0
    eye = np.asarray(sc.cam["eye"], np.float64)
    diag = np.linalg.norm(np.asarray(dims, np.float64) - 1.0)
    rays = np.nonzero(ent[:, 0] >= 0)[0]
    b = ent[rays].astype(np.float64)
    f = np.zeros((rays.size, OP.N_IN))
    f[:, 0] = 0.0
    f[:, 1:4] = (b + 0.5) / tb
    f[:, 4:7] = d[rays] / np.linalg.norm(d[rays], axis=1, keepdims=True)
    f[:, 7] = np.linalg.norm(4 * b + 2 - eye, axis=1) / diag
    bi = ent[rays].astype(np.int64)
    f[:, 8] = cnt[bi[:, 2] // 4, bi[:, 1] // 4, bi[:, 0] // 4] / 64.0
    f[:, 9] = scnt[bi[:, 2] // 16, bi[:, 1] // 16, bi[:, 0] // 16] / 64.0
    f[:, 10] = sc.iso
    f[:, 11] = rays.size / (W * H)
    return rays, f


def sphere_scene(orc):
    """A sphere in one corner: most rays enter the volume well before the box
    of blocks that hold the isovalue, so their walks start inside it."""
    from test_gpu_render import Scene
    dims = (72, 64, 56)
    vol = synth.volumes.sphere(dims, (54.0, 16.0, 40.0), 7.0)
    cam = synth.cameras.look_at((-50.0, 80.0, 90.0), (54.0, 16.0, 40.0), (0, 0, 1), 40.0, 80, 64)
    return Scene(orc, dims, vol, 8, 0.5, cam, 80, 64, lists=True)


@pytest.mark.parametrize("scene", ["noise", "sphere"])
def test_trace_features_and_labels(spr, orc, scene):
    """The first pass's features are those of the block where each ray enters
    the volume, also where the walk itself starts later, at the box of blocks
    that hold the isovalue (the sphere scene)."""
    sc = value_scene(orc, (40, 36, 32), 53, 80, 64, lists=True) if scene == "noise" else sphere_scene(orc)
    tr = spr.Trace(80 * 64 * 40)
    fb, rs, passes = render(spr, sc, spr.SPR_SPEC_ADAPTIVE, k_max=8, trace=tr)
    n = tr.n
    assert n == sum(p["n_active"] for p in passes)          # every live ray, every pass (mod 1)
    rays = tr.rays[:n].cpu().numpy().astype(np.int64)
    cons = tr.consumed[:n].cpu().numpy().astype(np.int64)
    lab = tr.labels[:n].cpu().numpy().astype(np.int64)
    feat = tr.features[:n].cpu().numpy().astype(np.float64)
    # labels: the oracle's visible lists, outside its ambiguity mask
    pix = sc.pix
    clear = pix["amb"][rays] == 0
    want = OP.labels_from_pixels(pix, rays, cons)
    assert np.array_equal(lab[clear], want[clear])
    assert clear.mean() > 0.95
    # first pass: nothing consumed, features from the oracle's geometry
    first = feat[:, 0] == 0.0
    assert np.all(cons[first] == 0)
    orays, of = features_at_entry(orc, sc, pix)
    pos = {int(rr): i for i, rr in enumerate(orays)}
    idx = np.array([pos[int(rr)] for rr in rays[first]])
    assert np.abs(feat[first] - of[idx]).max() < 2e-6
    # later passes consume exactly the counts taken before
    assert np.all(lab + np.minimum(cons, 10 ** 9) >= 1)


def test_learned_mode_needs_a_policy_and_valid_flags(spr, orc):
    import torch
    sc = value_scene(orc, (16, 16, 16), 54, 16, 16)
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, 16, 16)
    with pytest.raises(spr.SprError):
        spr.spr_set_speculation(r, spr.SPR_SPEC_LEARNED, k_max=8)
    p = OP.init_params(1).astype(np.float32)
    bad = p.copy()
    bad[7] = np.nan
    with pytest.raises(spr.SprError):
        spr.spr_set_policy(r, bad, 0.0)
    L = spr._lib.load()
    assert L.spr_set_policy(r.handle, p.ctypes.data_as(spr.api.ctypes.c_void_p), 0.0, 4) == spr._lib.SPR_ERR_INVALID_ARG
    spr.spr_set_policy(r, p, 0.0)
    spr.spr_set_speculation(r, spr.SPR_SPEC_LEARNED, k_max=8)
    r.close()
    v.close()


def test_trace_sampling_and_capacity(spr, orc):
    """With sample_mod m only rays whose id hashes to 0 mod m are recorded;
    a full buffer keeps its first samples and reports its capacity."""
    import torch
    sc = value_scene(orc, (40, 36, 32), 55, 80, 64)
    full = spr.Trace(80 * 64 * 40)
    render(spr, sc, spr.SPR_SPEC_ADAPTIVE, k_max=8, trace=full)
    n_full = full.n
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, sc.W, sc.H)
    spr.spr_set_cache_budget(r, 256 * sc.ovol.fine.shape[0])
    spr.spr_set_camera(r, sc.cam)
    spr.spr_set_isovalue(r, sc.iso)
    spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=8)
    sub = spr.Trace(n_full)
    spr.spr_set_trace(r, sub, 7)
    spr.spr_render_to_convergence(r, 100000)
    n_sub = spr.spr_trace_labels(r, sub)
    assert 0 < n_sub < n_full / 3
    rays_full = full.rays[:n_full].cpu().numpy()
    rays_sub = sub.rays[:n_sub].cpu().numpy()
    assert set(rays_sub.tolist()) <= set(rays_full.tolist())
    small = spr.Trace(100)
    spr.spr_set_trace(r, small, 1)
    spr.spr_set_camera(r, sc.cam)
    spr.spr_render_to_convergence(r, 100000)
    assert spr.spr_trace_labels(r, small) == 100
    # labels need a converged render
    spr.spr_set_camera(r, sc.cam)
    with pytest.raises(spr.SprError):
        spr.spr_trace_labels(r, small)
    r.close()
    v.close()
