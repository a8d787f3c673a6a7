"""Asynchronous renders and the render service (continuous batching).

A submitted render equals the synchronous render; the service admits queued
requests by free streams and device memory, merges requests of one volume and
size into batched renders, overlaps renders on the device, and every
request's image is bit-identical to the same request rendered alone (and,
outside the oracle's ambiguity mask, to the oracle)."""
import numpy as np
import pytest

import synth
from test_gpu_render import Scene, compare, value_scene

pytestmark = pytest.mark.gpu

FB_KEYS = ("depth", "rgba", "block", "status")


@pytest.fixture(scope="module")
def spr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_10212_gb300 as m
    return m


def make_renderer(spr, sc, slots=None, k_max=64):
    import torch
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    r = spr.spr_create_renderer(v, sc.W, sc.H)
    spr.spr_set_camera(r, sc.cam)
    spr.spr_set_isovalue(r, sc.iso)
    nb = sc.ovol.fine.shape[0]
    spr.spr_set_cache_budget(r, 256 * (slots if slots else max(8, nb)))
    spr.spr_set_speculation(r, spr.SPR_SPEC_ADAPTIVE, k_max=k_max)
    return v, r


def test_submit_equals_synchronous_render(spr, orc):
    import torch
    sc = value_scene(orc, (40, 36, 30), 21, 96, 64)
    v, r = make_renderer(spr, sc, slots=64)
    rs0, passes0 = spr.spr_render_to_convergence(r, 100000)
    fb0 = spr.spr_read_framebuffer(r)
    spr.spr_reset_cache(r)
    spr.spr_set_camera(r, sc.cam)
    stream = torch.cuda.Stream()
    spr.spr_render_submit(r, 100000, stream=stream)
    # settings wait until the render is collected
    with pytest.raises(spr.SprError):
        spr.spr_set_isovalue(r, sc.iso)
    seen = []
    while True:
        p, done = spr.spr_render_query(r)
        seen.append(p)
        if done:
            break
    rs1, passes1 = spr.spr_render_collect(r)
    assert seen == sorted(seen) and seen[-1] == rs1["passes"]
    fb1 = spr.spr_read_framebuffer(r)
    for k in fb0:
        assert np.array_equal(fb0[k], fb1[k]), k
    for k in ("passes", "blocks_decoded", "entries", "evictions", "n_rays", "n_hits", "converged"):
        assert rs0[k] == rs1[k], k
    assert [p["n_active"] for p in passes0] == [p["n_active"] for p in passes1]
    compare(sc, fb1)
    # idle again: settings are accepted, a query reports done
    spr.spr_set_isovalue(r, sc.iso)
    assert spr.spr_render_query(r) == (0, True)
    r.close()
    v.close()


def test_memory_estimate_matches_the_renderer(spr, orc):
    import torch
    sc = value_scene(orc, (48, 40, 36), 22, 80, 56)
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    for nv, slots in ((1, 64), (3, 500)):
        r = spr.spr_create_renderer(v, sc.W, sc.H)
        spr.spr_set_cache_budget(r, 256 * slots)
        spr.spr_set_view_count(r, nv)
        for i in range(nv):
            spr.spr_set_view(r, i, sc.cam, sc.iso)
        spr.spr_render_to_convergence(r, 100000)
        est = spr.spr_renderer_memory_estimate(v, sc.W, sc.H, nv, 256 * slots)
        assert spr.spr_renderer_memory(r) == est
        r.close()
    v.close()


def scenes_two_volumes(orc):
    """Requests over two volumes and two image sizes, mixed isovalues."""
    out = []
    vols = [((36, 30, 28), 31), ((28, 40, 24), 32)]
    for vi, (dims, seed) in enumerate(vols):
        vol = synth.volumes.value_noise(dims, seed=seed, ref=max(dims))
        for j, (W, H, q) in enumerate([(64, 48, 0.55), (64, 48, 0.7), (48, 40, 0.6), (64, 48, 0.45),
                                       (48, 40, 0.65)]):
            iso = float(np.float32(np.quantile(vol, q)))
            cam = synth.cameras.random_pose(dims, seed=seed * 10 + j, W=W, H=H, distance_factor=1.7)
            out.append((vi, Scene(orc, dims, vol, 8, iso, cam, W, H)))
    return out


def alone(spr, sc, cache_slots):
    v, r = make_renderer(spr, sc, slots=cache_slots)
    spr.spr_render_to_convergence(r, 100000)
    fb = spr.spr_read_framebuffer(r)
    r.close()
    v.close()
    return fb


def run_service(spr, reqs, memory_bytes, cache_slots, max_inflight, max_batch, stagger=0.0):
    import time

    import torch
    srv = spr.spr_server_create(memory_bytes, max_inflight=max_inflight, max_batch=max_batch)
    vols = {}
    for vi, sc in reqs:
        if vi not in vols:
            v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
            vols[vi] = (v, spr.spr_server_add_volume(srv, v, 256 * cache_slots))
    outs, results, peak = [], {}, 0
    t0 = time.perf_counter()
    for i, (vi, sc) in enumerate(reqs):
        n = sc.W * sc.H
        o = dict(depth=torch.full((n,), -1.0, device="cuda"),
                 rgba=torch.zeros(n, dtype=torch.int32, device="cuda"),
                 block=torch.zeros(n, dtype=torch.int32, device="cuda"),
                 status=torch.full((n,), 7, dtype=torch.uint8, device="cuda"))
        outs.append(o)
        while stagger and time.perf_counter() - t0 < i * stagger:
            for res in spr.spr_server_poll(srv):
                results[res["id"]] = res
        rid = spr.spr_server_submit(srv, vols[vi][1], sc.cam, sc.iso, sc.W, sc.H, outputs=o)
        assert rid == i
    inflight_peak = 0
    while len(results) < len(reqs):
        for res in spr.spr_server_poll(srv):
            results[res["id"]] = res
        info = spr.spr_server_info(srv)
        peak = max(peak, info["memory_used"])
        inflight_peak = max(inflight_peak, info["in_flight"])
        assert info["in_flight"] <= max_inflight
    info = spr.spr_server_info(srv)
    info["inflight_peak"] = inflight_peak
    torch.cuda.synchronize()
    srv.close()
    for v, _ in vols.values():
        v.close()
    fbs = []
    for o in outs:
        fbs.append({"depth": o["depth"].cpu().numpy(), "rgba": o["rgba"].cpu().numpy().view(np.uint32),
                    "block": o["block"].cpu().numpy().view(np.uint32), "status": o["status"].cpu().numpy()})
    return fbs, results, info, peak


@pytest.mark.parametrize("max_inflight,max_batch", [(1, 1), (3, 4), (4, 1)])
def test_service_results_equal_alone(spr, orc, max_inflight, max_batch):
    reqs = scenes_two_volumes(orc)
    fbs, results, info, _ = run_service(spr, reqs, 1 << 30, 300, max_inflight, max_batch)
    assert info["requests_done"] == len(reqs) and info["pending"] == 0 and info["in_flight"] == 0
    batches = [results[i]["batch"] for i in range(len(reqs))]
    if max_batch == 1:
        assert max(batches) == 1
    else:
        assert max(batches) > 1      # queued requests of one volume and size were merged
    if max_inflight > 1:
        # renders overlapped: several were on the device at once, and a
        # request was admitted while an earlier one was still running
        assert info["inflight_peak"] >= 2
        assert any(results[j]["t_admit"] < results[i]["t_done"]
                   for i in range(len(reqs)) for j in range(len(reqs))
                   if results[j]["t_admit"] > results[i]["t_admit"])
    for i, (vi, sc) in enumerate(reqs):
        res = results[i]
        assert res["status"] == 0
        assert res["t_arrival"] <= res["t_admit"] <= res["t_first_pass"] <= res["t_done"]
        assert res["passes"] >= 1
        want = alone(spr, sc, 300)
        for k in FB_KEYS:
            assert np.array_equal(fbs[i][k], want[k]), (i, k)
    # and the oracle, outside its ambiguity mask
    for i in (0, 7):
        fb = dict(fbs[i])
        vi, sc = reqs[i]
        fb["cell"] = alone_cells(spr, sc)
        compare(sc, fb)


def alone_cells(spr, sc):
    v, r = make_renderer(spr, sc, slots=300)
    spr.spr_render_to_convergence(r, 100000)
    cell = spr.spr_read_framebuffer(r)["cell"]
    r.close()
    v.close()
    return cell


def test_service_admits_by_memory(spr, orc):
    """A budget that holds one renderer at a time: requests still complete
    (idle renderers are released to admit the next shape), the pooled memory
    never exceeds the budget, and results are unchanged."""
    import torch
    reqs = scenes_two_volumes(orc)[:6]
    vi, sc = reqs[0]
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    one = max(spr.spr_renderer_memory_estimate(v, s.W, s.H, 1, 256 * 300) for _, s in reqs)
    v.close()
    budget = int(one * 1.5)
    fbs, results, info, peak = run_service(spr, reqs, budget, 300, 4, 1)
    assert peak <= budget
    assert info["renderers_destroyed"] >= 1
    for i, (vi, sc) in enumerate(reqs):
        assert results[i]["status"] == 0
        want = alone(spr, sc, 300)
        for k in FB_KEYS:
            assert np.array_equal(fbs[i][k], want[k]), (i, k)


def test_request_larger_than_budget_fails_cleanly(spr, orc):
    import torch
    sc = value_scene(orc, (24, 24, 24), 23, 32, 32)
    srv = spr.spr_server_create(1 << 16, max_inflight=2, max_batch=2)
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    vid = spr.spr_server_add_volume(srv, v, 256 * 64)
    spr.spr_server_submit(srv, vid, sc.cam, sc.iso, sc.W, sc.H)
    res = []
    while not res:
        res = spr.spr_server_poll(srv)
    assert res[0]["status"] == spr._lib.SPR_ERR_OUT_OF_MEMORY
    srv.close()
    v.close()


def test_staggered_arrivals_overlap(spr, orc):
    """Requests arriving while others run are admitted into free streams;
    first-pass times precede final times; results equal the alone renders."""
    reqs = scenes_two_volumes(orc)
    fbs, results, info, _ = run_service(spr, reqs, 1 << 30, 300, 3, 2, stagger=0.0005)
    for i, (vi, sc) in enumerate(reqs):
        res = results[i]
        assert res["status"] == 0 and res["t_first_pass"] <= res["t_done"]
        want = alone(spr, sc, 300)
        for k in FB_KEYS:
            assert np.array_equal(fbs[i][k], want[k]), (i, k)


def test_reserve_pools_a_renderer_within_the_budget(spr, orc):
    import torch
    sc = value_scene(orc, (28, 24, 20), 24, 40, 32)
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    one = spr.spr_renderer_memory_estimate(v, sc.W, sc.H, 1, 256 * 64)
    srv = spr.spr_server_create(int(one * 1.5), max_inflight=2, max_batch=2)
    vid = spr.spr_server_add_volume(srv, v, 256 * 64)
    spr.spr_server_reserve(srv, vid, sc.W, sc.H, 1)
    info = spr.spr_server_info(srv)
    assert info["renderers"] == 1 and info["memory_used"] == one
    with pytest.raises(spr.SprError):           # a second one does not fit
        spr.spr_server_reserve(srv, vid, sc.W, sc.H, 1)
    o = dict(depth=torch.zeros(sc.W * sc.H, device="cuda"))
    spr.spr_server_submit(srv, vid, sc.cam, sc.iso, sc.W, sc.H, outputs=o)
    res = []
    while not res:
        res = spr.spr_server_poll(srv)
    assert res[0]["status"] == 0
    assert spr.spr_server_info(srv)["renderers_created"] == 1   # the reserved one served it
    want = alone(spr, sc, 64)
    assert np.array_equal(o["depth"].cpu().numpy(), want["depth"])
    srv.close()
    v.close()


def test_submit_rejects_bad_requests(spr, orc):
    import torch
    sc = value_scene(orc, (20, 20, 20), 25, 16, 16)
    srv = spr.spr_server_create(1 << 26, max_inflight=1, max_batch=1)
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    vid = spr.spr_server_add_volume(srv, v, 256 * 64)
    with pytest.raises(spr.SprError):
        spr.spr_server_submit(srv, vid + 1, sc.cam, sc.iso, 16, 16)      # unknown volume
    cam = dict(sc.cam)
    cam["eye"] = np.array(cam["eye"], np.float32) + np.float32(1e-3)   # off the 1/256 grid
    with pytest.raises(spr.SprError):
        spr.spr_server_submit(srv, vid, cam, sc.iso, 16, 16)
    with pytest.raises(spr.SprError):
        spr.spr_server_submit(srv, vid, sc.cam, float("nan"), 16, 16)
    with pytest.raises(spr.SprError):
        spr.spr_server_create(1 << 20, max_inflight=0)
    assert spr.spr_server_info(srv)["pending"] == 0
    srv.close()
    v.close()
