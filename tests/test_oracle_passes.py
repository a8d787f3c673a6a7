"""Pins for the oracle's progressive pass simulator (Sec. 3, 4): the worked
example of Fig. 3, the speculation count rule, cache invariants, and
termination on rendered scenes."""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make_lists(W, H, lists, hits):
    """Per-pixel records as orc.render(lists=True) would return them."""
    import oracle
    n = W * H
    pix = np.zeros(n, dtype=oracle.PIXEL_DTYPE)
    off = np.zeros(n, dtype=np.int64)
    flat = []
    for p in range(n):
        lst = lists.get(p)
        off[p] = len(flat)
        if lst is None:
            continue
        pix["enters"][p] = 1
        pix["n_visible"][p] = len(lst)
        flat += lst
        if p in hits:
            pix["hit"][p] = 1
            pix["hit_index"][p] = hits[p]
        else:
            pix["hit_index"][p] = -1
    return pix, off, np.asarray(flat + [0], dtype=np.uint32)


def test_fig3_worked_example(orc):
    g = json.load(open(os.path.join(GOLDEN, "fig3_speculation.json")))
    W, H = g["slots"], 1
    # rays 2 and 3 hit in their first block; "ray one" (4) hits in its third
    # visible block, "ray two" (5) in its third of four
    lists = {2: [5], 3: [6], 4: [10, 11, 12], 5: [20, 21, 22, 23]}
    hits = {2: 0, 3: 0, 4: 2, 5: 2}
    pix, off, vis = make_lists(W, H, lists, hits)
    dims = (16, 16, 16)
    st, final = orc.simulate(W, H, dims, pix, off, vis, spec_mode=orc.SPEC_ADAPTIVE, k_max=64)
    assert st["n_active"][0] == g["rays_entering"]
    assert st["k"][0] == g["n_spec_pass1"]
    assert st["k"][1] == g["n_spec_pass2"]
    assert round(100 * st["n_entries"][1] / g["slots"]) == g["utilization_pass2_percent"]
    assert len(st) == g["passes_with_speculation"]
    st1, _ = orc.simulate(W, H, dims, pix, off, vis, spec_mode=orc.SPEC_FIXED, k=1)
    assert len(st1) == g["passes_without_speculation"]
    assert orc.spec_count(10 ** 6, 1, g["n_spec_cap"]) == g["n_spec_cap"]
    assert orc.spec_count(6, 4) == g["n_spec_pass1"]
    assert orc.spec_count(6, 2) == g["n_spec_pass2"]


def test_lru_eviction_sequence(orc):
    # 16 x 1 x 1 blocks: each visible block b also needs b+1.  One ray walks
    # blocks 0, 2, 4, ..., 14 one per pass; 8 slots hold 4 passes' worth.
    W, H = 1, 1
    lists = {0: [0, 2, 4, 6, 8, 10, 12, 14]}
    pix, off, vis = make_lists(W, H, lists, {})
    dims = (64, 4, 4)
    st, final = orc.simulate(W, H, dims, pix, off, vis, spec_mode=orc.SPEC_FIXED, k=1,
                             n_slots=8)
    assert list(st["n_requested"]) == [2] * 8 + [0]
    assert list(st["n_decoded"]) == [2] * 8 + [0]
    assert list(st["n_evicted"]) == [0, 0, 0, 0, 2, 2, 2, 2, 0]
    assert st["n_term_miss"][-1] == 1 and final[0] == 9


def _scene(orc, dims, seed, W, H, q=0.65):
    vol_f = synth.volumes.value_noise(dims, seed=seed, ref=max(dims))
    iso = float(np.float32(np.quantile(vol_f, q)))
    _, fine, _ = orc.ranges(vol_f, dims)
    vol = orc.Volume(vol_f, dims, fine)
    cam = synth.cameras.random_pose(dims, seed=seed + 1, W=W, H=H, distance_factor=1.6)
    pix, off, vis = orc.render(vol, cam, W, H, iso, lists=True)
    return pix, off, vis


@pytest.mark.parametrize("mode,k", [("adaptive", 64), ("fixed", 1), ("fixed", 4)])
def test_every_ray_terminates_once(orc, mode, k):
    dims = (32, 28, 30)
    W = H = 32
    pix, off, vis = _scene(orc, dims, 30, W, H)
    sm = orc.SPEC_ADAPTIVE if mode == "adaptive" else orc.SPEC_FIXED
    st, final = orc.simulate(W, H, dims, pix, off, vis, spec_mode=sm, k=k, k_max=k)
    enters = pix["enters"] == 1
    assert st["n_term_hit"].sum() == pix["hit"].sum()
    assert st["n_term_hit"].sum() + st["n_term_miss"].sum() == enters.sum()
    assert np.all(final[enters] >= 1) and np.all(final[~enters] == 0)
    n_act = st["n_active"]
    assert np.all(n_act[1:] == n_act[:-1] - st["n_term_hit"][:-1] - st["n_term_miss"][:-1])
    # with an unbounded cache every requested block is decoded exactly once
    assert st["n_evicted"].sum() == 0
    if sm == orc.SPEC_ADAPTIVE:
        assert np.all(st["n_entries"] <= W * H)


def test_tight_cache_splits_passes(orc):
    dims = (32, 28, 30)
    W = H = 32
    pix, off, vis = _scene(orc, dims, 31, W, H)
    full, _ = orc.simulate(W, H, dims, pix, off, vis, spec_mode=orc.SPEC_ADAPTIVE)
    tight, final = orc.simulate(W, H, dims, pix, off, vis, spec_mode=orc.SPEC_ADAPTIVE,
                                n_slots=40)
    assert np.all(tight["n_requested"] <= 40)
    assert tight["retries"].sum() > 0
    assert tight["n_term_hit"].sum() == full["n_term_hit"].sum()
    assert tight["n_decoded"].sum() >= full["n_decoded"].sum()
    assert tight["n_evicted"].sum() > 0


def test_per_ray_counts_worked_example(orc):
    """Per-ray counts (Sec. 6's per-ray speculation count) on the Fig. 3 rays,
    worked by hand: rays 2 and 3 take one block and hit; ray 4 takes three
    and hits in its third; ray 5 takes one per pass and hits in its third
    block in pass 3."""
    W, H = 6, 1
    lists = {2: [5], 3: [6], 4: [10, 11, 12], 5: [20, 21, 22, 23]}
    hits = {2: 0, 3: 0, 4: 2, 5: 2}
    pix, off, vis = make_lists(W, H, lists, hits)
    kray = np.ones((8, W), np.int32)
    kray[:, 4] = 3
    st, final = orc.simulate(W, H, (16, 16, 16), pix, off, vis, spec_mode=orc.SPEC_PER_RAY,
                             k_max=4, kray=kray)
    assert list(final) == [0, 0, 1, 1, 1, 3]
    assert list(st["n_entries"]) == [6, 1, 1]
    assert list(st["n_active"]) == [4, 1, 1]
    assert list(st["k"]) == [4, 4, 4]
    # unique visible blocks: {5, 6, 10, 11, 12, 20}, then {21}, then {22}
    assert list(st["n_visible"]) == [6, 1, 1]
    # the count is capped by k_max: with k_max = 1 ray 4 needs three passes
    st1, final1 = orc.simulate(W, H, (16, 16, 16), pix, off, vis, spec_mode=orc.SPEC_PER_RAY,
                               k_max=1, kray=kray)
    assert list(final1) == [0, 0, 1, 1, 3, 3]


def test_per_ray_uniform_counts_equal_fixed(orc):
    """Every ray taking the same count c is the fixed rule with k = c."""
    dims = (32, 28, 30)
    W = H = 32
    pix, off, vis = _scene(orc, dims, 32, W, H)
    for c in (1, 3, 8):
        fixed, ff = orc.simulate(W, H, dims, pix, off, vis, spec_mode=orc.SPEC_FIXED, k=c)
        kray = np.full((len(fixed) + 1, W * H), c, np.int32)
        per, fp = orc.simulate(W, H, dims, pix, off, vis, spec_mode=orc.SPEC_PER_RAY,
                               k_max=c, kray=kray)
        assert np.array_equal(fixed, per) and np.array_equal(ff, fp)


def test_per_ray_counts_closed_form(orc):
    """With a cache that never overflows, each ray is on its own: with
    cumulative counts C_P = k_1 + ... + k_P it finishes in the first pass
    where C_P > its hit index (a hit) or where its remaining list is shorter
    than its count (it left the volume), and takes min(count, remaining)
    entries in every pass until then."""
    dims = (32, 28, 30)
    W = H = 32
    pix, off, vis = _scene(orc, dims, 33, W, H)
    rng = np.random.default_rng(5)
    P = 200
    kray = rng.integers(1, 10, size=(P, W * H)).astype(np.int32)
    st, final = orc.simulate(W, H, dims, pix, off, vis, spec_mode=orc.SPEC_PER_RAY,
                             k_max=9, kray=kray)
    entries = np.zeros(P, np.int64)
    want = np.zeros(W * H, np.int32)
    for p in np.nonzero(pix["enters"])[0]:
        nv = int(pix["n_visible"][p])
        hi = int(pix["hit_index"][p]) if pix["hit"][p] else -1
        pos = 0
        for q in range(P):
            c = int(kray[q, p])
            take = min(c, nv - pos)
            entries[q] += take
            if (hi >= 0 and hi < pos + take) or take < c:
                want[p] = q + 1
                break
            pos += take
    assert np.array_equal(final, want)
    assert np.array_equal(st["n_entries"], entries[:len(st)])
    assert entries[len(st):].sum() == 0
    assert st["retries"].sum() == 0 and st["n_evicted"].sum() == 0
