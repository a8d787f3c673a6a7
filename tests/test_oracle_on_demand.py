"""The oracle's on-demand form (blocks decoded the first time a ray reaches
them, Sec. 3.5) against its dense form, and the volume encoder's slab
decomposition.

The dense form is pinned elsewhere (closed forms, brute force, the dense
march); here the on-demand form must give the same pixel records bit for
bit, decode exactly the blocks whose voxels the walk reads, and derive the
fine ranges of Sec. 3.1 from decoded neighbours exactly as orc_ranges does.
"""
import numpy as np
import pytest

import synth


def scene(orc, dims, seed, rate, q=0.6):
    vol = synth.volumes.value_noise(dims, seed=seed, ref=max(dims))
    iso = float(np.float32(np.quantile(vol, q)))
    comp = orc.encode_volume(vol, dims, rate)
    return vol, iso, comp


@pytest.mark.parametrize("dims,seed,rate", [((33, 17, 26), 4, 8), ((33, 17, 26), 5, 2),
                                            ((20, 12, 9), 6, 1), ((64, 40, 24), 7, 32)])
def test_on_demand_equals_dense(orc, dims, seed, rate):
    _, iso, comp = scene(orc, dims, seed, rate)
    dense = orc.Volume.from_compressed(comp, dims, rate)
    lazy = orc.Volume.on_demand(comp, dims, rate, lazy_fine=True)
    W, H = 48, 40
    cam = synth.cameras.random_pose(dims, seed=seed + 100, W=W, H=H, distance_factor=1.6)
    a = orc.render(dense, cam, W, H, iso, lists=True)
    b = orc.render(lazy, cam, W, H, iso, lists=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert a[0]["hit"].sum() > 50
    # walks continued past the hit (the speculative lists of Sec. 4.1)
    c = orc.render(dense, cam, W, H, iso, full_lists=True)
    d = orc.render(lazy, cam, W, H, iso, full_lists=True)
    assert np.array_equal(c, d)
    # without fine ranges the on-demand form reports no visible lists, as the
    # dense form without them does
    plain = orc.Volume.on_demand(comp, dims, rate)
    e = orc.render(plain, cam, W, H, iso)
    f = orc.render(orc.Volume(dense.decoded, dims), cam, W, H, iso)
    assert np.array_equal(e, f)
    assert np.all(e["n_visible"] == 0)
    # the independent dense march reads the same voxels
    assert np.array_equal(orc.march(dense, cam, W, H, iso), orc.march(lazy, cam, W, H, iso))


def test_sampled_pixels_and_threads(orc):
    dims, rate = (40, 36, 30), 2
    _, iso, comp = scene(orc, dims, 9, rate)
    dense = orc.Volume.from_compressed(comp, dims, rate)
    lazy = orc.Volume.on_demand(comp, dims, rate)
    W, H = 64, 48
    cam = synth.cameras.random_pose(dims, seed=109, W=W, H=H, distance_factor=1.4)
    px = np.random.default_rng(3).choice(W * H, size=500, replace=False)
    want = orc.render(dense, cam, W, H, iso, pixels=px)
    for nt in (1, 3):
        got = orc.render(lazy, cam, W, H, iso, pixels=px, nthreads=nt)
        want["n_visible"] = 0
        want["hit_index"] = -1
        assert np.array_equal(got, want)


def test_decodes_exactly_the_blocks_the_walk_reads(orc):
    """With the isovalue outside the data every ray walks to its exit; one
    pixel on one thread decodes each block holding a corner of a visited
    cell once (the memo never drops a block at these sizes), and nothing
    else."""
    dims, rate = (30, 22, 26), 4
    _, _, comp = scene(orc, dims, 11, rate)
    lazy = orc.Volume.on_demand(comp, dims, rate)
    W, H = 16, 12
    cam = synth.cameras.random_pose(dims, seed=111, W=W, H=H, distance_factor=1.5)
    nb = orc.nblocks(dims)
    checked = 0
    for p in range(W * H):
        cells = orc.trace_cells(dims, cam, W, H, p % W, p // W)
        orc.render(lazy, cam, W, H, 2.0, pixels=[p], nthreads=1)
        blocks = set()
        for c in cells:
            for k in range(8):
                x, y, z = c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + (k >> 2)
                blocks.add((x // 4) + nb[0] * ((y // 4) + nb[1] * (z // 4)))
        assert lazy.last_decodes == len(blocks), p
        checked += len(cells) > 0
    assert checked > 20
    # a camera looking away from the volume decodes nothing
    away = synth.cameras.look_at((-40.0, -40.0, -40.0), (-80.0, -90.0, -70.0), (0, 0, 1), 30.0, W, H)
    orc.render(lazy, away, W, H, 0.5)
    assert lazy.last_decodes == 0


def test_lazy_fine_ranges_match_orc_ranges(orc):
    """Visible lists from fine ranges formed on demand equal those from the
    precomputed grid, at several isovalues (so blocks both in and out of
    range are visited)."""
    dims, rate = (26, 31, 19), 8
    vol, _, comp = scene(orc, dims, 13, rate)
    dense = orc.Volume.from_compressed(comp, dims, rate)
    lazy = orc.Volume.on_demand(comp, dims, rate, lazy_fine=True)
    W, H = 32, 32
    cam = synth.cameras.random_pose(dims, seed=113, W=W, H=H, distance_factor=1.5)
    for q in (0.2, 0.5, 0.9):
        iso = float(np.float32(np.quantile(vol, q)))
        a = orc.render(dense, cam, W, H, iso, full_lists=True, lists=True)
        b = orc.render(lazy, cam, W, H, iso, full_lists=True, lists=True)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_slab_encoding_equals_whole_volume(orc):
    """The volume encoder on z slabs whose depth is a multiple of 4, the
    streams concatenated, equals the encoder on the whole volume (block ids
    run x, then y, then z); the last slab pads by edge replication."""
    dims = (23, 18, 30)
    u8 = (synth.volumes.value_noise(dims, seed=17, ref=30) * 255).astype(np.uint8)
    whole = orc.encode_volume(u8, dims, 2)
    parts = [orc.encode_volume(u8[z0:z0 + 8], (dims[0], dims[1], min(8, dims[2] - z0)), 2)
             for z0 in range(0, dims[2], 8)]
    assert np.array_equal(np.concatenate(parts), whole)
    # and block by block from the hand-padded block
    nb = orc.nblocks(dims)
    rng = np.random.default_rng(5)
    for b in rng.choice(nb[0] * nb[1] * nb[2], size=40, replace=False):
        bx, by, bz = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
        blk = np.zeros(64, np.float32)
        for z in range(4):
            for y in range(4):
                for x in range(4):
                    gx, gy, gz = (min(4 * bx + x, dims[0] - 1), min(4 * by + y, dims[1] - 1),
                                  min(4 * bz + z, dims[2] - 1))
                    blk[x + 4 * y + 16 * z] = np.float32(u8[gz, gy, gx]) / np.float32(255.0)
        assert np.array_equal(orc.encode_block(blk, 2), whole[16 * b:16 * b + 16])
