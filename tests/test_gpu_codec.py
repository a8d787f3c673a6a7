"""GPU parity of the FRC4 codec and the range grids (Sec. 3.1, 3.5): the CUDA
encoder, decoder and create_volume ranges against the oracle, bit for bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_10212_gb300 as m
    return m


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dims,rate", [((24, 20, 18), 1), ((24, 20, 18), 2), ((24, 20, 18), 8),
                                       ((17, 9, 30), 5), ((16, 16, 16), 32), ((64, 64, 64), 8)])
def test_encode_f32_matches_oracle(spr, orc, dims, rate):
    vol = synth.volumes.value_noise(dims, seed=3, ref=max(dims))
    want = orc.encode_volume(vol, dims, rate)
    got = spr.spr_encode_f32(_t(vol), rate).cpu().numpy()
    assert np.array_equal(got, want)


def test_encode_u8_matches_oracle(spr, orc):
    dims = (40, 36, 33)
    u8 = synth.volumes.gaussian_blobs(dims, seed=5, n=12)
    for rate in (1, 2, 3, 8):
        want = orc.encode_volume(u8, dims, rate)
        got = spr.spr_encode_u8(_t(u8), rate).cpu().numpy()
        assert np.array_equal(got, want), rate


def test_encode_rejects_non_finite(spr):
    import torch
    v = torch.zeros((8, 8, 8), dtype=torch.float32, device="cuda")
    v[3, 2, 1] = float("nan")
    with pytest.raises(spr.SprError) as e:
        spr.spr_encode_f32(v, 2)
    assert e.value.status == -1


@pytest.mark.parametrize("rate", [1, 2, 3, 8, 32])
def test_decode_random_streams_match_oracle(spr, orc, rate):
    rng = np.random.default_rng(rate)
    n = 3000
    streams = rng.integers(0, 256, size=(n, 8 * rate), dtype=np.uint8)
    got = spr.spr_decode_blocks(_t(streams.reshape(-1)), n, rate).cpu().numpy()
    for i in range(0, n, 7):
        want = orc.decode_block(streams[i], rate)
        assert np.array_equal(got[i].view(np.uint32), want.view(np.uint32)), i


def test_decode_list_and_bad_ids(spr, orc):
    import torch
    dims = (20, 16, 12)
    vol = synth.volumes.value_noise(dims, seed=4, ref=20)
    comp = orc.encode_volume(vol, dims, 4)
    nb = orc.nblocks(dims)
    n = nb[0] * nb[1] * nb[2]
    ids = torch.tensor([5, 0, n - 1, 17, 5], dtype=torch.int32, device="cuda")
    got = spr.spr_decode_blocks(_t(comp), n, 4, ids=ids).cpu().numpy()
    for row, b in zip(got, [5, 0, n - 1, 17, 5]):
        assert np.array_equal(row, orc.decode_block(comp[b * 32:(b + 1) * 32], 4))
    bad = torch.tensor([0, n], dtype=torch.int32, device="cuda")
    with pytest.raises(spr.SprError):
        spr.spr_decode_blocks(_t(comp), n, 4, ids=bad)


def _decode_as_volume(spr, comp, dims, rate):
    nb = tuple((d + 3) // 4 for d in dims)
    n = nb[0] * nb[1] * nb[2]
    blk = spr.spr_decode_blocks(_t(comp), n, rate)
    import torch
    v = blk.view(nb[2], nb[1], nb[0], 4, 4, 4).permute(0, 3, 1, 4, 2, 5)
    v = v.reshape(nb[2] * 4, nb[1] * 4, nb[0] * 4)[:dims[2], :dims[1], :dims[0]]
    return v.contiguous().cpu().numpy()


def test_decode_small_workload_volume(spr, orc):
    dims = (64, 64, 64)
    vol = synth.volumes.value_noise(dims, seed=1)
    comp = orc.encode_volume(vol, dims, 8)
    got = _decode_as_volume(spr, comp, dims, 8)
    want = orc.decode_volume(comp, dims, 8)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_decode_medium_workload_volume(spr, orc):
    """512^3 u8 Gaussian blobs at 2 bits/value: all 2,097,152 blocks."""
    dims = (512, 512, 512)
    u8 = synth.volumes.gaussian_blobs(dims, seed=2, device="cuda").cpu().numpy()
    comp = orc.encode_volume(u8, dims, 2)
    gpu_comp = __import__("paper_2309_10212_gb300").spr_encode_u8(_t(u8), 2).cpu().numpy()
    assert np.array_equal(gpu_comp, comp)
    got = _decode_as_volume(spr, comp, dims, 2)
    want = orc.decode_volume(comp, dims, 2)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_decode_mixing_layer_interface_blocks(spr, orc):
    """The blocks a paper-scale render decodes most: the interface of the
    2048x2048x1920 mixing layer (z = 956..963, full-scale generator, 2
    bits/value, 524,288 blocks), whose parses are the longest; encoder and
    decoder against the oracle, bit for bit."""
    dims = (2048, 2048, 1920)
    u8 = synth.volumes.mixing_layer_slab(dims, 956, 964, synth.volumes.mixing_layer_params(3),
                                         z_mid=960.0, device="cuda")
    sdims = (2048, 2048, 8)
    comp = orc.encode_volume(u8.cpu().numpy(), sdims, 2)
    gpu_comp = spr.spr_encode_u8(u8, 2).cpu().numpy()
    assert np.array_equal(gpu_comp, comp)
    got = _decode_as_volume(spr, comp, sdims, 2)
    want = orc.decode_volume(comp, sdims, 2)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # the slab holds the interface: a third of its blocks are not constant
    b = u8.cpu().numpy().reshape(2, 4, 512, 4, 512, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64)
    assert np.mean(b.max(axis=1) != b.min(axis=1)) > 0.2


@pytest.mark.parametrize("dims", [(16, 16, 16), (21, 13, 9), (65, 33, 18), (64, 64, 64)])
def test_range_grids_match_oracle(spr, orc, dims):
    vol = synth.volumes.value_noise(dims, seed=9, ref=max(dims))
    rate = 6
    comp = orc.encode_volume(vol, dims, rate)
    dec = orc.decode_volume(comp, dims, rate)
    _, fine_o, coarse_o = orc.ranges(dec, dims)
    v = spr.spr_create_volume(dims, rate, _t(comp))
    fine, coarse = spr.spr_volume_ranges(v)
    assert np.array_equal(fine, fine_o)
    assert np.array_equal(coarse, coarse_o)
    v2 = spr.spr_create_volume(dims, rate, comp)        # from host memory
    f2, c2 = spr.spr_volume_ranges(v2)
    assert np.array_equal(f2, fine_o) and np.array_equal(c2, coarse_o)
    v.close()
    v2.close()


def test_create_volume_argument_errors(spr):
    import torch
    with pytest.raises(spr.SprError) as e:
        spr.spr_create_volume((1, 8, 8), 2, torch.zeros(16, dtype=torch.uint8, device="cuda"))
    assert e.value.status == -1
    with pytest.raises(spr.SprError):
        spr.spr_create_volume((8, 8, 8), 2, torch.zeros(15, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("rate", [1, 2, 3, 8, 32])
def test_volume_decode_grouped_by_parse_length(spr, orc, rate):
    """spr_volume_decode_blocks (the renderer's decoder: entries grouped by
    their blocks' plane counts in steps of 256) against the plain decoder and
    the oracle, bit for bit: all blocks, a shuffled list with repeats and a
    ragged length, one entry, none, and an id beyond the volume."""
    import torch
    dims = (37, 29, 26)
    vol = synth.volumes.value_noise(dims, seed=rate, ref=40)
    vol[:12] = 0.0   # all-zero blocks (plane count 0) beside rough ones
    comp = orc.encode_volume(vol, dims, rate)
    nb = orc.nblocks(dims)
    n = nb[0] * nb[1] * nb[2]
    v = spr.spr_create_volume(dims, rate, _t(comp))
    full = spr.spr_volume_decode_blocks(v).cpu().numpy()
    plain = spr.spr_decode_blocks(_t(comp), n, rate).cpu().numpy()
    assert np.array_equal(full.view(np.uint32), plain.view(np.uint32))
    bpb = 8 * rate
    for b in range(0, n, 5):
        assert np.array_equal(full[b].view(np.uint32), orc.decode_block(comp[b * bpb:(b + 1) * bpb], rate).view(np.uint32)), b
    rng = np.random.default_rng(rate)
    ids = rng.integers(0, n, size=3 * 256 + 77).astype(np.int32)
    got = spr.spr_volume_decode_blocks(v, ids=_t(ids)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), plain[ids].view(np.uint32))
    one = spr.spr_volume_decode_blocks(v, ids=_t(ids[:1])).cpu().numpy()
    assert np.array_equal(one.view(np.uint32), plain[ids[:1]].view(np.uint32))
    assert spr.spr_volume_decode_blocks(v, ids=_t(ids[:0])).shape == (0, 64)
    with pytest.raises(spr.SprError):
        spr.spr_volume_decode_blocks(v, ids=torch.tensor([3, n], dtype=torch.int32, device="cuda"))


def test_volume_decode_mixing_layer_interface(spr, orc):
    """The renderer's decoder on the blocks that dominate a paper-scale
    render (the mixing layer's interface, 2 bits/value): a shuffled list of
    300,001 of its 524,288 blocks equals the plain decoder's output, and a
    sample equals the oracle's."""
    dims = (2048, 2048, 1920)
    u8 = synth.volumes.mixing_layer_slab(dims, 956, 964, synth.volumes.mixing_layer_params(3),
                                         z_mid=960.0, device="cuda")
    sdims = (2048, 2048, 8)
    comp = spr.spr_encode_u8(u8, 2)
    n = comp.numel() // 16
    v = spr.spr_create_volume(sdims, 2, comp)
    rng = np.random.default_rng(11)
    ids = rng.permutation(n)[:300001].astype(np.int32)
    got = spr.spr_volume_decode_blocks(v, ids=_t(ids)).cpu().numpy()
    plain = spr.spr_decode_blocks(comp, n, 2, ids=_t(ids)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), plain.view(np.uint32))
    c = comp.cpu().numpy()
    for k in range(0, len(ids), 997):
        b = int(ids[k])
        assert np.array_equal(got[k].view(np.uint32), orc.decode_block(c[b * 16:(b + 1) * 16], 2).view(np.uint32))
