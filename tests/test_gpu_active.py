"""The decode-every-active-block count (the alternative Sec. 5.3 measures the
progressive method against) against the oracle's ranges, and its bound on
what a render with an ample cache decodes."""
import numpy as np
import pytest

import synth
from test_gpu_render import gpu_render, value_scene

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


def counts_from_ranges(fine, nb, iso):
    act = ((fine[:, 0] <= iso) & (iso <= fine[:, 1])).reshape(nb[2], nb[1], nb[0])
    need = act.copy()
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                sh = np.zeros_like(act)
                sh[dz:, dy:, dx:] = act[:nb[2] - dz, :nb[1] - dy, :nb[0] - dx]
                need |= sh
    return int(act.sum()), int(need.sum())


@pytest.mark.parametrize("dims,seed,q", [((24, 20, 18), 3, 0.5), ((64, 64, 64), 5, 0.7),
                                         ((33, 17, 26), 4, 0.3)])
def test_active_counts_match_oracle(spr, orc, dims, seed, q):
    import torch
    vol = synth.volumes.value_noise(dims, seed=seed, ref=max(dims))
    iso = float(np.float32(np.quantile(vol, q)))
    comp = orc.encode_volume(vol, dims, 8)
    dec = orc.decode_volume(comp, dims, 8)
    _, fine, _ = orc.ranges(dec, dims)
    nb = tuple((d + 3) // 4 for d in dims)
    want = counts_from_ranges(np.asarray(fine, np.float32).reshape(-1, 2), nb, np.float32(iso))
    v = spr.spr_create_volume(dims, 8, torch.from_numpy(comp).cuda())
    got = spr.spr_count_active_blocks(v, iso)
    v.close()
    assert got == want
    assert 0 < got[0] <= got[1] <= int(np.prod(nb))


def test_render_decodes_at_most_the_needed_set(spr, orc):
    sc = value_scene(orc, (48, 40, 44), 21, 80, 64)
    import torch
    v = spr.spr_create_volume(sc.dims, sc.rate, torch.from_numpy(sc.comp).cuda())
    _, needed = spr.spr_count_active_blocks(v, sc.iso)
    v.close()
    for spec in (dict(mode="fixed", k=1), dict(mode="fixed", k=4), dict(k_max=64)):
        _, rs, _ = gpu_render(spr, sc, **spec)     # the cache holds every block: no evictions
        assert rs["evictions"] == 0
        assert 0 < rs["blocks_decoded"] <= needed
