"""The seeded input generators: the torch (device) form of the counter-based
noise hash gives the numpy form's values, so volumes generated on a GPU equal
those generated on the host."""
import numpy as np

import synth


def test_torch_hash_equals_numpy_hash():
    for seed, start in ((2, 0), (7, (1 << 32) - 3000), (123456789, 5 << 33)):
        a = synth.volumes.uniform_hash01(seed, 20000, start=start).astype(np.float32)
        b = synth.volumes.uniform_hash01_t(seed, 20000, start, "cpu").numpy()
        assert np.array_equal(a, b)


def test_fmix32_torch_equals_numpy():
    import torch
    x = np.random.Generator(np.random.PCG64(1)).integers(0, 1 << 32, size=5000, dtype=np.uint64)
    want = synth.volumes.fmix32(x)
    got = synth.volumes.fmix32_t(torch.from_numpy(x.astype(np.int64))).numpy().astype(np.uint64)
    assert np.array_equal(want, got)
