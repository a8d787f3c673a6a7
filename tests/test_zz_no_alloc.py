"""The allocation-free prefix sum (spr_exclusive_scan_u32_noalloc) against the
allocating one (spr_exclusive_scan_u32), called through the C ABI.

The file name sorts last so that the static scratch has been through every
other test's device work before these run; they also pass alone.  Integer
results: equality is the tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_N = 1 << 26   # the largest n the static scratch serves


@pytest.fixture(scope="module")
def spr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_10212_gb300 as m
    return m


def _input(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.integers(0, 1000, size=n).astype(np.int32)).cuda()


def _noalloc(spr, x):
    import torch
    out = torch.full_like(x, -1)
    total = torch.full((1,), -1, dtype=torch.int32, device=x.device)
    spr.spr_exclusive_scan_u32_noalloc(x, out, total)
    return out, total


# pairs of sizes called back to back: the second call must not see the
# first one's tile status, ticket or flags
@pytest.mark.parametrize("n1,n2", [(0, 1), (5, 2049), (3 * 2048 + 7, 2048),
                                   (1_000_003, 4096 * 3 + 5), (MAX_N, 12_345)])
def test_two_calls_in_a_row_match_the_allocating_scan(spr, n1, n2):
    import torch
    xs = [_input(n1, n1 + 1), _input(n2, n2 + 2)]
    got = [_noalloc(spr, x) for x in xs]
    torch.cuda.synchronize()
    for x, (out, total) in zip(xs, got):
        want, want_total = spr.spr_exclusive_scan_u32(x)
        assert torch.equal(out, want)
        assert int(total.item()) == int(want_total.item())


def test_in_place_and_repeated_on_one_input(spr):
    import torch
    x = _input(77_777, 3)
    want, want_total = spr.spr_exclusive_scan_u32(x)
    for _ in range(2):
        y = x.clone()
        total = torch.zeros(1, dtype=torch.int32, device="cuda")
        spr.spr_exclusive_scan_u32_noalloc(y, y, total)
        assert torch.equal(y, want)
        assert int(total.item()) == int(want_total.item())


def test_makes_no_allocator_call(spr):
    """With an allocator that refuses every request, the allocating scan
    fails with SPR_ERR_OUT_OF_MEMORY and this one still succeeds, asking
    the allocator for nothing."""
    import torch
    from paper_2309_10212_gb300 import _lib
    x = _input(50_000, 4)
    want, _ = spr.spr_exclusive_scan_u32(x)
    calls = []
    spr.spr_set_allocator(lambda nbytes, stream: calls.append(nbytes) or 0,
                          lambda ptr, nbytes, stream: None)
    try:
        out = torch.empty_like(x)
        total = torch.zeros(1, dtype=torch.int32, device="cuda")
        lib = _lib.load()
        rc = lib.spr_exclusive_scan_u32_noalloc(x.data_ptr(), out.data_ptr(), x.numel(),
                                                total.data_ptr(), None)
        assert rc == 0
        assert calls == []
        rc_alloc = lib.spr_exclusive_scan_u32(x.data_ptr(), out.data_ptr(), x.numel(),
                                              total.data_ptr(), None)
        assert rc_alloc == _lib.SPR_ERR_OUT_OF_MEMORY
        assert calls
    finally:
        spr.spr_set_allocator()
    torch.cuda.synchronize()
    out, _ = _noalloc(spr, x)
    assert torch.equal(out, want)


def test_rejects_n_beyond_the_static_scratch(spr):
    import torch
    from paper_2309_10212_gb300 import _lib
    x = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    out = torch.full_like(x, 7)
    rc = _lib.load().spr_exclusive_scan_u32_noalloc(x.data_ptr(), out.data_ptr(), x.numel(),
                                                    None, None)
    assert rc == _lib.SPR_ERR_INVALID_ARG
    assert b"static scratch limit" in _lib.load().spr_last_error()
    torch.cuda.synchronize()
    assert bool((out == 7).all())      # nothing was written
    y, _ = _noalloc(spr, x[:MAX_N])    # the limit itself is served
    assert int(y[-1].item()) == 0
