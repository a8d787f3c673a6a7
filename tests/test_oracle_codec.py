"""Pins for the oracle's FRC4 block codec (the stand-in for the ZFP fixed-rate
mode of Sec. 3.1/3.5).  Every check here compares the oracle with something
other than itself: hand-worked values, base -2 digits computed digit by
digit, polynomial counts, exact reversibility, the embedded-prefix property
of bit-plane coding, and error bounds."""
import numpy as np
import pytest


def negabinary_digits(x: int) -> int:
    """Base -2 representation of x, digit by digit (textbook definition)."""
    bits, k = 0, 0
    while x != 0:
        r = x & 1                 # remainder in {0, 1}
        bits |= r << k
        x = (x - r) // -2
        k += 1
    return bits


def test_negabinary_matches_base_minus_two(orc):
    rng = np.random.default_rng(0)
    vals = [0, 1, -1, 2, -2, 3, -3, 2 ** 24, -2 ** 24, 2 ** 27, -2 ** 27, 2 ** 27 - 1]
    vals += [int(v) for v in rng.integers(-2 ** 27, 2 ** 27, size=2000)]
    for v in vals:
        u = orc.int_to_negabinary(v)
        assert u == negabinary_digits(v), v
        assert orc.negabinary_to_int(u) == v
        assert u < 2 ** 30          # planes 29..0 suffice for |c| <= 2^27


def test_lift_hand_example(orc):
    # (1,3,5,9): d0 = 2, s0 = 1 + 1 = 2; d1 = 4, s1 = 5 + 2 = 7; dd = 5, ss = 2 + 2 = 4
    assert list(orc.fwd_lift4([1, 3, 5, 9])) == [4, 5, 2, 4]
    # negative differences use floor halves: (5,2,0,-3): d0=-3, s0=5+(-2)=3; d1=-3,
    # s1=0+(-2)=-2; dd=-5, ss=3+(-3)=0
    assert list(orc.fwd_lift4([5, 2, 0, -3])) == [0, -5, -3, -3]
    # a constant vector keeps only its mean
    assert list(orc.fwd_lift4([7, 7, 7, 7])) == [7, 0, 0, 0]


def test_lift_and_xform_exactly_reversible(orc):
    rng = np.random.default_rng(1)
    for _ in range(500):
        v = rng.integers(-2 ** 26, 2 ** 26, size=4)
        assert list(orc.inv_lift4(orc.fwd_lift4(v))) == list(v)
    for _ in range(300):
        c = rng.integers(-2 ** 24, 2 ** 24 + 1, size=64)
        f = orc.fwd_xform(c)
        assert np.abs(f).max() <= 2 ** 27
        assert np.array_equal(orc.inv_xform(f), c)
    # adversarial: alternating extremes grow the detail coefficients the most
    sign = np.array([(-1) ** (x + y + z) for z in range(4) for y in range(4) for x in range(4)])
    c = (sign * 2 ** 24).astype(np.int64)
    f = orc.fwd_xform(c)
    assert np.abs(f).max() <= 2 ** 27
    assert np.array_equal(orc.inv_xform(f), c)
    # a constant block transforms to its DC coefficient only
    f = orc.fwd_xform(np.full(64, 12345))
    assert f[0] == 12345 and np.all(f[1:] == 0)


def test_coefficient_order_levels(orc):
    perm = orc.coeff_order()
    assert sorted(perm) == list(range(64))
    assert perm[0] == 0
    level = {0: 0, 1: 1, 2: 2, 3: 2}
    lv = [level[p % 4] + level[(p // 4) % 4] + level[p // 16] for p in perm]
    assert lv == sorted(lv)
    # level histogram = coefficients of (1 + t + 2 t^2)^3
    poly = np.polynomial.polynomial.polypow([1, 1, 2], 3)
    assert [lv.count(s) for s in range(7)] == [int(x) for x in poly]
    # within a level, ties go by z, then y, then x
    for a, b in zip(perm, perm[1:]):
        la = level[a % 4] + level[(a // 4) % 4] + level[a // 16]
        lb = level[b % 4] + level[(b // 4) % 4] + level[b // 16]
        if la == lb:
            assert (a // 16, (a // 4) % 4, a % 4) < (b // 16, (b // 4) % 4, b % 4)


def _blocks(seed=2, n=200):
    rng = np.random.default_rng(seed)
    out = []
    x = np.arange(4)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    for _ in range(n):
        kind = rng.integers(0, 4)
        if kind == 0:      # smooth
            a = rng.normal(size=4)
            v = a[0] + 0.1 * (a[1] * X + a[2] * Y + a[3] * Z)
        elif kind == 1:    # noise
            v = rng.normal(size=(4, 4, 4))
        elif kind == 2:    # u8 quantised ramps
            v = np.round(255 * np.clip(0.3 + 0.05 * (X + 2 * Y - Z) + 0.02 * rng.normal(size=(4, 4, 4)), 0, 1)) / 255
        else:              # wide dynamic range
            v = rng.normal(size=(4, 4, 4)) * 2.0 ** rng.integers(-30, 30)
        out.append(np.transpose(v, (2, 1, 0)).reshape(64).astype(np.float32))  # x fastest
    return out


def test_rate32_reproduces_the_quantisation_grid(orc):
    for v in _blocks():
        s = orc.encode_block(v, 32)
        d = orc.decode_block(s, 32)
        nz = v[v != 0]
        emax = max(np.frexp(nz.astype(np.float64))[1].max(), -100)
        assert np.max(np.abs(d.astype(np.float64) - v)) <= 2.0 ** (emax - 25)


def test_round_half_even_quantisation(orc):
    # max value 1.0 -> emax = 1 -> grid 2^-23; 2^-24 is a tie that rounds to 0,
    # 3 * 2^-24 a tie that rounds to 4 * 2^-24
    v = np.zeros(64, np.float32)
    v[0] = 1.0
    v[1] = 2.0 ** -24
    v[2] = 3 * 2.0 ** -24
    v[3] = -3 * 2.0 ** -24
    d = orc.decode_block(orc.encode_block(v, 32), 32)
    assert d[0] == 1.0 and d[1] == 0.0
    assert d[2] == 4 * 2.0 ** -24 and d[3] == -4 * 2.0 ** -24


def test_constant_and_zero_blocks(orc):
    for c in [0.5, 1.0, 0.123456789, -7.25, 1e-20, 3e30, 200 / 255]:
        v = np.full(64, c, np.float32)
        for rate in (2, 4, 8):
            assert np.array_equal(orc.decode_block(orc.encode_block(v, rate), rate), v)
    z = np.zeros(64, np.float32)
    for rate in (1, 2, 32):
        s = orc.encode_block(z, rate)
        assert s.size == 8 * rate and not s.any()
        assert not orc.decode_block(s, rate).any()
    neg0 = np.full(64, -0.0, np.float32)
    assert not orc.encode_block(neg0, 2).any()


def test_embedded_prefix_property(orc):
    """Bit-plane coding is embedded: the rate-R stream is the first 64R bits
    of the rate-32 stream (beyond the common header)."""
    for v in _blocks(seed=3, n=120):
        full = np.unpackbits(orc.encode_block(v, 32), bitorder="little")
        for rate in (1, 2, 3, 5, 8, 16):
            part = np.unpackbits(orc.encode_block(v, rate), bitorder="little")
            assert np.array_equal(part, full[: 64 * rate]), rate


def test_error_falls_with_rate(orc):
    """Mean block-normalised RMS error falls with every extra bit per value, by
    about half per bit once the low planes are reached (a single block may
    fluctuate: truncating negabinary planes is not monotone per value)."""
    blocks = _blocks(seed=4, n=150)
    mean_err = []
    for rate in range(1, 17):
        errs = []
        for v in blocks:
            d = orc.decode_block(orc.encode_block(v, rate), rate).astype(np.float64)
            emax = np.frexp(v[v != 0].astype(np.float64))[1].max()
            errs.append(np.sqrt(np.mean((d - v) ** 2)) / 2.0 ** emax)
        mean_err.append(np.mean(errs))
    for r in range(1, len(mean_err)):
        assert mean_err[r] < mean_err[r - 1]
    for r in range(6, len(mean_err)):
        assert mean_err[r] < mean_err[r - 1] / 1.5


def test_decoder_accepts_any_bits(orc):
    rng = np.random.default_rng(5)
    for rate in (1, 2, 8, 32):
        for _ in range(50):
            s = rng.integers(0, 256, size=8 * rate, dtype=np.uint8)
            d = orc.decode_block(s, rate)
            assert d.shape == (64,)
            assert not np.isnan(d).any()


def test_volume_roundtrip_and_padding(orc):
    rng = np.random.default_rng(6)
    dims = (9, 6, 5)   # partial blocks on every axis
    vol = rng.random((dims[2], dims[1], dims[0])).astype(np.float32)
    comp = orc.encode_volume(vol, dims, 32)
    nb = orc.nblocks(dims)
    assert comp.size == nb[0] * nb[1] * nb[2] * 8 * 32
    dec = orc.decode_volume(comp, dims, 32)
    assert np.max(np.abs(dec - vol)) <= 2.0 ** -25
    # block (2,1,1) holds voxel x=8 only, repeated: its stream equals the
    # stream of a block built by edge replication
    blk = np.zeros((4, 4, 4), np.float32)
    for z in range(4):
        for y in range(4):
            for x in range(4):
                blk[z, y, x] = vol[min(4 + z, 4), min(4 + y, 5), min(8 + x, 8)]
    b = 2 + nb[0] * (1 + nb[1] * 1)
    assert np.array_equal(comp[b * 256:(b + 1) * 256], orc.encode_block(blk.reshape(64), 32))
    # u8 sources are read as u/255 in single precision
    u8 = rng.integers(0, 256, size=(dims[2], dims[1], dims[0]), dtype=np.uint8)
    c8 = orc.encode_volume(u8, dims, 8)
    cf = orc.encode_volume(u8.astype(np.float32) / np.float32(255.0), dims, 8)
    assert np.array_equal(c8, cf)
