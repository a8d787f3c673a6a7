"""Pins for the oracle's rays, traversal, intersection and ranges (Sec. 3.1-3.3,
3.7, 4.4).  The oracle is compared with: exact rational geometry computed
cell by cell with Fractions, closed-form isosurfaces of trilinear polynomial
fields (which trilinear interpolation reproduces exactly), an independent
dense march, and vectorised numpy range computations."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth


def single_ray(eye, d):
    """A 1x1 camera whose only ray has direction d exactly."""
    z = np.zeros(3, np.float32)
    return dict(eye=np.asarray(eye, np.float32), p00=np.asarray(d, np.float32), du=z, dv=z)


def brute_cells(dims, eye, d):
    """Cells whose box the ray crosses for a positive length, in order."""
    e = [Fr(float(x)) for x in eye]
    v = [Fr(float(x)) for x in d]
    lo, hi = Fr(0), None
    for a in range(3):
        if v[a] == 0:
            if not (0 <= e[a] <= dims[a] - 1):
                return []
            continue
        t0, t1 = (0 - e[a]) / v[a], (dims[a] - 1 - e[a]) / v[a]
        t0, t1 = min(t0, t1), max(t0, t1)
        lo = max(lo, t0)
        hi = t1 if hi is None else min(hi, t1)
    if hi is None or lo >= hi:
        return []
    out = []
    for z in range(dims[2] - 1):
        for y in range(dims[1] - 1):
            for x in range(dims[0] - 1):
                a, b = lo, hi
                ok = True
                for ax, c in enumerate((x, y, z)):
                    if v[ax] == 0:
                        if not (c < e[ax] < c + 1):
                            ok = False
                            break
                        continue
                    t0, t1 = (c - e[ax]) / v[ax], (c + 1 - e[ax]) / v[ax]
                    a, b = max(a, min(t0, t1)), min(b, max(t0, t1))
                if ok and a < b:
                    out.append((a, (x, y, z)))
    out.sort()
    return [c for _, c in out]


ADVERSARIAL = [
    ((-3.5, -3.5, -3.5), (1, 1, 1)),          # through lattice corners
    ((-2.0, 0.5, -2.0), (1, 0, 1)),           # along cell edges
    ((-1.25, -2.5, 0.75), (1, 2, 0)),         # through edges and corners in a plane
    ((0.5, 0.25, -1.0), (0, 0, 1)),           # axis aligned
    ((10.0, 3.5, 2.25), (-1, 0, 0)),          # axis aligned, negative
    ((9.0, 8.0, 7.0), (-1, -1, -1)),          # corner to corner, negative
    ((-0.5, 2.0, 3.0), (0.25, 0.125, -0.375)),
    ((2.5, 2.5, 2.5), (0.3, -0.7, 0.2)),      # eye inside the domain
    ((3.0, 3.0, 3.0), (1, 1, 0.5)),           # eye on a lattice point inside
]


def test_traversal_matches_rational_brute_force(orc):
    dims = (8, 7, 6)
    rng = np.random.default_rng(10)
    rays = list(ADVERSARIAL)
    for _ in range(150):
        eye = np.round(rng.uniform(-6, 14, size=3) * 256) / 256
        tgt = rng.uniform(0, 7, size=3)
        d = (tgt - eye).astype(np.float32)
        if rng.random() < 0.3:
            d[rng.integers(0, 3)] = 0.0
            if np.any((d == 0) & (eye == np.round(eye))):
                continue
        rays.append((tuple(eye), tuple(d)))
    checked = 0
    for eye, d in rays:
        cam = single_ray(eye, d)
        got = [tuple(c) for c in orc.trace_cells(dims, cam, 1, 1, 0, 0)]
        want = brute_cells(dims, np.asarray(eye, np.float32), np.asarray(d, np.float32))
        assert got == want, (eye, d)
        blk = orc.entry_blocks(dims, cam, 1, 1)[0]
        if want:
            x, y, z = want[0]
            nb = orc.nblocks(dims)
            assert blk == (x >> 2) + nb[0] * ((y >> 2) + nb[1] * (z >> 2))
            checked += 1
        else:
            assert blk == 0xFFFFFFFF
    assert checked > 100


def test_ray_directions_are_plain_float32(orc):
    cam = synth.cameras.small_pose((64, 64, 64), 16, 16)
    got = orc.ray_dirs(cam, 16, 16)
    for j in range(16):
        for i in range(16):
            fi, fj = np.float32(i) + np.float32(0.5), np.float32(j) + np.float32(0.5)
            want = (cam["p00"] + fi * cam["du"]) + fj * cam["dv"]   # float32, no FMA
            assert np.array_equal(got[i + 16 * j], want.astype(np.float32))


def test_camera_preconditions(orc):
    cam = synth.cameras.small_pose((64, 64, 64), 8, 8)
    assert orc.check_camera(cam, (64, 64, 64)) == 0
    bad = dict(cam)
    bad["eye"] = cam["eye"] + np.float32(1.0 / 1024)
    assert orc.check_camera(bad, (64, 64, 64)) != 0
    assert orc.check_camera(cam, (1, 64, 64)) != 0
    assert orc.check_camera(cam, (64, 64, 5000)) != 0


def trilinear_poly_field(dims, coef):
    """f = a + b x + c y + d z + e xy + f xz + g yz + h xyz on the voxel grid."""
    z, y, x = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]),
                          indexing="ij")
    a, b, c, d, e, f, g, h = coef
    return (a + b * x + c * y + d * z + e * x * y + f * x * z + g * y * z + h * x * y * z)


def poly_first_root(coef, iso, eye, d, t_lo, t_hi):
    from numpy.polynomial import Polynomial as P
    X = P([float(eye[0]), float(d[0])])
    Y = P([float(eye[1]), float(d[1])])
    Z = P([float(eye[2]), float(d[2])])
    a, b, c, dd, e, f, g, h = coef
    poly = a + b * X + c * Y + dd * Z + e * X * Y + f * X * Z + g * Y * Z + h * X * Y * Z - iso
    roots = [r.real for r in poly.roots() if abs(r.imag) < 1e-9 * (1 + abs(r.real))]
    roots = sorted(r for r in roots if t_lo - 1e-12 <= r <= t_hi + 1e-12)
    return (roots[0] if roots else None), poly


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_closed_form_trilinear_polynomial_isosurface(orc, seed):
    rng = np.random.default_rng(20 + seed)
    dims = (9, 7, 8)
    coef = list(np.round(rng.uniform(-2, 2, size=8) * 16) / 16)
    coef[7] = coef[7] / 4
    field = trilinear_poly_field(dims, coef).astype(np.float32)
    assert np.array_equal(field.astype(np.float64), trilinear_poly_field(dims, coef))
    iso = float(np.float32(np.median(field) + 0.1234567))
    vol = orc.Volume(field, dims)
    W = H = 24
    cam = synth.cameras.random_pose(dims, seed=100 + seed, W=W, H=H, distance_factor=1.3)
    pix = orc.render(vol, cam, W, H, iso)
    dirs = orc.ray_dirs(cam, W, H)
    n_cmp = 0
    for p in range(W * H):
        o = pix[p]
        d = dirs[p].astype(np.float64)
        e = cam["eye"].astype(np.float64)
        # domain interval in double precision (enough to bracket the roots)
        lo, hi = 0.0, np.inf
        for a in range(3):
            if d[a] == 0:
                continue
            t0, t1 = (0 - e[a]) / d[a], (dims[a] - 1 - e[a]) / d[a]
            lo, hi = max(lo, min(t0, t1)), min(hi, max(t0, t1))
        if not o["enters"]:
            assert lo >= hi - 1e-9 or not np.isfinite(hi)
            continue
        t_ref, poly = poly_first_root(coef, iso, e, d, lo, hi)
        if o["amb"]:
            continue
        if t_ref is None:
            assert not o["hit"], p
            continue
        slope = abs(poly.deriv()(t_ref)) / np.linalg.norm(d)
        if slope < 1e-3:
            continue
        assert o["hit"], p
        assert abs(o["t"] - t_ref) <= 1e-9 * (1 + abs(t_ref)), (p, o["t"], t_ref)
        assert abs(o["depth"] - t_ref * np.linalg.norm(d)) <= 1e-8 * (1 + o["depth"])
        hp = e + t_ref * d
        cell = np.clip(np.floor(hp), 0, np.array(dims) - 2).astype(int)
        assert tuple(o["cell"]) == tuple(cell), p
        n_cmp += 1
    assert n_cmp > 50


def test_grey_of_a_planar_field(orc):
    dims = (12, 10, 9)
    gvec = np.array([0.75, -0.5, 0.25])
    z, y, x = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]),
                          indexing="ij")
    field = (gvec[0] * x + gvec[1] * y + gvec[2] * z).astype(np.float32)
    iso = float(np.float32(2.3))
    W = H = 20
    cam = synth.cameras.random_pose(dims, seed=7, W=W, H=H, distance_factor=1.2)
    pix = orc.render(orc.Volume(field, dims), cam, W, H, iso)
    dirs = orc.ray_dirs(cam, W, H).astype(np.float64)
    hits = 0
    for p in np.nonzero(pix["hit"])[0]:
        d = dirs[p]
        cosv = abs(gvec @ d) / (np.linalg.norm(gvec) * np.linalg.norm(d))
        want = np.floor(255 * (0.1 + 0.9 * cosv) + 0.5)
        assert abs(pix["grey"][p] - want) <= 0 or abs(255 * (0.1 + 0.9 * cosv) % 1 - 0.5) < 1e-9
        # the linear root: g.(e + t d) = iso
        t = (iso - gvec @ cam["eye"].astype(np.float64)) / (gvec @ d)
        assert abs(pix["t"][p] - t) < 1e-9 * (1 + t)
        hits += 1
    assert hits > 50


def test_dense_march_agrees(orc):
    dims = (16, 16, 16)
    vol_f = synth.volumes.value_noise(dims, seed=11, ref=16)
    iso = float(np.float32(np.quantile(vol_f, 0.6)))
    W = H = 20
    cam = synth.cameras.random_pose(dims, seed=12, W=W, H=H, distance_factor=1.5)
    vol = orc.Volume(vol_f, dims)
    a = orc.render(vol, cam, W, H, iso)
    b = orc.march(vol, cam, W, H, iso)
    assert np.array_equal(a["enters"], b["enters"])
    clear = a["amb"] == 0
    assert clear.mean() > 0.9
    assert np.array_equal(a["hit"][clear], b["hit"][clear])
    both = clear & (a["hit"] == 1)
    assert both.sum() > 60
    assert np.max(np.abs(a["depth"][both] - b["depth"][both])) < 1e-3


def ranges_numpy(dec, dims):
    nb = [(d + 3) // 4 for d in dims]
    pad = np.full((nb[2] * 4, nb[1] * 4, nb[0] * 4), np.nan)
    pad[:dims[2], :dims[1], :dims[0]] = dec
    blk = pad.reshape(nb[2], 4, nb[1], 4, nb[0], 4)
    raw_mn = np.nanmin(blk, axis=(1, 3, 5))
    raw_mx = np.nanmax(blk, axis=(1, 3, 5))

    def plus_union(mn, mx):
        n2, n1, n0 = mn.shape
        P = np.full((n2 + 1, n1 + 1, n0 + 1), np.inf)
        Q = np.full((n2 + 1, n1 + 1, n0 + 1), -np.inf)
        P[:n2, :n1, :n0], Q[:n2, :n1, :n0] = mn, mx
        omn, omx = np.full(mn.shape, np.inf), np.full(mx.shape, -np.inf)
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    omn = np.minimum(omn, P[dz:dz + n2, dy:dy + n1, dx:dx + n0])
                    omx = np.maximum(omx, Q[dz:dz + n2, dy:dy + n1, dx:dx + n0])
        return omn, omx
    fmn, fmx = plus_union(raw_mn, raw_mx)
    nc = [(b + 3) // 4 for b in nb]
    cp = np.full((nc[2] * 4, nc[1] * 4, nc[0] * 4), np.nan)
    cq = np.full_like(cp, np.nan)
    cp[:nb[2], :nb[1], :nb[0]] = raw_mn
    cq[:nb[2], :nb[1], :nb[0]] = raw_mx
    cmn = np.nanmin(cp.reshape(nc[2], 4, nc[1], 4, nc[0], 4), axis=(1, 3, 5))
    cmx = np.nanmax(cq.reshape(nc[2], 4, nc[1], 4, nc[0], 4), axis=(1, 3, 5))
    kmn, kmx = plus_union(cmn, cmx)
    return (np.stack([raw_mn.ravel(), raw_mx.ravel()], 1), np.stack([fmn.ravel(), fmx.ravel()], 1),
            np.stack([kmn.ravel(), kmx.ravel()], 1))


@pytest.mark.parametrize("dims", [(16, 16, 16), (21, 13, 9), (33, 17, 18), (8, 8, 5)])
def test_ranges_match_numpy_and_cover_dual_grid(orc, dims):
    rng = np.random.default_rng(sum(dims))
    dec = rng.normal(size=(dims[2], dims[1], dims[0])).astype(np.float32)
    raw, fine, coarse = orc.ranges(dec, dims)
    r2, f2, c2 = ranges_numpy(dec.astype(np.float64), dims)
    assert np.array_equal(raw, r2.astype(np.float32))
    assert np.array_equal(fine, f2.astype(np.float32))
    assert np.array_equal(coarse, c2.astype(np.float32))
    nb = orc.nblocks(dims)
    nc = [(b + 3) // 4 for b in nb]
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                b = bx + nb[0] * (by + nb[1] * bz)
                dual = dec[4 * bz:4 * bz + 5, 4 * by:4 * by + 5, 4 * bx:4 * bx + 5]
                assert fine[b, 0] <= dual.min() and dual.max() <= fine[b, 1]
                c = (bx // 4) + nc[0] * ((by // 4) + nc[1] * (bz // 4))
                assert coarse[c, 0] <= fine[b, 0] and fine[b, 1] <= coarse[c, 1]


def test_visible_lists_follow_the_traversal(orc):
    dims = (24, 20, 28)
    vol_f = synth.volumes.value_noise(dims, seed=13, ref=24)
    iso = float(np.float32(np.quantile(vol_f, 0.7)))
    raw, fine, _ = orc.ranges(vol_f, dims)
    vol = orc.Volume(vol_f, dims, fine)
    W = H = 16
    cam = synth.cameras.random_pose(dims, seed=14, W=W, H=H, distance_factor=1.4)
    pix, off, vis = orc.render(vol, cam, W, H, iso, lists=True)
    nb = orc.nblocks(dims)
    assert not np.any(pix["amb"] & orc.AMB_INTERNAL)
    for p in range(W * H):
        lst = vis[off[p]:off[p] + pix["n_visible"][p]]
        if pix["hit"][p]:
            assert lst[pix["hit_index"][p]] == pix["block"][p]
        cells = orc.trace_cells(dims, cam, W, H, p % W, p // W)
        blocks = []
        for x, y, z in cells:
            b = (x >> 2) + nb[0] * ((y >> 2) + nb[1] * (z >> 2))
            if not blocks or blocks[-1] != b:
                blocks.append(b)
        assert len(set(blocks)) == len(blocks)
        want = [b for b in blocks if fine[b, 0] <= iso <= fine[b, 1]]
        assert list(lst) == want
