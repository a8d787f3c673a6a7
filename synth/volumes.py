"""Seeded synthetic volumes that stand in for the paper's data sets.

The paper evaluates on ten real volumes (Table 1) that are not available here.
These generators give seeded stand-ins with the shapes, value distributions
and surface structure of the three workloads the project measures:

* ``value_noise``   -- small: 4-octave value noise in [0, 1], float32;
* ``gaussian_blobs`` -- medium: a sum of 200 axis-aligned anisotropic
  Gaussians plus 10% uniform noise, normalised and stored as 8-bit values;
* ``mixing_layer``  -- paper scale: a two-fluid interface perturbed by seeded
  sinusoids and fractal value noise (amplitude 200 voxels), a stand-in for
  the Richtmyer-Meshkov data set, stored as 8-bit density.

Nothing here is part of the rendering method.  Integer hashing (MurmurHash3's
32-bit finaliser, ``fmix32``) runs in numpy; smooth interpolation runs in
torch so the large volumes can be generated on a GPU slab by slab.  Values
come back as numpy arrays of shape (Dz, Dy, Dx), or as torch tensors when a
device is given.
"""
from __future__ import annotations

import math

import numpy as np

M32 = np.uint64(0xFFFFFFFF)


def fmix32(x: np.ndarray) -> np.ndarray:
    """MurmurHash3 32-bit finaliser on uint32 arrays (computed in uint64)."""
    h = np.asarray(x, dtype=np.uint64) & M32
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & M32
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & M32
    h ^= h >> np.uint64(16)
    return h


def hash_coords(seed: int, octave: int, ix, iy, iz) -> np.ndarray:
    """A 32-bit hash of (seed, octave, ix, iy, iz), chained through fmix32."""
    h = fmix32(np.uint64(seed & 0xFFFFFFFF) ^ np.uint64(0x9E3779B9))
    h = fmix32(h ^ np.uint64(octave & 0xFFFFFFFF))
    h = fmix32(h ^ (np.asarray(ix, dtype=np.int64).astype(np.uint64) & M32))
    h = fmix32(h ^ (np.asarray(iy, dtype=np.int64).astype(np.uint64) & M32))
    h = fmix32(h ^ (np.asarray(iz, dtype=np.int64).astype(np.uint64) & M32))
    return h


def lattice(seed: int, octave: int, shape) -> np.ndarray:
    """Lattice values in [0, 1) of shape (nz, ny, nx)."""
    nz, ny, nx = shape
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (hash_coords(seed, octave, ix, iy, iz).astype(np.float64) / 4294967296.0)


def _torch():
    import torch
    return torch


def _smooth(t):
    return t * t * (3.0 - 2.0 * t)


def _interp_octave(lat, period: float, zs, ys, xs, torch, device):
    """Smoothstep-weighted trilinear interpolation of lattice `lat` (a torch
    tensor (nz, ny, nx)) at voxel coordinates zs x ys x xs (1-D tensors)."""
    def split(c):
        f = c / period
        i0 = torch.floor(f)
        return i0.long(), _smooth(f - i0)
    iz, wz = split(zs)
    iy, wy = split(ys)
    ix, wx = split(xs)
    wz = wz.view(-1, 1, 1)
    wy = wy.view(1, -1, 1)
    wx = wx.view(1, 1, -1)

    def g(dz, dy, dx):
        return lat[(iz + dz).view(-1, 1, 1), (iy + dy).view(1, -1, 1), (ix + dx).view(1, 1, -1)]
    c00 = g(0, 0, 0) * (1 - wx) + g(0, 0, 1) * wx
    c10 = g(0, 1, 0) * (1 - wx) + g(0, 1, 1) * wx
    c01 = g(1, 0, 0) * (1 - wx) + g(1, 0, 1) * wx
    c11 = g(1, 1, 0) * (1 - wx) + g(1, 1, 1) * wx
    return (c00 * (1 - wy) + c10 * wy) * (1 - wz) + (c01 * (1 - wy) + c11 * wy) * wz


def value_noise(dims=(64, 64, 64), seed: int = 1, octaves: int = 4, ref: int = 64,
                device=None):
    """Small workload: sum over octaves o of 2^-o * value noise with lattice
    period ref/(4*2^o) voxels, normalised to [0, 1); float32."""
    torch = _torch()
    dev = torch.device(device or "cpu")
    Dx, Dy, Dz = dims
    zs = torch.arange(Dz, dtype=torch.float64, device=dev)
    ys = torch.arange(Dy, dtype=torch.float64, device=dev)
    xs = torch.arange(Dx, dtype=torch.float64, device=dev)
    acc = torch.zeros((Dz, Dy, Dx), dtype=torch.float64, device=dev)
    total = 0.0
    for o in range(octaves):
        period = max(1.0, ref / (4.0 * 2 ** o))
        shape = (int(Dz / period) + 2, int(Dy / period) + 2, int(Dx / period) + 2)
        lat = torch.from_numpy(lattice(seed, o, shape)).to(dev)
        amp = 2.0 ** -o
        acc += amp * _interp_octave(lat, period, zs, ys, xs, torch, dev)
        total += amp
    out = (acc / total).to(torch.float32)
    return out if device is not None else out.numpy()


def uniform_hash01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Counter-based uniform numbers in [0, 1): fmix32(fmix32(seed) ^ index)."""
    idx = np.arange(start, start + n, dtype=np.uint64)
    h = fmix32(fmix32(np.uint64(seed) ^ np.uint64(0x51ED27)) ^ (idx & M32))
    h = fmix32(h ^ (idx >> np.uint64(32)))
    return h.astype(np.float64) / 4294967296.0


def _mul32_t(h, c: int):
    """(h * c) mod 2^32 for int64 tensors h < 2^32, in 16-bit halves so that
    no product leaves the int64 range."""
    lo, hi = h & 0xFFFF, h >> 16
    return ((lo * c) + (((hi * c) & 0xFFFF) << 16)) & 0xFFFFFFFF


def fmix32_t(h):
    """fmix32 on an int64 torch tensor of 32-bit values (same results)."""
    h = h & 0xFFFFFFFF
    h = h ^ (h >> 16)
    h = _mul32_t(h, 0x85EBCA6B)
    h = h ^ (h >> 13)
    h = _mul32_t(h, 0xC2B2AE35)
    return h ^ (h >> 16)


def uniform_hash01_t(seed: int, n: int, start: int, device):
    """uniform_hash01 computed with torch on `device` (float32 results equal
    the numpy version's after .astype(np.float32))."""
    torch = _torch()
    idx = torch.arange(start, start + n, dtype=torch.int64, device=device)
    s0 = int(fmix32(np.uint64(seed) ^ np.uint64(0x51ED27)))
    h = fmix32_t((idx & 0xFFFFFFFF) ^ s0)
    h = fmix32_t(h ^ (idx >> 32))
    return (h.to(torch.float64) / 4294967296.0).to(torch.float32)


def gaussian_blobs(dims=(512, 512, 512), seed: int = 2, n: int = 200, noise: float = 0.1,
                   device=None, return_u8: bool = True):
    """Medium workload: sum of `n` axis-aligned anisotropic Gaussians (centre
    uniform in the volume, sigma_x,y,z ~ U[4, 40], amplitude ~ U[0.5, 1],
    each truncated at 4 sigma) plus noise*U[0,1) per voxel, divided by its
    maximum and quantised to u8 = round(255 v).  Returns the u8 volume (the
    renderer sees u8/255)."""
    torch = _torch()
    dev = torch.device(device or "cpu")
    Dx, Dy, Dz = dims
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(0, 1, size=(n, 3)) * (np.array([Dx, Dy, Dz]) - 1)
    sigmas = rng.uniform(4, 40, size=(n, 3))
    amps = rng.uniform(0.5, 1.0, size=n)
    vol = torch.zeros((Dz, Dy, Dx), dtype=torch.float32, device=dev)
    for c, s, a in zip(centres, sigmas, amps):
        lo = [max(0, int(math.floor(c[i] - 4 * s[i]))) for i in range(3)]
        hi = [min(dims[i], int(math.ceil(c[i] + 4 * s[i])) + 1) for i in range(3)]
        g = []
        for i in range(3):
            x = torch.arange(lo[i], hi[i], dtype=torch.float32, device=dev)
            g.append(torch.exp(-0.5 * ((x - float(c[i])) / float(s[i])) ** 2))
        vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += float(a) * (
            g[2].view(-1, 1, 1) * g[1].view(1, -1, 1) * g[0].view(1, 1, -1))
    # per-voxel noise, generated slab by slab from a counter-based hash
    plane = Dx * Dy
    if dev.type == "cuda":
        step = max(1, (1 << 24) // plane)
        for z in range(0, Dz, step):
            z1 = min(Dz, z + step)
            u = uniform_hash01_t(seed, plane * (z1 - z), z * plane, dev)
            vol[z:z1] += noise * u.view(z1 - z, Dy, Dx)
    else:
        for z in range(Dz):
            u = uniform_hash01(seed, plane, start=z * plane).astype(np.float32)
            vol[z] += noise * torch.from_numpy(u).to(dev).view(Dy, Dx)
    vol /= vol.max()
    u8 = torch.round(vol * 255.0).clamp_(0, 255).to(torch.uint8)
    if not return_u8:
        u8 = u8.to(torch.float32) / 255.0
    return u8 if device is not None else u8.numpy()


def mixing_layer_params(seed: int = 3, scale: float = 1.0):
    """Seeded parameters of the interface height h(x, y, z).  At scale 1 (the
    2048x2048x1920 volume) |h| <= 200 voxels, sinusoid wavelengths lie in
    [64, 1024] and the noise's coarsest period is 512; smaller test volumes
    shrink all lengths by `scale`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    amp = 200.0 * scale
    n_sin = 6
    lam = scale * np.exp(rng.uniform(math.log(64.0), math.log(1024.0), size=n_sin))
    theta = rng.uniform(0, 2 * math.pi, size=n_sin)
    phase = rng.uniform(0, 2 * math.pi, size=n_sin)
    w = rng.uniform(0.5, 1.0, size=n_sin)
    sin_amp = 0.6 * amp * w / w.sum()
    return dict(lam=lam, theta=theta, phase=phase, sin_amp=sin_amp, fbm_amp=0.4 * amp,
                amp=amp, octaves=6, base_period=max(4.0, 512.0 * scale), seed=seed)


def mixing_layer_slab(dims, z0: int, z1: int, params=None, z_mid: float = 960.0,
                      width: float = 4.0, device=None):
    """u8 density for z in [z0, z1) of the paper-scale mixing layer:
    rho = 0.5 (1 + tanh((z - z_mid - h(x,y,z)) / width)), u8 = round(255 rho),
    with h = 6 sinusoids in (x, y) plus 6-octave 3-D fractal value noise,
    |h| <= amp (200 at full scale).  Beyond amp + 15*width voxels from z_mid
    the density rounds to exactly 0 or 255, so those slabs are filled
    directly."""
    torch = _torch()
    dev = torch.device(device or "cpu")
    p = params or mixing_layer_params()
    Dx, Dy, Dz = dims
    nz = z1 - z0
    out = torch.empty((nz, Dy, Dx), dtype=torch.uint8, device=dev)
    reach = p["amp"] + 15.0 * width
    lo = int(math.floor(z_mid - reach)) - z0
    hi = int(math.ceil(z_mid + reach)) - z0
    zi = torch.arange(z0, z1, device=dev)
    out[zi < z_mid] = 0
    out[zi >= z_mid] = 255
    a, b = max(0, lo), min(nz, hi)
    if a >= b:
        return out
    xs = torch.arange(Dx, dtype=torch.float64, device=dev)
    ys = torch.arange(Dy, dtype=torch.float64, device=dev)
    zs = torch.arange(z0 + a, z0 + b, dtype=torch.float64, device=dev)
    h2 = torch.zeros((Dy, Dx), dtype=torch.float64, device=dev)
    for lam, th, ph, am in zip(p["lam"], p["theta"], p["phase"], p["sin_amp"]):
        kx, ky = math.cos(th) / lam, math.sin(th) / lam
        h2 += am * torch.sin(2 * math.pi * (kx * xs.view(1, -1) + ky * ys.view(-1, 1)) + ph)
    fbm = torch.zeros((b - a, Dy, Dx), dtype=torch.float64, device=dev)
    total = 0.0
    for o in range(p["octaves"]):
        period = p["base_period"] / 2 ** o
        zlo = int(math.floor((z0 + a) / period))
        shape = (int((z0 + b) / period) - zlo + 2, int(Dy / period) + 2, int(Dx / period) + 2)
        nzl, nyl, nxl = shape
        iz, iy, ix = np.meshgrid(np.arange(zlo, zlo + nzl), np.arange(nyl), np.arange(nxl),
                                 indexing="ij")
        lat = torch.from_numpy(hash_coords(p["seed"], o, ix, iy, iz).astype(np.float64)
                               / 4294967296.0).to(dev)
        amp_o = 2.0 ** -o
        fbm += amp_o * _interp_octave(lat, period, zs - zlo * period, ys, xs, torch, dev)
        total += amp_o
    h = h2.view(1, Dy, Dx) + p["fbm_amp"] * (2.0 * fbm / total - 1.0)
    rho = 0.5 * (1.0 + torch.tanh((zs.view(-1, 1, 1) - z_mid - h) / width))
    out[a:b] = torch.round(rho * 255.0).clamp_(0, 255).to(torch.uint8)
    return out


def mixing_layer(dims=(2048, 2048, 1920), device=None, slab: int = 64, seed: int = 3):
    """The whole paper-scale u8 volume (8 GB at full size)."""
    torch = _torch()
    dev = torch.device(device or "cpu")
    Dx, Dy, Dz = dims
    p = mixing_layer_params(seed, scale=Dz / 1920.0)
    z_mid = Dz / 2.0
    vol = torch.empty((Dz, Dy, Dx), dtype=torch.uint8, device=dev)
    for z0 in range(0, Dz, slab):
        z1 = min(Dz, z0 + slab)
        vol[z0:z1] = mixing_layer_slab(dims, z0, z1, p, z_mid=z_mid, device=dev)
    return vol if device is not None else vol.numpy()


def sphere(dims, centre, radius: float) -> np.ndarray:
    """float32, 1 at the centre falling linearly to 0 at 2 x radius: the
    level 0.5 is the sphere of the given radius.  Placed off-centre it gives
    a volume whose blocks of that level fill a small corner."""
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims[::-1]], indexing="ij")
    d = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    return np.clip(1.0 - d / (2.0 * radius), 0.0, 1.0).astype(np.float32)


def u8_to_f32(u8):
    """The value the renderer sees for an 8-bit voxel: (float)u / 255.0f."""
    if isinstance(u8, np.ndarray):
        return u8.astype(np.float32) / np.float32(255.0)
    return u8.to(_torch().float32) / 255.0
