"""Seeded camera poses for the synthetic workloads.

A camera is four float32 triples: the eye and the pixel-grid basis
``p00, du, dv``; the ray of pixel (i, j) (j = 0 the bottom row) has direction
``(p00 + (i+0.5) du) + (j+0.5) dv``.  The basis is computed once in double
precision and rounded to float32, and the eye is snapped to a multiple of
1/256 voxel, so the same float32 values drive both the CUDA path and the
oracle.  The paper builds its initial rays by rasterising the volume's
bounding box (Sec. 3.2); these helpers only define the pinhole camera.
"""
from __future__ import annotations

import math

import numpy as np


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def snap_eye(eye) -> np.ndarray:
    e = np.round(np.asarray(eye, dtype=np.float64) * 256.0) / 256.0
    assert np.all(np.abs(e) < 32768.0)
    return e.astype(np.float32)


def look_at(eye, target, up, fovy_deg: float, W: int, H: int) -> dict:
    """Pinhole camera with vertical field of view fovy_deg."""
    e = snap_eye(eye)
    fwd = _unit(np.asarray(target, np.float64) - e.astype(np.float64))
    right = _unit(np.cross(fwd, np.asarray(up, np.float64)))
    upv = np.cross(right, fwd)
    half_h = math.tan(math.radians(fovy_deg) / 2.0)
    half_w = half_h * W / H
    p00 = fwd - right * half_w - upv * half_h
    du = right * (2.0 * half_w / W)
    dv = upv * (2.0 * half_h / H)
    return dict(eye=e, p00=p00.astype(np.float32), du=du.astype(np.float32),
                dv=dv.astype(np.float32))


def centre_and_diag(dims):
    d = np.asarray(dims, dtype=np.float64) - 1.0
    return d / 2.0, float(np.linalg.norm(d))


def orbit(dims, azimuth_deg: float, elevation_deg: float, radius_factor: float, W: int,
          H: int, fovy_deg: float = 45.0, up=(0.0, 0.0, 1.0)) -> dict:
    """A pose on an orbit around the volume centre, radius = factor x diagonal."""
    c, diag = centre_and_diag(dims)
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    u = np.asarray(up, np.float64)
    if abs(u[2]) > 0.5:
        dirv = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    else:
        dirv = np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])
    return look_at(c + radius_factor * diag * dirv, c, up, fovy_deg, W, H)


def random_pose(dims, seed: int, W: int, H: int, distance_factor: float = 2.0,
                fovy_deg: float = 45.0) -> dict:
    """Eye at centre + factor x diagonal along a seeded random direction."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    c, diag = centre_and_diag(dims)
    up = (0.0, 1.0, 0.0) if abs(v[1]) < 0.95 else (0.0, 0.0, 1.0)
    return look_at(c + distance_factor * diag * v, c, up, fovy_deg, W, H)


# the three measured workloads' poses
def small_pose(dims=(64, 64, 64), W: int = 256, H: int = 256) -> dict:
    return random_pose(dims, seed=4, W=W, H=H, distance_factor=2.0)


def medium_pose(i: int, dims=(512, 512, 512), W: int = 1280, H: int = 720) -> dict:
    return orbit(dims, azimuth_deg=22.5 * i, elevation_deg=20.0, radius_factor=1.5, W=W, H=H)


def paper_pose(dims=(2048, 2048, 1920), W: int = 1280, H: int = 720) -> dict:
    return orbit(dims, azimuth_deg=30.0, elevation_deg=20.0, radius_factor=1.4, W=W, H=H)
