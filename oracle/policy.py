"""Oracle of the speculation policy (the per-ray speculation count that the
paper leaves to future work, Sec. 6).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain numpy in
double precision, written from the definitions, never imported by the
product library.

* ``forward``: the perceptron 12 -> 64 -> 64 -> 2 with ReLU hidden layers,
  y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, parameters in the row-major
  [out][in] layout of the C ABI.  With ``bf16=True`` the weights, the inputs
  and the hidden activations are rounded to bfloat16 (round to nearest,
  ties to even) as the tensor-core inference stores them; the sums stay in
  double precision.
* ``loss`` / ``grad``: the training loss per sample with t = log2(min(label,
  64)), (y0 - t)^2 + pinball_tau(t - y1), averaged over the samples, and its
  gradient by the chain rule through the layers.
* ``policy_k``: the count max(min(ceil(2^(y1 + margin)), 32), floor_k)
  clamped to cap, where floor_k is the paper's uniform count for the pass.
* ``labels_from_pixels``: the visible blocks a ray still needs after taking
  ``consumed`` of them: up to and including its hit block (the hit's index in
  the ray's visible-block list + 1), or every visible block of a miss.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 12, 64, 2
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_HID * N_IN
OFF_W2 = OFF_B1 + N_HID
OFF_B2 = OFF_W2 + N_HID * N_HID
OFF_W3 = OFF_B2 + N_HID
OFF_B3 = OFF_W3 + N_OUT * N_HID
N_PARAMS = OFF_B3 + N_OUT   # 5122


def unpack(params):
    p = np.asarray(params, dtype=np.float64).reshape(-1)
    assert p.size == N_PARAMS
    W1 = p[OFF_W1:OFF_B1].reshape(N_HID, N_IN)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(N_HID, N_HID)
    b2 = p[OFF_B2:OFF_W3]
    W3 = p[OFF_W3:OFF_B3].reshape(N_OUT, N_HID)
    b3 = p[OFF_B3:]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, np.ravel(W3), b3]).astype(np.float64)


def bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float64: keep the top 16 bits of the float32 pattern after adding
    0x7FFF plus the lowest kept bit."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, X, bf16_round: bool = False, hidden: bool = False):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    if bf16_round:
        W1, W2, W3 = bf16(W1), bf16(W2), bf16(W3)
        X = bf16(X.astype(np.float32))
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    if bf16_round:
        h1 = bf16(h1.astype(np.float32))
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    if bf16_round:
        h2 = bf16(h2.astype(np.float32))
    y = h2 @ W3.T + b3
    if hidden:
        return y, (X, z1, h1, z2, h2)
    return y


def targets(labels):
    lab = np.clip(np.asarray(labels, dtype=np.float64), 1, 64)
    return np.log2(lab)


def loss(params, X, labels, tau: float):
    y = forward(params, X)
    t = targets(labels)
    e0 = y[:, 0] - t
    e1 = t - y[:, 1]
    return float(np.mean(e0 * e0)), float(np.mean(np.maximum(tau * e1, (tau - 1.0) * e1)))


def grad(params, X, labels, tau: float):
    """Gradient of the mean of both loss terms."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    y, (Xd, z1, h1, z2, h2) = forward(params, X, hidden=True)
    n = Xd.shape[0]
    t = targets(labels)
    dy = np.zeros_like(y)
    dy[:, 0] = 2.0 * (y[:, 0] - t) / n
    e1 = t - y[:, 1]
    dy[:, 1] = np.where(e1 > 0, -tau, 1.0 - tau) / n
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ Xd
    gb1 = dz1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def policy_k(y1, margin: float, cap: int, floor_k: int = 1):
    z = np.clip(np.asarray(y1, dtype=np.float64) + margin, -1.0, 12.0)
    k = np.clip(np.ceil(np.exp2(z)), 1, 32)
    return np.minimum(np.maximum(k, floor_k), cap).astype(np.int64)


def labels_from_pixels(pix, rays, consumed):
    """pix: the PIXEL_DTYPE array of ``oracle.render`` over all pixels."""
    rays = np.asarray(rays, dtype=np.int64)
    need = np.where(pix["hit"][rays] == 1, pix["hit_index"][rays] + 1, pix["n_visible"][rays])
    lab = need - np.asarray(consumed, dtype=np.int64)
    return np.maximum(lab, 1)


def init_params(seed: int = 0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_out, fan_in in ((N_HID, N_IN), (N_HID, N_HID), (N_OUT, N_HID)):
        bound = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, size=(fan_out, fan_in)))
        parts.append(rng.uniform(-bound, bound, size=fan_out))
    return pack(*parts)
