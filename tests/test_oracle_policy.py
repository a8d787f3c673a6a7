"""Pins of the speculation-policy oracle (oracle/policy.py) against what the
definitions fix: bfloat16 rounding cases worked by hand, closed-form network
outputs, the gradient against central finite differences of the loss, the
count rule on hand-picked values, and labels from visible-block lists."""
import numpy as np
import pytest

from oracle import policy as P


def test_bf16_rounding_worked_cases():
    one = 1.0
    cases = {
        one: one,
        one + 2.0 ** -8: one,                        # halfway, ties to the even mantissa (1.0)
        one + 2.0 ** -7 + 2.0 ** -8: one + 2.0 ** -6,  # halfway, even neighbour above
        one + 2.0 ** -8 + 2.0 ** -10: one + 2.0 ** -7,  # above halfway: up
        -(one + 2.0 ** -9): -one,                    # below halfway: down (sign kept)
        3.0: 3.0,
        0.0: 0.0,
    }
    for x, want in cases.items():
        assert P.bf16(np.float32(x)) == want, x


def test_bf16_matches_torch_on_random_floats():
    torch = pytest.importorskip("torch")
    x = np.random.Generator(np.random.PCG64(3)).normal(size=4000).astype(np.float32) * 37.0
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(P.bf16(x), want)


def test_forward_zero_weights_is_the_output_bias():
    p = np.zeros(P.N_PARAMS)
    p[P.OFF_B3:] = [0.7, -1.25]
    X = np.random.Generator(np.random.PCG64(1)).normal(size=(5, P.N_IN))
    y = P.forward(p, X)
    assert np.array_equal(y, np.tile([0.7, -1.25], (5, 1)))


def test_forward_identity_network_sums_the_positive_features():
    W1 = np.zeros((P.N_HID, P.N_IN))
    W1[:P.N_IN, :] = np.eye(P.N_IN)
    W2 = np.eye(P.N_HID)
    W3 = np.zeros((P.N_OUT, P.N_HID))
    W3[0, :P.N_IN] = 1.0
    W3[1, :P.N_IN] = -2.0
    p = P.pack(W1, np.zeros(P.N_HID), W2, np.zeros(P.N_HID), W3, np.array([0.5, 0.0]))
    X = np.array([[1.0, -2.0, 3.0, 0, 0, 0, 0, 0, 0, 0, 0.25, -0.5]])
    y = P.forward(p, X)
    assert y[0, 0] == 0.5 + 1.0 + 3.0 + 0.25
    assert y[0, 1] == -2.0 * (1.0 + 3.0 + 0.25)


def test_gradient_matches_finite_differences():
    rng = np.random.Generator(np.random.PCG64(7))
    p = P.init_params(5)
    X = rng.uniform(-1, 1, size=(24, P.N_IN))
    labels = rng.integers(1, 80, size=24)
    tau = 0.8
    g = P.grad(p, X, labels, tau)
    h = 1e-6
    idx = np.concatenate([rng.integers(0, P.N_PARAMS, size=60),
                          [P.OFF_B1, P.OFF_B2 + 3, P.OFF_B3, P.OFF_B3 + 1, P.OFF_W3 + 70]])
    for i in idx:
        e = np.zeros(P.N_PARAMS)
        e[i] = h
        lp = sum(P.loss(p + e, X, labels, tau))
        lm = sum(P.loss(p - e, X, labels, tau))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_policy_k_rule():
    assert P.policy_k(2.5, 0.0, 32) == 6          # 2^2.5 = 5.66
    assert P.policy_k(2.5, -1.0, 32) == 3         # 2^1.5 = 2.83
    assert P.policy_k(-3.0, 0.0, 32) == 1         # clamped below at 1
    assert P.policy_k(9.3, 0.0, 64) == 32         # the learned count stops at 32
    assert P.policy_k(4.2, 0.3, 64) == 23         # 2^4.5 = 22.6
    assert P.policy_k(2.5, 0.0, 64, floor_k=10) == 10   # never below the paper's uniform count
    assert P.policy_k(2.5, 0.0, 8, floor_k=10) == 8     # the attempt's cap wins


def test_labels_from_visible_lists():
    pix = np.zeros(4, dtype=[("hit", "<i4"), ("hit_index", "<i4"), ("n_visible", "<i4")])
    pix["hit"] = [1, 0, 1, 0]
    pix["hit_index"] = [4, -1, 0, -1]
    pix["n_visible"] = [9, 7, 3, 0]
    lab = P.labels_from_pixels(pix, [0, 0, 1, 2, 3], [0, 2, 7, 0, 0])
    assert lab.tolist() == [5, 3, 1, 1, 1]
