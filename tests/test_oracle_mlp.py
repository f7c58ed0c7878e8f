"""Pins for the oracle MLP (no GPU): a forward pass worked out by hand on small
integer weights, backward by central differences, the identity at o = 0, and
Adam's first step in closed form."""
import numpy as np

from oracle import mlp


def rand_theta(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(mlp.NPARAM) * scale


def test_sizes():
    assert mlp.NPARAM == 8 * 64 + 64 + 64 * 64 + 64 + 64 * 4 + 4 == 4996


def test_zero_output_layer_gives_reference_weights():
    th = rand_theta(0)
    P = mlp.unpack(th)
    off = 8 * 64 + 64 + 64 * 64 + 64
    th[off:] = 0.0                      # W3 = 0, b3 = 0 -> o = 0
    F = np.random.default_rng(1).standard_normal((5, 8))
    ref = np.array([1.0039, 1.0404, 1.1486, 1.3827])
    beta, _ = mlp.forward(th, F, ref)
    assert np.allclose(beta, ref[None, :], atol=0, rtol=1e-15)
    del P


def test_forward_by_hand():
    """Two feature rows through weights that are zero except for a few small
    integers; the hidden activations and the outputs o below were worked out by
    hand (ReLU zeroes a1[1] of row 0 and a2[0] of row 1), and beta follows from
    tanh(m/2) = (e^m - 1)/(e^m + 1) for integer m."""
    W1, b1, W2, b2 = np.zeros((64, 8)), np.zeros(64), np.zeros((64, 64)), np.zeros(64)
    W3, b3 = np.zeros((4, 64)), np.zeros(4)
    W1[0, 0], W1[0, 1], b1[0] = 1, 1, -1       # row 0: 1 + 2 - 1 = 2
    W1[1, 2], b1[1] = -1, 1                    # row 0: -3 + 1 = -2 -> 0
    W1[2, 7], b1[2] = 2, 5                     # row 0: -2 + 5 = 3
    W2[0, 0], W2[0, 2], b2[0] = 1, -1, 2       # row 0: 2 - 3 + 2 = 1
    W2[1, 1], W2[1, 2], b2[1] = 7, 1, -1       # row 0: 0 + 3 - 1 = 2
    W2[3, 0] = -1                              # row 0: -2 -> 0
    W3[0, 0] = 1                               # o0 = h2[0]
    W3[1, 1], W3[1, 0] = 1, -2                 # o1 = h2[1] - 2 h2[0]
    W3[2, 1], b3[2] = -1, 1                    # o2 = 1 - h2[1]
    W3[3, 3], b3[3] = 5, 3                     # o3 = 5 h2[3] + 3
    th = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    assert th.size == mlp.NPARAM
    F = np.zeros((2, 8))
    F[0, :] = [1, 2, 3, 0, 0, 0, 0, -1]
    ref = np.array([1.0, 1.25, 1.5, 2.0])
    beta, (Fc, a1, h1, a2, h2, t, _) = mlp.forward(th, F, ref)
    # row 1 (all features 0): h1 = relu(b1) = (0, 1, 5); a2 = (-5 + 2, 7 + 5 - 1, 0, 0)
    assert np.array_equal(h1[:, :4], [[2, 0, 3, 0], [0, 1, 5, 0]])
    assert np.array_equal(h2[:, :4], [[1, 2, 0, 0], [0, 11, 0, 0]])
    assert not h1[:, 4:].any() and not h2[:, 4:].any()
    o = np.array([[1, 0, -1, 3], [0, 11, -10, 3]], dtype=np.float64)
    fac = np.exp(2.0 * (np.exp(o) - 1.0) / (np.exp(o) + 1.0))
    assert np.allclose(beta, ref * fac, rtol=1e-14, atol=0)
    # o = 0 leaves the weight unchanged; o = 1 multiplies it by exp(2 (e-1)/(e+1))
    assert beta[0, 1] == 1.25 and beta[1, 0] == 1.0
    assert abs(beta[0, 0] - np.exp(2 * (np.e - 1) / (np.e + 1))) <= 1e-15


def test_backward_central_differences():
    th = rand_theta(2)
    rng = np.random.default_rng(3)
    F = rng.standard_normal((6, 8))
    ref = np.array([1.0, 1.04, 1.15, 1.38])
    G = rng.standard_normal((6, 4))
    L = lambda t: float(np.sum(G * mlp.forward(t, F, ref)[0]))
    _, cache = mlp.forward(th, F, ref)
    g = mlp.backward(th, cache, G)
    h = 1e-6
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (L(th + e) - L(th - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_adam_first_step_closed_form():
    # with m = v = 0 the first bias-corrected step is lr * g / (|g| + eps)
    th = rand_theta(4)
    g = np.random.default_rng(5).standard_normal(mlp.NPARAM)
    new, m, v = mlp.adam(th, g, np.zeros_like(th), np.zeros_like(th), 1, 1e-3)
    assert np.allclose(new, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
