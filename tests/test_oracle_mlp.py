"""Pins for the oracle MLP (no GPU): backward by central differences, the
identity at o = 0, and Adam's first step in closed form."""
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
