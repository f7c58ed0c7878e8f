"""FP64 reference of the weight-predicting MLP (test infrastructure only).

Not in the paper: the learned part of this build maps 8 features of an AMG
level to the k = 4 weights of Eq. polsmootheropt,

    h1 = relu(W1 f + b1)      (64)
    h2 = relu(W2 h1 + b2)     (64)
    o  = W3 h2 + b3           (4)
    beta = beta_ref * exp(2 * tanh(o / 2))

with beta_ref the optimal 4th-kind weights, so o = 0 reproduces them; the
factor exp(2 tanh(o/2)) has slope 1 at o = 0 and spans (e^-2, e^2), far wider
than any weight of a safe polynomial needs, so training is not held at a
bound of the parametrisation.  The
parameter vector is [W1 (64x8 row-major), b1, W2 (64x64), b2, W3 (4x64), b3]:
4996 numbers.  Adam is the textbook update with bias correction.
"""
from __future__ import annotations

import numpy as np

NF, NH, NO = 8, 64, 4
SIZES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NO, NH)),
         ("b3", (NO,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, off = {}, 0
    for name, shape in SIZES:
        m = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + m], dtype=np.float64).reshape(shape)
        off += m
    return out


def forward(theta, F, beta_ref):
    """F: (B, 8) features.  Returns beta (B, 4) and the cache for backward (no
    counterpart in the paper)."""
    P = unpack(theta)
    a1 = F @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    o = h2 @ P["W3"].T + P["b3"]
    t = np.tanh(0.5 * o)
    beta = np.asarray(beta_ref) * np.exp(2.0 * t)
    return beta, (F, a1, h1, a2, h2, t, beta)


def backward(theta, cache, gbeta):
    """dL/dtheta given dL/dbeta (B, 4), by the chain rule through the layers (no
    counterpart in the paper)."""
    P = unpack(theta)
    F, a1, h1, a2, h2, t, beta = cache
    go = gbeta * beta * (1.0 - t * t)                # d beta / d o = beta (1 - t^2)
    gW3 = go.T @ h2
    gb3 = go.sum(axis=0)
    gh2 = go @ P["W3"]
    ga2 = gh2 * (a2 > 0)
    gW2 = ga2.T @ h1
    gb2 = ga2.sum(axis=0)
    gh1 = ga2 @ P["W2"]
    ga1 = gh1 * (a1 > 0)
    gW1 = ga1.T @ F
    gb1 = ga1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def adam(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One textbook Adam step (step counts from 1).  Returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
