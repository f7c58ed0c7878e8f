"""One application of the polynomial-accelerated l1-Jacobi smoother (oracle).

Plain FP64 CSR code, natural row order, one library SpMV (scipy) per step and
no fusion.  Test infrastructure only.

Kinds (names follow Table 1 of Sec. 4):
  "l1jacobi"   k sweeps x <- x + M^{-1}(b - A x)                 (Eq. l1smooth)
  "cheb4"      4th-kind recurrence, rho(M^{-1}A) := rho          (Eq. polsmoother)
  "cheb4_opt"  same with x^(j) = x^(j-1) + beta_j z^(j)          (Eq. polsmootheropt)
  "weights"    as cheb4_opt with caller-supplied beta (learned weights)
  "cheb1_opt"  Algorithm 1 on [a_k*, 1] with rho(M^{-1}A) := 1
  "cheb1"      Algorithm 1 on [a_k*, 1] with rho := 1.1 * (10-step power estimate)

Degree convention: a degree-k application performs k products with A counting
the initial residual b - A x0 (absent when x0 = 0) and not counting a residual
update after the last step, whose result no later step reads.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import params

KINDS = ("l1jacobi", "cheb4", "cheb4_opt", "weights", "cheb1_opt", "cheb1")


def l1_diag(A):
    """M_i = a_ii + sum_{j != i} |a_ij|  (Eq. l1smooth)."""
    A = sp.csr_matrix(A)
    d = A.diagonal()
    absrow = np.asarray(abs(A).sum(axis=1)).ravel()
    return d + (absrow - np.abs(d))


def power_lambda(A, v0, iters=10, M=None):
    """Spectral estimate of M^{-1}A by ``iters`` power steps (the rho of kind
    CHEB1; Sec. 3 replaces rho(M^{-1}A) by 1 for the other kinds).

    v_0 = v0/||v0||_2; for i = 1..iters: w = M^{-1} A v_{i-1},
    lambda_i = ||w||_2, v_i = w / lambda_i.  Returns lambda_iters.  (The paper
    avoids eigen-estimates; the classic 1st-kind variant with
    rho = 1.1 * lambda is a configuration of this build.)"""
    M = l1_diag(A) if M is None else M
    v = np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = (A @ v) / M
        lam = np.linalg.norm(w)
        v = w / lam
    return lam


def cheb4(A, b, x0, k, beta=None, rho=1.0, M=None):
    """Eq. polsmoother (beta None: plain 4th kind, x^(j) = x^(j-1) + z^(j)) and
    Eq. polsmootheropt (x^(j) = x^(j-1) + beta_j z^(j), r still updated with
    the unweighted z^(j)):

        z^(0) = 0, r^(0) = b - A x^(0)
        z^(j) = (2j-3)/(2j+1) z^(j-1) + (8j-4)/(2j+1) (1/rho) M^{-1} r^(j-1)
        x^(j) = x^(j-1) + beta_j z^(j)
        r^(j) = r^(j-1) - A z^(j)
    """
    M = l1_diag(A) if M is None else M
    n = A.shape[0]
    if x0 is None:
        x = np.zeros(n)
        r = np.array(b, dtype=np.float64)
    else:
        x = np.array(x0, dtype=np.float64)
        r = b - A @ x
    z = np.zeros(n)
    for j in range(1, k + 1):
        z = (2 * j - 3) / (2 * j + 1) * z + (8 * j - 4) / (2 * j + 1) / rho * (r / M)
        bj = 1.0 if beta is None else beta[j - 1]
        x = x + bj * z
        if j < k:
            r = r - A @ z
    return x


def cheb1(A, b, x0, k, a, rho=1.0, M=None):
    """Algorithm 1 (ChebyshevAcceleration(A, b, x0, M, a, k)):

        r^(0) = (1/rho) M^{-1} (b - A x^(0)),  sigma_1 = theta/delta,
        rho_0 = 1/sigma_1,  d^(0) = r^(0)/theta,  x^(1) = x^(0) + d^(0)
        for j = 1..k-1:
            s^(j) = (1/rho) M^{-1} A d^(j-1)
            rho_j = (2 sigma_1 - rho_{j-1})^{-1}
            r^(j) = r^(j-1) - s^(j)
            d^(j) = rho_j rho_{j-1} d^(j-1) + (2 rho_j / delta) r^(j)
            x^(j+1) = x^(j) + d^(j)

    ``rho`` is rho(M^{-1}A) (1 for the l1-Jacobi reading of Sec. 3).
    theta, delta from Eq. optimal_parameters with interval [a, 1].
    """
    M = l1_diag(A) if M is None else M
    n = A.shape[0]
    theta, delta = params.theta_delta(a)
    if x0 is None:
        x = np.zeros(n)
        r = (np.asarray(b, dtype=np.float64) / M) / rho
    else:
        x = np.array(x0, dtype=np.float64)
        r = ((b - A @ x) / M) / rho
    sigma1 = theta / delta
    rho_prev = 1.0 / sigma1
    d = r / theta
    x = x + d
    for _ in range(1, k):
        s = ((A @ d) / M) / rho
        rho_j = 1.0 / (2.0 * sigma1 - rho_prev)
        r = r - s
        d = rho_j * rho_prev * d + (2.0 * rho_j / delta) * r
        x = x + d
        rho_prev = rho_j
    return x


def l1jacobi(A, b, x0, k, M=None):
    """k sweeps of x <- x + M^{-1}(b - A x)  (Sec. 2, Eq. l1smooth)."""
    M = l1_diag(A) if M is None else M
    x = np.zeros(A.shape[0]) if x0 is None else np.array(x0, dtype=np.float64)
    for _ in range(k):
        x = x + (b - A @ x) / M
    return x


class SmootherSpec:
    """Kind, degree and the scalars a kind needs on one level (the smoothers of
    Sec. 2.1-2.2 and the l1-Jacobi baseline of Eq. l1smooth)."""

    def __init__(self, kind, k, beta=None, rho=1.0, a=None):
        if kind not in KINDS:
            raise ValueError(kind)
        self.kind, self.k, self.rho = kind, int(k), float(rho)
        if kind == "cheb4_opt" and beta is None:
            beta = opt4_table(self.k)
        if kind == "weights" and beta is None:
            raise ValueError("kind 'weights' needs beta")
        self.beta = None if beta is None else np.asarray(beta, dtype=np.float64)
        if kind in ("cheb1", "cheb1_opt") and a is None:
            a = params.a_star(self.k)
        self.a = a


_OPT4_CACHE = {}


def opt4_table(k):
    """Cached optimal 4th-kind weights (Remez solution of Eq. prob1)."""
    if k not in _OPT4_CACHE:
        _OPT4_CACHE[k] = params.opt4_weights(k)
    return _OPT4_CACHE[k]


def smooth(A, b, x0, spec: SmootherSpec, M=None):
    """One smoother application (Eq. polsmoother, Eq. polsmootheropt,
    Algorithm 1 or Eq. l1smooth by kind): returns x after ``spec.k`` steps from x0
    (x0 None means the zero vector)."""
    kd = spec.kind
    if kd == "l1jacobi":
        return l1jacobi(A, b, x0, spec.k, M=M)
    if kd == "cheb4":
        return cheb4(A, b, x0, spec.k, None, spec.rho, M=M)
    if kd in ("cheb4_opt", "weights"):
        return cheb4(A, b, x0, spec.k, spec.beta, spec.rho, M=M)
    if kd in ("cheb1", "cheb1_opt"):
        return cheb1(A, b, x0, spec.k, spec.a, spec.rho, M=M)
    raise ValueError(kd)


def error_poly(spec: SmootherSpec, lam):
    """Closed-form error polynomial p(lambda) of one application, lambda an
    eigenvalue of M^{-1}A (Sec. 2.1-2.2)."""
    kd = spec.kind
    if kd == "l1jacobi":
        return params.p_jacobi(spec.k, lam)
    if kd == "cheb4":
        return params.p_cheb4(spec.k, np.asarray(lam) / spec.rho)
    if kd in ("cheb4_opt", "weights"):
        return params.p_opt4(spec.beta, np.asarray(lam) / spec.rho)
    return params.p_cheb1(spec.k, spec.a, lam, spec.rho)
