"""Reverse-mode derivatives of the smoother and of the V-cycle (oracle, FP64).

Test infrastructure only.  Each backward pass below differentiates the forward
recurrence of oracle.smoother line by line, in reverse order (plain
reverse-mode differentiation, storing the forward iterates), so it is
independent of the product's adjoint, which instead uses the symmetry of the
smoother operator.  No passage of the paper defines these derivatives; they
serve the learned-weight training of this build.

One smoother application is x = S(b, x0; beta).  Given gx = dL/dx the
functions return dL/db, dL/dx0 and (4th-kind family) dL/dbeta.
"""
from __future__ import annotations

import numpy as np

from . import params
from .smoother import SmootherSpec, l1_diag, smooth


def _cheb4_backward(A, b, x0, k, beta, rho, M, gx):
    """Eq. polsmoother / polsmootheropt, reversed.

    forward: r = b - A x0; z = 0; x = x0
             j = 1..k: z = a_j z + c_j M^{-1} r ; x = x + beta_j z ; (j<k) r = r - A z
    """
    n = A.shape[0]
    x0v = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64)
    a = [(2 * j - 3) / (2 * j + 1) for j in range(1, k + 1)]
    c = [(8 * j - 4) / (2 * j + 1) / rho for j in range(1, k + 1)]
    bet = np.ones(k) if beta is None else np.asarray(beta, dtype=np.float64)
    # forward, storing z_j
    r = b - A @ x0v
    z = np.zeros(n)
    zs = []
    for j in range(k):
        z = a[j] * z + c[j] * (r / M)
        zs.append(z)
        if j < k - 1:
            r = r - A @ z
    # reverse
    xbar = np.asarray(gx, dtype=np.float64)
    zbar = np.zeros(n)
    rbar = np.zeros(n)
    gbeta = np.zeros(k)
    for j in range(k - 1, -1, -1):
        if j < k - 1:            # r_j = r_{j-1} - A z_j
            zbar = zbar - A @ rbar
        gbeta[j] = xbar @ zs[j]  # x = x + beta_j z_j
        zbar = zbar + bet[j] * xbar
        rbar = rbar + c[j] * (zbar / M)   # z_j = a_j z_{j-1} + c_j M^{-1} r_{j-1}
        zbar = a[j] * zbar
    gb = rbar.copy()             # r_0 = b - A x0
    gx0 = xbar - A @ rbar
    return gb, gx0, gbeta


def _cheb1_backward(A, b, x0, k, a_int, rho, M, gx):
    """Algorithm 1, reversed (see oracle.smoother.cheb1 for the forward)."""
    n = A.shape[0]
    theta, delta = params.theta_delta(a_int)
    sigma1 = theta / delta
    rhos = [1.0 / sigma1]
    for _ in range(1, k):
        rhos.append(1.0 / (2.0 * sigma1 - rhos[-1]))
    # forward is not needed: every step is linear with fixed coefficients
    xbar = np.asarray(gx, dtype=np.float64)
    dbar = np.zeros(n)
    rbar = np.zeros(n)
    for j in range(k - 1, 0, -1):
        dbar = dbar + xbar                        # x^{j+1} = x^j + d^j
        c1, c2 = rhos[j] * rhos[j - 1], 2.0 * rhos[j] / delta
        rbar = rbar + c2 * dbar                   # d^j = c1 d^{j-1} + c2 r^j
        dprev = c1 * dbar
        sbar = -rbar                              # r^j = r^{j-1} - s^j
        dprev = dprev + (A @ ((sbar / M) / rho))  # s^j = (1/rho) M^{-1} A d^{j-1}
        dbar = dprev
    dbar = dbar + xbar                            # x^1 = x^0 + d^0
    rbar = rbar + dbar / theta                    # d^0 = r^0 / theta
    gb = (rbar / M) / rho                         # r^0 = (1/rho) M^{-1}(b - A x^0)
    gx0 = xbar - A @ gb
    return gb, gx0, None


def _jacobi_backward(A, b, x0, k, M, gx):
    xbar = np.asarray(gx, dtype=np.float64)
    gb = np.zeros(A.shape[0])
    for _ in range(k):                            # x <- x + M^{-1}(b - A x)
        t = xbar / M
        gb = gb + t
        xbar = xbar - A @ t
    return gb, xbar, None


def smooth_backward(A, b, x0, spec: SmootherSpec, gx, M=None):
    """(dL/db, dL/dx0, dL/dbeta or None) of one application x = S(b, x0) of the
    smoothers of Sec. 2.1-2.2 (Eq. polsmoother, Eq. polsmootheropt, Algorithm 1)."""
    M = l1_diag(A) if M is None else M
    kd = spec.kind
    if kd == "l1jacobi":
        return _jacobi_backward(A, b, x0, spec.k, M, gx)
    if kd in ("cheb1", "cheb1_opt"):
        return _cheb1_backward(A, b, x0, spec.k, spec.a, spec.rho, M, gx)
    beta = None if kd == "cheb4" else spec.beta
    return _cheb4_backward(A, b, x0, spec.k, beta, spec.rho, M, gx)


def vcycle_backward(amg, b, gx, level=0):
    """Reverse pass of OracleAMG.vcycle (Eq. amg): returns dL/db and a list of
    dL/dbeta per level (None for kinds without weights)."""
    nl = amg.n_levels
    gbeta = [None] * (nl - 1)

    def rec(l, bl, xbar):
        if l == nl - 1:
            y = amg.coarse_solve(xbar)            # the coarse operator is symmetric
            return y
        A, P, spec, M = amg.A[l], amg.P[l], amg.specs[l], amg.M[l]
        # forward (recomputed): pre, residual, restriction, coarse, prolongation
        x1 = smooth(A, bl, None, spec, M=M)
        res = bl - A @ x1
        bc = P.T @ res
        xc = amg.vcycle(bc, l + 1)
        x2 = x1 + P @ xc
        # reverse
        gb_post, gx2, gbt_post = smooth_backward(A, bl, x2, spec, xbar, M=M)
        gx1 = gx2.copy()
        gxc = P.T @ gx2
        gbc = rec(l + 1, bc, gxc)
        gres = P @ gbc
        gb = gb_post + gres
        gx1 = gx1 - A @ gres
        gb_pre, _, gbt_pre = smooth_backward(A, bl, None, spec, gx1, M=M)
        gb = gb + gb_pre
        if gbt_post is not None:
            g = gbt_post + gbt_pre
            gbeta[l] = g if gbeta[l] is None else gbeta[l] + g
        return gb

    gb = rec(level, np.asarray(b, dtype=np.float64), np.asarray(gx, dtype=np.float64))
    return gb, gbeta


def error_reduction_loss(amg, E0):
    """Mean over the columns e0 of E0 of ||E e0||_A^2 / ||e0||_A^2 with
    E = I - B A (one V-cycle of Eq. amg), and its gradient with respect to every
    level's weights (the loss has no counterpart in the paper; it drives the
    learned weights).  Returns (loss, [dL/dbeta_l])."""
    A = amg.A[0]
    m = E0.shape[1]
    loss = 0.0
    gsum = None
    for i in range(m):
        e0 = E0[:, i]
        Ae0 = A @ e0
        den = e0 @ Ae0
        z = amg.vcycle(Ae0)
        e1 = e0 - z
        Ae1 = A @ e1
        loss += (e1 @ Ae1) / den / m
        gz = -2.0 * Ae1 / den / m                 # dL/dz
        _, gb = vcycle_backward(amg, Ae0, gz)
        if gsum is None:
            gsum = [None if g is None else g.copy() for g in gb]
        else:
            gsum = [None if g is None else s + g for s, g in zip(gsum, gb)]
    return loss, gsum
