"""Polynomial parameters of the smoothers (oracle side, FP64, test infrastructure).

Sec. 2.1-2.3 of the paper.  Nothing here touches a matrix: these are the
scalar families p_k(lambda), the convergence functional of Proposition 1 and the
offline parameter tables a_k* and beta_{j,k}.
"""
from __future__ import annotations

import math
import numpy as np
from scipy.optimize import brentq, minimize_scalar

# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------


def W4(j, t):
    """4th-kind Chebyshev polynomial W_j(t), t = cos(theta), Sec. 2.1.

    Defined here as sin((j+1/2) theta) / sin(theta/2).  The paper prints
    cos/cos, which is the 3rd-kind polynomial; only sin/sin reproduces the
    recurrence of Eq. polsmoother and the bound of Eq. lottebound-4cheby
    (reading recorded with the design notes).  W_j(1) = 2j+1 (limit theta->0).
    """
    t = np.asarray(t, dtype=np.float64)
    th = np.arccos(np.clip(t, -1.0, 1.0))
    out = np.empty_like(th)
    small = th < 1e-7
    big = ~small
    out[big] = np.sin((j + 0.5) * th[big]) / np.sin(0.5 * th[big])
    # series of sin((j+1/2)th)/sin(th/2) about th=0: (2j+1)(1 - j(j+1) th^2/6)
    ths = th[small]
    out[small] = (2 * j + 1) * (1.0 - j * (j + 1) * ths * ths / 6.0)
    return out


def W4_deriv_at_one(j):
    """W_j'(1) = j(j+1)(2j+1)/3 (differentiate the series above in t=cos th:
    dt = -th dth near th=0)."""
    return j * (j + 1) * (2 * j + 1) / 3.0


def T1(k, y):
    """1st-kind Chebyshev polynomial tau_k(y) of Sec. 2.2 for real y, from
    identity (i): cos(k arccos y) on [-1,1], cosh(k arccosh |y|) with sign
    (+1 or (-1)^k) outside."""
    y = np.asarray(y, dtype=np.float64)
    out = np.empty_like(y)
    inside = np.abs(y) <= 1.0
    out[inside] = np.cos(k * np.arccos(y[inside]))
    pos = y > 1.0
    out[pos] = np.cosh(k * np.arccosh(y[pos]))
    neg = y < -1.0
    out[neg] = (-1.0) ** k * np.cosh(k * np.arccosh(-y[neg]))
    return out


def theta_delta(a):
    """Eq. optimal_parameters: theta = (1+a)/2, delta = (1-a)/2."""
    return 0.5 * (1.0 + a), 0.5 * (1.0 - a)


def tau_scaled(k, a, x):
    """tau_k^{[a,1]}(x) = tau_k((theta - x)/delta) / tau_k(theta/delta),
    Sec. 2.2 (the map of [a,b] onto [-1,1] with b=1, normalised at 0)."""
    th, de = theta_delta(a)
    x = np.asarray(x, dtype=np.float64)
    return T1(k, (th - x) / de) / T1(k, np.array([th / de]))[0]


def p_cheb4(k, lam):
    """Error polynomial of the 4th-kind smoother (Eq. polsmoother, rho=1):
    p_k(lambda) = W_k(1 - 2 lambda) / (2k+1)."""
    return W4(k, 1.0 - 2.0 * np.asarray(lam, dtype=np.float64)) / (2 * k + 1)


def p_opt4(beta, lam):
    """Error polynomial of the optimised-weight smoother (Eq. polsmootheropt):
    p_k(x) = sum_{j=0}^{k} (beta_j - beta_{j+1})/(2j+1) W_j(1-2x),
    beta_0 = 1, beta_{k+1} = 0 (Sec. 2.1)."""
    k = len(beta)
    b = np.concatenate([[1.0], np.asarray(beta, dtype=np.float64), [0.0]])
    t = 1.0 - 2.0 * np.asarray(lam, dtype=np.float64)
    out = np.zeros_like(t)
    for j in range(k + 1):
        out = out + (b[j] - b[j + 1]) / (2 * j + 1) * W4(j, t)
    return out


def p_cheb1(k, a, lam, rho=1.0):
    """Error polynomial of Algorithm 1 / Eq. polsmootheropt1kind:
    e^(k) = tau_k^{[a,1]}(lambda / rho) e^(0)."""
    return tau_scaled(k, a, np.asarray(lam, dtype=np.float64) / rho)


def p_jacobi(k, lam):
    """k plain l1-Jacobi sweeps: (1 - lambda)^k (Sec. 2, G = I - M^{-1}A)."""
    return (1.0 - np.asarray(lam, dtype=np.float64)) ** k


# ---------------------------------------------------------------------------
# The functional of Proposition 1
# ---------------------------------------------------------------------------


def f_objective(p, x):
    """x p(x)^2 / (1 - p(x)^2), the quantity whose sup over (0,1] is gamma
    (Proposition 1, Eq. prob1)."""
    return x * p * p / (1.0 - p * p)


def gamma_sup(pfun, pprime0, n_grid=200001):
    """gamma = sup_{0<x<=1} x p^2/(1-p^2) (Proposition 1).

    The limit at x -> 0+ equals 1/(2|p'(0)|) because p(0)=1 (Sec. 2.3); the
    remaining sup is taken on a dense grid and each grid maximum is refined by
    a bounded scalar maximisation."""
    # below x ~ 1e-4 the quotient loses digits to cancellation in 1 - p^2;
    # the limit there is taken analytically
    xs = np.concatenate([np.logspace(-4, -3, 300, endpoint=False),
                         np.linspace(1e-3, 1.0, n_grid)])
    f = f_objective(pfun(xs), xs)
    best = 1.0 / (2.0 * abs(pprime0))
    loc = np.where((f[1:-1] >= f[:-2]) & (f[1:-1] >= f[2:]))[0] + 1
    for i in loc:
        lo, hi = xs[i - 1], xs[i + 1]
        r = minimize_scalar(lambda x: -f_objective(pfun(np.array([x])), np.array([x]))[0],
                            bounds=(lo, hi), method="bounded",
                            options={"xatol": 1e-15})
        best = max(best, -r.fun, f[i])
    best = max(best, f[-1])
    return best


# ---------------------------------------------------------------------------
# Optimal 1st-kind interval endpoint a_k* (Sec. 2.3)
# ---------------------------------------------------------------------------


def phi_astar(k, x):
    """Left side of Eq. optimalparameter:
    8k(1-x^2)^{2k} + x[(1-x)^{4k} - (1+x)^{4k}]; its root in (0,1) is sqrt(a_k*)."""
    return 8 * k * (1 - x * x) ** (2 * k) + x * ((1 - x) ** (4 * k) - (1 + x) ** (4 * k))


def a_star(k):
    """a_k* = (root in (0,1) of Eq. optimalparameter)^2, found with Brent's
    method (the paper uses MATLAB's fzero, i.e. Brent's algorithm)."""
    r = brentq(lambda x: phi_astar(k, x), 1e-12, 1.0 - 1e-12, xtol=1e-300,
               rtol=4 * np.finfo(float).eps, maxiter=500)
    return r * r


def inv_two_c1(a, k):
    """1/(2|c_1^{(a,k)}|) from the binomial sums that close the derivation of
    Eq. c1 (Sec. 2.3).  Equals the sup of the Proposition 1 functional of
    tau_k^{[a,1]} on (0,a] (Lemma 1)."""
    num = sum(math.comb(2 * k, 2 * j) * a ** j for j in range(k + 1))
    den = 2 * k * sum(math.comb(2 * k, 2 * j + 1) * a ** j for j in range(k))
    return num / den


def value_at_one(a, k):
    """tau(1)^2/(1 - tau(1)^2) for tau = tau_k^{[a,1]} in the closed form of
    Sec. 2.3: 4 / ([q^k + q^{-k}]^2 - 4), q = (1+sqrt a)/(1-sqrt a)."""
    s = math.sqrt(a)
    q = (1 + s) / (1 - s)
    return 4.0 / ((q ** k + q ** (-k)) ** 2 - 4.0)


def cheb1_coeffs(a, k):
    """theta, delta and the scalars rho_0..rho_{k-1} of Algorithm 1:
    sigma_1 = theta/delta, rho_0 = 1/sigma_1, rho_j = (2 sigma_1 - rho_{j-1})^{-1}."""
    th, de = theta_delta(a)
    s1 = th / de
    rhos = [1.0 / s1]
    for _ in range(1, k):
        rhos.append(1.0 / (2.0 * s1 - rhos[-1]))
    return th, de, s1, rhos


# ---------------------------------------------------------------------------
# Optimal 4th-kind weights beta_{j,k} (minimax problem Eq. prob1)
# ---------------------------------------------------------------------------


def _phi_basis(k, x):
    """p_beta(x) = 1 + sum_j beta_j phi_j(x) with
    phi_j = W_j(1-2x)/(2j+1) - W_{j-1}(1-2x)/(2j-1): regroup the expansion of
    Eq. polsmootheropt by beta_j.  Returns the (len(x), k) matrix."""
    t = 1.0 - 2.0 * np.asarray(x, dtype=np.float64)
    cols = []
    for j in range(1, k + 1):
        cols.append(W4(j, t) / (2 * j + 1) - W4(j - 1, t) / (2 * j - 1))
    return np.stack(cols, axis=-1)


def _phi_basis_d0(k):
    """phi_j'(0) = -2 [W_j'(1)/(2j+1) - W_{j-1}'(1)/(2j-1)]."""
    return np.array([-2.0 * (W4_deriv_at_one(j) / (2 * j + 1)
                             - W4_deriv_at_one(j - 1) / (2 * j - 1))
                     for j in range(1, k + 1)])


def opt4_pprime0(beta):
    return float(_phi_basis_d0(len(beta)) @ np.asarray(beta, dtype=np.float64))


def opt4_weights(k, maxit=200, tol=1e-15, return_gamma=False):
    """beta_{1..k,k} minimising gamma(beta) = sup_{(0,1]} x p^2/(1-p^2) over
    the 4th-kind expansion of Eq. polsmootheropt (problem Eq. prob1).

    The paper takes these weights from Lottes' alternating minimisation, which
    it does not print.  This oracle solves the same minimax problem with a
    Remez exchange written from the equioscillation characterisation: at the
    optimum, x p^2/(1-p^2) reaches gamma at x->0+ (i.e. p'(0) = -1/(2 gamma)),
    at k-1 interior points and at x=1, where p alternates in sign:
    p(x_i) = (-1)^i sqrt(gamma/(x_i+gamma)).  Each exchange step solves that
    system for (beta, gamma) on the current reference and moves the reference
    to the new local maxima.  Start: the extrema of the plain 4th-kind
    polynomial (beta = 1).
    """
    if k == 1:
        ref = np.array([1.0])
    else:
        beta0 = np.ones(k)
        ref = _interior_maxima(beta0, k)
    d0 = _phi_basis_d0(k)
    signs = np.array([(-1.0) ** (i + 1) for i in range(k)])
    beta = None
    gam = None
    for _ in range(maxit):
        Phi = _phi_basis(k, ref)

        def beta_of(g):
            w = np.sqrt(g / (ref + g))
            return np.linalg.solve(Phi, signs * w - 1.0)

        def h(g):
            return d0 @ beta_of(g) + 1.0 / (2.0 * g)

        gs = np.logspace(-6, 0.5, 400)
        hv = np.array([h(g) for g in gs])
        # bracket the sign change nearest to the previous gamma (or the first)
        idx = np.where(np.sign(hv[:-1]) != np.sign(hv[1:]))[0]
        if len(idx) == 0:
            raise RuntimeError("Remez: no root for gamma")
        if gam is None:
            i = idx[0]
        else:
            i = idx[np.argmin(np.abs(gs[idx] - gam))]
        g_new = brentq(h, gs[i], gs[i + 1], xtol=1e-300, rtol=4 * np.finfo(float).eps)
        beta = beta_of(g_new)
        new_ref = _interior_maxima(beta, k) if k > 1 else np.array([1.0])
        moved = np.max(np.abs(new_ref - ref))
        ref = new_ref
        done = gam is not None and abs(g_new - gam) <= tol * g_new and moved < 1e-13
        gam = g_new
        if done:
            break
    if return_gamma:
        return beta, gam
    return beta


def _interior_maxima(beta, k):
    """The k-1 interior local maxima of x p^2/(1-p^2) plus the endpoint x=1:
    located on a grid, each refined by a bounded scalar maximisation."""
    xs = np.linspace(1e-4, 1.0, 20001)
    p = 1.0 + _phi_basis(k, xs) @ beta
    f = f_objective(p, xs)
    loc = np.where((f[1:-1] >= f[:-2]) & (f[1:-1] > f[2:]))[0] + 1
    if len(loc) > k - 1:
        loc = np.sort(loc[np.argsort(f[loc])[::-1][: k - 1]])
    if len(loc) < k - 1:
        raise RuntimeError("Remez: lost a reference point")
    pts = []
    for i in loc:
        fun = lambda x: -f_objective(1.0 + _phi_basis(k, np.array([x])) @ beta,
                                     np.array([x]))[0]
        r = minimize_scalar(fun, bounds=(xs[i - 1], xs[i + 1]), method="bounded",
                            options={"xatol": 1e-15})
        pts.append(r.x)
    return np.array(sorted(pts) + [1.0])


def gamma_opt4(beta):
    """gamma of the optimised 4th-kind polynomial with weights ``beta``: the
    objective of Eq. prob1 (Sec. 2.1)."""
    return gamma_sup(lambda x: p_opt4(beta, x), opt4_pprime0(beta))
