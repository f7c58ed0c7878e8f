"""Generate amgps_tables.h: the offline parameter tables of the smoothers.

Sec. 2 of the paper: the optimal polynomial parameters do not depend on the
matrix, so they are computed once and tabulated.  This script writes, for
degrees k = 1..16,

* a_k*        : the square of the root in (0,1) of Eq. optimalparameter,
                solved in 50-digit arithmetic;
* beta_{j,k}  : the weights of the optimised 4th-kind smoother
                (Eq. polsmootheropt), obtained by Newton's method on the
                equioscillation system of the minimax problem Eq. prob1 -- the
                route the paper attributes to Lottes: the functional
                x p^2/(1-p^2) equals gamma at x->0+ (p'(0) = -1/(2 gamma)),
                at k-1 interior maxima x_i (where its derivative vanishes) and
                at x = 1, with p(x_i) = (-1)^i sqrt(gamma/(x_i+gamma)).
                Unknowns: beta (k), gamma, x_1..x_{k-1}; Newton starts from
                the plain 4th-kind polynomial (beta = 1) and its maxima.

Run:  python paper_2407_09848_gb300/csrc/gen_tables.py   (needs mpmath)
The output is committed; the build does not run this script.
"""
import os
import sys

import mpmath as mp

KMAX = 16
mp.mp.dps = 50


def w_and_dw(k, t):
    """W_0..W_k at t and their t-derivatives, by the 4th-kind recurrence
    W_0 = 1, W_1 = 2t + 1, W_{j+1} = 2t W_j - W_{j-1}."""
    W = [mp.mpf(1), 2 * t + 1]
    D = [mp.mpf(0), mp.mpf(2)]
    for j in range(1, k):
        W.append(2 * t * W[j] - W[j - 1])
        D.append(2 * W[j] + 2 * t * D[j] - D[j - 1])
    return W, D


def p_and_dp(beta, x):
    """p(x) = sum_j (beta_j - beta_{j+1})/(2j+1) W_j(1-2x) and p'(x)."""
    k = len(beta)
    W, D = w_and_dw(k, 1 - 2 * x)
    b = [mp.mpf(1)] + list(beta) + [mp.mpf(0)]
    p = mp.mpf(0)
    dp = mp.mpf(0)
    for j in range(k + 1):
        c = (b[j] - b[j + 1]) / (2 * j + 1)
        p += c * W[j]
        dp += -2 * c * D[j]
    return p, dp


def equioscillation(k):
    def F(*v):
        beta, g = v[:k], v[k]
        xs = list(v[k + 1:]) + [mp.mpf(1)]
        _, dp0 = p_and_dp(beta, mp.mpf(0))
        out = [dp0 + 1 / (2 * g)]
        for i, x in enumerate(xs):
            s = (-1) ** (i + 1)
            p, dp = p_and_dp(beta, x)
            out.append(p - s * mp.sqrt(g / (x + g)))
            if i < k - 1:
                out.append(dp + s * mp.sqrt(g) / (2 * (x + g) ** mp.mpf(1.5)))
        return out
    return F


def plain_maxima(k):
    beta = [mp.mpf(1)] * k
    n = 4000
    xs = [mp.mpf(i) / n for i in range(1, n + 1)]
    fv = []
    for x in xs:
        p, _ = p_and_dp(beta, x)
        fv.append(x * p * p / (1 - p * p))
    return [xs[i] for i in range(1, n - 1) if fv[i] >= fv[i - 1] and fv[i] > fv[i + 1]]


def opt4(k):
    v0 = [mp.mpf(1)] * k + [mp.mpf(3) / (4 * k * (k + 1))] + plain_maxima(k)
    sol = mp.findroot(equioscillation(k), v0, solver="mdnewton",
                      tol=mp.mpf(10) ** -40, maxsteps=200)
    return [sol[j] for j in range(k)], sol[k]


def astar(k):
    phi = lambda x: 8 * k * (1 - x * x) ** (2 * k) + x * ((1 - x) ** (4 * k) - (1 + x) ** (4 * k))
    # phi(0) = 8k > 0 and phi(1) = -2^{4k} < 0 with a single sign change in
    # (0,1): plain bisection to far below double precision
    lo, hi = mp.mpf(0), mp.mpf(1)
    for _ in range(220):
        mid = (lo + hi) / 2
        if phi(mid) > 0:
            lo = mid
        else:
            hi = mid
    r = (lo + hi) / 2
    return r * r


def main(out_path):
    lines = ["/* Generated by gen_tables.py -- do not edit. */",
             "/* Offline smoother parameter tables, degrees 1..16 (see gen_tables.py). */",
             "#pragma once", "",
             f"#define AMGPS_TABLE_KMAX {KMAX}", "",
             "/* a_k* of Eq. optimalparameter, index k-1. */",
             "static const double AMGPS_ASTAR[AMGPS_TABLE_KMAX] = {"]
    for k in range(1, KMAX + 1):
        lines.append(f"  {mp.nstr(astar(k), 17, strip_zeros=False)},")
    lines += ["};", "",
              "/* beta_{j,k} of Eq. polsmootheropt: row k-1, entries j-1 (zero-padded). */",
              "/* gamma_k (Proposition 1) of each row in the trailing comment. */",
              "static const double AMGPS_OPT4_BETA[AMGPS_TABLE_KMAX][AMGPS_TABLE_KMAX] = {"]
    for k in range(1, KMAX + 1):
        beta, g = opt4(k)
        vals = [mp.nstr(b, 17, strip_zeros=False) for b in beta] + ["0.0"] * (KMAX - k)
        lines.append("  {" + ", ".join(vals) + "},  /* gamma = " + mp.nstr(g, 17) + " */")
    lines += ["};", ""]
    with open(out_path, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "amgps_tables.h"))
