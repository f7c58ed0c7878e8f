"""Pins for the oracle's scalar parameter code (no GPU).

Everything is compared with values the paper prints (tests/golden) or with
closed forms / textbook definitions that are independent of the code under test.
"""
import math

import numpy as np
import pytest

from conftest import load_constants
from oracle import params as P

ROWS = load_constants()


def printed_tol(v):
    """Half a unit in the last printed digit (15-16 significant digits)."""
    s = repr(v)
    digits = s.replace("0.", "").lstrip("0").replace(".", "")
    nsig = len(digits.split("e")[0])
    e = math.floor(math.log10(abs(v)))
    # plus a few units of double rounding on the computed side
    return 0.5 * 10.0 ** (e - nsig + 1) + 4e-15 * abs(v)


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"k{r[0]}")
def test_a_star_matches_printed(row):
    k, a_pr = row[0], row[1]
    # the printed roots come from the paper's own fzero run, whose stopping
    # tolerance leaves about one unit of error in the 15th digit
    assert abs(P.a_star(k) - a_pr) <= max(printed_tol(a_pr), 1e-14 * a_pr)


def test_a_star_k1_closed_form():
    # Eq. optimalparameter with k=1 reduces to 8 - 24 x^2 = 0
    assert abs(P.a_star(1) - 1.0 / 3.0) < 4e-16


@pytest.mark.parametrize("k", range(3, 16))
def test_theorem1_brackets(k):
    a = P.a_star(k)
    assert math.log(k) ** 2 / (9 * k * k) <= a <= math.log(k) ** 2 / (k * k)
    lam = P.inv_two_c1(a, k)
    assert math.log(k) / (6 * k * k) <= lam <= 1.03 * math.log(k) / (2 * k * k)


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"k{r[0]}")
def test_gamma_cheb1_opt(row):
    k, g_pr = row[0], row[3]
    a = P.a_star(k)
    g = P.inv_two_c1(a, k)
    assert abs(g - g_pr) <= printed_tol(g_pr)
    # a_k* balances the two branches of Eq. max2
    assert abs(P.value_at_one(a, k) - g) <= 1e-13 * g
    # and the sup of the Proposition 1 functional of the closed-form
    # tau_k^{[a*,1]} (built from T_k, not from the binomial sums) agrees
    tprime0 = (P.tau_scaled(k, a, np.array([1e-7])) - P.tau_scaled(k, a, np.array([-1e-7])))[0] / 2e-7
    gs = P.gamma_sup(lambda x: P.tau_scaled(k, a, x), tprime0)
    assert abs(gs - g_pr) <= 1e-8 * g_pr


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"k{r[0]}")
def test_gamma_cheb4(row):
    k, g_pr = row[0], row[2]
    # Eq. lottebound-4cheby: gamma = 3/(4k(k+1))
    assert abs(3.0 / (4 * k * (k + 1)) - g_pr) <= printed_tol(g_pr)
    pprime0 = -2.0 * P.W4_deriv_at_one(k) / (2 * k + 1)
    g = P.gamma_sup(lambda x: P.p_cheb4(k, x), pprime0)
    assert abs(g - g_pr) <= printed_tol(g_pr) + 1e-14


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"k{r[0]}")
def test_opt4_weights_reach_printed_gamma(row):
    k, g_pr = row[0], row[4]
    beta, g = P.opt4_weights(k, return_gamma=True)
    assert abs(g - g_pr) <= printed_tol(g_pr) + 2e-13 * g_pr
    # independent evaluation of the sup for the returned weights
    gs = P.gamma_opt4(beta)
    assert abs(gs - g_pr) <= 1e-9 * g_pr
    # the polynomial lies in Pi_k: p(0)=1 and |p|<1 on (0,1]
    xs = np.linspace(1e-6, 1.0, 100001)
    p = P.p_opt4(beta, xs)
    assert abs(P.p_opt4(beta, np.array([0.0]))[0] - 1.0) < 1e-14
    assert np.all(np.abs(p) < 1.0)


def test_opt4_k1_k2_closed_forms():
    b1, g1 = P.opt4_weights(1, return_gamma=True)
    assert abs(b1[0] - 9.0 / 8.0) < 1e-14 and abs(g1 - 1.0 / 3.0) < 1e-15
    _, g2 = P.opt4_weights(2, return_gamma=True)
    assert abs(g2 - (1.0 - 2.0 / math.sqrt(5.0))) < 1e-15


def test_opt4_with_unit_weights_is_plain_cheb4():
    # beta_j = 1 collapses the expansion of Eq. polsmootheropt to W_k/(2k+1)
    xs = np.linspace(0, 1, 1001)
    for k in range(1, 9):
        assert np.allclose(P.p_opt4(np.ones(k), xs), P.p_cheb4(k, xs), atol=1e-14)


def test_W4_is_fourth_kind():
    # textbook recurrence of the 4th kind: W0 = 1, W1 = 2t + 1, W_{j+1} = 2t W_j - W_{j-1}
    t = np.linspace(-1, 1, 2001)
    w_prev, w = np.ones_like(t), 2 * t + 1
    assert np.allclose(P.W4(0, t), w_prev, atol=1e-13)
    assert np.allclose(P.W4(1, t), w, atol=1e-13)
    for j in range(1, 16):
        w_prev, w = w, 2 * t * w - w_prev
        assert np.allclose(P.W4(j + 1, t), w, atol=1e-11 * (j + 1) ** 2)
        d = (P.W4(j + 1, np.array([1.0])) - P.W4(j + 1, np.array([1.0 - 1e-7])))[0] / 1e-7
        assert abs(d - P.W4_deriv_at_one(j + 1)) < 1e-4 * P.W4_deriv_at_one(j + 1)


def test_tau_recurrence_matches_closed_form():
    # Eq. recurrence-relation-shifted with sigma_0=1, sigma_1=theta/delta,
    # sigma_{k+1} = 2(theta/delta) sigma_k - sigma_{k-1}
    x = np.linspace(-0.2, 1.2, 1401)
    for a in (0.05, 0.2, 1 / 3):
        th, de = P.theta_delta(a)
        sig = [1.0, th / de]
        t_prev, t_cur = np.ones_like(x), 1 - x / th
        assert np.allclose(P.tau_scaled(1, a, x), t_cur, atol=1e-13)
        for k in range(1, 12):
            sig.append(2 * th / de * sig[k] - sig[k - 1])
            t_next = sig[k] / sig[k + 1] * (2 * (th - x) / de * t_cur - sig[k - 1] / sig[k] * t_prev)
            t_prev, t_cur = t_cur, t_next
            assert np.allclose(P.tau_scaled(k + 1, a, x), t_cur, atol=1e-11)


@pytest.mark.parametrize("k", [2, 3, 4, 6, 9])
def test_c1_formula_is_derivative_at_zero(k):
    # Eq. c1: c_1 = d/dx tau_k^{[a,1]} at 0, and 1/(2|c_1|) is the binomial ratio
    for a in (0.03, 0.1, 0.4):
        h = 1e-6
        d = (P.tau_scaled(k, a, np.array([h])) - P.tau_scaled(k, a, np.array([-h])))[0] / (2 * h)
        assert abs(1.0 / (2 * abs(d)) - P.inv_two_c1(a, k)) < 1e-7 * P.inv_two_c1(a, k)


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_lemma1_monotone_on_0_a(k):
    for a in (0.02, 0.15, 0.5, 0.9):
        x = np.linspace(1e-4 * a, a, 4000)
        tau = P.tau_scaled(k, a, x)
        f = P.f_objective(tau, x)
        assert np.all(f > 0)
        assert np.all(np.diff(f) < 1e-12 * f[:-1])


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_lemma2_g_increasing(k):
    xs = np.linspace(1e-4, 1 - 1e-4, 3000)
    g = np.array([P.inv_two_c1(x, k) for x in xs])
    assert np.all(np.diff(g) > 0)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_cheb1_coeffs_reproduce_tau(k):
    # the scalar recurrence of Algorithm 1 applied to an eigen-component must
    # give tau_k^{[a,1]}(lambda); scalar restatement of the vector algorithm
    a = P.a_star(k)
    th, de, s1, rhos = P.cheb1_coeffs(a, k)
    for lam in np.linspace(0.0, 1.0, 41):
        e0 = 1.0
        r = -lam * e0            # r = M^{-1}(b - A x) = -lambda e for b = 0
        d = r / th
        e = e0 + d
        for j in range(1, k):
            s = lam * d
            r = r - s
            d = rhos[j] * rhos[j - 1] * d + 2 * rhos[j] / de * r
            e = e + d
        assert abs(e - P.tau_scaled(k, a, np.array([lam]))[0]) < 1e-13
