"""Pins for the oracle smoothers (no GPU).

Each recurrence is compared with the closed-form error polynomial it is
supposed to realise (Sec. 2.1-2.2) on matrices whose eigen-decomposition is
known or computed densely: e_out = p(M^{-1}A) e_in.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import params as P
from oracle.smoother import SmootherSpec, l1_diag, power_lambda, smooth, error_poly

KIND_CASES = [("l1jacobi", None), ("cheb4", None), ("cheb4_opt", None),
              ("weights", "rand"), ("cheb1_opt", None), ("cheb1", 1.1), ("cheb4", 1.2)]


def make_spec(kind, extra, k, seed=0):
    if kind == "weights":
        beta = 1.0 + 0.3 * np.random.default_rng(seed).uniform(-1, 1, k)
        return SmootherSpec(kind, k, beta=beta)
    if kind == "cheb1" or (kind == "cheb4" and extra is not None):
        return SmootherSpec(kind, k, rho=extra)   # an explicit rho(M^{-1}A) estimate
    return SmootherSpec(kind, k)


@pytest.mark.parametrize("kind,extra", KIND_CASES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_diagonal_error_propagation(kind, extra, k):
    # A diagonal, M overridden so that M^{-1}A = diag(lambda) with lambda in (0,1]:
    # every component of the error is multiplied by p(lambda_i) exactly.
    rng = np.random.default_rng(1)
    n = 200
    lam = np.concatenate([np.linspace(1e-3, 1.0, n - 2), [1.0, 0.5]])
    a = rng.uniform(0.5, 3.0, n)
    A = sp.diags(a).tocsr()
    M = a / lam
    xs = rng.uniform(-1, 1, n)
    b = A @ xs
    spec = make_spec(kind, extra, k)
    for x0 in (None, rng.uniform(-1, 1, n)):
        e0 = (np.zeros(n) if x0 is None else x0) - xs
        x = smooth(A, b, x0, spec, M=M)
        expect = error_poly(spec, lam) * e0
        assert np.max(np.abs((x - xs) - expect)) <= 1e-13 * np.max(np.abs(e0))


@pytest.mark.parametrize("kind,extra", KIND_CASES)
@pytest.mark.parametrize("k", [1, 3, 5])
def test_periodic_laplacian_fourier(kind, extra, k):
    # circulant tridiag(-1, 2+s, -1): l1 diagonal is 4+s everywhere, the
    # eigenvectors are Fourier modes with lambda_j = (2+s-2cos(2 pi j/n))/(4+s)
    n, s = 96, 0.1
    main = np.full(n, 2.0 + s)
    off = -np.ones(n - 1)
    A = sp.diags([main, off, off], [0, 1, -1]).tolil()
    A[0, n - 1] = -1.0
    A[n - 1, 0] = -1.0
    A = A.tocsr()
    assert np.allclose(l1_diag(A), 4.0 + s)
    lam = (2.0 + s - 2.0 * np.cos(2 * np.pi * np.arange(n) / n)) / (4.0 + s)
    rng = np.random.default_rng(2)
    xs = rng.uniform(-1, 1, n)
    b = A @ xs
    spec = make_spec(kind, extra, k)
    x0 = rng.uniform(-1, 1, n)
    x = smooth(A, b, x0, spec)
    expect = np.fft.ifft(error_poly(spec, lam) * np.fft.fft(x0 - xs)).real
    assert np.max(np.abs((x - xs) - expect)) <= 1e-13


def dense_error_operator(A, spec):
    """p(M^{-1}A) from the eigen-decomposition of M^{-1/2} A M^{-1/2}."""
    Ad = A.toarray()
    M = l1_diag(A)
    Mh = np.sqrt(M)
    S = Ad / Mh[:, None] / Mh[None, :]
    mu, V = np.linalg.eigh(S)
    return (V * error_poly(spec, mu)) @ V.T / Mh[:, None] * Mh[None, :], mu


@pytest.mark.parametrize("kind,extra", KIND_CASES)
@pytest.mark.parametrize("k", [1, 2, 4])
def test_dirichlet_and_3d_brute_force(kind, extra, k):
    from paper_2407_09848_gb300 import problems as pr
    mats = [sp.diags([np.full(30, 2.0), -np.ones(29), -np.ones(29)], [0, 1, -1]).tocsr(),
            pr.to_csr(pr.poisson(4)), pr.to_csr(pr.varcoef(4, 1.5, 2.0, seed=3))]
    rng = np.random.default_rng(3)
    for A in mats:
        n = A.shape[0]
        spec = make_spec(kind, extra, k)
        G, mu = dense_error_operator(A, spec)
        assert mu.max() <= 1.0 + 1e-12 and mu.min() > 0   # Gershgorin: rho(M^{-1}A) <= 1
        xs = rng.uniform(-1, 1, n)
        b = A @ xs
        x0 = rng.uniform(-1, 1, n)
        x = smooth(A, b, x0, spec)
        assert np.allclose(x - xs, G @ (x0 - xs), atol=1e-13, rtol=0)
        x = smooth(A, b, None, spec)
        assert np.allclose(x - xs, G @ (-xs), atol=1e-13, rtol=0)


def test_l1_diag_by_hand():
    A = sp.csr_matrix(np.array([[4.0, -1.0, 2.0], [-1.0, 5.0, 0.0], [2.0, 0.0, 3.0]]))
    assert np.allclose(l1_diag(A), [7.0, 6.0, 5.0])


def test_power_lambda_closed_form():
    # with M^{-1}A = diag(lambda), v_i is proportional to lambda^i v0, so the
    # 10-step estimate is ||lambda^10 v0|| / ||lambda^9 v0||
    rng = np.random.default_rng(4)
    n = 50
    lam = rng.uniform(0.1, 0.95, n)
    a = rng.uniform(1, 2, n)
    A = sp.diags(a).tocsr()
    v0 = rng.uniform(-1, 1, n)
    est = power_lambda(A, v0, iters=10, M=a / lam)
    ref = np.linalg.norm(lam ** 10 * v0) / np.linalg.norm(lam ** 9 * v0)
    assert abs(est - ref) < 1e-14


def test_zero_start_equals_explicit_zero():
    from paper_2407_09848_gb300 import problems as pr
    A = pr.to_csr(pr.poisson(5))
    b = np.random.default_rng(5).uniform(-1, 1, A.shape[0])
    for kind, extra in KIND_CASES:
        spec = make_spec(kind, extra, 3)
        assert np.allclose(smooth(A, b, None, spec), smooth(A, b, np.zeros_like(b), spec),
                           atol=1e-15, rtol=0)
