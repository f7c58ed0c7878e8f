"""Pins for the oracle's reverse-mode derivatives (no GPU)."""
import numpy as np
import pytest

from oracle.adjoint import error_reduction_loss, smooth_backward, vcycle_backward
from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec, smooth
from paper_2407_09848_gb300 import problems as pr

KINDS = [("l1jacobi", {}), ("cheb4", {}), ("cheb4_opt", {}), ("cheb1_opt", {}),
         ("cheb1", {"rho": 1.07})]


def spec_of(kind, kw, k, seed=0):
    if kind == "weights":
        return SmootherSpec("weights", k, beta=1 + 0.3 * np.random.default_rng(seed).uniform(-1, 1, k))
    return SmootherSpec(kind, k, **kw)


@pytest.mark.parametrize("kind,kw", KINDS + [("weights", {})])
@pytest.mark.parametrize("k", [1, 2, 4])
def test_smooth_backward_central_differences(kind, kw, k):
    A = pr.to_csr(pr.varcoef(6, 1.0, 2.0, seed=5))
    n = A.shape[0]
    rng = np.random.default_rng(k)
    b, x0, gx, db, dx0 = rng.standard_normal((5, n))
    spec = spec_of(kind, kw, k)
    gb, gx0, gbeta = smooth_backward(A, b, x0, spec, gx)
    L = lambda bb, xx, sp: gx @ smooth(A, bb, xx, sp)
    h = 1e-3  # x is affine in b, x0 and beta: central differences are exact up to rounding
    fd_b = (L(b + h * db, x0, spec) - L(b - h * db, x0, spec)) / (2 * h)
    fd_x = (L(b, x0 + h * dx0, spec) - L(b, x0 - h * dx0, spec)) / (2 * h)
    scale = np.linalg.norm(gx) * np.linalg.norm(b)
    assert abs(fd_b - gb @ db) <= 1e-9 * scale
    assert abs(fd_x - gx0 @ dx0) <= 1e-9 * scale
    if spec.beta is not None:
        for j in range(k):
            e = np.zeros(k)
            e[j] = h
            sp_p = SmootherSpec("weights", k, beta=spec.beta + e)
            sp_m = SmootherSpec("weights", k, beta=spec.beta - e)
            fd = (L(b, x0, sp_p) - L(b, x0, sp_m)) / (2 * h)
            assert abs(fd - gbeta[j]) <= 1e-9 * scale


@pytest.mark.parametrize("kind,kw", KINDS + [("weights", {})])
def test_smooth_operator_is_symmetric(kind, kw):
    # x = x0 + Q (b - A x0) with Q = q(M^{-1}A) M^{-1} symmetric, so dL/db = Q gx
    # equals a smoother application to gx from zero, and dL/dx0 = gx - A dL/db
    A = pr.to_csr(pr.varcoef(7, 1.5, 3.0, seed=2))
    n = A.shape[0]
    rng = np.random.default_rng(3)
    b, x0, gx = rng.standard_normal((3, n))
    spec = spec_of(kind, kw, 3)
    gb, gx0, _ = smooth_backward(A, b, x0, spec, gx)
    q = smooth(A, gx, None, spec)
    assert np.max(np.abs(gb - q)) <= 1e-13 * np.max(np.abs(q))
    assert np.max(np.abs(gx0 - (gx - A @ q))) <= 1e-12 * np.max(np.abs(gx))


def test_dense_brute_force_gradient():
    # form Q column by column on 4^3 and compare dL/db = Q^T gx
    A = pr.to_csr(pr.poisson(4))
    n = A.shape[0]
    spec = spec_of("weights", {}, 4, seed=8)
    Q = np.stack([smooth(A, e, None, spec) for e in np.eye(n)], axis=1)
    gx = np.random.default_rng(1).standard_normal(n)
    gb, _, _ = smooth_backward(A, np.zeros(n), None, spec, gx)
    assert np.allclose(gb, Q.T @ gx, atol=1e-13, rtol=0)


def test_vcycle_backward_symmetric_and_fd():
    H = pr.build_hierarchy(pr.varcoef(8, 1.0, 3.0, seed=4), coarse_max=8)
    rng = np.random.default_rng(6)
    specs = [spec_of("weights", {}, 3, seed=l) for l in range(H.n_levels - 1)]
    amg = OracleAMG(H.A, H.P, specs)
    n = H.A[0].shape[0]
    b, gx = rng.standard_normal((2, n))
    gb, gbeta = vcycle_backward(amg, b, gx)
    assert np.allclose(gb, amg.vcycle(gx), atol=1e-12 * np.abs(gb).max())
    L = lambda: gx @ amg.vcycle(b)
    h = 1e-5
    for l in range(H.n_levels - 1):
        for j in range(3):
            base = specs[l].beta.copy()
            specs[l].beta = base.copy()
            specs[l].beta[j] += h
            lp = L()
            specs[l].beta[j] -= 2 * h
            lm = L()
            specs[l].beta = base
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gbeta[l][j]) <= 1e-7 * (abs(fd) + 1e-3)


def test_error_reduction_loss_gradient_fd():
    H = pr.build_hierarchy(pr.varcoef(8, 1.5, 2.0, seed=9), coarse_max=8)
    specs = [spec_of("weights", {}, 2, seed=10 + l) for l in range(H.n_levels - 1)]
    amg = OracleAMG(H.A, H.P, specs)
    E0 = np.random.default_rng(11).standard_normal((H.A[0].shape[0], 4))
    loss, g = error_reduction_loss(amg, E0)
    assert 0.0 < loss < 1.0  # one V-cycle reduces the A-norm of the error
    h = 1e-6
    for l in range(H.n_levels - 1):
        for j in range(2):
            base = specs[l].beta.copy()
            specs[l].beta = base.copy()
            specs[l].beta[j] += h
            lp, _ = error_reduction_loss(amg, E0)
            specs[l].beta[j] -= 2 * h
            lm, _ = error_reduction_loss(amg, E0)
            specs[l].beta = base
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[l][j]) <= 1e-6 * abs(g[l][j]) + 1e-9
