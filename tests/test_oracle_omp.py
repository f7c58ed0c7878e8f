"""The all-core C build of the oracle loops (oracle/c/amg_omp.c) on the CPU:
each smoother kind against its closed-form error polynomial on a circulant
matrix with Fourier eigenvectors, and against the numpy oracle: every
smoother kind from zero and from x0, the
V-cycle with aggregation and with smoothed-aggregation prolongators, both
coarse solvers, and PCG iteration counts.  The two restate the same steps in
the same order (one CSR pass per product, row order), so they agree to a few
units of rounding; the C build's dot products are summed per thread, so the
thread count is varied too."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import omp
from oracle.amg import OracleAMG
from oracle.sa import sa_hierarchy
from oracle.smoother import SmootherSpec, error_poly, power_lambda, smooth
from paper_2407_09848_gb300 import problems as pr

TOL = 1e-13


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def ragged():
    return pr.build_hierarchy(pr.varcoef(20, 1.0, 4.0, seed=11, ny=18, nz=13), coarse_max=100)


@pytest.mark.parametrize("kind,k,rho", [("l1jacobi", 2, 1.0), ("cheb4", 3, 1.0), ("cheb4_opt", 4, 1.0),
                                        ("cheb1_opt", 4, 1.0), ("cheb1", 3, 1.1)])
def test_smoother_closed_form_on_circulant(kind, k, rho):
    # tridiag(-1, 2+s, -1) with periodic wrap: M = (4+s) I, eigenvectors are
    # Fourier modes with lambda_j = (2+s-2cos(2 pi j/n))/(4+s), so the error
    # after one application is sum_j p(lambda_j) times its projection
    n, s = 64, 0.1
    off = -np.ones(n - 1)
    A = sp.diags([np.full(n, 2.0 + s), off, off], [0, 1, -1]).tolil()
    A[0, n - 1] = A[n - 1, 0] = -1.0
    A = A.tocsr()
    lam = (2.0 + s - 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)) / (4.0 + s)
    rng = np.random.default_rng(2)
    xs, x0 = rng.uniform(-1, 1, (2, n))
    b = A @ xs
    spec = SmootherSpec(kind, k, rho=rho)
    e = np.fft.ifft(error_poly(spec, lam) * np.fft.fft(x0 - xs)).real
    assert np.max(np.abs((omp.smooth(A, b, x0, spec) - xs) - e)) <= 1e-13


@pytest.mark.parametrize("kind,k", [("l1jacobi", 3), ("cheb4", 1), ("cheb4", 5), ("cheb4_opt", 4),
                                    ("weights", 3), ("cheb1_opt", 1), ("cheb1_opt", 4),
                                    ("cheb1", 3)])
def test_smoother_matches_numpy_oracle(ragged, kind, k):
    A = ragged.A[0]
    n = A.shape[0]
    rng = np.random.default_rng(5 + k)
    b, x0 = rng.uniform(-1, 1, (2, n))
    rho = 1.1 * power_lambda(A, pr.vec_uniform(n, seed=0)) if kind == "cheb1" else 1.0
    beta = 1.0 + 0.2 * rng.uniform(-1, 1, k) if kind == "weights" else None
    spec = SmootherSpec(kind, k, beta=beta, rho=rho)
    for start in (None, x0):
        assert relmax(omp.smooth(A, b, start, spec), smooth(A, b, start, spec)) <= TOL


@pytest.mark.parametrize("threads", [1, 3])
@pytest.mark.parametrize("coarse_sweeps", [0, 30])
def test_vcycle_matches_numpy_oracle(ragged, threads, coarse_sweeps):
    prev = omp.threads()
    omp.set_threads(threads)
    try:
        spec = SmootherSpec("cheb4_opt", 4)
        r = pr.rhs_uniform(ragged.A[0].shape[0], seed=3)
        z = omp.OmpAMG(ragged.A, ragged.P, spec, coarse_sweeps=coarse_sweeps).vcycle(r)
        zo = OracleAMG(ragged.A, ragged.P, spec, coarse_sweeps=coarse_sweeps).vcycle(r)
        assert relmax(z, zo) <= TOL
    finally:
        omp.set_threads(prev)


def test_vcycle_general_prolongator():
    # smoothed-aggregation P (several entries per row) exercises P^T as its
    # own CSR matrix
    st = pr.poisson(16, 14, 12)
    A0 = pr.to_csr(st)
    levels = pr.geometric_aggregates(st.shape, coarse_max=60)
    As, Ps, _ = sa_hierarchy(A0, [lv[0] for lv in levels], [lv[1] for lv in levels])
    spec = SmootherSpec("cheb1_opt", 3)
    r = pr.rhs_uniform(A0.shape[0], seed=1)
    assert relmax(omp.OmpAMG(As, Ps, spec).vcycle(r), OracleAMG(As, Ps, spec).vcycle(r)) <= TOL


@pytest.mark.parametrize("kind,k", [("cheb4_opt", 4), ("cheb4", 2), ("cheb1_opt", 3),
                                    ("l1jacobi", 4)])
def test_pcg_counts_match_numpy_oracle(kind, k):
    H = pr.build_hierarchy(pr.poisson(32), coarse_max=512)
    b = pr.rhs_uniform(H.A[0].shape[0], seed=0)
    spec = SmootherSpec(kind, k)
    x, it, rel, st = omp.OmpAMG(H.A, H.P, spec).pcg(b, rtol=1e-8)
    xo, ito, relo, _ = OracleAMG(H.A, H.P, spec).pcg(b, rtol=1e-8)
    assert st == 0 and it == ito and rel <= 1e-8
    assert abs(rel - relo) <= 1e-6 * relo
    assert relmax(x, xo) <= 1e-10
