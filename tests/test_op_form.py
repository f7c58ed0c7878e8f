"""Host logic of the stored-operator form of the smoothers (no GPU).

The library evaluates each smoother backwards (Clenshaw's scheme on the
three-term recurrence of its z_j: Sec. 2.1 Eq. polsmoother / polsmootheropt,
Sec. 2.2 Algorithm 1, and l1-Jacobi, Eq. l1smooth), one stored operator
tau I - sigma M^{-1} A per step.  Here the step coefficients that
amgps_op_coefs returns are applied in numpy exactly as the header documents
them, and one application must equal the oracle's forward recurrence to
rounding, for every kind, degree 2..16, rho and starting vector.  A wrong
sign, index or coefficient anywhere in the derivation changes the polynomial
and fails by orders of magnitude."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.smoother import SmootherSpec, l1_diag, smooth
from paper_2407_09848_gb300 import amgps, build
from paper_2407_09848_gb300 import problems as pr


@pytest.fixture(scope="module")
def lib():
    build.build()
    return amgps.lib()


@pytest.fixture(scope="module")
def system():
    A = pr.to_csr(pr.varcoef(10, sigma=1.0, ell=3.0, seed=3)).tocsr()
    rng = np.random.default_rng(11)
    n = A.shape[0]
    return A, l1_diag(A), rng.standard_normal(n), rng.standard_normal(n)


def op_apply(A, M, b, x0, coefs):
    """x = x0 + v_{k-2}: v_q = h s0 + g v_{q-2} + (tau I - sigma B) w_q."""
    tau, sigma, h, g = coefs
    B = sp.diags(1.0 / M) @ A
    s0 = (b - (A @ x0 if x0 is not None else 0.0)) / M
    v = []
    for q in range(len(tau)):
        w = s0 if q == 0 else v[q - 1]
        out = tau[q] * w - sigma[q] * (B @ w) + h[q] * s0
        if q >= 2:
            out = out + g[q] * v[q - 2]
        v.append(out)
    return (x0 if x0 is not None else 0.0) + v[-1]


CASES = [(kind, k, rho) for k in range(2, 17)
         for kind, rho in (("cheb4", 1.0), ("cheb4", 0.9), ("cheb4_opt", 1.0), ("cheb4_opt", 0.9),
                           ("weights", 0.95), ("cheb1", 1.0), ("cheb1", 0.9), ("cheb1_opt", 1.0),
                           ("l1jacobi", 1.0))]


@pytest.mark.parametrize("kind,k,rho", CASES, ids=lambda v: str(v))
def test_op_form_equals_oracle_recurrence(lib, system, kind, k, rho):
    A, M, b, x0 = system
    w = None
    beta = None
    if kind == "weights":
        w = 1.0 + 0.4 * np.sin(np.arange(1, k + 1))
        beta = w
    elif kind == "cheb4_opt":
        beta = amgps.opt4_weights(k)  # the library's table (pinned against the paper elsewhere)
    coefs = amgps.op_coefs(kind, k, w, rho)
    for start in (None, x0):
        spec = SmootherSpec(kind, k, beta=beta, rho=rho)
        ref = smooth(A, b, start, spec, M=M)
        got = op_apply(A, M, b, start, coefs)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= 1e-13, (kind, k, rho, start is None, err)


def test_op_coefs_shape_of_the_steps(lib):
    # the first step multiplies s0 alone; the second adds s0; from the third
    # on a step also takes v_{q-2}
    tau, sigma, h, g = amgps.op_coefs("cheb4_opt", 6)
    assert len(tau) == 5
    assert h[0] == 0.0 and g[0] == 0.0 and g[1] == 0.0
    assert np.all(g[2:] != 0.0) and np.all(h[1:] != 0.0)
    assert np.all(sigma > 0.0)


def test_op_coefs_l1jacobi_steps(lib):
    # l1-Jacobi (a_j = 0, c_j = 1): u_{k-1} = (2 I - B) s0, then
    # u_j = s0 + (I - B) u_{j+1}, with no u_{j+2} term
    tau, sigma, h, g = amgps.op_coefs("l1jacobi", 5)
    assert np.array_equal(tau, [2.0, 1.0, 1.0, 1.0]) and np.all(sigma == 1.0)
    assert np.array_equal(h, [0.0, 1.0, 1.0, 1.0]) and np.all(g == 0.0)


def test_op_coefs_rejects_degree_one(lib):
    with pytest.raises(amgps.AmgpsError):
        amgps.op_coefs("cheb4_opt", 1)
    with pytest.raises(amgps.AmgpsError):
        amgps.op_coefs("l1jacobi", 1)


@pytest.mark.parametrize("mistake", ["g_sign", "h_dropped", "tau_sigma_swapped", "sigma_sign",
                                     "steps_shifted", "last_c1_missing"])
def test_planted_coefficient_mistakes_are_caught(lib, system, mistake):
    # each plausible slip in the derivation (a sign, a dropped term, a swapped
    # or shifted coefficient, the c_1 scaling of the last step) moves the
    # result far outside the rounding-level agreement the test above demands
    A, M, b, x0 = system
    k = 5
    tau, sigma, h, g = (c.copy() for c in amgps.op_coefs("cheb4_opt", k))
    if mistake == "g_sign":
        g = -g
    elif mistake == "h_dropped":
        h[1] = 0.0
    elif mistake == "tau_sigma_swapped":
        tau[1], sigma[1] = sigma[1], tau[1]
    elif mistake == "sigma_sign":
        sigma[2] = -sigma[2]
    elif mistake == "steps_shifted":
        tau, sigma = np.roll(tau, 1), np.roll(sigma, 1)
    else:
        c1 = 4.0 / 3.0  # c_1 = (8 - 4) / (2 + 1) at rho = 1
        tau[-1], sigma[-1], h[-1], g[-1] = tau[-1] / c1, sigma[-1] / c1, h[-1] / c1, g[-1] / c1
    ref = smooth(A, b, x0, SmootherSpec("cheb4_opt", k, beta=amgps.opt4_weights(k)), M=M)
    got = op_apply(A, M, b, x0, (tau, sigma, h, g))
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) > 1e-6
