"""Pins for the oracle V-cycle and PCG (no GPU)."""
import numpy as np
import pytest

from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec, l1_diag, error_poly
from paper_2407_09848_gb300 import problems as pr

KINDS = [("l1jacobi", {}), ("cheb4", {}), ("cheb4_opt", {}), ("cheb1_opt", {}),
         ("cheb1", {"rho": 1.05})]


def hier(st, coarse_max):
    H = pr.build_hierarchy(st, coarse_max=coarse_max)
    return H.A, H.P


def dense_B(amg):
    n = amg.A[0].shape[0]
    I = np.eye(n)
    return np.stack([amg.vcycle(I[:, j]) for j in range(n)], axis=1)


def dense_G(A, spec):
    Ad = A.toarray()
    Mh = np.sqrt(l1_diag(A))
    mu, V = np.linalg.eigh(Ad / Mh[:, None] / Mh[None, :])
    return (V * error_poly(spec, mu)) @ V.T / Mh[:, None] * Mh[None, :]


def dense_B_reference(A_list, P_list, spec, level=0):
    """B_l from Eq. amg written with dense factors:
    I - B_l A_l = G (I - P_l B_{l+1} P_l^T A_l) G, G = p(M^{-1}A_l)
    (the post factor p(M^{-T} A) equals G because M is diagonal)."""
    A = A_list[level].toarray()
    if level == len(A_list) - 1:
        return np.linalg.inv(A)
    P = P_list[level].toarray()
    Bc = dense_B_reference(A_list, P_list, spec, level + 1)
    G = dense_G(A_list[level], spec)
    n = A.shape[0]
    E = G @ (np.eye(n) - P @ Bc @ P.T @ A) @ G
    return (np.eye(n) - E) @ np.linalg.inv(A)


@pytest.mark.parametrize("kind,kw", KINDS)
@pytest.mark.parametrize("k", [1, 2, 4])
def test_vcycle_equals_dense_composition(kind, kw, k):
    for st, cm in [(pr.poisson(4), 8), (pr.varcoef(4, 1.0, 2.0, seed=1), 8),
                   (pr.poisson(8), 8), (pr.aniso(6, 1e-2), 30)]:
        A, Pl = hier(st, cm)
        spec = SmootherSpec(kind, k, **kw)
        amg = OracleAMG(A, Pl, spec)
        B = dense_B(amg)
        Bref = dense_B_reference(A, Pl, spec)
        scale = np.abs(Bref).max()
        assert np.max(np.abs(B - Bref)) <= 1e-12 * scale
        # symmetric preconditioner
        assert np.max(np.abs(B - B.T)) <= 1e-12 * scale


@pytest.mark.parametrize("kind,kw", KINDS)
def test_vcycle_symmetric_larger(kind, kw):
    A, Pl = hier(pr.varcoef(16, 1.0, 4.0, seed=2), 64)
    amg = OracleAMG(A, Pl, SmootherSpec(kind, 3, **kw))
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((2, A[0].shape[0]))
    lhs, rhs = amg.vcycle(u) @ v, u @ amg.vcycle(v)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_two_level_exact_coarse_special_case():
    # with two levels the coarse correction is exactly P A_c^{-1} P^T
    A, Pl = hier(pr.poisson(6), 27)
    assert len(A) == 2
    spec = SmootherSpec("cheb4", 2)
    amg = OracleAMG(A, Pl, spec)
    Ad, Pd = A[0].toarray(), Pl[0].toarray()
    G = dense_G(A[0], spec)
    n = Ad.shape[0]
    E = G @ (np.eye(n) - Pd @ np.linalg.inv(Pd.T @ Ad @ Pd) @ Pd.T @ Ad) @ G
    B = dense_B(amg)
    assert np.allclose(np.eye(n) - B @ Ad, E, atol=1e-12)
    # the two-level error propagation contracts in the A-norm
    Ah = np.linalg.cholesky(Ad)
    assert np.linalg.norm(Ah.T @ E @ np.linalg.inv(Ah.T), 2) < 1.0


@pytest.mark.parametrize("kind,kw", KINDS)
def test_pcg_matches_dense_solve(kind, kw):
    A, Pl = hier(pr.varcoef(10, 1.0, 3.0, seed=4), 20)
    amg = OracleAMG(A, Pl, SmootherSpec(kind, 2, **kw))
    b = pr.rhs_uniform(A[0].shape[0], seed=1)
    x, it, rel, hist = amg.pcg(b, rtol=1e-10, maxit=200)
    xd = np.linalg.solve(A[0].toarray(), b)
    cond = np.linalg.cond(A[0].toarray())
    assert rel <= 1e-10
    assert np.linalg.norm(x - xd) <= 1e-10 * cond * np.linalg.norm(xd)
    assert np.linalg.norm(b - A[0] @ x) <= 1e-9 * np.linalg.norm(b)
    assert 0 < it < 200


def test_pcg_identity_preconditioner_is_cg():
    # a single-level hierarchy makes the preconditioner the exact inverse:
    # PCG converges in one iteration
    A, Pl = hier(pr.poisson(5), 1000)
    assert len(A) == 1
    amg = OracleAMG(A, Pl, [])
    b = pr.rhs_uniform(A[0].shape[0], seed=2)
    x, it, rel, _ = amg.pcg(b, rtol=1e-12)
    assert it == 1 and rel < 1e-12


def test_pcg_poisson32_opt4_k4_sanity():
    # the 32^3 configuration; iteration count vs the paper: parity unpinned
    # (different hierarchy, problem and hardware).  Sanity range only.
    A, Pl = hier(pr.poisson(32), 512)
    assert [a.shape[0] for a in A] == [32768, 4096, 512]
    amg = OracleAMG(A, Pl, SmootherSpec("cheb4_opt", 4))
    b = pr.rhs_uniform(32768, seed=0)
    x, it, rel, _ = amg.pcg(b, rtol=1e-8)
    assert rel <= 1e-8 and 5 <= it <= 20
    assert np.linalg.norm(b - A[0] @ x) <= 2e-8 * np.linalg.norm(b)


def test_flexible_pcg_matches_dense_solve_and_standard_on_linear_precond():
    # with an exactly linear symmetric preconditioner, r_{k+1}.z_k = 0 in exact
    # arithmetic, so the flexible and standard forms take the same iterations
    A, Pl = hier(pr.varcoef(10, 1.0, 3.0, seed=4), 20)
    amg = OracleAMG(A, Pl, SmootherSpec("cheb4_opt", 3))
    b = pr.rhs_uniform(A[0].shape[0], seed=1)
    x1, it1, _, _ = amg.pcg(b, rtol=1e-10)
    x2, it2, rel2, _ = amg.pcg(b, rtol=1e-10, flexible=True)
    assert it1 == it2 and rel2 <= 1e-10
    xd = np.linalg.solve(A[0].toarray(), b)
    assert np.linalg.norm(x2 - xd) <= 1e-8 * np.linalg.norm(xd)


def test_pcg_precond_hook_textbook_cases():
    # identity preconditioner: plain CG, which on an SPD matrix with m distinct
    # eigenvalues reaches the solution in m steps (exact arithmetic; here to
    # ~1e-12 with m = 3)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    d = np.repeat([1.0, 2.0, 5.0], 10)
    import scipy.sparse as sp
    A = sp.csr_matrix((Q * d) @ Q.T)
    As, Ps = pr.single_aggregate_hierarchy(A)
    amg = OracleAMG(As, Ps, SmootherSpec("cheb4", 1))
    b = rng.standard_normal(30)
    x, it, rel, _ = amg.pcg(b, rtol=1e-11, precond=lambda r: r.copy())
    assert it == 3 and rel <= 1e-11
    # exact inverse as preconditioner: one step
    Ainv = np.linalg.inv(A.toarray())
    x, it, rel, _ = amg.pcg(b, rtol=1e-11, precond=lambda r: Ainv @ r)
    assert it == 1
    assert np.allclose(x, Ainv @ b, atol=1e-12 * np.linalg.norm(Ainv @ b))


def test_fcg1_equals_pcg_on_fixed_spd_preconditioner():
    # for a fixed SPD preconditioner the one-reduction flexible CG generates the
    # same Krylov iterates as standard PCG (exact arithmetic); q stays A p
    A, Pl = hier(pr.varcoef(10, 1.0, 3.0, seed=4), 20)
    amg = OracleAMG(A, Pl, SmootherSpec("cheb4_opt", 3))
    b = pr.rhs_uniform(A[0].shape[0], seed=1)
    x1, it1, _, h1 = amg.pcg(b, rtol=1e-10)
    x2, it2, rel2, h2 = amg.fcg1(b, rtol=1e-10)
    assert it1 == it2 and rel2 <= 1e-10
    # residual histories agree until cancellation near convergence
    assert np.allclose(h1[:6], h2[:6], rtol=1e-8, atol=0)
    xd = np.linalg.solve(A[0].toarray(), b)
    assert np.linalg.norm(x2 - xd) <= 1e-8 * np.linalg.norm(xd)


def test_fcg1_textbook_cases():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    import scipy.sparse as sp
    A = sp.csr_matrix((Q * np.repeat([1.0, 2.0, 5.0], 10)) @ Q.T)
    As, Ps = pr.single_aggregate_hierarchy(A)
    amg = OracleAMG(As, Ps, SmootherSpec("cheb4", 1))
    b = rng.standard_normal(30)
    # identity preconditioner: CG, 3 distinct eigenvalues -> 3 steps
    _, it, rel, _ = amg.fcg1(b, rtol=1e-11, precond=lambda r: r.copy())
    assert it == 3 and rel <= 1e-11
    # exact inverse: one step
    Ainv = np.linalg.inv(A.toarray())
    x, it, _, _ = amg.fcg1(b, rtol=1e-11, precond=lambda r: Ainv @ r)
    assert it == 1 and np.allclose(x, Ainv @ b, atol=1e-12 * np.linalg.norm(Ainv @ b))
    # agrees with standard PCG under a non-trivial diagonal preconditioner (a
    # sign error in beta = z.Ap / p.Ap loses A-conjugacy and does not converge)
    M = np.diag(1.0 / np.linspace(1, 3, 30))
    _, it_ok, _, _ = amg.fcg1(b, rtol=1e-10, precond=lambda r: M @ r)
    _, it_pcg, _, _ = amg.pcg(b, rtol=1e-10, precond=lambda r: M @ r)
    assert it_ok == it_pcg


def test_coarse_l1jacobi_sweeps_dense_composition():
    # coarsest level solved by m l1-Jacobi sweeps from zero (Sec. 4): the
    # coarse operator is Q_m = sum_{j<m} (I - M^{-1}A_c)^j M^{-1}
    A, Pl = hier(pr.varcoef(8, 1.0, 2.0, seed=5), 64)
    assert len(A) == 2
    spec = SmootherSpec("cheb4_opt", 2)
    m = 7
    amg = OracleAMG(A, Pl, spec, coarse_sweeps=m)
    Ac = A[-1].toarray()
    Minv = np.diag(1.0 / l1_diag(A[-1]))
    E = np.eye(Ac.shape[0]) - Minv @ Ac
    Q = sum(np.linalg.matrix_power(E, j) for j in range(m)) @ Minv
    for i in range(Ac.shape[0]):
        e = np.zeros(Ac.shape[0])
        e[i] = 1.0
        assert np.allclose(amg.coarse_solve(e), Q[:, i], rtol=0, atol=1e-14)
    # two-level dense reference with Q_m in place of A_c^{-1}
    n = A[0].shape[0]
    B = dense_B(amg)
    Ad, Pd = A[0].toarray(), Pl[0].toarray()
    G = dense_G(A[0], spec)
    Eref = G @ (np.eye(n) - Pd @ Q @ Pd.T @ Ad) @ G
    assert np.max(np.abs(np.eye(n) - B @ Ad - Eref)) <= 1e-12
    assert np.max(np.abs(B - B.T)) <= 1e-12 * np.abs(B).max()


def test_coarse_sweeps_converge_to_exact_coarse_solve():
    A, Pl = hier(pr.poisson(8), 8)
    spec = SmootherSpec("cheb4", 2)
    exact = OracleAMG(A, Pl, spec)
    many = OracleAMG(A, Pl, spec, coarse_sweeps=3000)
    r = pr.rhs_uniform(A[0].shape[0], seed=3)
    assert np.allclose(many.vcycle(r), exact.vcycle(r), rtol=0, atol=1e-10)
    b = pr.rhs_uniform(A[0].shape[0], seed=1)
    _, it30, rel, _ = OracleAMG(A, Pl, spec, coarse_sweeps=30).pcg(b, rtol=1e-8)
    assert rel <= 1e-8 and it30 < 100


@pytest.mark.parametrize("flexible", [True, False])
def test_conjugacy_defect_under_a_variable_preconditioner(flexible):
    # With exact line searches r_{k+1} is orthogonal to p_k, and A p_k =
    # (r_k - r_{k+1}) / alpha_k, p_k.A p_k = r_k.z_k / alpha_k.  Hence for any
    # preconditioners B_k (z_k = B_k r_k) the local conjugacy defect is fixed
    # by the direction update alone:
    #   flexible (Polak-Ribiere):  alpha_k p_{k+1}.A p_k = z_{k+1}.r_k - r_{k+1}.z_k
    #   standard (Fletcher-Reeves): alpha_k p_{k+1}.A p_k = z_{k+1}.r_k
    # (the first is the local relation of inexact-preconditioned CG, Golub-Ye;
    # both vanish for a fixed symmetric B).  Steps s_k = x_{k+1} - x_k =
    # alpha_k p_k are read from runs stopped after 1, 2, ... iterations with the
    # same preconditioner sequence, and alpha_{k+1} = s.A s / (r_{k+1}.z_{k+1}).
    A, Pl = hier(pr.varcoef(6, 1.0, 3.0, seed=7), 30)
    amg = OracleAMG(A, Pl, SmootherSpec("cheb4", 1))
    A0 = A[0]
    n = A0.shape[0]
    b = pr.rhs_uniform(n, seed=5)
    D = np.random.default_rng(9).uniform(0.5, 2.0, (8, n))   # B_k = diag(D[k]), SPD, varying

    def run(m):
        calls = [0]

        def prec(r):
            d = D[calls[0]]
            calls[0] += 1
            return d * r
        x, it, _, _ = amg.pcg(b, rtol=0.0, maxit=m, flexible=flexible, precond=prec)
        assert it == m
        return x
    xs = [np.zeros(n)] + [run(m) for m in range(1, 6)]
    r = [b - A0 @ x for x in xs]
    z = [D[k] * r[k] for k in range(len(xs))]
    s = [xs[k + 1] - xs[k] for k in range(len(xs) - 1)]
    for k in range(len(s) - 1):
        alpha1 = (s[k + 1] @ (A0 @ s[k + 1])) / (r[k + 1] @ z[k + 1])
        lhs = s[k + 1] @ (A0 @ s[k])                     # alpha_{k+1} alpha_k p_{k+1}.A p_k
        defect = z[k + 1] @ r[k] - (r[k + 1] @ z[k] if flexible else 0.0)
        rhs = alpha1 * defect
        scale = abs(alpha1) * np.linalg.norm(z[k + 1]) * np.linalg.norm(r[k])
        assert abs(lhs - rhs) <= 1e-10 * scale, (k, lhs, rhs)
        if k >= 1:
            assert abs(rhs) > 1e-6 * scale               # the preconditioner change matters


@pytest.mark.parametrize("kind,k", [("cheb4_opt", 4), ("cheb4", 2), ("cheb1_opt", 6), ("cheb1", 4),
                                    ("l1jacobi", 1), ("cheb4_opt", 16)])
def test_stored_iteration_counts_match_the_oracle(kind, k):
    # the GPU tests compare against tests/golden/oracle_pcg_iterations.json;
    # a sample of its 32^3 entries must be what the oracle gives today
    import json
    import os
    from oracle.smoother import power_lambda
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_pcg_iterations.json")
    runs = {(r["grid"], r["kind"], r["degree"]): r for r in json.load(open(path))["runs"]}
    stored = runs[(32, kind, k)]["iterations"]
    A, Pl = hier(pr.poisson(32), 512)
    specs = []
    for Al in A[:-1]:
        if kind == "cheb1":
            lam = power_lambda(Al, pr.vec_uniform(Al.shape[0], seed=0), iters=10)
            specs.append(SmootherSpec(kind, k, rho=1.1 * lam))
        else:
            specs.append(SmootherSpec(kind, k))
    b = pr.rhs_uniform(A[0].shape[0], seed=0)
    _, it, rel, _ = OracleAMG(A, Pl, specs).pcg(b, rtol=1e-8, maxit=1000)
    assert rel <= 1e-8 and it == stored
