"""Smoothed aggregation on the GPU (Sec. 4): the device-built prolongator and
Galerkin product against the oracle, and the V-cycle / PCG / reverse mode
through general (non-aggregation) prolongators."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sa
from oracle.adjoint import vcycle_backward
from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec
from paper_2407_09848_gb300 import problems as pr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def solver(torch_cuda):
    from paper_2407_09848_gb300.amgps import Solver
    return Solver()


def max_abs_diff(X, Y):
    D = (sp.csr_matrix(X) - sp.csr_matrix(Y)).tocoo()
    return float(np.abs(D.data).max()) if D.nnz else 0.0


def dev(torch, v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()


PROBLEMS = {
    "poisson12": lambda: pr.poisson(12),
    "varcoef_ragged": lambda: pr.varcoef(13, 1.0, 3.0, seed=5, ny=12, nz=11),
    "aniso": lambda: pr.aniso(10, 1e-2),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_sa_level_matches_oracle(solver, name):
    st = PROBLEMS[name]()
    A = pr.to_csr(st)
    levels = pr.geometric_aggregates(st.shape, coarse_max=64)
    for agg, nc, _ in levels:
        P, Ac, om = solver.sa_level(A, agg, nc)
        Po, omo = sa.sa_prolongator(A, agg, nc)
        Aco = sa.galerkin(A, Po)
        assert om == pytest.approx(omo, rel=1e-15, abs=0)
        assert P.shape == Po.shape and Ac.shape == Aco.shape
        assert max_abs_diff(P, Po) <= 1e-15
        assert max_abs_diff(Ac, Aco) <= 1e-13 * np.abs(Aco.data).max()
        # rows come back sorted; a repeated call gives identical bits
        assert P.has_sorted_indices and Ac.has_sorted_indices
        P2, Ac2, _ = solver.sa_level(A, agg, nc)
        assert np.array_equal(Ac.data, Ac2.data) and np.array_equal(Ac.indices, Ac2.indices)
        assert np.array_equal(P.data, P2.data)
        A = Ac


def test_galerkin_generic_prolongator(solver):
    # a random P with rows of 1..40 entries (rows longer than a warp) and a
    # coarse level with wide rows
    rng = np.random.default_rng(7)
    st = pr.varcoef(9, 1.0, 2.0, seed=2, ny=8, nz=7)
    A = pr.to_csr(st)
    n, nc = A.shape[0], 60
    rows, cols = [], []
    for i in range(n):
        k = 40 if i % 97 == 0 else int(rng.integers(1, 6))
        c = rng.choice(nc, size=k, replace=False)
        rows += [i] * k
        cols += list(c)
    P = sp.csr_matrix((rng.uniform(-1, 1, len(rows)), (rows, cols)), shape=(n, nc))
    Ac = solver.galerkin(A, P)
    Aco = sa.galerkin(A, P)
    assert max_abs_diff(Ac, Aco) <= 1e-13 * np.abs(Aco.data).max()
    Ac2 = solver.galerkin(A, P)
    assert np.array_equal(Ac.data, Ac2.data)


def test_galerkin_wide_rows_and_row_limit(solver):
    # rows of 800 distinct columns take the wide form of the product kernels
    from paper_2407_09848_gb300.amgps import AmgpsError
    n = 800
    rng = np.random.default_rng(1)
    Q = rng.uniform(-1, 1, (n, n))
    A = sp.csr_matrix(Q @ Q.T + n * np.eye(n))
    P = sp.csr_matrix(rng.uniform(-1, 1, (n, 40)))
    Ac = solver.galerkin(A, P)
    Aco = sa.galerkin(A, P)
    assert max_abs_diff(Ac, Aco) <= 1e-13 * np.abs(Aco.data).max()
    # P = I: both products have rows of 800 columns; I^T A I = A exactly
    assert max_abs_diff(solver.galerkin(A, sp.identity(n, format="csr")), A) == 0.0
    # products with at most 16384 columns take the dense-accumulator form: a
    # row of 7000 columns is fine there (I^T B I = B exactly)
    m = 7000
    B = sp.identity(m, format="lil")
    B[0, :] = 1.0
    B = sp.csr_matrix(B)
    assert max_abs_diff(solver.galerkin(B, sp.identity(m, format="csr")), B) == 0.0
    # wider products use the hashed forms: a row of 20000 distinct columns
    # exceeds their limit (6144): AMGPS_E_ARG, and the context stays usable
    m = 20000
    B = sp.identity(m, format="lil")
    B[0, :] = 1.0
    with pytest.raises(AmgpsError) as ei:
        solver.galerkin(sp.csr_matrix(B), sp.identity(m, format="csr"))
    assert ei.value.name == "AMGPS_E_ARG"
    st = pr.poisson(6)
    (agg, nc, _), = pr.geometric_aggregates(st.shape, coarse_max=64)
    P, Ac, _ = solver.sa_level(pr.to_csr(st), agg, nc)
    assert Ac.shape == (nc, nc)


@pytest.fixture(scope="module")
def sa_case(torch_cuda, solver):
    # oracle-built SA hierarchy (host), loaded through the general-P path
    st = pr.varcoef(20, 1.0, 4.0, seed=11, ny=18, nz=13)
    levels = pr.geometric_aggregates(st.shape, coarse_max=200)
    As, Ps, _ = sa.sa_hierarchy(pr.to_csr(st), [a for a, _, _ in levels],
                                [nc for _, nc, _ in levels])
    from paper_2407_09848_gb300.amgps import Solver
    S = Solver().load(As, Ps)
    return torch_cuda, As, Ps, S


@pytest.mark.parametrize("kind,k", [("cheb4_opt", 4), ("cheb1_opt", 3), ("l1jacobi", 2)])
def test_vcycle_general_p_matches_oracle(sa_case, kind, k):
    torch, As, Ps, S = sa_case
    S.set_smoother(-1, kind, k)
    ora = OracleAMG(As, Ps, SmootherSpec(kind, k))
    r = pr.vec_uniform(As[0].shape[0], seed=3)
    z = torch.empty(As[0].shape[0], dtype=torch.float64, device="cuda")
    S.vcycle(dev(torch, r), z)
    zo = ora.vcycle(r)
    assert np.linalg.norm(z.cpu().numpy() - zo) <= 1e-12 * np.linalg.norm(zo)
    S.set_smoother(-1, "cheb4_opt", 4)


def test_pcg_general_p_iterations_identical(sa_case):
    torch, As, Ps, S = sa_case
    b = pr.rhs_uniform(As[0].shape[0], seed=0)
    x = torch.empty(As[0].shape[0], dtype=torch.float64, device="cuda")
    it, rel = S.pcg(dev(torch, b), x, rtol=1e-10)
    _, ito, _, _ = OracleAMG(As, Ps, SmootherSpec("cheb4_opt", 4)).pcg(b, rtol=1e-10)
    assert it == ito and rel <= 1e-10


def test_vcycle_backward_general_p(sa_case):
    torch, As, Ps, S = sa_case
    k = 3
    rng = np.random.default_rng(9)
    betas = 1 + 0.2 * rng.uniform(-1, 1, (len(As) - 1, k))
    specs = []
    for l in range(len(As) - 1):
        S.set_smoother(l, "weights", k, weights=betas[l])
        specs.append(SmootherSpec("weights", k, beta=betas[l]))
    r, gz = rng.uniform(-1, 1, (2, As[0].shape[0]))
    gr, gw = S.vcycle_backward(dev(torch, r), dev(torch, gz))
    rr, rw = vcycle_backward(OracleAMG(As, Ps, specs), r, gz)
    assert np.linalg.norm(gr.cpu().numpy() - rr) <= 1e-12 * np.linalg.norm(rr)
    for l in range(len(As) - 1):
        assert np.max(np.abs(gw[l, :k] - rw[l])) <= 1e-12 * np.max(np.abs(rw[l]))
    S.set_smoother(-1, "cheb4_opt", 4)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_mixed_precision_general_p_converges(sa_case, prec):
    torch, As, Ps, _ = sa_case
    from paper_2407_09848_gb300.amgps import Solver
    S = Solver().load(As, Ps, prec=prec)
    b = pr.rhs_uniform(As[0].shape[0], seed=0)
    x = torch.empty(As[0].shape[0], dtype=torch.float64, device="cuda")
    it, rel = S.pcg(dev(torch, b), x, rtol=1e-9)
    true = np.linalg.norm(b - As[0] @ x.cpu().numpy()) / np.linalg.norm(b)
    assert rel <= 1e-9 and true <= 2e-9
    # with the paper's setting: coarse l1-Jacobi sweeps run in the mixed
    # engine, one-reduction flexible CG outside
    S.set_coarse_sweeps(30)
    S.set_flexible("fcg1")
    it2, rel2 = S.pcg(dev(torch, b), x, rtol=1e-9)
    true2 = np.linalg.norm(b - As[0] @ x.cpu().numpy()) / np.linalg.norm(b)
    assert rel2 <= 1e-9 and true2 <= 2e-9 and it2 <= 2 * it
    S.close()


@pytest.mark.parametrize("grid", [32, 64])
def test_device_built_sa_hierarchy_pcg(solver, grid):
    # hierarchy built on the GPU; iteration count equal to the oracle's on the
    # oracle-built hierarchy
    torch = pytest.importorskip("torch")
    from paper_2407_09848_gb300.amgps import Solver
    st = pr.poisson(grid)
    levels = pr.geometric_aggregates(st.shape, coarse_max=512)
    As, Ps, _ = solver.sa_hierarchy(pr.to_csr(st), levels)
    Aso, Pso, _ = sa.sa_hierarchy(pr.to_csr(st), [a for a, _, _ in levels],
                                  [nc for _, nc, _ in levels])
    for X, Y in zip(As, Aso):
        assert max_abs_diff(X, Y) <= 1e-12 * np.abs(Y.data).max()
    S = Solver().load(As, Ps)
    b = pr.rhs_uniform(As[0].shape[0], seed=0)
    x = torch.empty(As[0].shape[0], dtype=torch.float64, device="cuda")
    it, rel = S.pcg(dev(torch, b), x, rtol=1e-8)
    _, ito, _, _ = OracleAMG(Aso, Pso, SmootherSpec("cheb4_opt", 4)).pcg(b, rtol=1e-8)
    assert it == ito and rel <= 1e-8
    S.close()


@pytest.mark.parametrize("grid", [32, 64])
def test_paper_setting_iterations_match_oracle(solver, grid):
    # Sec. 4's solver setting on the device-built SA hierarchy: 30 l1-Jacobi
    # coarse sweeps, one-reduction flexible CG, tolerance 1e-7; counts equal
    # the oracle's on its own host-built hierarchy
    torch = pytest.importorskip("torch")
    from paper_2407_09848_gb300.amgps import Solver
    st = pr.poisson(grid)
    levels = pr.geometric_aggregates(st.shape, coarse_max=512)
    As, Ps, _ = solver.sa_hierarchy(pr.to_csr(st), levels)
    Aso, Pso, _ = sa.sa_hierarchy(pr.to_csr(st), [a for a, _, _ in levels],
                                  [nc for _, nc, _ in levels])
    S = Solver().load(As, Ps)
    S.set_coarse_sweeps(30)
    S.set_flexible("fcg1")
    b = pr.rhs_uniform(As[0].shape[0], seed=0)
    x = torch.empty(As[0].shape[0], dtype=torch.float64, device="cuda")
    for kind, k in (("cheb4_opt", 4), ("cheb1_opt", 4), ("l1jacobi", 4)):
        S.set_smoother(-1, kind, k)
        it, rel = S.pcg(dev(torch, b), x, rtol=1e-7)
        xo, ito, _, _ = OracleAMG(Aso, Pso, SmootherSpec(kind, k), coarse_sweeps=30).fcg1(b, rtol=1e-7)
        assert it == ito and rel <= 1e-7, (kind, it, ito)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
    S.close()
