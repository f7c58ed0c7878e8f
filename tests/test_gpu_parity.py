"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerance: relative 2-norm difference <= 1e-12 per FP64 smoother application
and per V-cycle, and the largest element-wise difference <= 1e-12 of the
oracle's largest element; identical PCG iteration counts.  Inputs are seeded
(problems.py); sizes span many 32-row slices with a ragged last slice.
"""
import numpy as np
import pytest

from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec, power_lambda, smooth
from paper_2407_09848_gb300 import problems as pr
from parity import assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    build.build()
    return torch


def to_dev(torch, v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()


def to_np(t):
    return t.detach().cpu().numpy()


class Case:
    def __init__(self, torch, st, coarse_max=512, prec="f64"):
        from paper_2407_09848_gb300.amgps import Solver
        self.H = pr.build_hierarchy(st, coarse_max=coarse_max)
        self.A, self.P = self.H.A, self.H.P
        self.S = Solver().load(self.A, self.P, prec=prec)
        self.torch = torch


@pytest.fixture(scope="module")
def ragged(torch_cuda):
    # 20 x 18 x 13 = 4680 rows (146.25 slices): ragged tail on every level
    return Case(torch_cuda, pr.varcoef(20, 1.0, 4.0, seed=11, ny=18, nz=13), coarse_max=100)


@pytest.fixture(scope="module")
def poisson32(torch_cuda):
    return Case(torch_cuda, pr.poisson(32))


KINDS = ["l1jacobi", "cheb4", "cheb4_opt", "weights", "cheb1_opt", "cheb1"]


def weights_for(k, seed):
    return 1.0 + 0.25 * np.random.default_rng(seed).uniform(-1, 1, k)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("level", [0, 1])
def test_smoother_parity(ragged, kind, k, level):
    torch = ragged.torch
    S, A = ragged.S, ragged.A[level]
    n = A.shape[0]
    rng = np.random.default_rng(100 + 7 * k + level)
    b = rng.uniform(-1, 1, n)
    x0 = rng.uniform(-1, 1, n)
    rho = 1.0
    beta = None
    if kind == "weights":
        beta = weights_for(k, k)
        S.set_smoother(level, "weights", k, weights=beta)
    elif kind == "cheb1":
        rho = 1.1 * power_lambda(A, pr.vec_uniform(n, seed=0), iters=10)
        S.set_smoother(level, "cheb1", k, rho=rho)
    else:
        S.set_smoother(level, "cheb4_opt", 4)
    spec = SmootherSpec(kind, k, beta=beta, rho=rho)
    for start in (None, x0):
        bd = to_dev(torch, b)
        xd = torch.zeros(n, dtype=torch.float64, device="cuda") if start is None else to_dev(torch, start)
        S.smooth(level, kind, k, bd, xd, x_is_zero=start is None)
        got = to_np(xd)
        ref = smooth(A, b, start, spec)
        assert_parity(got, ref, TOL, kind, k, level, start is None)
    S.set_smoother(-1, "cheb4_opt", 4)


@pytest.mark.parametrize("level", [0, 1])
def test_power_iteration_parity(ragged, level):
    torch = ragged.torch
    A = ragged.A[level]
    v0 = pr.vec_uniform(A.shape[0], seed=0)
    lam = ragged.S.estimate_lambda(level, to_dev(torch, v0), iters=10)
    ref = power_lambda(A, v0, iters=10)
    assert abs(lam - ref) <= TOL * ref
    assert 0.0 < lam <= 1.0 + 1e-12


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("k", [1, 2, 4])
def test_vcycle_parity(ragged, kind, k):
    torch = ragged.torch
    S, A, P = ragged.S, ragged.A, ragged.P
    specs = []
    for l in range(len(A) - 1):
        if kind == "weights":
            beta = weights_for(k, 50 + l)
            S.set_smoother(l, kind, k, weights=beta)
            specs.append(SmootherSpec(kind, k, beta=beta))
        elif kind == "cheb1":
            rho = 1.1 * power_lambda(A[l], pr.vec_uniform(A[l].shape[0], seed=0), iters=10)
            S.set_smoother(l, kind, k, rho=rho)
            specs.append(SmootherSpec(kind, k, rho=rho))
        else:
            S.set_smoother(l, kind, k)
            specs.append(SmootherSpec(kind, k))
    ora = OracleAMG(A, P, specs)
    r = pr.rhs_uniform(A[0].shape[0], seed=3)
    z = torch.empty(A[0].shape[0], dtype=torch.float64, device="cuda")
    S.vcycle(to_dev(torch, r), z)
    ref = ora.vcycle(r)
    assert_parity(to_np(z), ref, TOL, kind, k)
    # replay through the captured graph gives the identical result
    z2 = torch.empty_like(z)
    S.vcycle(to_dev(torch, r), z2)
    assert torch.equal(z, z2)
    S.set_smoother(-1, "cheb4_opt", 4)


@pytest.mark.parametrize("kind,k", [("cheb4_opt", 4), ("cheb4", 3), ("cheb1_opt", 2), ("l1jacobi", 2)])
def test_pcg_iterations_identical_32(poisson32, kind, k):
    torch = poisson32.torch
    S, A, P = poisson32.S, poisson32.A, poisson32.P
    S.set_smoother(-1, kind, k)
    ora = OracleAMG(A, P, SmootherSpec(kind, k))
    b = pr.rhs_uniform(A[0].shape[0], seed=0)
    x = torch.empty(A[0].shape[0], dtype=torch.float64, device="cuda")
    it, relres = S.pcg(to_dev(torch, b), x, rtol=1e-8)
    xo, ito, relo, _ = ora.pcg(b, rtol=1e-8)
    assert it == ito, (it, ito)
    assert relres <= 1e-8 and abs(relres - relo) <= 1e-6 * relo
    assert rel(to_np(x), xo) <= 1e-9
    S.set_smoother(-1, "cheb4_opt", 4)


def test_pcg_iterations_identical_ragged(ragged):
    torch = ragged.torch
    S, A, P = ragged.S, ragged.A, ragged.P
    S.set_smoother(-1, "cheb4_opt", 3)
    ora = OracleAMG(A, P, SmootherSpec("cheb4_opt", 3))
    b = pr.rhs_uniform(A[0].shape[0], seed=5)
    x = torch.empty(A[0].shape[0], dtype=torch.float64, device="cuda")
    it, relres = S.pcg(to_dev(torch, b), x, rtol=1e-10)
    _, ito, _, _ = ora.pcg(b, rtol=1e-10)
    assert it == ito
    # bitwise reproducible: a second solve repeats every iteration exactly
    x2 = torch.empty_like(x)
    it2, rel2 = S.pcg(to_dev(torch, b), x2, rtol=1e-10)
    assert it2 == it and rel2 == relres and torch.equal(x, x2)
    S.set_smoother(-1, "cheb4_opt", 4)


def test_pcg_host_equals_device(poisson32):
    torch = poisson32.torch
    S = poisson32.S
    n = S.sizes[0]
    b = pr.rhs_uniform(n, seed=0)
    xd = torch.empty(n, dtype=torch.float64, device="cuda")
    it, r = S.pcg(to_dev(torch, b), xd)
    xh = np.zeros(n)
    it2, r2 = S.pcg_host(b.copy(), xh)
    assert it2 == it and r2 == r and np.array_equal(xh, to_np(xd))
    bp = torch.from_numpy(b.copy()).pin_memory()
    xp = torch.zeros(n, dtype=torch.float64).pin_memory()
    it3, r3 = S.pcg_host(bp, xp)
    assert it3 == it and np.array_equal(xp.numpy(), xh)


def test_explicit_slices_and_irregular_aggregates(torch_cuda):
    # a non-stencil SPD matrix: random sparse symmetric pattern, diagonally
    # dominant; random aggregates of sizes 1..11 -> explicit SELL slices and
    # children lists longer than the eight lanes of the restriction group
    import scipy.sparse as sp
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    rng = np.random.default_rng(9)
    n = 2000
    R = sp.random(n, n, density=0.004, random_state=9, format="csr")
    R = R + R.T
    R.data = -np.abs(R.data)
    d = np.asarray(abs(R).sum(axis=1)).ravel() + rng.uniform(0.1, 1.0, n)
    A0 = (R + sp.diags(d)).tocsr()
    A0.sort_indices()
    sizes = []
    tot = 0
    while tot < n:
        s = int(min(rng.integers(1, 12), n - tot))
        sizes.append(s)
        tot += s
    agg = np.repeat(np.arange(len(sizes)), sizes)
    rng.shuffle(agg)
    nc = len(sizes)
    P0 = sp.csr_matrix((np.ones(n), agg.astype(np.int32), np.arange(n + 1)), shape=(n, nc))
    A1 = (P0.T @ A0 @ P0).tocsr()
    A1.sort_indices()
    S = Solver().load([A0, A1], [P0])
    _, nnz, stored = S.level_info(0)
    assert stored >= nnz
    for kind in ("cheb4_opt", "cheb1_opt", "l1jacobi"):
        S.set_smoother(0, kind, 3)
        ora = OracleAMG([A0, A1], [P0], SmootherSpec(kind, 3))
        r = rng.uniform(-1, 1, n)
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        S.vcycle(to_dev(torch, r), z)
        assert_parity(to_np(z), ora.vcycle(r), TOL)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        it, _ = S.pcg(to_dev(torch, r), x, rtol=1e-9)
        _, ito, _, _ = ora.pcg(r, rtol=1e-9)
        assert it == ito


def test_single_level_and_tiny(torch_cuda):
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    for st in (pr.poisson(1), pr.poisson(3, 2, 1), pr.poisson(5)):
        H = pr.build_hierarchy(st, coarse_max=512)
        assert H.n_levels == 1
        S = Solver().load(H.A, H.P)
        n = H.levels[0].A.shape[0]
        b = pr.rhs_uniform(n, seed=1)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        it, relres = S.pcg(to_dev(torch, b), x, rtol=1e-12)
        assert it == 1 and relres <= 1e-12
        xd = np.linalg.solve(H.levels[0].A.toarray(), b)
        assert rel(to_np(x), xd) <= 1e-13
    # two levels with a 1-row coarsest level
    H = pr.build_hierarchy(pr.poisson(2), coarse_max=1)
    assert [lv.A.shape[0] for lv in H.levels] == [8, 1]
    S = Solver().load(H.A, H.P)
    ora = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4))
    r = pr.rhs_uniform(8, seed=2)
    z = torch.empty(8, dtype=torch.float64, device="cuda")
    S.vcycle(to_dev(torch, r), z)
    assert_parity(to_np(z), ora.vcycle(r), TOL)


def test_status_codes(torch_cuda):
    import scipy.sparse as sp
    from paper_2407_09848_gb300.amgps import AmgpsError, Solver
    torch = torch_cuda
    S = Solver()
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(AmgpsError) as e:
        S.pcg(b, x)
    assert e.value.name == "AMGPS_E_STATE"
    H = pr.build_hierarchy(pr.poisson(4), coarse_max=8)
    bad = H.A[0].copy()
    bad.data[0] = -1.0  # negative diagonal
    with pytest.raises(AmgpsError) as e:
        S.load([bad] + H.A[1:], H.P)
    assert e.value.name == "AMGPS_E_NOT_SPD"
    P2 = sp.csr_matrix(H.P[0])[:, :-1]  # one coarse column short of A_1
    with pytest.raises(AmgpsError) as e:
        S.load(H.A, [P2])
    assert e.value.name == "AMGPS_E_ARG"
    indef = sp.csr_matrix(np.array([[1.0, 2.0], [2.0, 1.0]]))
    with pytest.raises(AmgpsError) as e:
        S.load([indef], [])
    assert e.value.name == "AMGPS_E_NOT_SPD"
    S.load(H.A, H.P)
    n = H.A[0].shape[0]
    b = to_dev(torch, pr.rhs_uniform(n, seed=0))
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(AmgpsError) as e:
        S.pcg(b, x, rtol=1e-14, maxit=1)
    assert e.value.name == "AMGPS_E_NOCONV"
    it, rr = S.pcg(b, x, rtol=1e-14, maxit=1, raise_on_noconv=False)
    assert it == 1 and rr > 1e-14
    with pytest.raises(AmgpsError) as e:
        S.smooth(0, "weights", 3, b, x)
    assert e.value.name == "AMGPS_E_STATE"
    with pytest.raises(AmgpsError) as e:
        S.smooth(len(H.A) - 1, "cheb4", 2, b[:8], x[:8])
    assert e.value.name == "AMGPS_E_ARG"
    with pytest.raises(AmgpsError):
        S.set_smoother(0, "cheb4", 17)
    bz = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, rr = S.pcg(bz, x)
    assert it == 0 and torch.count_nonzero(x) == 0


def test_profile_counts(poisson32):
    torch = poisson32.torch
    S = poisson32.S
    n = S.sizes[0]
    S.profile(True)
    for c in range(3):
        S.profile_read(c, reset=True)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    it, _ = S.pcg(to_dev(torch, pr.rhs_uniform(n, seed=0)), x)
    S.profile(False)
    n_step, ms, by = S.profile_read(0, reset=True)
    # CHEB4_OPT k=4 from a zero start: 3 SpMV steps pre, 4 post per V-cycle
    assert n_step == 7 * it and ms > 0 and by > 0
    n_sp, ms_sp, _ = S.profile_read(2, reset=True)
    assert n_sp == it and ms_sp > 0


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("grid", ["varcoef48", "poisson512"])
def test_tma_step_equals_direct_step(torch_cuda, prec, grid):
    # the TMA-fed kernel evaluates the same arithmetic in the same order as the
    # direct-load kernel: results must agree bit for bit (a 512-wide grid plans
    # its -nx..+nx offsets as one window)
    from paper_2407_09848_gb300.amgps import Solver, tma_plan_stats
    torch = torch_cuda
    st = (pr.varcoef(48, 1.0, 4.0, seed=3, ny=40, nz=36) if grid == "varcoef48"
          else pr.poisson(512, 24, 20))
    H = pr.build_hierarchy(st, coarse_max=512)
    assert tma_plan_stats(H.levels[0].A, prec)[0] > 0
    S = Solver().load(H.A, H.P, prec=prec)
    rng = np.random.default_rng(12)
    for level in (0, 1):
        n = H.levels[level].A.shape[0]
        b = to_dev(torch, rng.uniform(-1, 1, n))
        x0 = to_dev(torch, rng.uniform(-1, 1, n))
        for kind, k in [("cheb4_opt", 4), ("cheb4", 2), ("cheb1_opt", 3), ("l1jacobi", 3),
                        ("cheb1", 2), ("weights", 3)]:
            if kind == "weights" and level != 0:
                continue
            if kind == "cheb1":
                S.set_smoother(level, "cheb1", k, rho=1.05)
            if kind == "weights":
                S.set_smoother(level, "weights", 3, weights=[1.1, 0.9, 1.3])
            for zero in (True, False):
                outs = []
                for tma in ("always", False):
                    S.set_tma(tma)
                    x = x0.clone()
                    S.smooth(level, kind, k, b, x, x_is_zero=zero)
                    outs.append(x)
                S.synchronize()
                assert torch.equal(outs[0], outs[1]), (prec, level, kind, k, zero)
    S.set_tma("always")
    z1 = torch.empty(H.levels[0].A.shape[0], dtype=torch.float64, device="cuda")
    z2 = torch.empty_like(z1)
    r = to_dev(torch, rng.uniform(-1, 1, H.levels[0].A.shape[0]))
    S.vcycle(r, z1)
    S.set_tma(False)
    S.vcycle(r, z2)
    S.synchronize()
    assert torch.equal(z1, z2)


@pytest.mark.parametrize("prec", ["f64", "bf16"])
def test_flexible_pcg_iterations_identical(torch_cuda, prec):
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    H = pr.build_hierarchy(pr.varcoef(24, 1.5, 4.0, seed=7), coarse_max=200)
    S = Solver().load(H.A, H.P, prec=prec)
    S.set_flexible(True)
    b = pr.rhs_uniform(H.A[0].shape[0], seed=2)
    x = torch.empty(H.A[0].shape[0], dtype=torch.float64, device="cuda")
    it, rel = S.pcg(to_dev(torch, b), x, rtol=1e-9)
    true = np.linalg.norm(b - H.A[0] @ to_np(x)) / np.linalg.norm(b)
    assert rel <= 1e-9 and true <= 2e-9
    if prec == "f64":
        _, ito, _, _ = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4)).pcg(b, rtol=1e-9,
                                                                            flexible=True)
        assert it == ito


@pytest.mark.parametrize("prec", ["f64", "bf16"])
def test_fcg1_iterations_identical(torch_cuda, prec):
    # the one-reduction flexible CG: FP64 iteration counts equal the oracle's,
    # x agrees with the oracle's iterate; BF16 smoothers still reach 1e-9
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    H = pr.build_hierarchy(pr.varcoef(24, 1.5, 4.0, seed=7), coarse_max=200)
    S = Solver().load(H.A, H.P, prec=prec)
    S.set_flexible("fcg1")
    b = pr.rhs_uniform(H.A[0].shape[0], seed=2)
    x = torch.empty(H.A[0].shape[0], dtype=torch.float64, device="cuda")
    it, rel = S.pcg(to_dev(torch, b), x, rtol=1e-9)
    true = np.linalg.norm(b - H.A[0] @ to_np(x)) / np.linalg.norm(b)
    assert rel <= 1e-9 and true <= 2e-9
    if prec == "f64":
        xo, ito, _, _ = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4)).fcg1(b, rtol=1e-9)
        assert it == ito
        assert np.linalg.norm(to_np(x) - xo) <= 1e-7 * np.linalg.norm(xo)
        # after two iterations (far from cancellation) the iterates agree to 1e-12
        it2, _ = S.pcg(to_dev(torch, b), x, rtol=1e-9, maxit=2, raise_on_noconv=False)
        xo2, _, _, _ = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4)).fcg1(b, rtol=1e-9,
                                                                               maxit=2)
        assert it2 == 2
        assert np.linalg.norm(to_np(x) - xo2) <= 1e-12 * np.linalg.norm(xo2)
    S.set_flexible("cg")
    it_cg, _ = S.pcg(to_dev(torch, b), x, rtol=1e-9)
    assert abs(it_cg - it) <= 1


def test_coarse_l1jacobi_sweeps(torch_cuda):
    # the paper's coarse solver (m l1-Jacobi sweeps from zero) against the
    # oracle: V-cycle, PCG counts, reverse mode; switching back restores the
    # dense coarse solve (the coarse-level graph is rebuilt)
    from oracle.adjoint import vcycle_backward
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    H = pr.build_hierarchy(pr.varcoef(20, 1.0, 4.0, seed=11, ny=18, nz=13), coarse_max=200)
    S = Solver().load(H.A, H.P)
    n = H.A[0].shape[0]
    r = pr.vec_uniform(n, seed=4)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    z0 = torch.empty_like(z)
    S.vcycle(to_dev(torch, r), z0)
    for m in (1, 30):
        S.set_coarse_sweeps(m)
        ora = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4), coarse_sweeps=m)
        S.vcycle(to_dev(torch, r), z)
        assert_parity(to_np(z), ora.vcycle(r), TOL)
        b = pr.rhs_uniform(n, seed=0)
        x = torch.empty_like(z)
        it, relres = S.pcg(to_dev(torch, b), x, rtol=1e-9)
        _, ito, _, _ = ora.pcg(b, rtol=1e-9)
        assert it == ito and relres <= 1e-9
    gz = pr.vec_uniform(n, seed=8)
    gr, _ = S.vcycle_backward(to_dev(torch, r), to_dev(torch, gz))
    rr, _ = vcycle_backward(OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4), coarse_sweeps=30), r, gz)
    assert rel(gr.cpu().numpy(), rr) <= TOL
    S.set_coarse_sweeps(0)
    S.vcycle(to_dev(torch, r), z)
    S.synchronize()
    assert torch.equal(z, z0)
    S.close()


def test_more_input_and_option_errors(torch_cuda):
    # every case is rejected on the host before a launch (no device fault)
    from paper_2407_09848_gb300.amgps import AmgpsError, Solver, lib
    torch = torch_cuda
    H = pr.build_hierarchy(pr.poisson(8), coarse_max=64)
    S = Solver().load(H.A, H.P)
    n = H.A[0].shape[0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    bn = to_dev(torch, pr.rhs_uniform(n, seed=0))
    bn[3] = float("nan")
    with pytest.raises(AmgpsError) as e:
        S.pcg(bn, x)
    assert e.value.name == "AMGPS_E_NAN"
    for opt, val in ((1, 3), (2, 3), (3, -1), (3, 1001), (9, 0)):
        assert lib().amgps_set_option(S._h, opt, val) == 1  # AMGPS_E_ARG
    # zero right-hand side through every outer CG form
    bz = torch.zeros(n, dtype=torch.float64, device="cuda")
    for form in ("cg", "flexible", "fcg1"):
        S.set_flexible(form)
        it, rr = S.pcg(bz, x)
        assert it == 0 and torch.count_nonzero(x) == 0
    S.set_flexible("cg")
    # smoothed aggregation: aggregate index out of range, empty aggregate
    A0 = pr.to_csr(pr.poisson(6))
    (agg, nc, _), = pr.geometric_aggregates((6, 6, 6), coarse_max=64)
    bad = agg.copy()
    bad[0] = nc
    with pytest.raises(AmgpsError) as e:
        S.sa_level(A0, bad, nc)
    assert e.value.name == "AMGPS_E_ARG"
    with pytest.raises(AmgpsError) as e:
        S.sa_level(A0, agg, nc + 1)  # coarse index nc has no fine point
    assert e.value.name == "AMGPS_E_ARG"
    # smoother-only PCG needs a level with a smoother
    H1 = pr.build_hierarchy(pr.poisson(3), coarse_max=512)
    S1 = Solver().load(H1.A, H1.P)
    b1 = to_dev(torch, pr.rhs_uniform(27, seed=1))
    x1 = torch.zeros(27, dtype=torch.float64, device="cuda")
    with pytest.raises(AmgpsError) as e:
        S1.pcg_smoother("cheb4_opt", 2, b1, x1)
    assert e.value.name == "AMGPS_E_ARG"
    S1.close()
    S.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_coarse_kernel_equals_launches(torch_cuda, prec):
    """The persistent kernel of the coarse levels gives the bits of their
    launched kernels: V-cycles of several kinds (and with the coarse-sweeps
    solver), and a PCG solve's iteration count and iterate.  It really runs:
    a V-cycle then launches one kernel for all levels below the first."""
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    # 43,200 rows: no level is large enough for the TMA-fed step, so every
    # level below the first runs in the persistent kernel
    H = pr.build_hierarchy(pr.varcoef(40, 1.0, 4.0, seed=5, ny=36, nz=30), coarse_max=64)
    assert H.n_levels >= 4
    on, off = Solver().load(H.A, H.P, prec=prec), Solver().load(H.A, H.P, prec=prec)
    on.set_coarse_kernel(True)
    off.set_coarse_kernel(False)
    n = H.A[0].shape[0]
    r = to_dev(torch, pr.rhs_uniform(n, seed=8))
    for kind, k, sweeps in [("cheb4_opt", 4, 0), ("cheb1_opt", 3, 0), ("l1jacobi", 2, 0),
                            ("cheb4", 2, 30)]:
        zs = []
        for S in (on, off):
            S.set_smoother(-1, kind, k)
            S.set_coarse_sweeps(sweeps)
            z = torch.empty(n, dtype=torch.float64, device="cuda")
            S.vcycle(r, z)       # builds the graph (and the persistent kernel)
            S.profile_read(3, reset=True)
            S.vcycle(r, z)
            torch.cuda.synchronize()
            zs.append((z, S.profile_read(3, reset=True)[0]))
        assert torch.equal(zs[0][0], zs[1][0]), (prec, kind, k, sweeps)
        assert zs[0][1] < zs[1][1], (zs[0][1], zs[1][1])
    for S in (on, off):
        S.set_smoother(-1, "cheb4_opt", 4)
        S.set_coarse_sweeps(0)
    xs = []
    for S in (on, off):
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        it, rel = S.pcg(r, x, rtol=1e-8)
        xs.append((it, rel, x))
    assert xs[0][0] == xs[1][0] and xs[0][1] == xs[1][1] and torch.equal(xs[0][2], xs[1][2])


def test_coarse_kernel_option_falls_back_on_general_transfers(torch_cuda):
    """A smoothed-aggregation hierarchy (general P, stored transfers) is not
    taken by the persistent kernel: with the option on, the V-cycle keeps its
    launches and gives the same bits and the same launch count."""
    from oracle.sa import sa_hierarchy
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    st = pr.poisson(24, 20, 18)
    A0 = pr.to_csr(st)
    levels = pr.geometric_aggregates(st.shape, coarse_max=60)
    As, Ps, _ = sa_hierarchy(A0, [lv[0] for lv in levels], [lv[1] for lv in levels])
    on, off = Solver().load(As, Ps), Solver().load(As, Ps)
    on.set_coarse_kernel(True)
    n = A0.shape[0]
    r = to_dev(torch, pr.rhs_uniform(n, seed=2))
    out = []
    for S in (on, off):
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        S.vcycle(r, z)
        S.profile_read(3, reset=True)
        S.vcycle(r, z)
        torch.cuda.synchronize()
        out.append((z, S.profile_read(3, reset=True)[0]))
    assert torch.equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_allocation_limit_reports_nomem_and_recovers(torch_cuda):
    """Failure injected on the host: a context limited to 1 MiB of device
    memory refuses a hierarchy with AMGPS_E_NOMEM before reaching the CUDA
    allocator, keeps no hierarchy (and none of the partial buffers), and
    loads and solves once the limit is lifted."""
    from paper_2407_09848_gb300.amgps import AmgpsError, Solver
    torch = torch_cuda
    H = pr.build_hierarchy(pr.poisson(24), coarse_max=100)
    Solver().load(H.A, H.P).close()   # the load's kernels are on the device now
    S = Solver()
    S.set_alloc_limit(1 << 20)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(AmgpsError) as e:
        S.load(H.A, H.P)
    assert e.value.name == "AMGPS_E_NOMEM" and "AMGPS_OPT_ALLOC_LIMIT" in str(e.value)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0   # the partial buffers were released
    with pytest.raises(AmgpsError) as e:
        S.level_info(0)
    assert e.value.name == "AMGPS_E_STATE"
    S.set_alloc_limit(0)
    S.load(H.A, H.P)
    n = H.A[0].shape[0]
    b = to_dev(torch, pr.rhs_uniform(n, seed=0))
    x = torch.empty_like(b)
    it, rel = S.pcg(b, x, rtol=1e-8)
    assert rel <= 1e-8 and it > 0
