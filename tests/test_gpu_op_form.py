"""GPU parity of the stored-operator form of the polynomial smoothers.

On FP64 levels of at least 131,072 rows the library evaluates each
polynomial smoother backwards (Clenshaw's scheme, one stored operator
tau I - sigma M^{-1} A per step).  It is the same polynomial as the forward
recurrences of Sec. 2.1 (Eq. polsmoother, Eq. polsmootheropt) and Sec. 2.2
(Algorithm 1), so it must meet the oracle at the FP64 tolerance of every
smoother application (relative 2-norm and largest element <= 1e-12), give
identical PCG iteration counts, and run the same bits through the TMA-fed and
the direct kernels.  Two levels just pass the 608-tile threshold of the
TMA-fed kernel (a ragged last slice; a 512-wide grid whose +-nx offsets share
one window); a third (64^3) takes the form through the direct kernel only.
"""
import numpy as np
import pytest

from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec, l1_diag, smooth
from paper_2407_09848_gb300 import problems as pr
from parity import assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-12
GRIDS = {
    # 81 x 72 x 63 = 367,416 rows: 717 planned tiles, ragged last slice
    "varcoef81": lambda: pr.varcoef(81, 1.0, 4.0, seed=5, ny=72, nz=63),
    # 512 x 24 x 28 = 344,064 rows: 672 tiles, merged +-nx window
    "poisson512": lambda: pr.poisson(512, 24, 28),
    # 64^3 = 262,144 rows: 512 tiles, below the TMA threshold (direct kernel)
    "varcoef64": lambda: pr.varcoef(64, 1.0, 4.0, seed=9),
}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module", params=sorted(GRIDS))
def case(request, torch_cuda):
    from paper_2407_09848_gb300.amgps import Solver, tma_plan_stats
    H = pr.build_hierarchy(GRIDS[request.param](), coarse_max=512)
    tiles = tma_plan_stats(H.levels[0].A, "f64")[0]
    assert (tiles < 4 * 152) == (request.param == "varcoef64")
    S = Solver().load(H.A, H.P)
    return request.param, H, S


def dev(torch, v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()


SPECS = [("cheb4_opt", 2), ("cheb4_opt", 3), ("cheb4_opt", 4), ("cheb4_opt", 6),
         ("cheb4_opt", 16), ("cheb4", 3), ("weights", 4), ("cheb1", 2), ("cheb1", 4),
         ("cheb1_opt", 3), ("l1jacobi", 2), ("l1jacobi", 5)]


def set_spec(S, kind, k):
    """The level-0 smoother of the case and the oracle's spec of it."""
    from paper_2407_09848_gb300.amgps import opt4_weights
    if kind == "weights":
        w = [1.2, 0.8, 1.1, 1.4][:k]
        S.set_smoother(0, "weights", k, weights=w)
        return SmootherSpec("weights", k, beta=np.array(w))
    if kind == "cheb1":
        S.set_smoother(0, "cheb1", k, rho=1.05)
        return SmootherSpec("cheb1", k, rho=1.05)
    S.set_smoother(0, kind, k)
    beta = opt4_weights(k) if kind == "cheb4_opt" else None
    return SmootherSpec(kind, k, beta=beta)


def run_smooth(torch, S, kind, k, b, x0, zero, form):
    S.set_step_form(form)
    x = x0.clone()
    S.profile(True)
    S.profile_read(0, reset=True)
    S.smooth(0, kind, k, b, x, x_is_zero=zero)
    S.synchronize()
    flops = S.profile_flops(0)
    launches = S.profile_read(0, reset=True)[0]
    S.profile(False)
    return x, flops, launches


@pytest.mark.parametrize("kind,k", SPECS, ids=lambda v: str(v))
def test_op_form_smooth_matches_oracle(torch_cuda, case, kind, k):
    torch = torch_cuda
    name, H, S = case
    A = H.levels[0].A
    n = A.shape[0]
    rng = np.random.default_rng(7 + k)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    spec = set_spec(S, kind, k)
    M = l1_diag(A)
    try:
        for zero in (True, False):
            ref = smooth(A, b, None if zero else x0, spec, M=M)
            x1, f1, n1 = run_smooth(torch, S, kind, k, dev(torch, b), dev(torch, x0), zero, 1)
            x0f, f0, n0 = run_smooth(torch, S, kind, k, dev(torch, b), dev(torch, x0), zero, 0)
            assert_parity(x1.cpu().numpy(), ref, TOL, (name, kind, k, zero, "operators"))
            assert_parity(x0f.cpu().numpy(), ref, TOL, (name, kind, k, zero, "recurrence"))
            # the forms ran: k - 1 operator steps (+ the s0 step from x0) against
            # the recurrence's k - 1 (+ 1), with fewer flops
            assert n1 == (k - 1 if zero else k), (n1, k, zero)
            assert f1 < f0
            assert not torch.equal(x1, x0f)
    finally:
        S.set_step_form(1)
        S.set_smoother(0, "cheb4_opt", 4)


@pytest.mark.parametrize("kind,k", [("cheb4_opt", 4), ("cheb4_opt", 5), ("cheb4", 2),
                                    ("cheb1", 3), ("weights", 3)], ids=lambda v: str(v))
def test_op_form_tma_equals_direct(torch_cuda, case, kind, k):
    torch = torch_cuda
    name, H, S = case
    n = H.levels[0].A.shape[0]
    rng = np.random.default_rng(3 * k)
    b, x0 = dev(torch, rng.uniform(-1, 1, n)), dev(torch, rng.uniform(-1, 1, n))
    set_spec(S, kind, k)
    try:
        for zero in (True, False):
            outs = []
            for tma in (True, False):
                S.set_tma(tma)
                x = x0.clone()
                S.smooth(0, kind, k, b, x, x_is_zero=zero)
                outs.append(x)
            S.synchronize()
            assert torch.equal(outs[0], outs[1]), (name, kind, k, zero)
    finally:
        S.set_tma(True)
        S.set_smoother(0, "cheb4_opt", 4)


def test_op_form_vcycle_and_pcg(torch_cuda, case):
    torch = torch_cuda
    name, H, S = case
    A = H.levels[0].A
    n = A.shape[0]
    S.set_smoother(-1, "cheb4_opt", 4)
    ora = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4))
    rng = np.random.default_rng(21)
    r = rng.uniform(-1, 1, n)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    S.profile(True)
    S.profile_read(0, reset=True)
    S.vcycle(dev(torch, r), z)
    S.synchronize()
    flops = S.profile_flops(0)
    inst = S.profile_fp64_inst(0)
    launches, _, _ = S.profile_read(0, reset=True)
    S.profile(False)
    assert_parity(z.cpu().numpy(), ora.vcycle(r), TOL, (name, "vcycle"))
    # a k = 4 cycle on level 0: three steps from zero, the s0 step and three
    # more after the prolongation; flops 14 nnz + 7 n (see amgps_profile_flops),
    # FP64 instructions 7 x stored entries + 6 n (vector terms 0, 1, 2 from
    # zero; 1, 0, 1, 1 after the prolongation)
    assert launches == 7
    assert flops == 14.0 * A.nnz + 7.0 * n
    assert inst == 7.0 * S.level_info(0)[2] + 6.0 * n
    b = rng.uniform(-1, 1, n)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    it1, rel1 = S.pcg(dev(torch, b), x, rtol=1e-8)
    xs = x.cpu().numpy()
    _, it_ora, _, _ = ora.pcg(b, rtol=1e-8)
    S.set_step_form(0)
    try:
        it0, _ = S.pcg(dev(torch, b), x, rtol=1e-8)
    finally:
        S.set_step_form(1)
    assert it1 == it_ora == it0, (it1, it_ora, it0)
    assert np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8


def test_op_form_falls_back_when_operators_do_not_fit(torch_cuda, case):
    # a level whose stored operators would pass the allocation limit keeps the
    # recurrence form (same bits as form 0) and reports no error; without the
    # limit the operators are built.  A fresh context: the load builds the
    # three operators of the default k = 4 (arrays are kept for reuse, so a
    # context that already ran a higher degree would need no allocation).
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    name, H, _ = case
    n = H.levels[0].A.shape[0]
    rng = np.random.default_rng(5)
    b, x0 = dev(torch, rng.uniform(-1, 1, n)), dev(torch, rng.uniform(-1, 1, n))
    S = Solver().load(H.A, H.P)
    try:
        S.set_alloc_limit(1)  # every further allocation fails
        S.set_smoother(0, "cheb4_opt", 8)  # 7 operators: more than the 3 built at load
        xa, _, _ = run_smooth(torch, S, "cheb4_opt", 8, b, x0, False, 1)
        xb, _, _ = run_smooth(torch, S, "cheb4_opt", 8, b, x0, False, 0)
        assert torch.equal(xa, xb)
        S.set_alloc_limit(0)
        S.set_smoother(0, "cheb4_opt", 8)
        xc, _, nc = run_smooth(torch, S, "cheb4_opt", 8, b, x0, False, 1)
        assert nc == 8 and not torch.equal(xc, xb)
    finally:
        S.close()


def test_step_form_option_values(torch_cuda, case):
    from paper_2407_09848_gb300.amgps import AmgpsError
    _, _, S = case
    for bad in (-1, 2):
        with pytest.raises(AmgpsError) as e:
            S.set_step_form(bad)
        assert e.value.name == "AMGPS_E_ARG"
    S.set_step_form(1)


def test_op_form_on_explicit_slices(torch_cuda):
    # a non-stencil SPD matrix large enough for the stored-operator form:
    # random symmetric pattern (explicit SELL slices, the operators' diagonal
    # found by column), one warp per slice (direct kernel), two levels
    import scipy.sparse as sp
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    rng = np.random.default_rng(31)
    n = 1 << 18
    m = 4 * n  # random off-diagonal entries (duplicates and the diagonal merge below)
    R = sp.coo_matrix((rng.uniform(0.0, 1.0, m), (rng.integers(0, n, m), rng.integers(0, n, m))),
                      shape=(n, n)).tocsr()
    R.setdiag(0.0)
    R.eliminate_zeros()
    R = R + R.T
    R.data = -np.abs(R.data)
    d = np.asarray(abs(R).sum(axis=1)).ravel() + rng.uniform(0.1, 1.0, n)
    A0 = (R + sp.diags(d)).tocsr()
    A0.sort_indices()
    agg = (rng.permutation(n) // 256).astype(np.int32)  # 1024 aggregates
    P0 = sp.csr_matrix((np.ones(n), agg, np.arange(n + 1)), shape=(n, 1024))
    A1 = (P0.T @ A0 @ P0).tocsr()
    A1.sort_indices()
    S = Solver().load([A0, A1], [P0])
    M = l1_diag(A0)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    try:
        for kind, k in (("cheb4_opt", 4), ("cheb1_opt", 3), ("l1jacobi", 3)):
            spec = set_spec(S, kind, k)
            for zero in (True, False):
                ref = smooth(A0, b, None if zero else x0, spec, M=M)
                x1, _, n1 = run_smooth(torch, S, kind, k, dev(torch, b), dev(torch, x0), zero, 1)
                x0f, _, _ = run_smooth(torch, S, kind, k, dev(torch, b), dev(torch, x0), zero, 0)
                assert_parity(x1.cpu().numpy(), ref, TOL, ("explicit", kind, k, zero))
                assert n1 == (k - 1 if zero else k) and not torch.equal(x1, x0f)
            ora = OracleAMG([A0, A1], [P0], spec)
            z = torch.empty(n, dtype=torch.float64, device="cuda")
            S.vcycle(dev(torch, b), z)
            assert_parity(z.cpu().numpy(), ora.vcycle(b), TOL, ("explicit vcycle", kind, k))
    finally:
        S.close()
