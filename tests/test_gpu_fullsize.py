"""Element-wise parity at the benchmark's full size (256^3 Poisson, FP64, the
TMA-fed kernels the benchmark times): one smoother application per kind and
one V-cycle against the oracle, whole vectors compared by their relative
2-norm and by their largest element-wise difference, and single steps compared
region by region on the rows of the first and last pipelined tile and of the
slices the TMA plan leaves to direct loads."""
import numpy as np
import pytest

from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec, l1_diag, smooth
from paper_2407_09848_gb300 import problems as pr
from parity import assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def full():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    from paper_2407_09848_gb300.amgps import Solver
    build.build()
    H = pr.build_hierarchy(pr.poisson(256), coarse_max=512)
    return torch, H, Solver().load(H.A, H.P)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind,k", [("cheb4_opt", 4), ("cheb1_opt", 4), ("cheb4", 3)])
def test_smoother_full_size(full, kind, k):
    torch, H, S = full
    A = H.A[0]
    n = A.shape[0]
    rng = np.random.default_rng(17)
    b, x0 = rng.uniform(-1, 1, (2, n))
    M = l1_diag(A)
    for start in (None, x0):
        x = torch.zeros(n, dtype=torch.float64, device="cuda") if start is None else \
            torch.from_numpy(start.copy()).cuda()
        S.smooth(0, kind, k, torch.from_numpy(b).cuda(), x, x_is_zero=start is None)
        xo = smooth(A, b, start, SmootherSpec(kind, k), M=M)
        assert_parity(x.cpu().numpy(), xo, TOL, kind, k, start is None)


def test_vcycle_full_size(full):
    torch, H, S = full
    S.set_smoother(-1, "cheb4_opt", 4)
    n = H.A[0].shape[0]
    r = pr.vec_uniform(n, seed=23)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    S.vcycle(torch.from_numpy(r).cuda(), z)
    zo = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4)).vcycle(r)
    assert_parity(z.cpu().numpy(), zo, TOL)


@pytest.mark.parametrize("k,from_zero", [(1, False), (2, True)])
def test_single_step_tile_edges(full, k, from_zero):
    """One fused step (degree 1 from x0, or the one step after the first
    elementwise step from zero): every row of the first and last TMA tile and
    of the leftover slices against the oracle, each region on its own."""
    from paper_2407_09848_gb300.amgps import tma_plan
    torch, H, S = full
    A = H.A[0]
    n = A.shape[0]
    plan = tma_plan(A, "f64")
    rows = plan["rows"]
    first, last = int(plan["tiles"][:, 0].min()), int(plan["tiles"][:, 0].max())
    gen_rows = (plan["gen"].astype(np.int64)[:, None] * 32 + np.arange(32)).ravel()
    gen_rows = gen_rows[gen_rows < n]
    assert len(plan["tiles"]) >= 4 * 152 and gen_rows.size > 0
    rng = np.random.default_rng(29)
    b, x0 = rng.uniform(-1, 1, (2, n))
    x = torch.zeros(n, dtype=torch.float64, device="cuda") if from_zero else \
        torch.from_numpy(x0.copy()).cuda()
    S.smooth(0, "cheb4_opt", k, torch.from_numpy(b).cuda(), x, x_is_zero=from_zero)
    got = x.cpu().numpy()
    ref = smooth(A, b, None if from_zero else x0, SmootherSpec("cheb4_opt", k), M=l1_diag(A))
    for name, idx in (("first tile", np.arange(first, first + rows)),
                      ("last tile", np.arange(last, min(last + rows, n))),
                      ("leftover slices", gen_rows)):
        assert_parity(got[idx], ref[idx], TOL, name, k, from_zero)
    assert_parity(got, ref, TOL, "all rows", k, from_zero)
