"""Element-wise parity at the benchmark's full size (256^3 Poisson, FP64, the
TMA-fed kernels the benchmark times): one smoother application per kind and
one V-cycle against the oracle, whole vectors compared."""
import numpy as np
import pytest

from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec, l1_diag, smooth
from paper_2407_09848_gb300 import problems as pr

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
        assert rel(x.cpu().numpy(), xo) <= TOL, (kind, k, start is None)


def test_vcycle_full_size(full):
    torch, H, S = full
    S.set_smoother(-1, "cheb4_opt", 4)
    n = H.A[0].shape[0]
    r = pr.vec_uniform(n, seed=23)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    S.vcycle(torch.from_numpy(r).cuda(), z)
    zo = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4)).vcycle(r)
    assert rel(z.cpu().numpy(), zo) <= TOL
