"""Mixed precision (FP32 / BF16 matrix values on the smoother and transfer path,
FP32 V-cycle vectors, FP64 outer PCG and coarsest solve): errors against the
FP64 oracle are stated here as bounds, and PCG must still reach a true relative
residual of 1e-8."""
import numpy as np
import pytest

from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec, smooth
from paper_2407_09848_gb300 import problems as pr

pytestmark = pytest.mark.gpu

# stated per-application relative errors vs the FP64 oracle (2-norm)
BOUND = {"f32": 2e-6, "bf16": 2e-2}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    build.build()
    return torch


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module", params=["f32", "bf16"])
def mixed(request, torch_cuda):
    from paper_2407_09848_gb300.amgps import Solver
    H = pr.build_hierarchy(pr.varcoef(24, 1.0, 4.0, seed=21, ny=22, nz=20), coarse_max=200)
    return request.param, H, Solver().load(H.A, H.P, prec=request.param), torch_cuda


def test_mixed_smoother_and_vcycle_error(mixed):
    prec, H, S, torch = mixed
    n = H.levels[0].A.shape[0]
    b = pr.rhs_uniform(n, seed=4)
    spec = SmootherSpec("cheb4_opt", 4)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    S.smooth(0, "cheb4_opt", 4, torch.from_numpy(b).cuda(), x, x_is_zero=True)
    e_s = rel(x.cpu().numpy(), smooth(H.A[0], b, None, spec))
    z = torch.empty_like(x)
    S.vcycle(torch.from_numpy(b).cuda(), z)
    e_v = rel(z.cpu().numpy(), OracleAMG(H.A, H.P, spec).vcycle(b))
    print(f"{prec}: smoother rel err {e_s:.2e}, V-cycle rel err {e_v:.2e}")
    assert e_s <= BOUND[prec] and e_v <= BOUND[prec]
    assert e_s > 0  # the path really runs in reduced precision


def test_mixed_pcg_reaches_1e8(mixed):
    prec, H, S, torch = mixed
    n = H.levels[0].A.shape[0]
    b = pr.rhs_uniform(n, seed=0)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    it, relres = S.pcg(torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=200)
    true = np.linalg.norm(b - H.A[0] @ x.cpu().numpy()) / np.linalg.norm(b)
    _, it64, _, _ = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4)).pcg(b, rtol=1e-8)
    print(f"{prec}: PCG iterations {it} (FP64 oracle {it64}), relres {relres:.2e}, true {true:.2e}")
    assert relres <= 1e-8 and true <= 1.5e-8
    assert it <= it64 + 3
