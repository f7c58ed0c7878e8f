"""GPU reverse mode through the C-ABI against the oracle's reverse mode."""
import numpy as np
import pytest

from oracle.adjoint import smooth_backward, vcycle_backward
from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec
from paper_2407_09848_gb300 import problems as pr
from parity import assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def case():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    from paper_2407_09848_gb300.amgps import Solver
    build.build()
    H = pr.build_hierarchy(pr.varcoef(40, 1.0, 4.0, seed=13, ny=36, nz=30), coarse_max=200)
    return torch, H, Solver().load(H.A, H.P)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(torch, v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


@pytest.mark.parametrize("kind", ["weights", "cheb4_opt", "cheb4", "cheb1_opt", "l1jacobi"])
@pytest.mark.parametrize("k", [1, 3, 4])
@pytest.mark.parametrize("level", [0, 1])
def test_smooth_backward_matches_oracle(case, kind, k, level):
    torch, H, S = case
    A = H.A[level]
    n = A.shape[0]
    rng = np.random.default_rng(31 * k + level)
    b, x0, gx = rng.uniform(-1, 1, (3, n))
    beta = 1 + 0.2 * rng.uniform(-1, 1, k)
    if kind == "weights":
        S.set_smoother(level, "weights", k, weights=beta)
        spec = SmootherSpec("weights", k, beta=beta)
    else:
        spec = SmootherSpec(kind, k)
    for start in (None, x0):
        gb, gx0, gw = S.smooth_backward(level, kind, k, dev(torch, b),
                                        None if start is None else dev(torch, start),
                                        dev(torch, gx))
        rb, rx0, rw = smooth_backward(A, b, start, spec, gx)
        assert_parity(gb.cpu().numpy(), rb, TOL, "dL/db")
        assert_parity(gx0.cpu().numpy(), rx0, TOL, "dL/dx0")
        if rw is not None:
            assert np.max(np.abs(gw - rw)) <= TOL * np.max(np.abs(rw))
        else:
            assert np.all(gw == 0)
    S.set_smoother(-1, "cheb4_opt", 4)


@pytest.mark.parametrize("k", [2, 4])
def test_vcycle_backward_matches_oracle(case, k):
    torch, H, S = case
    rng = np.random.default_rng(5 + k)
    nl = H.n_levels
    betas = 1 + 0.2 * rng.uniform(-1, 1, (nl - 1, k))
    specs = []
    for l in range(nl - 1):
        S.set_smoother(l, "weights", k, weights=betas[l])
        specs.append(SmootherSpec("weights", k, beta=betas[l]))
    ora = OracleAMG(H.A, H.P, specs)
    n = H.A[0].shape[0]
    r, gz = rng.uniform(-1, 1, (2, n))
    gr, gw = S.vcycle_backward(dev(torch, r), dev(torch, gz))
    rr, rw = vcycle_backward(ora, r, gz)
    assert_parity(gr.cpu().numpy(), rr, TOL, "dL/dr")
    for l in range(nl - 1):
        assert np.max(np.abs(gw[l, :k] - rw[l])) <= TOL * np.max(np.abs(rw[l]))
        assert np.all(gw[l, k:] == 0)
    S.set_smoother(-1, "cheb4_opt", 4)


def test_autograd_gradcheck(case):
    torch, H, S = case
    from paper_2407_09848_gb300.autograd import SmootherFn, VCycleFn
    n = H.A[1].shape[0]
    rng = np.random.default_rng(2)
    b = dev(torch, rng.uniform(-1, 1, n)).requires_grad_()
    x0 = dev(torch, rng.uniform(-1, 1, n)).requires_grad_()
    beta = torch.tensor([1.05, 0.95, 1.2], dtype=torch.float64, requires_grad=True)
    f = lambda bb, xx, ww: SmootherFn.apply(bb, xx, ww, S, 1)
    assert torch.autograd.gradcheck(f, (b, x0, beta), eps=1e-6, atol=1e-8, rtol=1e-6,
                                    fast_mode=True)
    n0 = H.A[0].shape[0]
    r = dev(torch, rng.uniform(-1, 1, n0)).requires_grad_()
    betas = torch.from_numpy(1 + 0.1 * rng.uniform(-1, 1, (H.n_levels - 1, 2))).requires_grad_()
    g = lambda rr, bb: VCycleFn.apply(rr, bb, S)
    assert torch.autograd.gradcheck(g, (r, betas), eps=1e-6, atol=1e-8, rtol=1e-6, fast_mode=True)
    S.set_smoother(-1, "cheb4_opt", 4)
