"""The allocation-free smoother entry point (amgps_smooth_noalloc) against
amgps_smooth.

Some callers may not allocate device memory when they call the smoother (an
outside allocator owns the device memory, or allocation is forbidden in that
phase of their loop).  amgps_smooth_noalloc runs the same kernels with its work
vectors in a static device array of 65536 rows; this test calls it through the
C ABI twice in a row and checks each result against amgps_smooth's within the
parity tolerance of the other GPU tests, that a larger level is refused, and
that the calls leave the device's free memory and torch's allocator untouched
(the scratch array is claimed when the context is created).  The file name
makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2407_09848_gb300 import problems as pr

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    build.build()
    return torch


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_smooth_noalloc_matches_smooth(torch_cuda, prec):
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    H = pr.build_hierarchy(pr.varcoef(20, 1.0, 4.0, seed=11, ny=18, nz=13), coarse_max=100)
    S = Solver().load(H.A, H.P, prec=prec)
    S.set_smoother(1, "weights", 3, weights=[1.05, 0.97, 1.2])
    rng = np.random.default_rng(7)
    for call in range(2):
        for level, kind, k in [(0, "cheb4_opt", 4), (0, "cheb1_opt", 3), (1, "weights", 3),
                               (0, "l1jacobi", 2), (1, "cheb4", 1)]:
            n = H.levels[level].A.shape[0]
            b = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
            x0 = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
            for zero in (True, False):
                ref = x0.clone()
                S.smooth(level, kind, k, b, ref, x_is_zero=zero)
                got = x0.clone()
                S.smooth_noalloc(level, kind, k, b, got, x_is_zero=zero)
                torch.cuda.synchronize()
                e = rel(got.cpu().numpy(), ref.cpu().numpy())
                assert e <= TOL, (call, level, kind, k, zero, e)


def test_smooth_noalloc_rejects_large_level(torch_cuda):
    from paper_2407_09848_gb300.amgps import AmgpsError, Solver
    torch = torch_cuda
    H = pr.build_hierarchy(pr.poisson(48), coarse_max=512)
    assert H.levels[0].A.shape[0] > 65536 >= H.levels[1].A.shape[0]
    S = Solver().load(H.A, H.P)
    n0 = H.levels[0].A.shape[0]
    b = torch.ones(n0, dtype=torch.float64, device="cuda")
    x = torch.zeros(n0, dtype=torch.float64, device="cuda")
    with pytest.raises(AmgpsError) as e:
        S.smooth_noalloc(0, "cheb4_opt", 4, b, x, x_is_zero=True)
    assert e.value.name == "AMGPS_E_ARG" and "65536" in str(e.value)
    n1 = H.levels[1].A.shape[0]
    b1 = torch.ones(n1, dtype=torch.float64, device="cuda")
    x1 = torch.zeros(n1, dtype=torch.float64, device="cuda")
    x2 = torch.zeros(n1, dtype=torch.float64, device="cuda")
    S.smooth_noalloc(1, "cheb4_opt", 4, b1, x1, x_is_zero=True)
    S.smooth(1, "cheb4_opt", 4, b1, x2, x_is_zero=True)
    assert rel(x1.cpu().numpy(), x2.cpu().numpy()) <= TOL


def test_smooth_noalloc_allocates_nothing(torch_cuda):
    """Free device memory (cudaMemGetInfo) and torch's allocated bytes are the
    same before the first allocation-free call on a fresh context and after
    several of them.  The kernels are loaded first through amgps_smooth (the
    CUDA runtime loads a kernel's module on its first launch)."""
    from paper_2407_09848_gb300.amgps import Solver
    torch = torch_cuda
    H = pr.build_hierarchy(pr.poisson(24, 22, 20), coarse_max=100)
    S = Solver().load(H.A, H.P)
    n = H.levels[0].A.shape[0]
    rng = np.random.default_rng(3)
    b = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    x0 = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    calls = [("cheb4_opt", 4, True), ("cheb4_opt", 4, False), ("cheb1_opt", 3, False),
             ("l1jacobi", 2, True)]
    outs = [x0.clone() for _ in calls]
    refs = [x0.clone() for _ in calls]
    for (kind, k, zero), r in zip(calls, refs):
        S.smooth(0, kind, k, b, r, x_is_zero=zero)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    used0 = torch.cuda.memory_allocated()
    for rep in range(3):
        for (kind, k, zero), o in zip(calls, outs):
            o.copy_(x0)
            S.smooth_noalloc(0, kind, k, b, o, x_is_zero=zero)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, rep
        assert torch.cuda.memory_allocated() == used0, rep
    for o, r in zip(outs, refs):
        assert rel(o.cpu().numpy(), r.cpu().numpy()) <= TOL
