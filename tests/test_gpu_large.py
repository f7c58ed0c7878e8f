"""Largest size exercised: 512^3 Poisson (134,217,728 rows, 939 M stored matrix
entries: every value array passes 2^31 bytes).  Too large for the oracle, so
the checks are properties: the true residual, an iteration count near the
256^3 one, and a repeated solve reproducing every bit."""
import numpy as np
import pytest

from paper_2407_09848_gb300 import problems as pr

pytestmark = pytest.mark.gpu


def test_poisson_512_pcg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    from paper_2407_09848_gb300.amgps import Solver
    build.build()
    H = pr.build_hierarchy(pr.poisson(512), coarse_max=512)
    S = Solver().load(H.A, H.P)
    n = H.A[0].shape[0]
    assert n == 512 ** 3 and S.level_info(0)[2] * 8 > 2 ** 31
    b = pr.rhs_uniform(n, seed=0)
    bd = torch.from_numpy(b).cuda()
    x = torch.empty_like(bd)
    it, rel = S.pcg(bd, x, rtol=1e-8)
    true = np.linalg.norm(b - H.A[0] @ x.cpu().numpy()) / np.linalg.norm(b)
    assert rel <= 1e-8 and true <= 1.01e-8
    assert 30 <= it <= 60
    x2 = torch.empty_like(bd)
    it2, rel2 = S.pcg(bd, x2, rtol=1e-8)
    assert it2 == it and rel2 == rel and torch.equal(x, x2)
    S.close()
