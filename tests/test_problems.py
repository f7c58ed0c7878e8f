"""Checks of the seeded input generators (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2407_09848_gb300 import problems as pr


@pytest.mark.parametrize("st", [pr.poisson(8), pr.poisson(5, 7, 9), pr.aniso(6, 1e-3),
                                pr.varcoef(10, 1.0, 3.0, seed=1), pr.varcoef(7, 2.0, 2.0, seed=2)],
                         ids=["p8", "p579", "aniso6", "var10", "var7"])
def test_galerkin_equals_PtAP(st):
    H = pr.build_hierarchy(st, coarse_max=20)
    for l in range(H.n_levels - 1):
        A, P = H.levels[l].A, H.levels[l].P
        Ac = (P.T @ A @ P).toarray()
        assert np.allclose(H.levels[l + 1].A.toarray(), Ac, rtol=0, atol=1e-12 * np.abs(Ac).max())
        # P: exactly one unit entry per row, agg matches
        assert np.all(np.diff(P.indptr) == 1) and np.all(P.data == 1.0)
        assert np.array_equal(P.indices, H.levels[l].agg)
    for lv in H.levels:
        A = lv.A
        assert abs(A - A.T).max() == 0
        assert A.indices.dtype == np.int32
        assert np.linalg.eigvalsh(A.toarray()).min() > 0


def test_poisson_stencil_values():
    A = pr.to_csr(pr.poisson(6))
    d = A.diagonal()
    assert np.all(d == 6.0)
    off = A - sp.diags(d)
    assert set(np.unique(off.data)) == {-1.0}
    # interior rows sum to zero, boundary rows to the number of eliminated neighbours
    rs = np.asarray(A.sum(axis=1)).ravel().reshape(6, 6, 6)
    assert rs[1:-1, 1:-1, 1:-1].max() == 0 and rs[0, 0, 0] == 3


def test_coarse_poisson_values():
    H = pr.build_hierarchy(pr.poisson(8), coarse_max=8)
    A1 = H.levels[1].A
    assert np.allclose(A1[0, 0], 48 - 24) and np.allclose(A1[0, 1], -4)


def test_seeded_and_grf_normalised():
    assert np.array_equal(pr.rhs_uniform(100, 3), pr.rhs_uniform(100, 3))
    g = pr.grf((20, 18, 16), 3.0, seed=7)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1) < 1e-12
