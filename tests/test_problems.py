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


@pytest.mark.parametrize("spectrum", ["equispaced", "boundary", "gap"])
def test_spectral_test_matrix_has_the_stated_spectrum(spectrum):
    N = 64
    A, b = pr.spectral_test_matrix(N, spectrum)
    Ad = A.toarray()
    assert A.nnz == N * N and np.array_equal(Ad, Ad.T)
    ev = np.linalg.eigvalsh(Ad)
    h = N // 2
    if spectrum == "equispaced":
        d = np.arange(1, N + 1) / N
    elif spectrum == "boundary":
        d = np.concatenate([10.0 ** np.linspace(-8, -1, h), 1 - 10.0 ** np.linspace(-8, -1, h)])
    else:
        d = np.concatenate([10.0 ** np.linspace(-8, -1, h),
                            10.0 ** np.linspace(1, np.log10(np.pi), h)])
    assert np.max(np.abs(ev - np.sort(d))) <= 1e-13 * d.max()
    assert np.allclose(b, Ad.sum(axis=1), rtol=0, atol=1e-14 * N)
    if spectrum == "equispaced":
        # the eigenvectors are the discrete sine modes: A v_j = (j/N) v_j
        i = np.arange(1, N + 1)
        j = 5
        v = np.sin(i * j * np.pi / (N + 1))
        assert np.allclose(Ad @ v, (j / N) * v, rtol=0, atol=1e-13)


def test_single_aggregate_hierarchy_is_galerkin():
    A, _ = pr.spectral_test_matrix(16, "equispaced")
    As, Ps = pr.single_aggregate_hierarchy(A)
    assert As[1].shape == (1, 1) and Ps[0].shape == (16, 1)
    assert np.isclose(As[1][0, 0], A.sum())
