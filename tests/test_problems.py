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


def test_aniso_weak_direction_is_z():
    # reading 10: x/y neighbours -1, z neighbours -eps, diagonal 4 + 2 eps inside
    nz, ny, nx = 5, 6, 7
    A = pr.to_csr(pr.aniso(nx, 1e-3, ny=ny, nz=nz)).tolil()
    i = lambda x, y, z: (z * ny + y) * nx + x
    c = i(3, 3, 2)
    assert A[c, i(4, 3, 2)] == -1.0 and A[c, i(3, 4, 2)] == -1.0
    assert A[c, i(3, 3, 3)] == -1e-3 and abs(A[c, c] - (4 + 2e-3)) <= 4e-16 * 4


def test_varcoef_faces_are_harmonic_means_and_boundary_faces_the_cell_value():
    # reading 10: k = exp(sigma g); interior face 2 k_i k_j / (k_i + k_j); a
    # boundary face takes the cell's own k, so the diagonal is the sum of the
    # six face coefficients
    nx, ny, nz, sigma, ell, seed = 9, 8, 7, 1.5, 3.0, 4
    k = np.exp(sigma * pr.grf((nz, ny, nx), ell, seed))
    A = pr.to_csr(pr.varcoef(nx, sigma, ell, seed=seed, ny=ny, nz=nz)).tolil()
    i = lambda x, y, z: (z * ny + y) * nx + x
    hm = lambda a, b: 2 * a * b / (a + b)
    for (x, y, z) in [(0, 0, 0), (4, 3, 2), (8, 7, 6), (0, 5, 3)]:
        c = i(x, y, z)
        face = 0.0
        for dx, dy, dz in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            X, Y, Z = x + dx, y + dy, z + dz
            if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                f = hm(k[z, y, x], k[Z, Y, X])
                assert abs(A[c, i(X, Y, Z)] + f) <= 1e-14 * f
            else:
                f = k[z, y, x]
            face += f
        assert abs(A[c, c] - face) <= 1e-13 * face


def test_grf_correlation_length():
    # reading 11: covariance exp(-r^2 / (2 ell^2)); the sample correlation of
    # the field at lag ell along an axis is close to exp(-1/2), at lag 2 ell to
    # exp(-2) (a filter width off by a factor 2 moves these far outside)
    ell = 3.0
    g = pr.grf((48, 48, 96), ell, seed=11)
    def corr(lag):
        a, b = g[..., :-lag], g[..., lag:]
        return float(np.mean(a * b) / np.sqrt(np.mean(a * a) * np.mean(b * b)))
    assert abs(corr(3) - np.exp(-0.5)) < 0.06
    assert abs(corr(6) - np.exp(-2.0)) < 0.06
    assert corr(1) > corr(3) > corr(6)


def test_vectors_are_seeded_and_in_range():
    b = pr.rhs_uniform(10000, seed=0)
    assert b.min() >= -1 and b.max() <= 1 and abs(b.mean()) < 0.05
    assert not np.array_equal(b, pr.rhs_uniform(10000, seed=1))
    E = pr.vec_normal(5000, seed=2, count=3)
    assert E.shape == (3, 5000) and abs(E.std() - 1) < 0.05
    assert np.array_equal(E, pr.vec_normal(5000, seed=2, count=3))
