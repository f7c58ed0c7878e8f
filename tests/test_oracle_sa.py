"""Pins for the smoothed-aggregation oracle (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sa
from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec
from paper_2407_09848_gb300 import problems as pr


def lap1d(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()


def test_1d_pairs_closed_form():
    # tridiag(-1, 2, -1) with pair aggregates: the Gershgorin bound of D^{-1}A
    # is 2, omega = 2/3; a point keeps 1 - omega (2 - 1)/2 = 2/3 in its own
    # aggregate and gets omega/2 = 1/3 from the neighbouring one (interior)
    n = 12
    A = lap1d(n)
    agg = np.arange(n) // 2
    P, om = sa.sa_prolongator(A, agg, n // 2)
    assert om == pytest.approx(2 / 3, abs=1e-16)
    Pd = P.toarray()
    for i in range(1, n - 1):
        J = i // 2
        other = J - 1 if i % 2 == 0 else J + 1
        assert Pd[i, J] == pytest.approx(2 / 3, abs=1e-15)
        assert Pd[i, other] == pytest.approx(1 / 3, abs=1e-15)
        assert np.count_nonzero(Pd[i]) == 2
    # the end points border one aggregate only (Dirichlet): 1 - omega/2 = 2/3
    assert Pd[0, 0] == pytest.approx(2 / 3, abs=1e-15) and np.count_nonzero(Pd[0]) == 1


def test_constant_preserved_where_rows_sum_to_zero():
    # interior Poisson rows annihilate constants, so (P 1_c)_i = 1 there
    st = pr.poisson(10)
    A = pr.to_csr(st)
    (agg, nc, _), = pr.geometric_aggregates(st.shape, coarse_max=200)
    P, _ = sa.sa_prolongator(A, agg, nc)
    rs = np.asarray(A.sum(axis=1)).ravel()
    one = P @ np.ones(nc)
    assert np.all(np.abs(one[rs == 0] - 1) <= 1e-14)
    assert np.all(one[rs > 0] < 1)


@pytest.mark.parametrize("st", [pr.poisson(8), pr.varcoef(7, 1.0, 3.0, seed=3, ny=6, nz=5),
                                pr.aniso(6, 1e-2)], ids=["p8", "var765", "aniso6"])
def test_galerkin_dense_brute_force_and_spd(st):
    A = pr.to_csr(st)
    (agg, nc, _), *_ = pr.geometric_aggregates(st.shape, coarse_max=20)
    P, om = sa.sa_prolongator(A, agg, nc)
    Ad, Pd = A.toarray(), P.toarray()
    # dense P from the definition, entry by entry
    Dinv = 1.0 / np.diag(Ad)
    Pref = np.zeros((A.shape[0], nc))
    for i in range(A.shape[0]):
        Pref[i, agg[i]] += 1.0
        for j in range(A.shape[0]):
            if Ad[i, j] != 0:
                Pref[i, agg[j]] -= om * Dinv[i] * Ad[i, j]
    assert np.max(np.abs(Pd - Pref)) <= 1e-15
    # Gershgorin bound >= the largest eigenvalue of D^{-1} A
    lam = np.max(np.linalg.eigvals(Ad * Dinv[:, None]).real)
    assert lam <= 4 / (3 * om) * (1 + 1e-14)
    Ac = sa.galerkin(A, P).toarray()
    Acd = np.zeros((nc, nc))
    for I in range(nc):
        for J in range(nc):
            Acd[I, J] = Pref[:, I] @ Ad @ Pref[:, J]
    assert np.max(np.abs(Ac - Acd)) <= 1e-13 * np.abs(Acd).max()
    assert np.array_equal(Ac, Ac.T) or np.max(np.abs(Ac - Ac.T)) <= 1e-15 * np.abs(Ac).max()
    assert np.linalg.eigvalsh(0.5 * (Ac + Ac.T)).min() > 0


def test_sa_two_level_contracts_and_beats_unsmoothed():
    st = pr.poisson(8)
    A = pr.to_csr(st)
    (agg, nc, _), *_ = pr.geometric_aggregates(st.shape, coarse_max=100)
    P, _ = sa.sa_prolongator(A, agg, nc)
    Pu = sa.tentative(agg, nc)
    spec = SmootherSpec("cheb4_opt", 2)
    Ad = A.toarray()
    Lh = np.linalg.cholesky(Ad)

    def anorm_E(Pm):
        amg = OracleAMG([A, sa.galerkin(A, Pm)], [Pm], spec)
        n = A.shape[0]
        B = np.stack([amg.vcycle(e) for e in np.eye(n)], axis=1)
        E = np.eye(n) - B @ Ad
        return np.linalg.norm(Lh.T @ E @ np.linalg.inv(Lh.T), 2)
    e_sa, e_ua = anorm_E(P), anorm_E(Pu)
    assert e_sa < 1 and e_sa < e_ua


def test_sa_hierarchy_pcg_32():
    st = pr.poisson(32)
    levels = pr.geometric_aggregates(st.shape, coarse_max=512)
    As, Ps, _ = sa.sa_hierarchy(pr.to_csr(st), [a for a, _, _ in levels],
                                [nc for _, nc, _ in levels])
    assert [a.shape[0] for a in As] == [32768, 4096, 512]
    b = pr.rhs_uniform(32768, seed=0)
    x, it, rel, _ = OracleAMG(As, Ps, SmootherSpec("cheb4_opt", 4)).pcg(b, rtol=1e-8)
    assert rel <= 1e-8 and it <= 8
    assert np.linalg.norm(b - As[0] @ x) <= 2e-8 * np.linalg.norm(b)


def test_geometric_aggregates_match_unsmoothed_hierarchy():
    st = pr.varcoef(9, 1.0, 2.0, seed=1, ny=7, nz=6)
    H = pr.build_hierarchy(st, coarse_max=20)
    levels = pr.geometric_aggregates(st.shape, coarse_max=20)
    assert len(levels) == H.n_levels - 1
    for (agg, nc, shp), lv, nxt in zip(levels, H.levels[:-1], H.levels[1:]):
        assert np.array_equal(agg, lv.agg) and nc == nxt.A.shape[0] and shp == nxt.shape


def test_stored_sa_iteration_counts_match_the_oracle():
    # the GPU tests compare against tests/golden/oracle_sa_pcg_iterations.json;
    # its 32^3 entries must be what the oracle gives today
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_sa_pcg_iterations.json")
    runs = [r for r in json.load(open(path))["runs"] if r["grid"] == 32]
    assert len(runs) == 3
    st = pr.poisson(32)
    levels = pr.geometric_aggregates(st.shape, coarse_max=512)
    As, Ps, om = sa.sa_hierarchy(pr.to_csr(st), [a for a, _, _ in levels],
                                 [nc for _, nc, _ in levels])
    b = pr.rhs_uniform(32768, seed=0)
    for r in runs:
        assert [a.shape[0] for a in As] == r["levels"] and [a.nnz for a in As] == r["nnz"]
        assert np.allclose(om, r["omega"], rtol=1e-15, atol=0)
        _, it, rel, _ = OracleAMG(As, Ps, SmootherSpec(r["kind"], r["degree"])).pcg(b, rtol=1e-8)
        assert rel <= 1e-8 and it == r["iterations"]
