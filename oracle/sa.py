"""Smoothed-aggregation prolongator and Galerkin coarse operator (oracle).

Test infrastructure only.  FP64, scipy.sparse products as library steps.

Sec. 4 builds the hierarchy from a tentative prolongator P_hat (piecewise
constant on aggregates) smoothed by one damped Jacobi step,

    P = (I - omega D^{-1} A) P_hat,   D = diag(A),   omega = 4 / (3 lambda_max),

with lambda_max an estimate of the largest eigenvalue of D^{-1} A, and the
coarse matrices by the Galerkin product A_c = P^T A P (Eq. amg's setting).
Readings: the aggregates are supplied by the caller (the paper's aggregates
come from weighted matching or VBM, of size up to 8; geometric 2x2x2 blocks
stand in for them); the lambda_max estimate is the row-sum (Gershgorin) bound
max_i sum_j |a_ij| / a_ii, an upper bound of the spectrum of D^{-1} A that
needs no iteration.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def tentative(agg, n_coarse):
    """P_hat of Sec. 4: one unit entry per fine row, in column agg[i]."""
    agg = np.asarray(agg, dtype=np.int64)
    n = agg.size
    return sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, n_coarse))


def lambda_bound(A):
    """max_i sum_j |a_ij| / a_ii  (>= every eigenvalue of D^{-1} A): the estimate of
    lambda_max of D^{-1} A in omega = 4/(3 lambda_max), Sec. 4."""
    A = sp.csr_matrix(A)
    return float(np.max(np.asarray(abs(A).sum(axis=1)).ravel() / A.diagonal()))


def sa_prolongator(A, agg, n_coarse):
    """Returns (P, omega): P = (I - omega D^{-1} A) P_hat (Sec. 4)."""
    A = sp.csr_matrix(A)
    omega = 4.0 / (3.0 * lambda_bound(A))
    Ph = tentative(agg, n_coarse)
    P = Ph - omega * (sp.diags(1.0 / A.diagonal()) @ (A @ Ph))
    return sp.csr_matrix(P), omega


def galerkin(A, P):
    """A_c = P^T A P, the Galerkin product of Sec. 2."""
    P = sp.csr_matrix(P)
    return sp.csr_matrix(P.T @ (sp.csr_matrix(A) @ P))


def sa_hierarchy(A0, aggs, n_coarse):
    """Levels A_0..A_L and prolongators P_0..P_{L-1} from per-level aggregates
    (smoothed aggregation of Sec. 4, Galerkin products of Sec. 2)."""
    As, Ps, omegas = [sp.csr_matrix(A0)], [], []
    for agg, nc in zip(aggs, n_coarse):
        P, om = sa_prolongator(As[-1], agg, nc)
        Ps.append(P)
        omegas.append(om)
        As.append(galerkin(As[-1], P))
    return As, Ps, omegas
