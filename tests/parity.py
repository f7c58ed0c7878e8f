"""Comparison of a GPU result with the oracle's, shared by the parity tests.

Two measures, both bounded by the same tolerance: the relative 2-norm of the
difference over the whole vector, and the largest element-wise difference
relative to the largest element of the oracle's vector.  The second one sees
an error confined to a few rows (one 32-row slice, the edge of a pipelined
tile) that the 2-norm of a 16.8 M-row vector dilutes below the tolerance.
"""
import numpy as np


def errors(got, ref):
    """(relative 2-norm, relative max-element) difference of got against ref."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = got - ref
    n2 = float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300))
    ninf = float(np.max(np.abs(d)) / max(np.max(np.abs(ref)), 1e-300)) if d.size else 0.0
    return n2, ninf


def assert_parity(got, ref, tol, *what):
    n2, ninf = errors(got, ref)
    assert n2 <= tol and ninf <= tol, (*what, "rel2", n2, "relmax", ninf)
    return n2, ninf
