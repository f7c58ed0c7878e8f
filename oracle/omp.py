"""All-core CPU build of the oracle loops (test infrastructure only).

`oracle/c/amg_omp.c` restates the numpy oracle's smoother (Eq. l1smooth,
Eq. polsmoother, Eq. polsmootheropt, Algorithm 1), V-cycle (Eq. amg) and PCG
(Sec. 4) in plain C with OpenMP row loops, for timing the oracle on every host
core.  This module compiles it (gcc, on first use or when the source is newer)
and calls it through ctypes.  The parameters each kind needs (a_k*, the optimal
beta_j) come from the numpy oracle's `params`; P^T and the coarsest level's
Cholesky factor come from scipy / numpy, as in `oracle.amg`.  It is checked
against the numpy oracle by `tests/test_oracle_omp.py`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np
import scipy.sparse as sp

from .smoother import SmootherSpec

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "amg_omp.c")
LIB = os.path.join(HERE, "c", "libora_omp.so")
# plain IEEE FP64: no contraction of a*b + c into a fused multiply-add, so
# each operation rounds as numpy's does
CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC"]


def build(force=False):
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc"] + CFLAGS + [SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


class _Csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class _Spec(C.Structure):
    _fields_ = [("kind", C.c_int), ("k", C.c_int), ("has_beta", C.c_int),
                ("beta", C.c_double * 16), ("a", C.c_double), ("rho", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.ora_hier_create.restype = C.c_void_p
        L.ora_hier_create.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_int]
        L.ora_hier_free.argtypes = [C.c_void_p]
        L.ora_vcycle.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.ora_pcg.restype = C.c_int
        L.ora_pcg.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                              C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.ora_smooth.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
        L.ora_l1diag.argtypes = [C.c_void_p, C.c_void_p]
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_get_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(t):
    lib().ora_set_threads(int(t))


def threads():
    return int(lib().ora_get_threads())


def _csr(A, keep):
    A = sp.csr_matrix(A)
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    va = np.ascontiguousarray(A.data, dtype=np.float64)
    keep += [rp, ci, va]
    return _Csr(A.shape[0], A.shape[1], rp.ctypes.data, ci.ctypes.data, va.ctypes.data)


def _spec(s: SmootherSpec):
    kind = {"l1jacobi": 0, "cheb4": 1, "cheb4_opt": 1, "weights": 1, "cheb1": 2,
            "cheb1_opt": 2}[s.kind]
    out = _Spec()
    out.kind, out.k, out.rho = kind, s.k, s.rho
    out.has_beta = 0 if s.beta is None else 1
    if s.beta is not None:
        for j, v in enumerate(s.beta):
            out.beta[j] = float(v)
    out.a = float(s.a) if s.a is not None else 0.0
    return out


def smooth(A, b, x0, spec: SmootherSpec):
    """One smoother application, as oracle.smoother.smooth."""
    keep = []
    a = _csr(A, keep)
    n = A.shape[0]
    M = np.zeros(n)
    lib().ora_l1diag(C.byref(a), M.ctypes.data)
    x = np.zeros(n)
    work = np.zeros(3 * n)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x0c = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    s = _spec(spec)
    lib().ora_smooth(C.byref(a), M.ctypes.data, C.byref(s), b.ctypes.data,
                     None if x0c is None else x0c.ctypes.data, x.ctypes.data, work.ctypes.data)
    return x


class OmpAMG:
    """The hierarchy of oracle.amg.OracleAMG (same A_l, P_l, specs, coarse
    solver), run by the C loops."""

    def __init__(self, A_list, P_list, specs, coarse_sweeps=0):
        self._keep = []
        A_list = [sp.csr_matrix(A) for A in A_list]
        P_list = [sp.csr_matrix(P) for P in P_list]
        nl = len(A_list)
        if isinstance(specs, SmootherSpec):
            specs = [specs] * (nl - 1)
        self.n = A_list[0].shape[0]
        self._A = (_Csr * nl)(*[_csr(A, self._keep) for A in A_list])
        self._P = (_Csr * max(nl - 1, 1))(*[_csr(P, self._keep) for P in P_list])
        self._PT = (_Csr * max(nl - 1, 1))(*[_csr(P.T.tocsr(), self._keep) for P in P_list])
        self._S = (_Spec * max(nl - 1, 1))(*[_spec(s) for s in specs])
        self._L = np.ascontiguousarray(np.linalg.cholesky(A_list[-1].toarray()))
        self._h = lib().ora_hier_create(nl, C.cast(self._A, C.c_void_p), C.cast(self._P, C.c_void_p),
                                        C.cast(self._PT, C.c_void_p), C.cast(self._S, C.c_void_p),
                                        self._L.ctypes.data, int(coarse_sweeps))
        if not self._h:
            raise MemoryError("ora_hier_create failed")

    def close(self):
        if self._h:
            lib().ora_hier_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vcycle(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n)
        lib().ora_vcycle(self._h, b.ctypes.data, x.ctypes.data)
        return x

    def pcg(self, b, rtol=1e-8, maxit=1000):
        """(x, iterations, recurrence residual ratio, status): status 0
        converged, 1 maxit, 2 p.Ap <= 0, 3 out of memory."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n)
        it, rel = C.c_int(), C.c_double()
        st = lib().ora_pcg(self._h, b.ctypes.data, x.ctypes.data, float(rtol), int(maxit),
                           C.byref(it), C.byref(rel))
        return x, it.value, rel.value, st
