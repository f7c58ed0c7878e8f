"""Python binding of libamgps (include/amgps.h): argument marshalling only.

Every step of the smoother, V-cycle and PCG runs in the library's CUDA
kernels; this module checks shapes/dtypes, passes raw pointers and turns
status codes into exceptions.  Device vectors are torch CUDA tensors (FP64,
contiguous); PyTorch provides memory and the caller's stream, nothing else.
The library must be built (``paper_2407_09848_gb300.build.build()``); there is
no fallback path: a missing library raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamgps.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "amgps.h")

KIND = {"l1jacobi": 0, "cheb4": 1, "cheb4_opt": 2, "cheb1": 3, "cheb1_opt": 4, "weights": 5}
PREC = {"f64": 0, "f32": 1, "bf16": 2}
STATUS = {0: "AMGPS_OK", 1: "AMGPS_E_ARG", 2: "AMGPS_E_NOT_SPD", 3: "AMGPS_E_NOCONV",
          4: "AMGPS_E_NAN", 5: "AMGPS_E_CUDA", 6: "AMGPS_E_TIMEOUT", 7: "AMGPS_E_STATE",
          8: "AMGPS_E_NOMEM"}
PROF_STEP, PROF_RESTRICT, PROF_SPMV, PROF_COUNT, PROF_COARSE = 0, 1, 2, 3, 4
OPT_TMA, OPT_FLEXIBLE, OPT_COARSE_SWEEPS, OPT_COARSE_KERNEL, OPT_ALLOC_LIMIT = 1, 2, 3, 4, 5
OPT_STEP_FORM = 6


class AmgpsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class CSR(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class CSRBuf(C.Structure):
    """Library-allocated host CSR (amgps_csr_buf)."""
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.POINTER(C.c_int32)), ("col", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double))]


_lib = None

_SIGS = {
    "amgps_version": ([], C.c_int),
    "amgps_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_void_p], C.c_int),
    "amgps_destroy": ([C.c_void_p], C.c_int),
    "amgps_last_error": ([C.c_void_p], C.c_char_p),
    "amgps_hierarchy_load": ([C.c_void_p, C.c_int, C.POINTER(CSR), C.POINTER(CSR), C.c_int], C.c_int),
    "amgps_level_info": ([C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                          C.POINTER(C.c_int64)], C.c_int),
    "amgps_set_smoother": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_double], C.c_int),
    "amgps_estimate_lambda": ([C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "amgps_smooth": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "amgps_smooth_noalloc": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int],
                             C.c_int),
    "amgps_vcycle": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "amgps_smooth_backward": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "amgps_vcycle_backward": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
                              C.c_int),
    "amgps_pcg": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int),
                   C.POINTER(C.c_double)], C.c_int),
    "amgps_pcg_smoother": ([C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                            C.POINTER(C.c_int), C.POINTER(C.c_double)], C.c_int),
    "amgps_pcg_host": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int),
                        C.POINTER(C.c_double)], C.c_int),
    "amgps_synchronize": ([C.c_void_p], C.c_int),
    "amgps_vcycle_loss_grad": ([C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p],
                               C.c_int),
    "amgps_error_cycles": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int], C.c_int),
    "amgps_mlp_forward": ([C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p], C.c_int),
    "amgps_mlp_backward": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "amgps_mlp_adam": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.c_float,
                        C.c_float, C.c_float, C.c_void_p], C.c_int),
    "amgps_round_bf16": ([C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "amgps_step_coefs": ([C.c_int, C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                          C.c_void_p, C.POINTER(C.c_double)], C.c_int),
    "amgps_tma_plan": ([C.POINTER(CSR), C.c_int, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p,
                        C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "amgps_sell_layout": ([C.POINTER(CSR), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                           C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p], C.c_int),
    "amgps_opt4_weights": ([C.c_int, C.c_void_p], C.c_int),
    "amgps_cheb1_astar": ([C.c_int, C.POINTER(C.c_double)], C.c_int),
    "amgps_profile_enable": ([C.c_void_p, C.c_int], C.c_int),
    "amgps_set_option": ([C.c_void_p, C.c_int, C.c_int64], C.c_int),
    "amgps_tma_plan_stats": ([C.POINTER(CSR), C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                              C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "amgps_csr_buf_free": ([C.POINTER(CSRBuf)], None),
    "amgps_galerkin": ([C.c_void_p, C.POINTER(CSR), C.POINTER(CSR), C.POINTER(CSRBuf)], C.c_int),
    "amgps_sa_level": ([C.c_void_p, C.POINTER(CSR), C.c_void_p, C.c_int64, C.POINTER(C.c_double),
                        C.POINTER(CSRBuf), C.POINTER(CSRBuf)], C.c_int),
    "amgps_profile_read": ([C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                            C.POINTER(C.c_double)], C.c_int),
    "amgps_profile_flops": ([C.c_void_p, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "amgps_profile_fp64_inst": ([C.c_void_p, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "amgps_op_coefs": ([C.c_int, C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                        C.c_void_p, C.c_void_p], C.c_int),
}


def lib():
    """Load libamgps.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2407_09848_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def header_symbols():
    """Names of the entry points declared in include/amgps.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(amgps_[a-z0-9_]+)\s*\(", text)))


def opt4_weights(k):
    """The library's tabulated optimal 4th-kind weights (host call, no GPU)."""
    out = np.zeros(k)
    st = lib().amgps_opt4_weights(k, out.ctypes.data)
    if st:
        raise AmgpsError(st, "bad degree")
    return out


def cheb1_astar(k):
    a = C.c_double()
    st = lib().amgps_cheb1_astar(k, C.byref(a))
    if st:
        raise AmgpsError(st, "bad degree")
    return a.value


def _fptr(t, n, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous() and t.numel() == n):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor of {n} entries")
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _raise_global(st):
    if st:
        raise AmgpsError(st, lib().amgps_last_error(None).decode())


def mlp_forward(params, feats, beta_ref, beta, acts):
    """Library MLP forward (FP32 device tensors; see amgps_mlp_forward)."""
    B = feats.numel() // 8
    _raise_global(lib().amgps_mlp_forward(
        _fptr(params, 4996, "params"), _fptr(feats, B * 8, "feats"), B, _fptr(beta_ref, 4, "beta_ref"),
        _fptr(beta, B * 4, "beta"), _fptr(acts, B * 132, "acts"), _stream()))


def mlp_backward(params, feats, acts, beta, gbeta, work, grads):
    B = feats.numel() // 8
    _raise_global(lib().amgps_mlp_backward(
        _fptr(params, 4996, "params"), _fptr(feats, B * 8, "feats"), _fptr(acts, B * 132, "acts"),
        _fptr(beta, B * 4, "beta"), B, _fptr(gbeta, B * 4, "gbeta"), _fptr(work, B * 132, "work"),
        _fptr(grads, 4996, "grads"), _stream()))


def mlp_adam(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    _raise_global(lib().amgps_mlp_adam(
        _fptr(params, 4996, "params"), _fptr(grads, 4996, "grads"), _fptr(m, 4996, "m"),
        _fptr(v, 4996, "v"), int(step), float(lr), float(b1), float(b2), float(eps), _stream()))


def tma_plan_stats(A, prec="f64"):
    """Host-only: (tiles, generic_slices, stage_bytes, nstages) of the TMA plan."""
    keep = []
    csr = _csr_struct(A, keep)
    t, g, sb, ns = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
    st = lib().amgps_tma_plan_stats(C.byref(csr), PREC[prec], C.byref(t), C.byref(g), C.byref(sb),
                                    C.byref(ns))
    if st:
        raise AmgpsError(st, lib().amgps_last_error(None).decode())
    return t.value, g.value, sb.value, ns.value


def round_bf16(x):
    """Host-only: BF16 bit patterns (uint16) of FP64 values as the loader rounds them."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.size, np.uint16)
    stat = lib().amgps_round_bf16(x.ctypes.data, x.size, out.ctypes.data)
    if stat:
        raise AmgpsError(stat, lib().amgps_last_error(None).decode())
    return out


def step_coefs(kind, degree, weights=None, rho=0.0):
    """Host-only: (c1, c2, beta, rhoinv) of one application, arrays indexed by
    step j = 0..degree (see amgps_step_coefs)."""
    c1, c2, beta = (np.zeros(degree + 1) for _ in range(3))
    ri = C.c_double()
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    stat = lib().amgps_step_coefs(KIND[kind], int(degree), None if w is None else w.ctypes.data,
                                  float(rho), c1.ctypes.data, c2.ctypes.data, beta.ctypes.data,
                                  C.byref(ri))
    if stat:
        raise AmgpsError(stat, lib().amgps_last_error(None).decode())
    return c1, c2, beta, ri.value


def op_coefs(kind, degree, weights=None, rho=0.0):
    """Host-only: (tau, sigma, h, g) of the stored-operator steps of one
    application, arrays of degree - 1 entries (see amgps_op_coefs)."""
    tau, sigma, h, g = (np.zeros(degree - 1) for _ in range(4))
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    stat = lib().amgps_op_coefs(KIND[kind], int(degree), None if w is None else w.ctypes.data,
                                float(rho), tau.ctypes.data, sigma.ctypes.data, h.ctypes.data,
                                g.ctypes.data)
    if stat:
        raise AmgpsError(stat, lib().amgps_last_error(None).decode())
    return tau, sigma, h, g


def tma_plan(A, prec="f64"):
    """Host-only: the TMA plan of a square matrix (see amgps_tma_plan) as a dict:
    the scalar fields, g_start / g_elems / g_smem / d arrays, tiles (ntiles x 2:
    first row, value index) and gen (slices left to the direct kernel)."""
    keep = []
    csr = _csr_struct(A, keep)
    info = np.zeros(32, np.int32)
    nt, ng = C.c_int64(), C.c_int64()
    stat = lib().amgps_tma_plan(C.byref(csr), PREC[prec], info.ctypes.data, C.byref(nt), None,
                                C.byref(ng), None)
    if stat:
        raise AmgpsError(stat, lib().amgps_last_error(None).decode())
    tiles = np.zeros((max(nt.value, 1), 2), np.int64)
    gen = np.zeros(max(ng.value, 1), np.int32)
    stat = lib().amgps_tma_plan(C.byref(csr), PREC[prec], info.ctypes.data, C.byref(nt),
                                tiles.ctypes.data, C.byref(ng), gen.ctypes.data)
    if stat:
        raise AmgpsError(stat, lib().amgps_last_error(None).decode())
    keys = ("rows", "w", "ngroups", "d0", "vals_bytes", "vec_bytes", "win_bytes",
            "stage_bytes", "nstages")
    out = {k: int(v) for k, v in zip(keys, info[:9])}
    out.update(g_start=info[9:13].copy(), g_elems=info[13:17].copy(), g_smem=info[17:21].copy(),
               d=info[21:29].copy(), tiles=tiles[:nt.value], gen=gen[:ng.value])
    return out


def sell_layout(A):
    """Host-only: the SELL-32 layout of a square matrix, as a dict of numpy
    arrays (vbase, width, cref, val, col, off); see amgps_sell_layout."""
    keep = []
    csr = _csr_struct(A, keep)
    ns, st, no = C.c_int64(), C.c_int64(), C.c_int64()
    z = None
    stat = lib().amgps_sell_layout(C.byref(csr), C.byref(ns), C.byref(st), C.byref(no),
                                   z, z, z, z, z, z)
    if stat:
        raise AmgpsError(stat, lib().amgps_last_error(None).decode())
    out = {"vbase": np.zeros(ns.value, np.int64), "width": np.zeros(ns.value, np.int32),
           "cref": np.zeros(ns.value, np.int32), "val": np.zeros(st.value, np.float64),
           "col": np.zeros(st.value, np.int32), "off": np.zeros(max(no.value, 1), np.int32)}
    ptr = lambda a: a.ctypes.data
    stat = lib().amgps_sell_layout(C.byref(csr), C.byref(ns), C.byref(st), C.byref(no),
                                   ptr(out["vbase"]), ptr(out["width"]), ptr(out["cref"]),
                                   ptr(out["val"]), ptr(out["col"]), ptr(out["off"]))
    if stat:
        raise AmgpsError(stat, lib().amgps_last_error(None).decode())
    out["off"] = out["off"][:no.value]
    return out


def _csr_struct(A, keep):
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int32)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    keep.extend([rowptr, col, val])
    return CSR(A.shape[0], A.shape[1], A.nnz, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data)


def _from_buf(b):
    """Copy a library-allocated CSR into scipy and release it."""
    import scipy.sparse as sp
    n, nnz, ncol = b.n_rows, b.nnz, b.n_cols
    try:
        rp = np.ctypeslib.as_array(b.rowptr, shape=(n + 1,)).copy()
        col = np.ctypeslib.as_array(b.col, shape=(max(nnz, 1),))[:nnz].copy()
        val = np.ctypeslib.as_array(b.val, shape=(max(nnz, 1),))[:nnz].copy()
    finally:
        lib().amgps_csr_buf_free(C.byref(b))
    return sp.csr_matrix((val, col, rp), shape=(n, ncol))


def _sorted_csr(A):
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    return A if A.has_sorted_indices else A.sorted_indices()


def _dptr(t, n=None, name="vector"):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
    return C.c_void_p(t.data_ptr())


class Solver:
    """One libamgps context on one device."""

    def __init__(self, device=0, stream=None):
        import torch
        self._h = C.c_void_p()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        st = lib().amgps_create(C.byref(self._h), int(device), C.c_void_p(stream))
        if st:
            raise AmgpsError(st, lib().amgps_last_error(None).decode())
        self.device = device
        self.n_levels = 0
        self.sizes = []

    def _check(self, st):
        if st:
            raise AmgpsError(st, lib().amgps_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib().amgps_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, A_list, P_list, prec="f64"):
        keep = []
        nl = len(A_list)
        As = (CSR * nl)(*[_csr_struct(A, keep) for A in A_list])
        Ps = (CSR * max(nl - 1, 1))(*([_csr_struct(P, keep) for P in P_list] or [CSR()]))
        self._check(lib().amgps_hierarchy_load(self._h, nl, As, Ps, PREC[prec]))
        self.n_levels = nl
        self.sizes = [A.shape[0] for A in A_list]
        self.prec = prec
        return self

    def galerkin(self, A, P):
        """A_c = P^T A P on the device (amgps_galerkin); returns scipy CSR."""
        keep = []
        a, p = _csr_struct(_sorted_csr(A), keep), _csr_struct(_sorted_csr(P), keep)
        out = CSRBuf()
        self._check(lib().amgps_galerkin(self._h, C.byref(a), C.byref(p), C.byref(out)))
        return _from_buf(out)

    def sa_level(self, A, agg, n_coarse):
        """Smoothed-aggregation level on the device (amgps_sa_level):
        returns (P, A_c, omega) with P, A_c scipy CSR."""
        keep = []
        a = _csr_struct(_sorted_csr(A), keep)
        g = np.ascontiguousarray(agg, dtype=np.int32)
        if g.size != a.n_rows:
            raise ValueError("agg needs one entry per row of A")
        om = C.c_double()
        P, Ac = CSRBuf(), CSRBuf()
        self._check(lib().amgps_sa_level(self._h, C.byref(a), g.ctypes.data, int(n_coarse),
                                         C.byref(om), C.byref(P), C.byref(Ac)))
        return _from_buf(P), _from_buf(Ac), om.value

    def sa_hierarchy(self, A0, levels):
        """Smoothed-aggregation hierarchy built on the device from the
        aggregate maps [(agg, n_coarse, ...), ...] of each level; returns
        (A_list, P_list, omegas) ready for load()."""
        As, Ps, oms = [_sorted_csr(A0)], [], []
        for lv in levels:
            P, Ac, om = self.sa_level(As[-1], lv[0], lv[1])
            Ps.append(P)
            As.append(Ac)
            oms.append(om)
        return As, Ps, oms

    def level_info(self, level):
        n, nnz, stored = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(lib().amgps_level_info(self._h, level, C.byref(n), C.byref(nnz), C.byref(stored)))
        return n.value, nnz.value, stored.value

    def set_smoother(self, level, kind, degree, weights=None, rho=0.0):
        w = None
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.float64)
            if w.size != degree:
                raise ValueError("weights must have `degree` entries")
        self._check(lib().amgps_set_smoother(self._h, level, KIND[kind], degree,
                                             None if w is None else w.ctypes.data, float(rho)))

    def estimate_lambda(self, level, v0, iters=10):
        lam = C.c_double()
        self._check(lib().amgps_estimate_lambda(self._h, level, _dptr(v0, self._n(level), "v0"),
                                                iters, C.byref(lam)))
        return lam.value

    def _n(self, level):
        return self.sizes[level] if 0 <= level < len(self.sizes) else None

    def smooth(self, level, kind, degree, b, x, x_is_zero=False):
        n = self._n(level)
        self._check(lib().amgps_smooth(self._h, level, KIND[kind], degree, _dptr(b, n, "b"),
                                       _dptr(x, n, "x"), 1 if x_is_zero else 0))

    def smooth_noalloc(self, level, kind, degree, b, x, x_is_zero=False):
        """amgps_smooth without device allocation (static 65536-row scratch)."""
        n = self._n(level)
        self._check(lib().amgps_smooth_noalloc(self._h, level, KIND[kind], degree, _dptr(b, n, "b"),
                                               _dptr(x, n, "x"), 1 if x_is_zero else 0))

    def vcycle(self, r, z):
        n = self._n(0)
        self._check(lib().amgps_vcycle(self._h, _dptr(r, n, "r"), _dptr(z, n, "z")))

    def smooth_backward(self, level, kind, degree, b, x0, gx, want_x0=True, want_weights=True):
        """Reverse mode of one smoother application: (gb, gx0 or None, gweights or None)."""
        import torch
        n = self._n(level)
        gb = torch.empty(n, dtype=torch.float64, device=gx.device)
        gx0 = torch.empty_like(gb) if want_x0 else None
        gw = np.zeros(degree) if want_weights else None
        self._check(lib().amgps_smooth_backward(
            self._h, level, KIND[kind], degree, _dptr(b, n, "b"),
            None if x0 is None else _dptr(x0, n, "x0"), _dptr(gx, n, "gx"), _dptr(gb, n, "gb"),
            None if gx0 is None else _dptr(gx0, n, "gx0"),
            None if gw is None else gw.ctypes.data))
        return gb, gx0, gw

    def vcycle_backward(self, r, gz, want_r=True):
        """Reverse mode of one V-cycle: (gr or None, [dL/dbeta_l] per non-coarsest level)."""
        import torch
        n = self._n(0)
        gr = torch.empty(n, dtype=torch.float64, device=gz.device) if want_r else None
        gw = np.zeros((max(self.n_levels - 1, 1), 16))
        self._check(lib().amgps_vcycle_backward(self._h, _dptr(r, n, "r"), _dptr(gz, n, "gz"),
                                                None if gr is None else _dptr(gr, n, "gr"),
                                                gw.ctypes.data))
        return gr, gw[: self.n_levels - 1]

    def loss_grad(self, E0):
        """Mean A-norm error reduction of one V-cycle over the rows of E0
        (m x n_0 CUDA float64) and its weight gradient: (loss, (levels-1, 16))."""
        m = E0.shape[0]
        loss = C.c_double()
        gw = np.zeros((max(self.n_levels - 1, 1), 16))
        self._check(lib().amgps_vcycle_loss_grad(self._h, _dptr(E0, m * self._n(0), "E0"), m,
                                                 C.byref(loss), gw.ctypes.data))
        return loss.value, gw[: self.n_levels - 1]

    def error_cycles(self, E, cycles):
        """E <- (I - B A)^cycles E, in place, for each row of E (m x n_0 CUDA float64)."""
        m = E.shape[0]
        self._check(lib().amgps_error_cycles(self._h, _dptr(E, m * self._n(0), "E"), m, int(cycles)))

    def pcg(self, b, x, rtol=1e-8, maxit=1000, raise_on_noconv=True):
        n = self._n(0)
        it, rel = C.c_int(), C.c_double()
        st = lib().amgps_pcg(self._h, _dptr(b, n, "b"), _dptr(x, n, "x"), rtol, maxit,
                             C.byref(it), C.byref(rel))
        if st == 3 and not raise_on_noconv:
            return it.value, rel.value
        self._check(st)
        return it.value, rel.value

    def pcg_smoother(self, kind, degree, b, x, rtol=1e-5, maxit=10000, raise_on_noconv=True):
        """PCG preconditioned by one level-0 smoother application (no coarse levels)."""
        n = self._n(0)
        it, rel = C.c_int(), C.c_double()
        st = lib().amgps_pcg_smoother(self._h, KIND[kind], degree, _dptr(b, n, "b"), _dptr(x, n, "x"),
                                      rtol, maxit, C.byref(it), C.byref(rel))
        if st == 3 and not raise_on_noconv:
            return it.value, rel.value
        self._check(st)
        return it.value, rel.value

    def pcg_host(self, b, x, rtol=1e-8, maxit=1000):
        """b, x: host arrays (numpy float64, or pinned CPU torch tensors)."""
        n = self._n(0)
        bp, xp = self._host_ptr(b, n), self._host_ptr(x, n)
        it, rel = C.c_int(), C.c_double()
        self._check(lib().amgps_pcg_host(self._h, bp, xp, rtol, maxit, C.byref(it), C.byref(rel)))
        return it.value, rel.value

    @staticmethod
    def _host_ptr(a, n):
        try:
            import torch
            if isinstance(a, torch.Tensor):
                if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
                    raise TypeError("host tensor must be contiguous float64 CPU with n entries")
                return C.c_void_p(a.data_ptr())
        except ImportError:
            pass
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                and (n is None or a.size == n)):
            raise TypeError("host array must be contiguous float64 with n entries")
        return C.c_void_p(a.ctypes.data)

    def set_tma(self, on):
        """Step kernel choice: True (default: TMA-fed kernel on levels large
        enough for it), False (direct kernel everywhere), "always" (TMA-fed
        kernel wherever a level's layout allows it)."""
        v = 2 if on == "always" else (1 if on else 0)
        self._check(lib().amgps_set_option(self._h, OPT_TMA, v))

    def set_alloc_limit(self, nbytes):
        """Most device bytes the context may allocate for a hierarchy (0: no limit);
        a load that would pass it fails with AMGPS_E_NOMEM and keeps nothing."""
        self._check(lib().amgps_set_option(self._h, OPT_ALLOC_LIMIT, int(nbytes)))

    def set_step_form(self, form):
        """Polynomial smoothers on the large FP64 levels: 1 (default) the
        stored-operator form (Clenshaw steps, one stored operator per step),
        0 the recurrence form; equal to rounding."""
        self._check(lib().amgps_set_option(self._h, OPT_STEP_FORM, int(form)))

    def set_coarse_kernel(self, on):
        """Coarse levels (below the TMA-fed ones): True one persistent kernel,
        False (default) one launch per kernel; identical results."""
        self._check(lib().amgps_set_option(self._h, OPT_COARSE_KERNEL, 1 if on else 0))

    def set_coarse_sweeps(self, m):
        """Coarsest-level solve: 0 = dense inverse (default), m > 0 = m
        l1-Jacobi sweeps from zero (the paper's coarse solver)."""
        self._check(lib().amgps_set_option(self._h, OPT_COARSE_SWEEPS, int(m)))

    OUTER = {"cg": 0, "flexible": 1, "fcg1": 2}

    def set_flexible(self, on):
        """Outer CG form of pcg / pcg_smoother: False or "cg" (standard),
        True or "flexible" (Polak-Ribiere beta), "fcg1" (flexible CG with one
        reduction per iteration)."""
        v = self.OUTER[on] if isinstance(on, str) else (1 if on else 0)
        self._check(lib().amgps_set_option(self._h, OPT_FLEXIBLE, v))

    def synchronize(self):
        self._check(lib().amgps_synchronize(self._h))

    def profile(self, on=True):
        self._check(lib().amgps_profile_enable(self._h, 1 if on else 0))

    def profile_flops(self, cls):
        """Algorithmic FP64 flops of the class's timed launches since its last
        reset (read before profile_read(cls, reset=True))."""
        f = C.c_double()
        self._check(lib().amgps_profile_flops(self._h, cls, C.byref(f)))
        return f.value

    def profile_fp64_inst(self, cls):
        """FP64 thread instructions of the class's timed launches since its
        last reset (read before profile_read(cls, reset=True))."""
        f = C.c_double()
        self._check(lib().amgps_profile_fp64_inst(self._h, cls, C.byref(f)))
        return f.value

    def profile_read(self, cls, reset=False):
        n, ms, by = C.c_int64(), C.c_double(), C.c_double()
        self._check(lib().amgps_profile_read(self._h, cls, 1 if reset else 0, C.byref(n),
                                             C.byref(ms), C.byref(by)))
        return n.value, ms.value, by.value
