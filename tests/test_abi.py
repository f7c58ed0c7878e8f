"""The C-ABI library builds, loads and exports every declared entry point;
its host-only table calls agree with the oracle and the paper (no GPU)."""
import os
import numpy as np
import pytest

from conftest import load_constants
from paper_2407_09848_gb300 import amgps, build

ROWS = load_constants()


@pytest.fixture(scope="module")
def lib():
    build.build()
    return amgps.lib()


def test_every_declared_symbol_is_exported(lib):
    names = amgps.header_symbols()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name


def test_version(lib):
    assert lib.amgps_version() >= 1


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"k{r[0]}")
def test_astar_table(lib, row):
    from oracle import params
    k, a_pr = row[0], row[1]
    a = amgps.cheb1_astar(k)
    # the oracle solves in double precision: a few units of rounding
    assert abs(a - params.a_star(k)) <= 2e-15 * a
    assert abs(a - a_pr) <= 1e-14 * a_pr


@pytest.mark.parametrize("row", ROWS[:10], ids=lambda r: f"k{r[0]}")
def test_opt4_table_agrees_with_oracle(lib, row):
    # two independent solvers of Eq. prob1 (the library's table: high-precision
    # Newton on the equioscillation system; the oracle: a Remez exchange)
    from oracle import params, smoother
    k, g_pr = row[0], row[4]
    beta_lib = amgps.opt4_weights(k)
    beta_ora = smoother.opt4_table(k)
    assert np.max(np.abs(beta_lib - beta_ora)) <= 1e-12
    g = params.gamma_opt4(beta_lib)
    assert abs(g - g_pr) <= 1e-9 * g_pr


def test_table_degree_bounds(lib):
    with pytest.raises(amgps.AmgpsError):
        amgps.opt4_weights(17)
    with pytest.raises(amgps.AmgpsError):
        amgps.cheb1_astar(0)


def test_create_reports_missing_gpu(lib):
    import ctypes
    import torch
    h = ctypes.c_void_p()
    st = lib.amgps_create(ctypes.byref(h), 0, None)
    if torch.cuda.is_available():
        assert st == 0
        lib.amgps_destroy(h)
    else:
        assert st == 5  # AMGPS_E_CUDA, reported without touching a device
        assert lib.amgps_last_error(None)
        assert not h.value


def test_null_arguments_rejected_on_host(lib):
    import ctypes
    assert lib.amgps_create(None, 0, None) == 1
    assert lib.amgps_smooth(None, 0, 2, 4, None, None, 1) == 1
    assert lib.amgps_pcg(None, None, None, 1e-8, 10, None, None) == 1
    assert lib.amgps_destroy(None) == 0
    assert lib.amgps_opt4_weights(4, None) == 1


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_tma_plan_covers_and_checks_copies(lib, prec):
    # host-only: the plan proves every bulk copy in bounds / aligned (else E_ARG)
    from paper_2407_09848_gb300 import problems as pr
    for st in (pr.poisson(16), pr.poisson(33, 17, 9), pr.varcoef(24, 1.0, 4.0, seed=1),
               pr.poisson(64)):
        H = pr.build_hierarchy(st)
        for lv in H.levels[:-1]:
            n = lv.A.shape[0]
            tiles, gen, stage, nst = amgps.tma_plan_stats(lv.A, prec)
            nslices = (n + 31) // 32
            per = (512 if prec == "f64" else 1024) // 32
            assert tiles * per + gen == nslices
            if tiles:
                budget = 230400 if prec == "f64" else 115200  # one CTA per SM for FP64, two otherwise
                assert 2 <= nst <= 8 and nst * stage + 128 <= budget and stage % 128 == 0
                assert prec != "f64" or nst % 2 == 0  # a multiple of the two consumer groups
    # 64^3: (almost) every tile whose +-4096-row windows stay inside the vector
    # qualifies; the exceptions are tiles where the slice pattern changes
    H = pr.build_hierarchy(pr.poisson(64))
    tiles, gen, _, _ = amgps.tma_plan_stats(H.levels[0].A, prec)
    rows = 512 if prec == "f64" else 1024
    per = rows // 32
    assert tiles * per + gen == 8192 and tiles >= (262144 - 2 * 4096) // rows - 64 // per - 2


def test_tma_plan_rejects_bad_csr(lib):
    import scipy.sparse as sp
    A = sp.csr_matrix(np.array([[2.0, -1.0], [-1.0, 2.0]]))
    A.indices[0] = 5  # column out of range
    with pytest.raises(amgps.AmgpsError):
        amgps.tma_plan_stats(A, "f64")


def test_layout_of_wide_smoothed_aggregation_levels(lib):
    # host-only: a smoothed-aggregation coarse level (the oracle's product, up to
    # 168 offsets per row) goes through the SELL builder's wide uniform path;
    # stencils wider than the TMA window limit are left to the direct kernel
    import scipy.sparse as sp
    from oracle import sa
    from paper_2407_09848_gb300 import problems as pr
    st = pr.poisson(32)
    levels = pr.geometric_aggregates(st.shape, coarse_max=512)
    As, _, _ = sa.sa_hierarchy(pr.to_csr(st), [a for a, _, _ in levels],
                               [nc for _, nc, _ in levels])
    for A in As[1:]:
        A = sp.csr_matrix(A)
        assert np.diff(A.indptr).max() > 8
        tiles, gen, _, _ = amgps.tma_plan_stats(A, "f64")
        assert tiles == 0 and gen == (A.shape[0] + 31) // 32
    # a duplicated entry in a wide row is rejected
    A = sp.csr_matrix(As[1]).sorted_indices()
    r0 = A.indptr[100]
    dup = A.copy()
    dup.indices[r0 + 1] = dup.indices[r0]
    with pytest.raises(amgps.AmgpsError):
        amgps.tma_plan_stats(dup, "f64")


def test_header_compiles_as_c(tmp_path):
    # the boundary is a C ABI: include/amgps.h must stay valid C11, and the
    # quick-start calls must type-check against it
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "quick.c"
    src.write_text(
        '#include "amgps.h"\n#include <stddef.h>\n'
        "int quick(int nl, const amgps_csr* A, const amgps_csr* P, const double* b, double* x) {\n"
        "  amgps_ctx* ctx;\n"
        "  if (amgps_create(&ctx, 0, NULL) != AMGPS_OK) return -1;\n"
        "  amgps_hierarchy_load(ctx, nl, A, P, AMGPS_F64);\n"
        "  amgps_set_smoother(ctx, -1, AMGPS_CHEB4_OPT, 4, NULL, 0.0);\n"
        "  amgps_set_option(ctx, AMGPS_OPT_FLEXIBLE, 2);\n"
        "  int it; double rel;\n"
        "  amgps_pcg(ctx, b, x, 1e-8, 1000, &it, &rel);\n"
        "  amgps_csr_buf Ac = {0};\n"
        "  amgps_galerkin(ctx, A, P, &Ac);\n"
        "  amgps_csr_buf_free(&Ac);\n"
        "  amgps_destroy(ctx);\n"
        "  return it;\n}\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-c", "-I", inc, str(src), "-o",
                        str(tmp_path / "quick.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_malformed_csr_rejected_on_host(lib):
    # host-only: every malformed CSR form returns AMGPS_E_ARG from the validator
    # that hierarchy_load shares, before any layout or device work
    import ctypes as C

    def plan(n_rows, n_cols, rowptr, col, val):
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        vv = np.ascontiguousarray(val, dtype=np.float64)
        nnz = int(len(ci))
        csr = amgps.CSR(n_rows, n_cols, nnz, rp.ctypes.data, ci.ctypes.data, vv.ctypes.data)
        t, g, sb, ns = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
        st = lib.amgps_tma_plan_stats(C.byref(csr), 0, C.byref(t), C.byref(g), C.byref(sb),
                                      C.byref(ns))
        return st, lib.amgps_last_error(None).decode()

    good = ([0, 2, 4], [0, 1, 0, 1], [2.0, -1.0, -1.0, 2.0])
    assert plan(2, 2, *good)[0] == 0
    cases = {
        "empty matrix": (0, 0, [0], [0], [0.0]),
        "not square": (2, 3, *good),
        "bad rowptr ends": (2, 2, [0, 2, 3], *good[1:]),
        "rowptr not monotone": (3, 3, [0, 3, 1, 4], [0, 1, 2, 2], [2.0, -1.0, -1.0, 2.0]),
        "duplicate entry": (2, 2, [0, 3, 4], [0, 1, 0, 1], [2.0, -1.0, -1.0, 2.0]),
        "column index out of range": (2, 2, [0, 2, 4], [0, 2, 0, 1], good[2]),
        "negative column": (2, 2, [0, 2, 4], [0, -1, 0, 1], good[2]),
        "non-finite value": (2, 2, [0, 2, 4], good[1], [2.0, np.nan, -1.0, 2.0]),
        "infinite value": (2, 2, [0, 2, 4], good[1], [2.0, -1.0, np.inf, 2.0]),
    }
    for name, args in cases.items():
        st, msg = plan(*args)
        assert st == 1, (name, st, msg)  # AMGPS_E_ARG
        assert msg, name
    assert lib.amgps_tma_plan_stats(None, 0, None, None, None, None) == 1
    assert plan(2, 2, *good)[0] == 0 and lib.amgps_tma_plan_stats(
        C.byref(amgps.CSR(2, 2, 4, 0, 0, 0)), 0, None, None, None, None) == 1  # null arrays


def test_binding_constants_match_header():
    # the Python binding's status, kind, precision and option numbers are the
    # enumerators of include/amgps.h
    import re
    txt = open(amgps.HEADER).read()
    enum = {m.group(1): int(m.group(2))
            for m in re.finditer(r"\b(AMGPS_[A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    for code, name in amgps.STATUS.items():
        assert enum[name] == code, name
    assert {n for n in enum if n.startswith("AMGPS_E_") or n == "AMGPS_OK"} == set(
        amgps.STATUS.values())
    for kind, v in amgps.KIND.items():
        assert enum["AMGPS_" + kind.upper()] == v, kind
    for prec, v in amgps.PREC.items():
        assert enum["AMGPS_" + prec.upper()] == v, prec
    assert (enum["AMGPS_OPT_TMA"], enum["AMGPS_OPT_FLEXIBLE"], enum["AMGPS_OPT_COARSE_SWEEPS"],
            enum["AMGPS_OPT_COARSE_KERNEL"], enum["AMGPS_OPT_ALLOC_LIMIT"]) == (
        amgps.OPT_TMA, amgps.OPT_FLEXIBLE, amgps.OPT_COARSE_SWEEPS, amgps.OPT_COARSE_KERNEL,
        amgps.OPT_ALLOC_LIMIT)


def test_fp64_stage_count_is_even(lib):
    # a banded matrix whose seven offsets chain into one window of 2400 + 512
    # elements (gaps of at most 544) leaves room for three 60.2 KB FP64 stages
    # of 512-row tiles (values 28,672 B, r_in and x_in 8,192 B, window
    # 23,296 B); the planner keeps two, a multiple of the FP64 shape's two
    # consumer groups
    import scipy.sparse as sp
    from paper_2407_09848_gb300 import problems as pr
    offs = [-1200, -656, -112, 0, 112, 656, 1200]
    n = 9600
    A = sp.diags([np.full(n - abs(o), 8.0 if o == 0 else -1.0) for o in offs], offs).tocsr()
    tiles, gen, stage, nst = amgps.tma_plan_stats(A, "f64")
    assert tiles > 0 and stage == 60160 and nst == 2
    tiles, gen, stage, nst = amgps.tma_plan_stats(pr.to_csr(pr.poisson(256, 8, 8)), "f64")
    assert nst == 4


def _sell_spmv(L, n, x):
    """y = A x evaluated from the SELL-32 arrays the way the device rows read
    them: explicit columns, or row + offset clamped to [0, n-1] in uniform
    slices; lanes past n are dropped."""
    y = np.zeros(n)
    lanes = np.arange(32)
    for s in range(len(L["vbase"])):
        rows = 32 * s + lanes
        live = rows < n
        for k in range(int(L["width"][s])):
            e = int(L["vbase"][s]) + 32 * k + lanes
            if L["cref"][s] >= 0:
                c = np.clip(rows + int(L["off"][L["cref"][s] + k]), 0, n - 1)
            else:
                c = L["col"][e]
            y[rows[live]] += L["val"][e][live] * x[c[live]]
    return y


def _sell_entries(L, n):
    """(row, col, val) of every stored nonzero of the layout."""
    out = []
    lanes = np.arange(32)
    for s in range(len(L["vbase"])):
        rows = 32 * s + lanes
        for k in range(int(L["width"][s])):
            e = int(L["vbase"][s]) + 32 * k + lanes
            v = L["val"][e]
            if L["cref"][s] >= 0:
                assert np.all(L["col"][e] == -1)
                c = rows + int(L["off"][L["cref"][s] + k])
            else:
                c = L["col"][e]
                assert np.all((c >= 0) & (c < n))     # padding keeps an in-range column
            nz = v != 0
            assert np.all(rows[nz] < n) and np.all((c[nz] >= 0) & (c[nz] < n))
            out.append(np.stack([rows[nz], c[nz]], 1))
            out.append(v[nz])
    rc = np.concatenate(out[0::2]) if out else np.zeros((0, 2), int)
    vals = np.concatenate(out[1::2]) if out else np.zeros(0)
    return rc, vals


def test_sell_layout_reproduces_the_matrix(lib):
    # host-only: the layout hierarchy_load uploads holds every entry of A once,
    # bit for bit, and the device's row semantics evaluated on it give A x
    import scipy.sparse as sp
    from oracle import sa
    from paper_2407_09848_gb300 import problems as pr
    mats = {"poisson16": pr.to_csr(pr.poisson(16)),
            "poisson33x17x9": pr.to_csr(pr.poisson(33, 17, 9)),
            "varcoef": pr.to_csr(pr.varcoef(20, 1.0, 3.0, seed=2, ny=13, nz=11)),
            "aniso": pr.to_csr(pr.aniso(12, 1e-3)),
            "lap1d_70": sp.diags([-np.ones(69), 2 * np.ones(70), -np.ones(69)], [-1, 0, 1]).tocsr()}
    st = pr.poisson(16)
    lev = pr.geometric_aggregates(st.shape, coarse_max=8)
    As, _, _ = sa.sa_hierarchy(pr.to_csr(st), [a for a, _, _ in lev], [c for _, c, _ in lev])
    for i, A in enumerate(As[1:]):
        mats[f"sa_level{i + 1}"] = sp.csr_matrix(A)
    rng = np.random.default_rng(4)
    R = sp.random(300, 300, density=0.03, random_state=5, data_rvs=lambda m: rng.uniform(-1, 1, m))
    R = (R + R.T + sp.diags(np.full(300, 20.0))).tolil()
    R[7, :] = rng.uniform(-1, 1, 300)                 # one dense row: a wide explicit slice
    R[7, 7] = 50.0
    mats["random_explicit"] = sp.csr_matrix(R)
    kinds = set()
    for name, A in mats.items():
        A = sp.csr_matrix(A)
        A.sum_duplicates()
        A.eliminate_zeros()
        n = A.shape[0]
        L = amgps.sell_layout(A)
        assert len(L["vbase"]) == (n + 31) // 32
        kinds |= {"uniform" if c >= 0 else "explicit" for c in L["cref"]}
        rc, vals = _sell_entries(L, n)
        B = sp.csr_matrix((vals, (rc[:, 0], rc[:, 1])), shape=A.shape)
        assert B.nnz == A.nnz == len(vals), name            # no entry stored twice
        B.sort_indices()
        A.sort_indices()
        assert np.array_equal(B.indptr, A.indptr) and np.array_equal(B.indices, A.indices), name
        assert np.array_equal(B.data, A.data), name         # values copied bit for bit
        x = rng.uniform(-1, 1, n)
        y = _sell_spmv(L, n, x)
        assert np.max(np.abs(y - A @ x)) <= 1e-13 * np.abs(A).sum(axis=1).max(), name
    assert kinds == {"uniform", "explicit"}
    # a wide smoothed-aggregation level stays uniform (no column stream)
    Lw = amgps.sell_layout(mats["sa_level1"])
    assert np.all(Lw["cref"] >= 0) and Lw["width"].max() > 32


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tma_plan_stage_emulation(lib, prec):
    # host-only: replay the producer's copies of every planned tile into a
    # stage (values block, the tile's own rows, one window of u per group) and
    # the consumers' shared-memory reads (entry k of tile row i at window index
    # d[k] + i): each planned row must give (A u)_row, its own-row read (d0) must
    # be u_row, and tiles plus left-over slices must cover every slice once
    from paper_2407_09848_gb300 import problems as pr
    rng = np.random.default_rng(11)
    planned = 0
    for st in (pr.poisson(64, 40, 12), pr.varcoef(48, 1.0, 3.0, seed=3, ny=40, nz=9),
               pr.aniso(40, 1e-3), pr.poisson(480, 4, 4), pr.poisson(300, 3, 3),
               pr.poisson(512, 4, 4), pr.varcoef(520, 1.0, 3.0, seed=4, ny=4, nz=3)):
        A = pr.to_csr(st)
        n = A.shape[0]
        L = amgps.sell_layout(A)
        P = amgps.tma_plan(A, prec)
        rows, w = P["rows"], P["w"]
        spt = rows // 32
        covered = np.zeros(len(L["vbase"]), int)
        covered[P["gen"]] += 1
        u = rng.uniform(-1, 1, n)
        Au = A @ u
        planned += len(P["tiles"])
        for r0, vb in P["tiles"]:
            assert r0 % rows == 0 and r0 + rows <= n
            s0 = r0 // 32
            covered[s0:s0 + spt] += 1
            assert np.all(L["cref"][s0:s0 + spt] == L["cref"][s0])   # one uniform pattern
            vals = L["val"][vb:vb + w * rows]                         # the values copy
            win = np.zeros(int(P["win_bytes"]) // (8 if prec == "f64" else 4))
            for g in range(P["ngroups"]):
                a, m, o = int(P["g_start"][g]), int(P["g_elems"][g]), int(P["g_smem"][g])
                assert 0 <= r0 + a and r0 + a + m <= n                # copies stay inside u
                win[o:o + m] = u[r0 + a:r0 + a + m]
            i = np.arange(rows)
            cs, lane = i // 32, i % 32
            acc = np.zeros(rows)
            for k in range(w):
                acc += vals[cs * w * 32 + k * 32 + lane] * win[P["d"][k] + i]
            assert np.max(np.abs(acc - Au[r0:r0 + rows])) <= 1e-13 * np.abs(A).sum(axis=1).max()
            assert np.array_equal(win[P["d0"] + i], u[r0:r0 + rows])
        assert np.all(covered == 1)
    assert planned > 90


def test_tma_plan_merges_the_windows_of_512_wide_grids(lib):
    # host-only: with R-row FP64 tiles the -nx..+nx offsets of a grid up to
    # R + 65 wide share one window (for R < nx the gap the window copies along
    # is at most 64 elements), so a 7-point level has three window groups and,
    # with no 1/M slot in FP64 stages, four stages at 512-wide; one column
    # wider the gap exceeds the slack, five groups exceed the plan's four and
    # no tile is planned
    from paper_2407_09848_gb300 import problems as pr
    rows = amgps.tma_plan(pr.to_csr(pr.poisson(64, 16, 16)), "f64")["rows"]
    for nx in (rows - 31, 512, rows + 1, rows + 65):
        P = amgps.tma_plan(pr.to_csr(pr.poisson(nx, 16, 16)), "f64")
        assert P["ngroups"] == 3 and len(P["tiles"]) > 0, nx
        assert P["g_elems"][1] >= 2 * nx + rows  # rows -nx .. nx + rows - 1 of the tile
        if nx == 512:
            assert P["nstages"] == 4
    P = amgps.tma_plan(pr.to_csr(pr.poisson(rows + 66, 16, 16)), "f64")
    assert len(P["tiles"]) == 0
    # 256-wide grids keep their windows and four stages
    P = amgps.tma_plan(pr.to_csr(pr.poisson(256, 16, 16)), "f64")
    assert P["ngroups"] == 3 and P["nstages"] == 4


@pytest.mark.parametrize("kind", ["cheb4", "cheb4_opt", "weights", "cheb1_opt", "cheb1",
                                  "cheb4_rho"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 9, 16])
def test_step_coefs_realise_the_error_polynomials(lib, kind, k):
    # host-only: run the library's step scalars through the kernels' recurrences
    # on one eigen-component (M^{-1}A = lambda, b = 0, error e0 = 1): the error
    # after one application must be the closed-form polynomial of Sec. 2.1 /
    # Algorithm 1 (the oracle's parameter code)
    from oracle import params as P
    # the 4th-kind closed form (via arccos) holds on [0, 1]; tau_k also beyond
    lam = np.linspace(0.0, 1.0 if kind.startswith("cheb4") or kind == "weights" else 1.3, 131)
    weights = 1.0 + 0.2 * np.sin(np.arange(1, k + 1)) if kind == "weights" else None
    rho = {"cheb1": 1.07, "cheb4_rho": 1.2}.get(kind, 0.0)
    explicit_rho = kind == "cheb4_rho"
    kind = "cheb4" if explicit_rho else kind
    c1, c2, beta, rhoinv = amgps.step_coefs(kind, k, weights, rho)
    if kind in ("cheb4", "cheb4_opt", "weights"):
        x, z, r = np.ones_like(lam), np.zeros_like(lam), -lam   # r = M^{-1}(b - A x)
        for j in range(1, k + 1):
            z = c1[j] * z + c2[j] * r
            x = x + beta[j] * z
            r = r - lam * z
        if kind == "cheb4":
            ref = P.p_cheb4(k, lam / (1.2 if explicit_rho else 1.0))
            assert np.all(beta[1:] == 1.0)
        else:
            # the library's tabulated weights (pinned to the oracle's Remez
            # solution by test_opt4_table_agrees_with_oracle)
            b = amgps.opt4_weights(k) if kind == "cheb4_opt" else weights
            ref = P.p_opt4(b, lam)
    else:
        a = P.a_star(k)
        rr = 1.07 if kind == "cheb1" else 1.0
        assert rhoinv == pytest.approx(1.0 / rr, rel=1e-15)
        r = rhoinv * (-lam)
        d = c2[0] * r
        x = 1.0 + d
        for j in range(1, k):
            r = r - rhoinv * lam * d
            d = c1[j] * d + c2[j] * r
            x = x + d
        ref = P.p_cheb1(k, a, lam, rr)
    assert np.max(np.abs(x - ref)) <= 5e-12 * max(1.0, np.abs(ref).max())


def _bf16_value(bits):
    import struct
    from fractions import Fraction
    return Fraction(struct.unpack("<f", struct.pack("<I", int(bits) << 16))[0])


def _bf16_reference(x):
    """Nearest BF16 to x, ties to the even pattern, by exact rational comparison
    of the two BF16 neighbours that bracket x (BF16 = the high 16 bits of an
    FP32 pattern)."""
    import struct
    from fractions import Fraction
    X = Fraction(x)
    f = struct.unpack("<I", struct.pack("<f", float(np.float32(x))))[0] >> 16
    cands = [c & 0xFFFF for c in (f - 1, f, f + 1)]
    cands = [c for c in cands if (c & 0x7F80) != 0x7F80]          # finite patterns only
    best = min(cands, key=lambda c: (abs(_bf16_value(c) - X), c & 1))
    return best


def test_bf16_rounding_is_direct_and_ties_to_even(lib):
    # reading 13: FP64 -> BF16 directly, round to nearest, ties to even; an
    # intermediate FP32 rounding would turn a value just above a BF16 midpoint
    # into the midpoint itself and round it the wrong way
    import struct
    rng = np.random.default_rng(13)
    xs = list(rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000))
    for b in rng.integers(0x0080, 0x7F00, 300):       # around BF16 values and midpoints
        lo, hi = _bf16_value(b), _bf16_value(b + 1)
        mid = float((lo + hi) / 2)
        xs += [mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf), float(lo), -mid]
        # just above the midpoint but within half an FP32 ulp of it: FP32
        # rounding lands exactly on the midpoint (the double-rounding trap)
        f32_ulp = float(np.spacing(np.float32(mid)))
        xs.append(mid + 0.25 * f32_ulp)
        xs.append(mid - 0.25 * f32_ulp)
    xs += [0.0, -0.0, 6.0, -1.0, 1.0 / 3.0, 3.0e38, -3.0e38, 1e-38]
    got = amgps.round_bf16(np.array(xs))
    want = np.array([_bf16_reference(x) for x in xs], dtype=np.uint16)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(xs[i], hex(got[i]), hex(want[i])) for i in bad[:5]]
    # Poisson's values are exact in BF16
    assert np.array_equal(amgps.round_bf16(np.array([6.0, -1.0, 24.0, -4.0])),
                          np.array([0x40C0, 0xBF80, 0x41C0, 0xC080], dtype=np.uint16))
    with pytest.raises(amgps.AmgpsError):
        amgps.round_bf16(np.array([1.0, np.inf]))


def test_binding_rejects_non_device_vectors():
    # host-side: the binding passes only contiguous FP64 CUDA tensors of the
    # right length to the library (a host pointer never reaches a kernel)
    import torch
    with pytest.raises(TypeError):
        amgps._dptr(torch.zeros(8, dtype=torch.float64), 8, "b")           # host tensor
    with pytest.raises(TypeError):
        amgps._dptr(np.zeros(8), 8, "b")                                  # not a tensor
    with pytest.raises(TypeError):
        amgps._dptr(torch.zeros(8, dtype=torch.float32), 8, "b")
    with pytest.raises(TypeError):
        amgps._dptr(torch.zeros((4, 4), dtype=torch.float64).t(), 16, "b")  # non-contiguous
