"""Experiments of the paper reproduced on the GPU path.

smoother_only: the remark of Sec. 2.3 -- PCG iteration counts (tol 1e-5,
b = A 1) when the preconditioner is one application of the optimised
1st-kind (Algorithm 1) or 4th-kind (Eq. polsmootheropt) polynomial smoother
alone, on A = Q D Q^T with equispaced, boundary-clustered and gapped spectra,
for several sizes and degrees.  The paper shows these counts only as images.

sa_solve: PCG on a smoothed-aggregation hierarchy built on the GPU (a short
fixed command for profiling that path).

degree_sweep: PCG iterations and time per iteration against the degree
(k = 1..12, five kinds) on the grid^3 Poisson problem.

CLI:  python -m paper_2407_09848_gb300.experiments smoother_only
      python -m paper_2407_09848_gb300.experiments sa_solve [grid]
      python -m paper_2407_09848_gb300.experiments degree_sweep [grid]
"""
from __future__ import annotations

import json
import sys

from . import problems as pr


def smoother_only(sizes=(128, 256, 512, 1024), degrees=(1, 2, 3, 4, 5, 6, 8, 10, 12),
                  spectra=("equispaced", "boundary", "gap"), rtol=1e-5):
    import torch
    from .amgps import Solver
    out = []
    for spec in spectra:
        for N in sizes:
            A, b = pr.spectral_test_matrix(N, spec)
            As, Ps = pr.single_aggregate_hierarchy(A)
            S = Solver().load(As, Ps)
            bd = torch.from_numpy(b).cuda()
            x = torch.empty_like(bd)
            for k in degrees:
                row = {"spectrum": spec, "N": N, "degree": k}
                for kind in ("cheb1_opt", "cheb4_opt"):
                    it, rel = S.pcg_smoother(kind, k, bd, x, rtol=rtol, maxit=20000,
                                             raise_on_noconv=False)
                    row[kind] = it
                out.append(row)
            S.close()
    return out


def sa_solve(grid=256, kind="cheb4_opt", degree=4, solves=2, rtol=1e-8):
    """Smoothed-aggregation hierarchy of the grid^3 Poisson problem built on
    the GPU, then `solves` PCG solves (the first one warms up): iterations and
    the last solve's time.  A fixed, short command for profiling the SA path."""
    import time
    import torch
    from .amgps import Solver
    st = pr.poisson(grid)
    builder = Solver()
    As, Ps, _ = builder.sa_hierarchy(pr.to_csr(st), pr.geometric_aggregates(st.shape, 512))
    builder.close()
    S = Solver().load(As, Ps)
    S.set_smoother(-1, kind, degree)
    b = torch.from_numpy(pr.rhs_uniform(As[0].shape[0], seed=0)).cuda()
    x = torch.empty_like(b)
    out = {}
    for _ in range(solves):
        torch.cuda.synchronize()
        t = time.perf_counter()
        it, rel = S.pcg(b, x, rtol=rtol)
        torch.cuda.synchronize()
        out = {"grid": grid, "kind": kind, "degree": degree, "iterations": it, "relres": rel,
               "ms": 1e3 * (time.perf_counter() - t)}
    S.close()
    return out


def degree_sweep(grid=256, degrees=(1, 2, 3, 4, 5, 6, 8, 10, 12),
                 kinds=("cheb4_opt", "cheb1_opt", "cheb4", "cheb1", "l1jacobi"), rtol=1e-8):
    """The supplementary trend of the paper (Sec. 4 and its supplement):
    PCG iterations and time per iteration against the polynomial degree, on
    the grid^3 Poisson problem with unsmoothed aggregation, FP64.  CHEB1 uses
    rho = 1.1 x the 10-step power estimate of each level."""
    import time
    import torch
    from .amgps import Solver
    H = pr.build_hierarchy(pr.poisson(grid), coarse_max=512)
    S = Solver().load(H.A, H.P)
    b = torch.from_numpy(pr.rhs_uniform(H.A[0].shape[0], seed=0)).cuda()
    x = torch.empty_like(b)
    rows = []
    for kind in kinds:
        for k in degrees:
            if kind == "cheb1":
                for l in range(H.n_levels - 1):
                    v0 = torch.from_numpy(pr.vec_uniform(H.A[l].shape[0], seed=0)).cuda()
                    S.set_smoother(l, "cheb1", k, rho=1.1 * S.estimate_lambda(l, v0, iters=10))
            else:
                S.set_smoother(-1, kind, k)
            S.pcg(b, x, rtol=rtol, maxit=2000)
            torch.cuda.synchronize()
            t = time.perf_counter()
            it, rel = S.pcg(b, x, rtol=rtol, maxit=2000)
            torch.cuda.synchronize()
            ms = 1e3 * (time.perf_counter() - t)
            rows.append({"kind": kind, "degree": k, "iterations": it, "ms": round(ms, 3),
                         "ms_per_iteration": round(ms / max(it, 1), 4)})
    S.close()
    return rows


def main(argv):
    if len(argv) >= 1 and argv[0] == "smoother_only":
        print(json.dumps(smoother_only()))
        return 0
    if len(argv) >= 1 and argv[0] == "degree_sweep":
        grid = int(argv[1]) if len(argv) > 1 else 256
        print(json.dumps(degree_sweep(grid)))
        return 0
    if len(argv) >= 1 and argv[0] == "sa_solve":
        grid = int(argv[1]) if len(argv) > 1 else 256
        print(json.dumps(sa_solve(grid)))
        return 0
    print(__doc__)
    return 2


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
