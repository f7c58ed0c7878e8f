"""Write tests/golden/oracle_sa_pcg_iterations.json: PCG iteration counts of
the FP64 oracle on smoothed-aggregation hierarchies (calls only oracle/ and
the input generators).

For each grid: Poisson 7-point, geometric 2x2x2 aggregates to <= 512 rows,
P = (I - omega D^{-1} A) P_hat and A_c = P^T A P by oracle/sa.py, b = U[-1,1]
(seed 0), x0 = 0, PCG to ||r|| <= 1e-8 ||b||, for the listed smoother kinds
and degrees.  The GPU builds the same hierarchy itself (amgps_sa_level) and
must reach the same counts.

Run: python tests/golden/make_oracle_sa_iterations.py [--grids 32,64,256]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(ROOT, "tests", "golden", "oracle_sa_pcg_iterations.json")
RUNS = [("cheb4_opt", 4), ("cheb1_opt", 2), ("l1jacobi", 4)]


def run_grid(grid):
    from oracle import sa
    from oracle.amg import OracleAMG
    from oracle.smoother import SmootherSpec
    from paper_2407_09848_gb300 import problems as pr
    st = pr.poisson(grid)
    levels = pr.geometric_aggregates(st.shape, coarse_max=512)
    t = time.time()
    As, Ps, oms = sa.sa_hierarchy(pr.to_csr(st), [a for a, _, _ in levels],
                                  [nc for _, nc, _ in levels])
    t_setup = time.time() - t
    b = pr.rhs_uniform(As[0].shape[0], seed=0)
    rows = []
    for kind, k in RUNS:
        t = time.time()
        _, it, rel, _ = OracleAMG(As, Ps, SmootherSpec(kind, k)).pcg(b, rtol=1e-8, maxit=1000)
        rows.append({"grid": grid, "kind": kind, "degree": k, "iterations": it, "relres": rel,
                     "levels": [a.shape[0] for a in As], "nnz": [a.nnz for a in As],
                     "omega": oms, "oracle_setup_seconds": t_setup,
                     "oracle_seconds": time.time() - t})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grids", default="32,64,256")
    a = ap.parse_args()
    grids = [int(g) for g in a.grids.split(",")]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(grids)) as pool:
        res = pool.map(run_grid, grids, chunksize=1)
    old = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            old = {(r["grid"], r["kind"], r["degree"]): r for r in json.load(f)["runs"]}
    for rows in res:
        for r in rows:
            old[(r["grid"], r["kind"], r["degree"])] = r
    runs = sorted(old.values(), key=lambda r: (r["grid"], r["kind"], r["degree"]))
    with open(OUT, "w") as f:
        json.dump({"problem": "poisson 7-point, smoothed aggregation (2x2x2 aggregates, omega = "
                              "4/(3 row-sum bound of D^-1 A)) to <=512, b=U[-1,1] seed 0, x0=0, "
                              "rtol=1e-8 (recurrence residual), FP64 oracle",
                   "runs": runs}, f, indent=1)


if __name__ == "__main__":
    main()
