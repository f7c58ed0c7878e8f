"""Write tests/golden/oracle_pcg_iterations.json: PCG iteration counts of the
FP64 oracle on the seeded Poisson problems (calls only oracle/ and the input
generators).

For each grid (32^3, 256^3), smoother kind and degree k = 1..6: Poisson 7-point,
2x2x2 aggregation to <= 512 rows, b = U[-1,1] (seed 0), x0 = 0, PCG to
||r|| <= 1e-8 ||b||.  Kind "cheb1" uses rho_l = 1.1 * (10-step power estimate
from v0 = U[-1,1], seed 0, on each level).  The counts are the expected values
for the GPU path (identical iteration counts) and the scale factor of the
oracle's bounded timing sample in the benchmark.

Run: python tests/golden/make_oracle_iterations.py [--grids 32,256] [--jobs 6]

Runs are merged into the stored file by (grid, kind, degree).  The committed
file was written by the default run plus
  --kinds cheb4,cheb4_opt,cheb1_opt,l1jacobi --degrees 8,10,12,16 --grids 32
  --kinds cheb4,cheb4_opt,cheb1_opt,l1jacobi --degrees 8,10,12 --grids 256
  --kinds l1jacobi --degrees 1,2,3,4,5,6
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(ROOT, "tests", "golden", "oracle_pcg_iterations.json")
KINDS = ["cheb1", "cheb4", "cheb4_opt", "cheb1_opt"]
DEGREES = [1, 2, 3, 4, 5, 6]
ALL_KINDS = KINDS + ["l1jacobi"]

_H = {}


def _hier(grid):
    from paper_2407_09848_gb300 import problems as pr
    if grid not in _H:
        _H.clear()
        _H[grid] = pr.build_hierarchy(pr.poisson(grid), coarse_max=512)
    return _H[grid]


def run_one(args):
    grid, kind, k = args
    from oracle.amg import OracleAMG
    from oracle.smoother import SmootherSpec, power_lambda
    from paper_2407_09848_gb300 import problems as pr
    H = _hier(grid)
    specs = []
    for lv in H.levels[:-1]:
        if kind == "cheb1":
            lam = power_lambda(lv.A, pr.vec_uniform(lv.A.shape[0], seed=0), iters=10)
            specs.append(SmootherSpec(kind, k, rho=1.1 * lam))
        else:
            specs.append(SmootherSpec(kind, k))
    ora = OracleAMG(H.A, H.P, specs)
    b = pr.rhs_uniform(H.levels[0].A.shape[0], seed=0)
    t = time.time()
    _, it, rel, _ = ora.pcg(b, rtol=1e-8, maxit=1000)
    return {"grid": grid, "kind": kind, "degree": k, "iterations": it, "relres": rel,
            "oracle_seconds": time.time() - t}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grids", default="32,256")
    ap.add_argument("--kinds", default=",".join(KINDS))
    ap.add_argument("--degrees", default=",".join(map(str, DEGREES)))
    ap.add_argument("--jobs", type=int, default=4)
    a = ap.parse_args()
    grids = [int(g) for g in a.grids.split(",")]
    kinds = [k for k in a.kinds.split(",") if k in ALL_KINDS]
    degrees = [int(k) for k in a.degrees.split(",")]
    tasks = [(g, kd, k) for g in grids for kd in kinds for k in degrees]
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.jobs) as pool:
        rows = pool.map(run_one, tasks, chunksize=1)
    old = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            old = {(r["grid"], r["kind"], r["degree"]): r for r in json.load(f)["runs"]}
    for r in rows:
        old[(r["grid"], r["kind"], r["degree"])] = r
    runs = sorted(old.values(), key=lambda r: (r["grid"], r["kind"], r["degree"]))
    with open(OUT, "w") as f:
        json.dump({"problem": "poisson 7-point, 2x2x2 aggregation to <=512, b=U[-1,1] seed 0, "
                              "x0=0, rtol=1e-8 (recurrence residual), FP64 oracle",
                   "runs": runs}, f, indent=1)


if __name__ == "__main__":
    main()
