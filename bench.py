#!/usr/bin/env python3
"""Benchmark of the hot path: V-cycle-preconditioned CG to ||r|| <= 1e-8 ||b||.

Workload (default): 3-D Poisson 7-point on a 256^3 grid (16.8 M unknowns,
Dirichlet), 2x2x2 aggregation down to <= 512 unknowns (6 levels), l1-Jacobi +
optimised 4th-kind Chebyshev smoother of degree 4 (Eq. polsmootheropt) before
and after the coarse correction, dense Cholesky on the coarsest level, FP64.
One step = one full PCG solve from x0 = 0 with the inputs resident on the GPU.

Printed (one JSON line on rank 0): time to solution (ms, lower is better,
timed with no per-kernel events), the roofline of the dominant kernel (the
fused smoother step on the finest level, from a separate pass of the same
solves with CUDA events around each of its launches), the end-to-end time
through the host-buffer C-ABI call, the CPU oracle baseline, clocks during the
timed region and the kernel launch count.

CPU baseline and reference arm: the all-core C build of the oracle loops
(oracle/c/amg_omp.c, OpenMP on every host core) solving the same system.
--impl reference times it as the reference of this build, each step one whole
PCG solve of the same workload.
"""
import os

# numpy's BLAS pools stay single-threaded (the C oracle build sets its own
# OpenMP thread count through its library call, not through this variable)
for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG-AMG time-to-1e-8 and smoother HBM GB/s: plain FP64 vs learned/mixed form"
GOLDEN_ITERS = os.path.join(ROOT, "tests", "golden", "oracle_pcg_iterations.json")
GOLDEN_SA = os.path.join(ROOT, "tests", "golden", "oracle_sa_pcg_iterations.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_step_poisson256_traffic.json")
STEP_SOURCES = [os.path.join(ROOT, "paper_2407_09848_gb300", "csrc", f)
                for f in ("kernels_tma.cu", "kernels_smooth.cu", "kernels_common.cuh",
                          "amgps_internal.h")]
LEARNED = os.path.join(ROOT, "paper_2407_09848_gb300", "data", "learned_weights_lognormal64.npz")


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--kind", default="cheb4_opt")
    ap.add_argument("--degree", type=int, default=4)
    ap.add_argument("--prec", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--step-form", type=int, default=1, choices=[0, 1],
                    help="FP64 polynomial steps: 1 stored operators (default), 0 recurrence")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed-precision (192^3) and learned+mixed (256^3) comparisons")
    ap.add_argument("--cpu-oracle", default=None, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def workload_name(a):
    return f"poisson{a.grid}^3_{a.kind}_k{a.degree}_{a.prec}"


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(value, dist=None):
    """Largest `value` over all ranks (replicas report the slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def step_source_hash():
    h = hashlib.sha256()
    for p in STEP_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def host_info():
    """Logical CPUs and CPU model of the host the CPU oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def golden_iterations(grid, kind, degree):
    if not os.path.exists(GOLDEN_ITERS):
        return None
    with open(GOLDEN_ITERS) as f:
        for r in json.load(f)["runs"]:
            if r["grid"] == grid and r["kind"] == kind and r["degree"] == degree:
                return int(r["iterations"])
    return None


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_smi_id(torch, dev):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    try:
        props = torch.cuda.get_device_properties(dev)
        bus = getattr(props, "pci_bus_id", None)
        dom = getattr(props, "pci_domain_id", 0)
        if bus is not None:
            out = subprocess.run(["nvidia-smi", "--query-gpu=index,pci.bus_id", "--format=csv,noheader"],
                                 capture_output=True, text=True, timeout=20).stdout
            for line in out.splitlines():
                idx, bid = [x.strip() for x in line.split(",")]
                parts = bid.split(":")
                if len(parts) >= 2 and int(parts[-2], 16) == bus and int(parts[0], 16) == dom:
                    return int(idx)
    except Exception:
        pass
    if vis:
        return vis.split(",")[dev]
    return dev


def build_problem(a):
    from paper_2407_09848_gb300 import problems as pr
    H = pr.build_hierarchy(pr.poisson(a.grid), coarse_max=512, name=f"poisson{a.grid}")
    b = pr.rhs_uniform(H.levels[0].A.shape[0], seed=0)
    return H, b


def configure(S, H, kind, degree, torch):
    from paper_2407_09848_gb300 import problems as pr
    if kind == "cheb1":
        for l in range(H.n_levels - 1):
            v0 = torch.from_numpy(pr.vec_uniform(H.levels[l].A.shape[0], seed=0)).cuda()
            lam = S.estimate_lambda(l, v0, iters=10)
            S.set_smoother(l, "cheb1", degree, rho=1.1 * lam)
    else:
        S.set_smoother(-1, kind, degree)


def oracle_specs(H, kind, degree):
    from oracle.smoother import SmootherSpec, power_lambda
    from paper_2407_09848_gb300 import problems as pr
    specs = []
    for lv in H.levels[:-1]:
        if kind == "cheb1":
            lam = power_lambda(lv.A, pr.vec_uniform(lv.A.shape[0], seed=0), iters=10)
            specs.append(SmootherSpec(kind, degree, rho=1.1 * lam))
        else:
            specs.append(SmootherSpec(kind, degree))
    return specs


def omp_oracle(A, P, specs):
    """The all-core C build of the oracle loops on this hierarchy."""
    from oracle import omp
    return omp.OmpAMG(A, P, specs)


def time_omp_solves(ora, b, rtol, count, warmup=1, budget_s=30.0):
    """Wall seconds of whole PCG solves by the C oracle: `warmup` untimed, then
    up to `count` timed ones (fewer once `budget_s` of timed work is spent,
    at least one).  Returns (times, iterations, relres)."""
    for _ in range(warmup):
        ora.pcg(b, rtol=rtol, maxit=1000)
    times, it, rel = [], 0, 0.0
    while len(times) < count:
        t = time.perf_counter()
        _, it, rel, _ = ora.pcg(b, rtol=rtol, maxit=1000)
        times.append(time.perf_counter() - t)
        if sum(times) >= budget_s:
            break
    return times, it, rel


def problem_stencil(spec):
    """The seeded stencil of a problem spec (dict): poisson / varcoef / aniso."""
    from paper_2407_09848_gb300 import problems as pr
    if spec["problem"] == "poisson":
        return pr.poisson(spec["grid"])
    if spec["problem"] == "varcoef":
        return pr.varcoef(spec["grid"], spec["sigma"], spec["ell"], seed=spec.get("seed", 0))
    return pr.aniso(spec["grid"], spec["eps"])


def cpu_oracle_main(spec):
    """Entry of the CPU-oracle subprocess (--cpu-oracle): builds the problem
    of `spec` and prints cpu_oracle_baseline's dict as one JSON line.  A fresh
    interpreter that never imports torch or initialises CUDA, so the OpenMP
    pool spans every host core, as in the reference arm."""
    from paper_2407_09848_gb300 import problems as pr
    H = pr.build_hierarchy(problem_stencil(spec), coarse_max=512)
    b = pr.rhs_uniform(H.levels[0].A.shape[0], seed=0)
    specs = oracle_specs(H, spec["kind"], spec["degree"])
    out = cpu_oracle_baseline(H.A, H.P, specs, b, spec["rtol"], spec["label"],
                              count=spec.get("count", 3), warmup=spec.get("warmup", 1))
    print(json.dumps(out))
    return 0


def cpu_oracle_subprocess(spec, timeout=900):
    """cpu_oracle_baseline of `spec` run in a spawned interpreter (see
    cpu_oracle_main); None with the reason when it fails."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-oracle", json.dumps(spec)],
                       capture_output=True, text=True, timeout=timeout, cwd=ROOT)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"unavailable": f"CPU oracle subprocess rc={r.returncode}: {r.stderr[-300:]}"}
    return json.loads(lines[-1])


def cpu_oracle_baseline(A, P, specs, b, rtol, label, count=3, warmup=1):
    """CPU baseline: median of whole solves by the all-core C oracle build,
    plus its single-thread time for one PCG iteration scaled by the iteration
    count (stated as extrapolated)."""
    from oracle import omp
    ora = omp_oracle(A, P, specs)
    threads = omp.threads()
    times, it, rel = time_omp_solves(ora, b, rtol, count=count, warmup=warmup)
    omp.set_threads(1)
    try:
        t = time.perf_counter()
        ora.pcg(b, rtol=1e-300, maxit=1)  # one V-cycle, one product with A_0, the CG updates
        t1 = time.perf_counter() - t
    finally:
        omp.set_threads(threads)
    ora.close()
    return {"value": 1e3 * statistics.median(times), "unit": "ms", "cores": threads,
            "kind": "oracle",
            "sample": f"{len(times)} whole PCG solves of {label} by the all-core C build of the "
                      f"oracle loops (OpenMP, {threads} threads), median",
            "iterations": it, "relres": rel, "host": host_info(),
            "single_thread": {"value": 1e3 * t1 * it, "unit": "ms", "cores": 1,
                              "extrapolated_from": f"one PCG iteration ({1e3 * t1:.1f} ms) x {it} "
                                                   f"iterations"}}


def timed_solve(S, bd, x, rtol, torch, reps=2):
    """(iterations, ms, relres) of one PCG solve, best of `reps` after one warm-up."""
    S.pcg(bd, x, rtol=rtol, maxit=2000)
    best = None
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        it, rel = S.pcg(bd, x, rtol=rtol, maxit=2000)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return it, best, rel


def step_roofline_of_solve(S, bd, x, rtol, torch, workload, prec):
    """HBM roofline of the level-0 step over one profiled solve (CUDA events
    around each level-0 step launch)."""
    from paper_2407_09848_gb300.amgps import PROF_STEP
    S.profile(True)
    S.profile_read(PROF_STEP, reset=True)
    S.pcg(bd, x, rtol=rtol, maxit=2000)
    torch.cuda.synchronize()
    S.profile(False)
    n_step, ms_step, by_step = S.profile_read(PROF_STEP, reset=True)
    return step_hbm_roofline(n_step, ms_step, by_step, committed_traffic(workload, prec))


def run_mixed_c1(a, torch, H, b):
    """256^3 Poisson, CHEB4_OPT k = 4: FP32 and BF16 matrix values on the
    smoother and transfer path (FP32 vectors and accumulation, FP64 PCG and
    coarse solve), with the level-0 step's HBM roofline."""
    import numpy as np
    from paper_2407_09848_gb300.amgps import Solver
    bd = torch.from_numpy(b).cuda()
    out = {"workload": f"poisson{a.grid}^3, CHEB4_OPT k4, rtol {a.rtol}"}
    for prec in ("f32", "bf16"):
        S = Solver().load(H.A, H.P, prec=prec)
        S.set_smoother(-1, "cheb4_opt", 4)
        x = torch.empty_like(bd)
        it, ms, rel = timed_solve(S, bd, x, a.rtol, torch)
        true = float(np.linalg.norm(b - H.levels[0].A @ x.cpu().numpy()) / np.linalg.norm(b))
        wl = f"poisson{a.grid}^3_cheb4_opt_k4_{prec}"
        out[prec] = {"iterations": it, "ms": round(ms, 3), "relres": rel, "true_relres": true,
                     "roofline": step_roofline_of_solve(S, bd, x, a.rtol, torch, wl, prec)}
        S.close()
    return out


def run_mixed_c2(a, torch, cpu=True):
    """192^3 variable coefficient (k = exp(g), GRF sigma 1, ell 8): FP64 vs
    FP32 / BF16 values on the smoother and transfer path (CHEB4_OPT k = 4),
    each with the level-0 step's HBM roofline, and the all-core C oracle's
    FP64 solve of the same system."""
    import numpy as np
    from paper_2407_09848_gb300 import problems as pr
    from paper_2407_09848_gb300.amgps import Solver
    H = pr.build_hierarchy(pr.varcoef(192, 1.0, 8.0, seed=0), coarse_max=512)
    b = pr.rhs_uniform(H.levels[0].A.shape[0], seed=0)
    bd = torch.from_numpy(b).cuda()
    out, ref = {}, None
    for prec in ("f64", "f32", "bf16"):
        S = Solver().load(H.A, H.P, prec=prec)
        x = torch.empty_like(bd)
        it, ms, rel = timed_solve(S, bd, x, a.rtol, torch)
        xs = x.cpu().numpy()
        true = float(np.linalg.norm(b - H.levels[0].A @ xs) / np.linalg.norm(b))
        if ref is None:
            ref = xs
        out[prec] = {"iterations": it, "ms": round(ms, 3), "relres": rel, "true_relres": true,
                     "solution_rel_diff_vs_f64": float(np.linalg.norm(xs - ref) / np.linalg.norm(ref)),
                     "roofline": step_roofline_of_solve(S, bd, x, a.rtol, torch,
                                                        "varcoef192^3_cheb4_opt_k4", prec)}
        S.close()
    if cpu:
        out["cpu_oracle_f64"] = cpu_oracle_subprocess(
            {"problem": "varcoef", "grid": 192, "sigma": 1.0, "ell": 8.0, "kind": "cheb4_opt",
             "degree": 4, "rtol": a.rtol, "label": "the 192^3 variable-coefficient system",
             "count": 1, "warmup": 0})
    return {"workload": "varcoef192^3 sigma1 ell8, CHEB4_OPT k4, rtol 1e-8", **out}


def run_sa_c1(a, torch):
    """256^3 Poisson with a smoothed-aggregation hierarchy built on the GPU
    (amgps_sa_level: SA prolongator + Galerkin SpGEMM per level) against the
    unsmoothed-aggregation hierarchy of the headline run; FP64, CHEB4_OPT k4
    and l1-Jacobi k4."""
    import numpy as np
    from paper_2407_09848_gb300 import problems as pr
    from paper_2407_09848_gb300.amgps import Solver
    st = pr.poisson(a.grid)
    levels = pr.geometric_aggregates(st.shape, coarse_max=512)
    A0 = pr.to_csr(st)
    builder = Solver()
    t0 = time.perf_counter()
    As, Ps, oms = builder.sa_hierarchy(A0, levels)
    t_build = time.perf_counter() - t0
    builder.close()
    t0 = time.perf_counter()
    S = Solver().load(As, Ps, prec="f64")
    t_load = time.perf_counter() - t0
    b = pr.rhs_uniform(A0.shape[0], seed=0)
    bd = torch.from_numpy(b).cuda()
    x = torch.empty_like(bd)
    out = {"workload": f"poisson{a.grid}^3 smoothed aggregation, rtol {a.rtol}",
           "levels": [m.shape[0] for m in As], "nnz_per_row": [round(m.nnz / m.shape[0], 1) for m in As],
           "operator_complexity": round(sum(m.nnz for m in As) / As[0].nnz, 3),
           "omega": [round(o, 6) for o in oms],
           "setup_s": {"sa_levels_on_gpu_incl_transfers": round(t_build, 3), "load": round(t_load, 3)}}
    gold = {}
    if os.path.exists(GOLDEN_SA):
        with open(GOLDEN_SA) as f:
            gold = {(r["grid"], r["kind"], r["degree"]): r["iterations"] for r in json.load(f)["runs"]}
    for kind, k in (("cheb4_opt", 4), ("l1jacobi", 4)):
        S.set_smoother(-1, kind, k)
        it, ms, rel = timed_solve(S, bd, x, a.rtol, torch)
        true = float(np.linalg.norm(b - A0 @ x.cpu().numpy()) / np.linalg.norm(b))
        out[f"{kind}_k{k}"] = {"iterations": it, "ms": round(ms, 3), "relres": rel,
                               "true_relres": true,
                               "oracle_iterations": gold.get((a.grid, kind, k))}
    # the paper's solver setting (Sec. 4): 30 l1-Jacobi sweeps on the coarsest
    # level, flexible CG with one reduction per iteration, tolerance 1e-7 (on
    # the residual here; the paper states it on the error)
    S.set_coarse_sweeps(30)
    S.set_flexible("fcg1")
    paper = {}
    for kind, k in (("cheb4_opt", 4), ("cheb1_opt", 4), ("l1jacobi", 4)):
        S.set_smoother(-1, kind, k)
        it, ms, rel = timed_solve(S, bd, x, 1e-7, torch)
        paper[f"{kind}_k{k}"] = {"iterations": it, "ms": round(ms, 3), "relres": rel}
    out["paper_setting_coarse30_fcg1_rtol1e-7"] = paper
    S.close()
    return out


def run_learned_c4(a, torch, cpu=True):
    """256^3 log-normal (sigma 2, ell 16) and anisotropic (eps 1e-3 in z):
    plain FP64 with the optimal 4th-kind weights vs learned weights with
    BF16 / FP32 values (FP64 PCG and coarse solve), and the all-core C
    oracle's FP64 solve with the optimal weights."""
    import numpy as np
    from paper_2407_09848_gb300 import learn
    from paper_2407_09848_gb300 import problems as pr
    from paper_2407_09848_gb300.amgps import Solver
    if not os.path.exists(LEARNED):
        return {"unavailable": "no trained weights file"}
    net = learn.WeightMLP(seed=0).load(LEARNED)
    res = {"workload": "256^3, PCG to 1e-8; learned = MLP trained on 512 log-normal 64^3 problems"}
    for name, st in (("lognormal_s2_l16", pr.varcoef(256, 2.0, 16.0, seed=0)),
                     ("aniso_eps1e-3", pr.aniso(256, 1e-3))):
        H = pr.build_hierarchy(st, coarse_max=512)
        b = pr.rhs_uniform(H.levels[0].A.shape[0], seed=0)
        bd = torch.from_numpy(b).cuda()
        S64 = Solver().load(H.A, H.P, prec="f64")
        feats = learn.level_features(S64, H)
        betas = net.predict(feats)
        ref = learn.amgps.opt4_weights(4)
        safe = [learn.make_safe(bb, ref) for bb in betas]
        # the optimal weights judge the network on this hierarchy (set-up)
        t0 = time.perf_counter()
        used, rho_l, rho_o, keep = learn.judge(S64, betas)
        t_judge = time.perf_counter() - t0
        x = torch.empty_like(bd)
        row = {"predicted_weights": [list(map(float, bb)) for bb in betas],
               "safe_weights": [list(map(float, w)) for w, _ in safe],
               "t_towards_prediction": [float(t) for _, t in safe],
               "judge": {"pcg_factor_learned": rho_l, "pcg_factor_optimal": rho_o,
                         "learned_kept": bool(keep), "setup_s": round(t_judge, 3)},
               "used_weights": [list(map(float, w)) for w in used]}
        S64.set_smoother(-1, "cheb4_opt", 4)
        it, ms, rel = timed_solve(S64, bd, x, a.rtol, torch)
        row["f64_opt"] = {"iterations": it, "ms": round(ms, 3), "relres": rel}
        # the network's safe weights without the judge, for the record
        for l, (w, _) in enumerate(safe):
            S64.set_smoother(l, "weights", 4, weights=w)
        it, ms, rel = timed_solve(S64, bd, x, a.rtol, torch)
        row["f64_learned_unjudged"] = {"iterations": it, "ms": round(ms, 3), "relres": rel}
        S64.close()
        for prec in ("bf16", "f32"):
            S = Solver().load(H.A, H.P, prec=prec)
            it, ms, rel = timed_solve(S, bd, x, a.rtol, torch)
            row[f"{prec}_opt"] = {"iterations": it, "ms": round(ms, 3), "relres": rel}
            for l, w in enumerate(used):
                S.set_smoother(l, "weights", 4, weights=w)
            it, ms, rel = timed_solve(S, bd, x, a.rtol, torch)
            row[f"{prec}_learned"] = {"iterations": it, "ms": round(ms, 3), "relres": rel}
            S.close()
        row["speedup_bf16_learned_vs_f64_opt"] = round(row["f64_opt"]["ms"] / row["bf16_learned"]["ms"], 3)
        if cpu:
            pspec = ({"problem": "varcoef", "grid": 256, "sigma": 2.0, "ell": 16.0}
                     if name.startswith("lognormal") else {"problem": "aniso", "grid": 256,
                                                           "eps": 1e-3})
            row["cpu_oracle_f64_opt"] = cpu_oracle_subprocess(
                {**pspec, "kind": "cheb4_opt", "degree": 4, "rtol": a.rtol,
                 "label": f"the 256^3 {name} system", "count": 1, "warmup": 0})
        res[name] = row
    return res


def workload_config(a, H):
    """The workload both arms run (identical keys and values in both lines)."""
    return {"workload": workload_name(a), "grid": a.grid, "n": int(H.levels[0].A.shape[0]),
            "levels": H.n_levels, "nnz": int(H.levels[0].A.nnz), "kind": a.kind,
            "degree": a.degree, "prec": a.prec, "rtol": a.rtol,
            "l2": "inputs larger than L2 (finest matrix 0.94 GB, 129 MB L2)",
            "parallelism": "replicas" if dist_env()[1] > 1 else "none"}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import omp
    H, b = build_problem(a)
    ora = omp_oracle(H.A, H.P, oracle_specs(H, a.kind, a.degree))
    threads = omp.threads()
    for _ in range(a.warmup):
        ora.pcg(b, rtol=a.rtol, maxit=1000)
    times = []
    for _ in range(a.steps):
        t = time.perf_counter()
        _, its, rel, st = ora.pcg(b, rtol=a.rtol, maxit=1000)
        times.append(time.perf_counter() - t)
    ora.close()
    value_ms = 1e3 * statistics.mean(times)
    sample = (f"each step one whole PCG solve of {workload_name(a)} by the all-core C build of the "
              f"oracle loops (OpenMP, {threads} threads); value = mean over {a.steps} steps")
    out = {"impl": "reference", "metric": METRIC, "value": value_ms, "unit": "ms",
           "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": value_ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(a, H),
           "result": {"iterations": its, "relres": rel, "converged": st == 0,
                      "step_ms_min": 1e3 * min(times), "step_ms_max": 1e3 * max(times)},
           "cpu_baseline": {"value": value_ms, "unit": "ms", "cores": threads, "kind": "oracle",
                            "sample": sample, "host": host_info()},
           "e2e": {"value": value_ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def profiled_pass(S, bd, x, a, torch, smi):
    """The same solves again with CUDA events around each level-0 step launch
    (class 0), each level-0 residual + restriction (1), each PCG SpMV (2) and
    the levels below 0 (4).  Returns per-class (launches, ms, bytes) summed over
    the pass, its solve count and the clock summary sampled during it."""
    from paper_2407_09848_gb300.amgps import PROF_COARSE, PROF_RESTRICT, PROF_SPMV, PROF_STEP
    classes = (PROF_STEP, PROF_RESTRICT, PROF_SPMV, PROF_COARSE)
    S.profile(True)
    for c in classes:
        S.profile_read(c, reset=True)
    torch.cuda.synchronize()
    with ClockSampler(smi) as clk:
        for _ in range(a.steps):
            S.pcg(bd, x, rtol=a.rtol)
        torch.cuda.synchronize()
    S.profile(False)
    flops = S.profile_flops(PROF_STEP)  # before the reset below
    inst = S.profile_fp64_inst(PROF_STEP)
    out = {c: S.profile_read(c, reset=True) for c in classes}
    out["step_flops"] = flops
    out["step_fp64_inst"] = inst
    return out, a.steps, clk.summary()


def step_hbm_roofline(n_step, ms_step, by_step, traffic=None, kernel=None):
    peak, peak_src = measured_peak()
    achieved = (by_step / 1e9) / (ms_step / 1e3) if ms_step > 0 else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic,
            "kernel": kernel or "fused smoother step on level 0 (k_step_tma + leftover k_step)",
            "launches": n_step, "avg_launch_us": 1e3 * ms_step / max(n_step, 1),
            "bytes_per_launch": by_step / max(n_step, 1), "peak_source": peak_src}


def committed_traffic(workload, prec, step_form=1):
    """ncu DRAM bytes per launch of the level-0 step from the committed capture,
    when it was taken on the current sources of the step kernels in the same
    step form."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        tr = json.load(f)
    entries = tr if isinstance(tr, list) else [tr]
    for e in entries:
        if (e.get("source_sha256") == step_source_hash() and e.get("workload") == workload
                and e.get("prec", "f64") == prec and e.get("step_form", 0) == step_form):
            return e.get("dram_bytes_per_launch")
    return None


def run_ours(a):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2407_09848_gb300 import build as bld
    bld.build()
    from paper_2407_09848_gb300.amgps import PROF_COARSE, PROF_RESTRICT, PROF_SPMV, PROF_STEP, Solver

    H, b = build_problem(a)
    n = H.levels[0].A.shape[0]
    S = Solver(local).load(H.A, H.P, prec=a.prec)
    S.set_step_form(a.step_form)
    configure(S, H, a.kind, a.degree, torch)
    bd = torch.from_numpy(b).cuda()
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(a.warmup):
        its, rel = S.pcg(bd, x, rtol=a.rtol)
    torch.cuda.synchronize()

    # ---- timed region: K solves, CUDA events on the caller's stream, no
    # per-kernel events inside ----
    S.profile(False)
    S.profile_read(3, reset=True)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    smi = gpu_smi_id(torch, local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(smi) as clk:
        ev0.record(stream)
        for _ in range(a.steps):
            its, rel = S.pcg(bd, x, rtol=a.rtol)
        ev1.record(stream)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    total_ms = ev0.elapsed_time(ev1)
    launches, _, _ = S.profile_read(3, reset=True)
    ms_per = max_over_ranks(total_ms / a.steps, pg)
    true_res = float(np.linalg.norm(b - H.levels[0].A @ x.cpu().numpy()) / np.linalg.norm(b))
    clk = clk.summary()

    # ---- per-kernel split and roofline: a separate pass of the same solves ----
    prof, nprof, clk_prof = profiled_pass(S, bd, x, a, torch, smi)
    n_step, ms_step, by_step = prof[PROF_STEP]
    ms_rr, ms_sp, ms_coarse = prof[PROF_RESTRICT][1], prof[PROF_SPMV][1], prof[PROF_COARSE][1]
    traffic = committed_traffic(workload_name(a), a.prec, a.step_form)
    hbm = step_hbm_roofline(n_step, ms_step, by_step, traffic)
    hbm["share_of_solve_time"] = (ms_step / nprof) / ms_per if ms_per else None
    roof = hbm
    if a.prec == "f64" and a.kind in ("cheb4", "cheb4_opt", "weights") and n_step:
        # FP64 path: the step is bound by the FP64 pipe.  Flops per launch: the
        # library's algorithmic count over the profiled level-0 steps
        # (amgps_profile_flops: a multiply-add 2, a lone multiply 1, 2 per
        # nonzero for the products), averaged per launch.  In the
        # stored-operator form a k = 4 cycle's seven level-0 steps total
        # 14 nnz + 7 n (2 nnz + n per launch); the recurrence form's are
        # 2 nnz + 5 n per launch.  Peak: 304 FP64 FMA thread-instructions per
        # clock (152 SMs x 2, ncu peak_sustained) x 2 flops x the SM clock
        # sampled during the profiled pass.
        fl = prof["step_flops"] / n_step
        mhz = clk_prof.get("sm_mhz") or 2070.0
        fpeak = 304 * 2 * mhz * 1e6 / 1e12
        fach = fl / (1e-3 * ms_step / n_step) / 1e12
        # FP64 issue: thread instructions per launch (one per stored entry and
        # per vector term) against 304 per clock; a lone multiply is one flop
        # but a whole issue slot, so this is the pipe's utilisation
        inst = prof["step_fp64_inst"] / n_step
        issue = inst / (1e-3 * ms_step / n_step) / (304 * mhz * 1e6)
        roof = {"bound": "alu", "achieved": fach, "peak": fpeak, "unit": "TFLOP/s",
                "frac": fach / fpeak, "traffic": traffic, "kernel": hbm["kernel"],
                "flops_per_launch": fl, "fp64_inst_per_launch": inst,
                "fp64_issue_frac": issue,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2 flops x sampled SM clock",
                "launches": n_step, "avg_launch_us": hbm["avg_launch_us"],
                "share_of_solve_time": hbm["share_of_solve_time"], "hbm": hbm}
    roof["measured_in"] = (f"a pass of {nprof} solves after the timed region, CUDA events around "
                           f"each level-0 step launch on the library stream")
    roof["step_form"] = ("stored operators (Clenshaw steps)" if a.step_form == 1
                         else "recurrence (z, r, x)")
    roof["clocks"] = clk_prof

    # ---- end to end through the host-buffer C-ABI call ----
    bh = torch.from_numpy(b.copy()).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    S.pcg_host(bh, xh, rtol=a.rtol)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        S.pcg_host(bh, xh, rtol=a.rtol)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / a.steps

    # ---- smoother sweep of the 256^3 configuration (one solve each) ----
    sweep = None
    if not a.no_sweep and rank == 0:
        sweep = []
        for kind in ("cheb1", "cheb4", "cheb4_opt", "cheb1_opt", "l1jacobi"):
            for k in range(1, 7):
                configure(S, H, kind, k, torch)
                S.pcg(bd, x, rtol=a.rtol, maxit=1000)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                it_k, _ = S.pcg(bd, x, rtol=a.rtol, maxit=1000)
                torch.cuda.synchronize()
                sweep.append({"kind": kind, "degree": k, "iterations": it_k,
                              "ms": round(1e3 * (time.perf_counter() - t0), 3),
                              "oracle_iterations": golden_iterations(a.grid, kind, k)})
        configure(S, H, a.kind, a.degree, torch)
        # outer CG forms at the timed configuration: standard, flexible
        # (Polak-Ribiere), flexible with one reduction per iteration
        outer = []
        for form in ("cg", "flexible", "fcg1"):
            S.set_flexible(form)
            S.pcg(bd, x, rtol=a.rtol, maxit=1000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it_f, rel_f = S.pcg(bd, x, rtol=a.rtol, maxit=1000)
            torch.cuda.synchronize()
            outer.append({"form": form, "iterations": it_f,
                          "ms": round(1e3 * (time.perf_counter() - t0), 3), "relres": rel_f})
        S.set_flexible("cg")
        sweep = {"smoothers": sweep, "outer_cg_forms": outer}

    # ---- comparisons: mixed precision (256^3 Poisson, 192^3 variable
    # coefficient), learned + mixed (256^3), smoothed aggregation ----
    extras = None
    if not a.no_extras and rank == 0:
        S.close()
        extras = {"mixed_c1": run_mixed_c1(a, torch, H, b),
                  "mixed_c2": run_mixed_c2(a, torch, cpu=not a.no_cpu),
                  "learned_c4": run_learned_c4(a, torch, cpu=not a.no_cpu),
                  "smoothed_aggregation": run_sa_c1(a, torch)}

    # ---- CPU baseline: the all-core C oracle build on the same solve ----
    cpu = None
    if not a.no_cpu and rank == 0:
        cpu = cpu_oracle_subprocess({"problem": "poisson", "grid": a.grid, "kind": a.kind,
                                     "degree": a.degree, "rtol": a.rtol,
                                     "label": workload_name(a), "count": 3, "warmup": 1})

    out = {"metric": METRIC, "value": ms_per, "unit": "ms", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_per, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": a.prec, "data": "synthetic",
           "config": workload_config(a, H),
           "result": {"iterations": its, "relres": rel, "true_relres": true_res,
                      "oracle_iterations": golden_iterations(a.grid, a.kind, a.degree)},
           "roofline": roof,
           "cpu_baseline": cpu,
           "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 8 * n,
                   "d2h_bytes_per_step": 8 * n},
           "gpu_launches": launches,
           "clocks": clk,
           "kernel_ms": {"k_step_level0": ms_step / nprof, "k_resid_restrict_level0": ms_rr / nprof,
                         "k_spmv_dot": ms_sp / nprof, "coarse_levels": ms_coarse / nprof,
                         "measured_in": "the profiled pass (per solve)"},
           "sweep": sweep,
           "comparisons": extras}
    if rank == 0:
        print(json.dumps(out))
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    a = parse_args()
    if a.cpu_oracle:
        return cpu_oracle_main(json.loads(a.cpu_oracle))
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
