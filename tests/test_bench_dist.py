"""bench.py's multi-process plumbing on the CPU (gloo, world size 2): the
replicas report the slowest rank, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks(10.0 + rank, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 11.0, 1: 11.0}


def test_single_process_and_reference_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    old = dict(os.environ)
    try:
        os.environ.update(RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
        import argparse
        args = argparse.Namespace(impl="reference", steps=1, warmup=0, grid=8, kind="cheb4_opt",
                                  degree=4, prec="f64", rtol=1e-8)
        assert bench.run_reference(args) == 0   # non-zero ranks exit without work
    finally:
        os.environ.clear()
        os.environ.update(old)


def test_reference_arm_json_line():
    # the oracle arm on the CPU: one JSON line with the benchmark contract's keys
    import json
    import subprocess
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--grid", "32", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in r, key
    assert r["impl"] == "reference" and r["value"] > 0 and r["higher_is_better"] is False
    # the all-core C oracle build: every host core, whole solves per step
    assert r["cpu_baseline"]["cores"] >= 1 and r["cpu_baseline"]["kind"] == "oracle"
    assert r["result"]["iterations"] == 11 and r["result"]["converged"]
    assert r["e2e"]["h2d_bytes_per_step"] == 0 and r["e2e"]["value"] == r["value"]


def test_clock_summary_parses_nvidia_smi_lines():
    # the clocks key of the bench line: median SM clock under load, the
    # maximum, and every throttle reason seen active in any sample
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "1965, 2070, 1398.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
               "garbage"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = []
    assert c.summary()["samples"] == 0 and c.summary()["sm_mhz"] is None


def test_cpu_baseline_times_whole_solves_of_the_c_oracle():
    sys.path.insert(0, ROOT)
    import bench
    from oracle import omp
    from oracle.amg import OracleAMG
    from paper_2407_09848_gb300 import problems as pr
    H = pr.build_hierarchy(pr.poisson(16), coarse_max=64)
    b = pr.rhs_uniform(H.A[0].shape[0], seed=0)
    specs = bench.oracle_specs(H, "cheb4_opt", 4)
    cb = bench.cpu_oracle_baseline(H.A, H.P, specs, b, 1e-8, "16^3", count=2, warmup=0)
    _, it, _, _ = OracleAMG(H.A, H.P, specs).pcg(b, rtol=1e-8)
    assert cb["kind"] == "oracle" and cb["cores"] == omp.threads() and cb["unit"] == "ms"
    assert cb["iterations"] == it and cb["value"] > 0 and cb["host"]["nproc"] == os.cpu_count()
    assert cb["single_thread"]["cores"] == 1 and "extrapolated_from" in cb["single_thread"]
    assert omp.threads() == cb["cores"]  # the single-thread sample restores the pool


def test_reference_arm_line_has_the_workload_config(capsys):
    sys.path.insert(0, ROOT)
    import bench
    import json
    args = bench.parse_args(["--impl", "reference", "--grid", "16", "--steps", "2", "--warmup", "1"])
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    H, _ = bench.build_problem(args)
    assert line["impl"] == "reference" and line["config"] == bench.workload_config(args, H)
    assert line["steps"] == 2 and line["value"] == line["ms_per_step"] > 0
    assert line["result"]["converged"] and line["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_oracle_runs_in_a_fresh_interpreter():
    # the bench's CPU baselines run in a spawned interpreter that imports no
    # torch, so the OpenMP pool is the host's whole core set
    sys.path.insert(0, ROOT)
    import bench
    out = bench.cpu_oracle_subprocess({"problem": "poisson", "grid": 16, "kind": "cheb4_opt",
                                       "degree": 4, "rtol": 1e-8, "label": "16^3", "count": 1,
                                       "warmup": 0})
    assert out["kind"] == "oracle" and out["iterations"] > 0 and out["value"] > 0
    assert out["cores"] == len(os.sched_getaffinity(0))
