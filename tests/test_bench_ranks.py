"""The multi-rank path of bench.py on the CPU. Under torchrun the bench runs one process per GPU;
the ranks are replicas (each solves its own instance of the workload, no data-path collective),
the job's time is the slowest rank's and its work the sum over ranks. That host-side logic is
checked here with two gloo ranks launched the way torchrun launches them (RANK, WORLD_SIZE,
MASTER_ADDR, MASTER_PORT in the environment); no GPU is involved."""
import json
import os
import socket
import subprocess
import sys

import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
rank, world, local = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
try:
    ms = bench.max_over_ranks(dist, 1.0 + 2.0 * rank)        # rank 0: 1 ms, rank 1: 3 ms
    units = bench.job_units(dist, 100.0 + rank)             # 100 and 101 DOF
    p = bench.problem_for_rank(rank)
    print(json.dumps({"rank": rank, "world": world, "local": local, "ms": ms, "units": units,
                      "N": p.N, "M": p.M, "k": p.k}), flush=True)
finally:
    dist.destroy_process_group()
"""


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ)
    env.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port), BENCH_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
    return env


def test_two_gloo_ranks_reduce_like_the_bench():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=_env(r, 2, port), cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for pr in procs:
        try:
            out, err = pr.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert pr.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for r, o in enumerate(outs):
        assert (o["rank"], o["world"], o["local"]) == (r, 2, r)
        assert o["ms"] == 3.0            # the slowest rank's time, on every rank
        assert o["units"] == 201.0       # the work of both ranks
    # replicas: every rank solves an instance of the same shape
    assert (outs[0]["N"], outs[0]["M"], outs[0]["k"]) == (outs[1]["N"], outs[1]["M"], outs[1]["k"])


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 2.5) == 2.5
    assert bench.job_units(None, 7.0) == 7.0


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun the oracle arm runs and prints on rank 0; the other ranks exit 0 without work
    env = _env(1, 2, _free_port())
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=180)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_reference_arm_times_the_whole_oracle_solve():
    # one rank: every step is the oracle's solve of all N levels, and ms_per_step is that measured
    # time (value = N M / time), not an extrapolation from a sample of levels
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--workload", "heat1d"], cwd=ROOT, capture_output=True, text=True, timeout=180)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert "all 64 of 64 time levels" in line["cpu_baseline"]["sample"]
    dof = line["config"]["dof"]
    assert abs(line["ms_per_step"] - 1e3 * dof / line["value"]) <= 1e-9 * line["ms_per_step"]
    assert line["e2e"]["value"] == line["value"]


def test_stored_ncu_traffic_applies_to_its_own_workload_only():
    # the DRAM traffic bench.py reports beside a roofline comes from an ncu capture of one
    # workload; another workload's launch of the same kernel moves different bytes
    sys.path.insert(0, ROOT)
    import bench
    captured = "heat2d_255x255_N256_bdf4"
    assert captured in bench.NCU_TRAFFIC
    for name, (value, src, _sha) in bench.NCU_TRAFFIC[captured].items():
        assert bench.traffic_for(name, captured) in (None, value)   # null once the source changed
        assert bench.traffic_for(name, "periodic2d_256x256_N256_bdf4") is None
        assert bench.traffic_for(name, "fem_example1_M1023_N128_k3") is None
    assert bench.traffic_for("no_such_kernel", captured) is None


def test_oracle_sample_reports_the_error_of_given_solutions():
    # the bench line's accuracy figure: each GPU solution against the oracle's levels
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    from oracle import grid, sequential
    p = workloads.c1_heat1d()
    ref = sequential.solve_sequential(p.k, p.alpha, p.tau, grid.operator(p), p.v, p.f(), p.fderiv())
    info = bench.oracle_sample(p, budget_s=1.0, results={"same": ref, "off": ref * (1 + 1e-9)})
    n_s = info["levels_compared"]
    assert 8 <= n_s <= p.N
    assert info["rel_err_vs_oracle"]["same"] == 0.0
    assert abs(info["rel_err_vs_oracle"]["off"] - 1e-9) <= 1e-12


def test_second_cpu_reference_sample():
    # the diagonalised WR solve on the host (bench's cpu_diag_wr entry): the GPU's sweep count from
    # U_0 = v, its accuracy reported against the oracle beside the GPU solutions'
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    p = workloads.c1_heat1d()
    info, U = bench.diag_wr_sample(p, 3)
    assert info["value"] > 0 and info["cores"] >= 1 and U.shape == (p.N, p.M)
    errs = bench.oracle_sample(p, budget_s=1.0, results={"cpu_diag_wr": U})["rel_err_vs_oracle"]
    assert errs["cpu_diag_wr"] <= 1e-10
    assert bench.diag_wr_sample(workloads.fem_problem(mx=15, N=16, k=2), 3) is None   # FD only


def test_every_profiled_kernel_has_algorithmic_bytes():
    # bench.py's roofline divides a kernel's algorithmic bytes by its CUDA-event time: every name
    # the library's per-kernel profiler can report needs an entry
    import re
    sys.path.insert(0, ROOT)
    import bench
    csrc = os.path.join(ROOT, "paper_2007_13125_gb300", "csrc")
    names = set()
    for fn in os.listdir(csrc):
        if not fn.endswith(".cu"):
            continue
        text = open(os.path.join(csrc, fn)).read()
        for m in re.finditer(r"prof_begin\(([^;]*);", text):
            names |= set(re.findall(r'"([a-z0-9_]+)"', m.group(1)))
        for m in re.finditer(r"const char\* name = ([^;]*);", text):
            names |= set(re.findall(r'"([a-z0-9_]+)"', m.group(1)))
    assert len(names) >= 25
    missing = sorted(n for n in names if bench.algo_bytes(n, 64, 63) <= 0)
    assert not missing, missing


def test_oracle_check_of_returned_solutions():
    # the mix64 / serve lines compare a bounded subset of returned solutions with the oracle
    sys.path.insert(0, ROOT)
    import bench
    from oracle import grid, sequential
    p = workloads.small_problem(dim=1, mx=31, N=32, k=2, alpha=0.5, kappa=0.1)
    ref = sequential.solve_sequential(p.k, p.alpha, p.tau, grid.operator(p), p.v, p.f(), p.fderiv())
    big = workloads.c2_heat2d()     # N M = 16.6 M: skipped as too large for a bounded CPU run
    out = bench.oracle_check([(p, ref), (big, None), (p, ref * (1 + 1e-9))])
    assert out["checked"] == 2
    assert out["per_problem"][0]["rel_err"] == 0.0
    assert abs(out["max_rel_err_by_kind"]["1d_cq"] - 1e-9) < 1e-12
