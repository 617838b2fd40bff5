"""Benchmark of the parallel-in-time solve on the 2D heat workload.

Workload (one "step" = one whole solve through the hot path): 2D heat on the unit square,
255 x 255 interior points, N = 256 steps, T = 1, BDF4 with starting-step corrections,
kappa = 0.05, f = e^{-t} sin(pi x) sin(2 pi y), v a 64 x 64-mode random sine series (seed 1).
A step forms F_hat from (v, f, d^l f(0)) and runs WR sweeps from U_0^n = v (pint_solve_v: the
first sweep's residual F_hat - beta_n v - A v is formed from v, U_0 is never written) until the
solver's a-posteriori error estimate is below tol = 1e-8 (the estimate includes the rounding
floor of the FP32 inner solves; relative l2 error <= 1e-8 against the sequential FP64 solution
is checked at this size and tolerance by tests/test_gpu_parity.py).

value   = space-time DOF (N * M) per second of the MIXED path, inputs resident in HBM.
e2e     = the same through host buffers (pinned H2D of v, f, d^l f(0); D2H of U) per step.
The FP64 diagonalised path (Algorithm 1 in FP64) is timed beside it on the same GPU.

``--impl reference`` times the CPU oracle (sequential FP64 BDF4 with a sparse LU) on a
bounded sample of the same workload, on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "space-time DOF/s to rel err 1e-8 (mixed vs FP64 diag); p50/p99 solve latency"
UNIT = "DOF/s"
TOL = 1e-8

# algorithmic bytes per launch of each kernel, as a function of (N, M)
def algo_bytes(name: str, N: int, M: int, K: int = 1) -> float:
    NM, JM = N * M, (N // 2 + 1) * M
    table = {
        "resid_fwd_ff": 16 * NM + 8 * JM,       # read U, F_hat (double-float); write half spectrum
        "resid_v0_ff": 8 * NM + 8 * JM,         # first sweep from v: read F_hat; write half spectrum
        "inv_update_v0_ff": 8 * JM + 8 * NM,    # first sweep: read spectrum; write U (double-float)
        "inv_update_ff": 8 * JM + 16 * NM,      # read spectrum; read + write U (double-float)
        "dst_f32": 16 * JM,                     # read + write spectrum (complex float)
        "dst_tc_f32": 16 * JM,                  # the same transform as tensor-core products
        "dst_tc_y_f32": 16 * JM,                # the y transform of 3D grids, the same way
        "axis_solve_tc_f32": 16 * JM,           # the z solve of 3D grids, two tensor-core passes
        "axis_solve_f32": 16 * JM,
        "rhs_f64": 16 * NM,                     # read f, write F_hat
        "rhs_head_f64": 16 * K * M,             # F_hat's first k levels: read f, write
        "cvt_d2ff": 16 * NM,
        "cvt_ff2d": 16 * NM,
        "initial_guess": 8 * NM,
        "direct_fwd_f64": 8 * NM + 16 * JM,
        "direct_inv_f64": 16 * JM + 16 * NM,
        "dst_f64": 32 * JM,
        "axis_solve_f64": 32 * JM,
        "toeplitz_f64": 16 * NM,                # read U, write the history product
        "toeplitz_ff": 16 * NM,                 # read U (hi, lo), write the history (hi, lo)
        "trivar_solve_f32": 32 * JM,            # read + write spectrum, read the two LU factors
        "trivar_solve_f64": 64 * JM,
        "trivar_factor": 16 * JM,               # write the two LU factors (FP32)
        "nl_linearise": 8 * NM,                 # read U
        "nl_rhs": 32 * NM,                      # read F_hat, U; write the linearised F_hat, U_{l-1}
        "nl_norms": 16 * NM,                    # read U, U_{l-1}
        "small_solve_ff": 16 * NM,              # one-CTA solve: read F_hat, write U (the rest stays on chip)
        "cvt_bcast_d2ff": 8 * NM,               # write U_0 = v on every level (double-float)
        "cvt_d2f": 12 * NM,                     # read FP64, write FP32
        "cvt_f2d": 12 * NM,
        "tri_y_f32": 16 * JM,                   # read + write spectrum (complex float)
        "pcr_y_f32": 16 * JM,                   # the same systems by parallel cyclic reduction
        "axis_solve_per_f32": 16 * JM,
        "fft_per_f32": 16 * JM,
        "axis_solve_per_f64": 32 * JM,
        "fft_per_f64": 32 * JM,
        "direct_fwd_f32": 4 * NM + 8 * JM,      # read F (FP32), write half spectrum
        "direct_inv_f32": 8 * JM + 8 * NM,      # read spectrum, U old; write U (FP32)
        "window_rhs": 16 * NM,                  # read f, write F_hat
    }
    return float(table.get(name, 0.0))


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of a workload (`ncu --set full` of `bench.py --once mixed`), per workload and kernel, valid while
# the kernel's source is unchanged (sha1 of its translation unit); other workloads report null
NCU_TRAFFIC = {
    "heat2d_255x255_N256_bdf4": {
        "resid_fwd_ff": (317.82e6, "kernels_resid.cu", "bef7a9dcb9ea6525c6c50e53b5f4b76293ad46a2"),
        "resid_v0_ff": (167.23e6, "kernels_resid.cu", "bef7a9dcb9ea6525c6c50e53b5f4b76293ad46a2"),
        "inv_update_v0_ff": (141.95e6, "kernels_time.cu", "4f1bc2da689b12f51d0599e98cff88feff864466"),
        "inv_update_ff": (277.48e6, "kernels_time.cu", "4f1bc2da689b12f51d0599e98cff88feff864466"),
        "dst_f32": (76.07e6, "kernels_space.cu", "75607f77d5b73a2e1fbb1c5ca20a86e16298a900"),
        "dst_tc_f32": (75.21e6, "kernels_dst_tc.cu", "cc4217510b4500885aa87744fecb930383c9a098"),
        "axis_solve_f32": (78.60e6, "kernels_space.cu", "75607f77d5b73a2e1fbb1c5ca20a86e16298a900"),
    },
    "heat3d_127x127x63_N32_k4_a1.0": {
        "dst_tc_y_f32": (217.41e6, "kernels_dst_tc.cu", "cc4217510b4500885aa87744fecb930383c9a098"),
    },
}


def traffic_for(name: str, workload: str):
    import hashlib
    ent = NCU_TRAFFIC.get(workload, {}).get(name)
    if not ent:
        return None
    path = os.path.join(ROOT, "paper_2007_13125_gb300", "csrc", ent[1])
    try:
        h = hashlib.sha1(open(path, "rb").read()).hexdigest()
    except OSError:
        return None
    return ent[0] if h == ent[2] else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    The sampler is started (and its first sample awaited) before the warm-up, so that starting
    nvidia-smi does not fall inside the timed region; every line is stamped with the host time
    at which it arrived and stop(t0, t1) keeps the samples of [t0, t1] (the nearest one when the
    region is shorter than the sampling interval)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None
        self.ready = threading.Event()

    def start(self, wait_s: float = 5.0):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        self.ready.wait(wait_s)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))
            self.ready.set()

    def stop(self, t0: float, t1: float) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        lag = 2 * self.INTERVAL_MS / 1000.0
        time.sleep(lag)  # the sample covering t1 arrives a little later
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        inside = [ln for t, ln in self.lines if t0 <= t <= t1 + lag]
        where = "timed region"
        if not inside and self.lines:
            t_mid = 0.5 * (t0 + t1)
            inside = [min(self.lines, key=lambda tl: abs(tl[0] - t_mid))[1]]
            where = "nearest sample to the timed region"
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": where}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


WORKLOADS = {"heat2d": workloads.c2_heat2d, "heat1d": workloads.c1_heat1d,
             "subdiff1d": workloads.c3_subdiff1d,
             # Example 1's data (Sec. 4) with P1 finite elements at the paper's scale on a
             # power-of-two mesh: 1023 nodes, N = 128, T = 0.5, BDF3, kappa = 0.5
             "fem1d": lambda: workloads.fem_problem(mx=1023, N=128, k=3, alpha=1.0, kappa=0.5, T=0.5,
                                                    data="example1"),
             # periodic boundary conditions (FFT in space), the heat2d scale: 256 x 256, N = 256
             "periodic2d": lambda: workloads.periodic_problem(dim=2, mx=256, my=256, N=256, k=4, alpha=1.0,
                                                              kappa=0.05, seed=1, modes=32),
             # 3D heat on the unit cube: 127^3 interior points, N = 128, BDF4 (2.1 GB per FP64 array)
             "heat3d": lambda: workloads.heat3d_problem(m=127, N=128, k=4, alpha=1.0, kappa=0.05, seed=1,
                                                        modes=8),
             # 127 x 127 x 63 points, N = 32 (~1 GB on the device; the half spectrum, 138 MB, is
             # larger than L2): the size of the 3D profiler captures
             "heat3d_small": lambda: workloads.heat3d_problem(m=127, mz=63, N=32, k=4, alpha=1.0, kappa=0.05,
                                                              seed=1, modes=8)}
# Example 4 (Sec. 4.3, Allen-Cahn, eps = 1) with P1 elements at the paper's scale on a power-of-two
# mesh: 1023 nodes, N = 128 (the paper: 999 nodes, N = 100), T = 0.4, alpha = 0.75, CQ-BDF3, kappa = 0.1
NL_WORKLOADS = {"allencahn1d": lambda: workloads.allen_cahn_problem("fem", mx=1023, N=128, k=3, alpha=0.75,
                                                                    kappa=0.1, T=0.4, eps=1.0,
                                                                    data="example4")}
# outer tolerance = the metric's 1e-8 (the outer rule does not trust the first update's ratio on its own);
# inner solves to 1e-10
NL_NEWTON_TOL, NL_TOL = 1e-8, 1e-10
WORKLOAD = "heat2d"


def max_over_ranks(pg, ms: float, device=None) -> float:
    """The job's time for a step: the slowest rank's (all_reduce MAX); unchanged on one rank."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_units(pg, units: float, device=None) -> float:
    """Units (space-time DOF) that all ranks processed (all_reduce SUM): the ranks are replicas
    with their own problems, so the job's work grows with the rank count (weak scaling)."""
    if pg is None:
        return units
    import torch
    t = torch.tensor([units], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def problem_for_rank(rank: int):
    # weak scaling: every rank solves its own instance (replicas; no exchange step)
    return (NL_WORKLOADS if WORKLOAD in NL_WORKLOADS else WORKLOADS)[WORKLOAD]()


def oracle_sample(p, budget_s: float = 15.0, results=None, full: bool = False):
    """Time the CPU oracle on the first n_s time levels of the workload (bounded; all N levels
    when full). results: optional {label: GPU solution [N][M]}; each is compared with the oracle's
    solution on the levels the sample covers (the schemes are causal, so those levels are exact).
    The returned dict carries the measured seconds and the levels run ("seconds", "levels")."""
    if p.dim == 3 and p.M > 300_000:
        # the oracle's sparse LU of a 3D operator this large (fill-in) exceeds a bounded sample
        raise RuntimeError(f"not run: sparse LU of the 3D operator ({p.M} unknowns) exceeds a bounded CPU sample")
    from oracle import fem, grid, nonlinear, sequential
    f_full = p.f()
    fd = p.fderiv()
    if isinstance(p, workloads.NlProblem):
        Mass, A, w = nonlinear.space_ops(p.space, p.mx)

        def run(n_s):
            t0 = time.perf_counter()
            Fh = nonlinear.nl_rhs(p.k, p.alpha, p.tau, Mass, A, w, p.g, p.v, f_full[:n_s], fd)
            Ur = nonlinear.solve_sequential_nl(p.k, p.alpha, p.tau, Mass, A, w, p.g, Fh)
            return time.perf_counter() - t0, Ur

        n_s = p.N if full else _levels_in_budget(run, p.N, budget_s)
        t, Ur = run(n_s)
        return _with_errors({"value": p.M * n_s / t, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "seconds": t, "levels": n_s,
                             "sample": f"sequential FP64 semilinear CQ-BDF{p.k} (Newton per step, sparse LU) over the "
                                       f"first {n_s} of {p.N} time levels of the workload, {t:.2f} s"}, results, Ur)
    if getattr(p, "space", "fd") == "fem":
        _, Mh, Kh = fem.fem_matrices(p.mx)

        def run(n_s):
            t0 = time.perf_counter()
            Ur = fem.solve_sequential_fem(p.k, p.alpha, p.tau, Mh, Kh, p.v, f_full[:n_s], fd)
            return time.perf_counter() - t0, Ur
    else:
        A = grid.operator(p)

        def run(n_s):
            t0 = time.perf_counter()
            Ur = sequential.solve_sequential(p.k, p.alpha, p.tau, A, p.v, f_full[:n_s], fd)
            return time.perf_counter() - t0, Ur

    n_s = p.N if full else _levels_in_budget(run, p.N, budget_s)
    t, Ur = run(n_s)
    scheme = f"BDF{p.k}" if p.alpha == 1.0 else f"CQ-BDF{p.k} (alpha = {p.alpha})"
    return _with_errors({"value": p.M * n_s / t, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "seconds": t, "levels": n_s,
                         "sample": f"sequential FP64 {scheme} (sparse LU, SuperLU single-threaded) over "
                                   f"{'all' if n_s == p.N else 'the first'} {n_s} of {p.N} time levels of the "
                                   f"workload, {t:.2f} s"}, results, Ur)


def _levels_in_budget(run, N: int, budget_s: float) -> int:
    """Levels of the oracle that fit in budget_s, from the time of its first 8 levels."""
    t8, _ = run(min(8, N))
    per = t8 / min(8, N)
    return int(max(min(8, N), min(N, budget_s / max(per, 1e-9))))


def diag_wr_sample(p, sweeps):
    """The second CPU reference: the diagonalised WR solve of the whole workload in FP64 with
    NumPy/SciPy FFTs on all host cores (oracle/diag_wr.py), F_hat formation and the same number of
    sweeps as the GPU's MIXED solve from U_0^n = v. Finite differences, Dirichlet, 1D/2D only.
    Returns (info, U) or None."""
    if isinstance(p, workloads.NlProblem) or p.dim > 2 or getattr(p, "space", "fd") != "fd" or p.N * p.M > 50_000_000:
        return None
    from oracle import diag_wr, grid, sequential
    f_t, fd = p.f(), p.fderiv()
    A = grid.laplacian(p.mx, p.my, p.dim)
    t0 = time.perf_counter()
    Fh = sequential.all_at_once_rhs(p.k, p.alpha, p.tau, A, p.v, f_t, fd)
    U = np.tile(p.v, (p.N, 1))
    for _ in range(sweeps):
        U, _c = diag_wr.sweep(p.k, p.alpha, p.kappa, p.tau, p.mx, p.my, p.dim, Fh, U, A)
    t = time.perf_counter() - t0
    return ({"value": p.dof / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "cpu diagonalised WR (FP64)",
             "sample": f"the whole workload: F_hat and {sweeps} sweeps from U_0 = v with NumPy/SciPy FFTs "
                       f"(SciPy FFT workers = all cores; the stencil product single-threaded), {t:.2f} s"}, U)


def _with_errors(info, results, Ur):
    """Add the space-time relative l2 error of each GPU solution against the oracle's levels."""
    if results:
        n_s = Ur.shape[0]
        ref = float(np.linalg.norm(Ur))
        info["rel_err_vs_oracle"] = {k: float(np.linalg.norm(np.asarray(U)[:n_s] - Ur) / ref)
                                     for k, U in results.items()}
        info["levels_compared"] = n_s
    return info


def run_reference(args):
    """The oracle arm: every step is the oracle's whole sequential solve of the workload (all N
    levels; about 2.7 s for heat2d on one Arm core), timed on the host; ms_per_step is the median
    measured step time and value = N * M / that time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    p = problem_for_rank(0)
    secs = []
    info = None
    for i in range(args.warmup + args.steps):
        info = oracle_sample(p, full=True)
        if i >= args.warmup:
            secs.append(info["seconds"])
    t_step = statistics.median(secs)
    value = p.dof / t_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": p.name, "dof": p.dof},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": info["sample"] + f"; median of {len(secs)} timed steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _device_inputs(p, dev):
    import torch
    v = torch.tensor(p.v, device=dev)
    ph = torch.tensor(p.f_space, device=dev)
    f = torch.outer(torch.tensor(p.f_time, device=dev), ph).contiguous()
    fd = (torch.outer(torch.tensor(p.f_derivs0, device=dev), ph).contiguous() if p.k >= 2
          else torch.zeros((0, p.M), dtype=torch.float64, device=dev))
    return v, f, fd


def _kind(p) -> str:
    return f"{p.dim}d_{'bdf' if p.alpha == 1.0 else 'cq'}"


def oracle_check(pairs, budget_s: float = 40.0):
    """Compare returned solutions with the oracle's sequential solution: pairs = [(Problem, U)], in
    a fixed order; problems too large for a bounded CPU run (BDF: N M > 4e6; CQ: N^2 M > 4e9) are
    skipped, and checking stops once budget_s of oracle time is spent. Returns the space-time relative
    l2 error of each checked problem and the largest error per kind (1d/2d, bdf/cq)."""
    from oracle import grid, sequential
    out, t_used = [], 0.0
    for p, U in pairs:
        if p.N * p.M > 4e6 or (p.alpha != 1.0 and p.N * p.N * p.M > 4e9):
            continue
        if t_used > budget_s:
            break
        t0 = time.perf_counter()
        ref = sequential.solve_sequential(p.k, p.alpha, p.tau, grid.operator(p), p.v, p.f(), p.fderiv())
        t_used += time.perf_counter() - t0
        out.append({"problem": p.name, "kind": _kind(p), "dof": p.dof,
                     "rel_err": float(np.linalg.norm(np.asarray(U) - ref) / np.linalg.norm(ref))})
    worst = {}
    for r in out:
        worst[r["kind"]] = max(worst.get(r["kind"], 0.0), r["rel_err"])
    return {"checked": len(out), "max_rel_err_by_kind": worst, "oracle_s": round(t_used, 2),
            "max_rel_err": max((r["rel_err"] for r in out), default=None), "per_problem": out}


def run_mix(args) -> int:
    """64 mixed problems (1D/2D, per-axis 127/255/511, N 64..2048, k 1..6, alpha, kappa), one graph
    launch per step for all of them (pint_batch_solve)."""
    import torch
    from paper_2007_13125_gb300 import Plan, pint
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    dev = torch.device("cuda", local)
    probs = workloads.c4_batch(64, seed=2)
    plans, Fs, Us, vs = [], [], [], []
    for p in probs:
        pl = Plan.for_problem(p, "mixed")
        v, f, fd = _device_inputs(p, dev)
        F = torch.empty_like(f)
        pl.form_rhs(v, f, fd, F)
        torch.cuda.synchronize()
        del f, fd
        plans.append(pl); Fs.append(F); Us.append(torch.empty_like(F)); vs.append(v)
    dof = sum(p.dof for p in probs)

    def step():
        # every problem from U_0^n = v (the first sweep reads v)
        return pint.batch_solve_v(plans, Fs, vs, Us, tol=TOL, max_sweeps=30)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        st, sweeps, upd = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the same 64 solves one at a time (each its own graph launch, the GPU otherwise idle): the batch
    # graph's independent branches should beat the sum of these
    solo = []
    for pl, F, v, U in zip(plans, Fs, vs, Us):
        pl.solve_v(F, v, U, tol=TOL, max_sweeps=30)      # warm (graph built)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record()
        pl.solve_v(F, v, U, tol=TOL, max_sweeps=30)
        b.record()
        torch.cuda.synchronize()
        solo.append(a.elapsed_time(b))
    kinds = {"heat": sum(1 for p in probs if p.alpha == 1.0), "subdiffusion": sum(1 for p in probs if p.alpha != 1.0)}
    # the returned solutions of a seeded subset against the oracle (the last step's results)
    check = oracle_check([(p, U.cpu().numpy()) for p, U in zip(probs, Us)]) if not args.no_cpu_baseline else None
    line = {"metric": METRIC, "value": dof / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
            "config": {"workload": "mix64_seed2", "problems": len(probs), "dof": dof, "kinds": kinds,
                       "device_bytes": sum(pl.workspace_bytes() for pl in plans) + 16 * dof,
                       "sweeps": {"min": min(sweeps), "max": max(sweeps), "mean": sum(sweeps) / len(sweeps)},
                       "status": st,
                       "solo_sum_ms": sum(solo), "batch_over_solo_speedup": sum(solo) / ms,
                       "solo_ms": {p.name: round(t, 3) for p, t in zip(probs, solo)},
                       "tuning": {p.name: pl.tuning() for p, pl in zip(probs, plans)},
                       "solo_note": "each problem alone (one graph launch per solve, host wait after each); "
                                    "the batch runs them as independent branches of one graph",
                       "launch_mode": "one CUDA graph for all 64 solves (independent branches)",
                       "rel_err_vs_oracle": check}}
    print(json.dumps(line), flush=True)
    for pl in plans:
        pl.close()
    return 0


def run_serve(args) -> int:
    """Poisson arrivals (mean 200 / s, seed 3) of problems from the mixed distribution, served with
    continuous batching under a 120 GB device budget; inputs are device arrays of the client."""
    import torch
    from paper_2007_13125_gb300 import pint
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    dev = torch.device("cuda", local)
    arr = workloads.c5_arrivals(args.requests, rate=200.0, seed=3)
    inputs = [_device_inputs(p, dev) for _, p in arr]
    torch.cuda.synchronize()
    infos = []
    # the client receives every solution: one reusable pinned host buffer of the largest size
    out_buf = torch.empty(max(p.dof for _, p in arr), dtype=torch.float64).pin_memory().numpy()
    with pint.Server(120 << 30, max_active=16) as srv:
        t0 = time.perf_counter()
        tickets = []
        for (ta, p), (v, f, fd) in zip(arr, inputs):
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(p, v, f, fd, tol=TOL))
        kept = []   # a copy of the solutions the oracle can check (bounded, in arrival order)
        for (_, p), t in zip(arr, tickets):
            st, info = srv.poll(t, out_buf[:p.dof], timeout_us=600_000_000)
            infos.append((st, info.t_submit, info.t_start, info.t_done, info.sweeps))
            if st == 0 and len(kept) < 12 and p.N * p.M <= 4e6 and (p.alpha == 1.0 or p.N * p.N * p.M <= 4e9):
                kept.append((p, out_buf[:p.dof].reshape(p.N, p.M).copy()))
        t_client = time.perf_counter() - t0
        stats = srv.stats()
    lat = sorted(1e3 * (d - s) for _, s, _, d, _ in infos)
    wait = sorted(1e3 * (a - s) for _, s, a, _, _ in infos)
    span = max(d for *_, d, _ in infos) - min(s for _, s, *_ in infos)
    dof = sum(p.dof for _, p in arr)
    ok = sum(1 for st, *_ in infos if st == 0)
    line = {"metric": METRIC, "value": dof / span, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * span, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+df64", "data": "synthetic",
            "config": {"workload": "serve_poisson200_seed3", "requests": len(arr), "completed_ok": ok,
                       "dof": dof, "offered_dof_per_s": dof / arr[-1][0],
                       "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
                       "queue_wait_ms_p50": float(np.percentile(wait, 50)),
                       "queue_wait_ms_p99": float(np.percentile(wait, 99)),
                       "budget_bytes": 120 << 30, "peak_device_bytes": stats["peak_hbm"], "max_active": 16,
                       "client_span_s": t_client, "client_dof_per_s": dof / t_client,
                       "rel_err_vs_oracle": oracle_check(kept) if not args.no_cpu_baseline else None,
                       "completion": "value: solutions complete on the device (first submit to last completion); "
                                     "client_*: until the client has copied every solution to its pinned host buffer "
                                     "(solutions wait on the device until polled)"}}
    print(json.dumps(line), flush=True)
    return 0


def run_nl(args) -> int:
    """Algorithm 3 on a semilinear workload: one step = F_hat of the semilinear scheme, U_0 = v and
    the modified Newton iteration (inner WR solves to NL_TOL) until the outer estimate is below
    NL_NEWTON_TOL. value = N M / device time per step (MIXED, inputs resident)."""
    import torch
    from paper_2007_13125_gb300 import Plan, pint
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    p = problem_for_rank(rank)
    N, M = p.N, p.M
    v_h, f_h, fd_h = p.v, p.f(), p.fderiv()
    v = torch.tensor(v_h, device=dev)
    f = torch.tensor(f_h, device=dev)
    fd = torch.tensor(fd_h, device=dev)
    F = torch.empty((N, M), dtype=torch.float64, device=dev)
    U = torch.empty((N, M), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = Plan.for_problem(p, "mixed")
    last = {}

    def step(vv=v, ff=f, ffd=fd):
        plan.nl_form_rhs(p.g, vv, ff, ffd, F, stream)
        plan.initial_guess(vv, U, stream)
        last["nl"] = plan.nl_solve(p.g, F, U, newton_tol=NL_NEWTON_TOL, max_steps=20, tol=NL_TOL, max_sweeps=40,
                                   stream=stream)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)

    def timed(steps, per_step=False):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        lat = []
        e0.record(stream)
        for _ in range(steps):
            if per_step:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            step()
            if per_step:
                b.record(stream)
                lat.append((a, b))
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        ms = max_over_ranks(pg, ms, dev)
        return ms, [a.elapsed_time(b) for a, b in lat]

    clk = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clk.start()
    for _ in range(args.warmup):
        step()
    barrier()
    t_clk0 = time.monotonic()
    ms, lat = timed(args.steps, per_step=True)
    clocks = clk.stop(t_clk0, time.monotonic())
    st, sweeps, upds = last["nl"]
    # launches per step: 2 (source) + 1 (U_0); per outer step 4 (linearise, rhs, factor, norms) and
    # the inner solve graph: control init, conversion in / out, per sweep the sweep kernels + check
    per_sweep = 3 + (1 if p.alpha != 1.0 else 0) + 1
    launches = args.steps * (3 + sum(4 + 3 + s * per_sweep for s in sweeps))

    # per-kernel CUDA-event times: the same step with sweeps launched one by one
    pint.set_profiling(True)
    pint.kernel_stats(reset=True)
    timed(max(3, args.steps // 2))
    kstats = pint.kernel_stats(reset=True)
    pint.set_profiling(False)

    # end to end: inputs from pinned host memory and U back, inside the timed region
    v_pin = torch.tensor(v_h).pin_memory()
    f_pin = torch.tensor(f_h).pin_memory()
    fd_pin = torch.tensor(fd_h).pin_memory()
    U_pin = torch.empty((N, M), dtype=torch.float64).pin_memory()

    def e2e_step():
        v.copy_(v_pin, non_blocking=True)
        f.copy_(f_pin, non_blocking=True)
        fd.copy_(fd_pin, non_blocking=True)
        step()
        U_pin.copy_(U, non_blocking=True)

    e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ke = max(10, args.steps)
    e0.record(stream)
    for _ in range(ke):
        e2e_step()
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1) / ke

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    per_kernel = {}
    tot_all = sum(t for _, t in kstats.values()) or 1.0
    for name, (n, tot) in kstats.items():
        avg_ms = tot / max(n, 1)
        b = algo_bytes(name, N, M, p.k)
        per_kernel[name] = {"launches": n, "avg_us": round(1e3 * avg_ms, 2), "share": round(tot / tot_all, 3),
                            "algo_GBps": round(b / (avg_ms * 1e-3) / 1e9, 1) if b else None}
    roofline = None
    if kstats:
        name, (n, tot) = max(kstats.items(), key=lambda kv: kv[1][1])
        ach = algo_bytes(name, N, M, p.k) / (tot / n * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(ach / hbm_peak, 4), "traffic": traffic_for(name, p.name),
                    "peak_source": peak_src + " hbm_gbs (STREAM-style copy)",
                    "algo_bytes_per_launch": algo_bytes(name, N, M, p.k),
                    "note": f"1D problem of {N * M * 8 / 1e6:.1f} MB per FP64 array: latency-bound, no bandwidth claim"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            step()
            torch.cuda.synchronize(dev)
            cpu = oracle_sample(p, results={"mixed": U.cpu().numpy()})
        except Exception as e:
            cpu = {"error": str(e)}
    dof_total = job_units(pg, p.dof, dev)
    line = {
        "metric": METRIC, "value": dof_total / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
        "config": {"workload": p.name, "dim": 1, "mx": p.mx, "N": N, "k": p.k, "alpha": p.alpha, "kappa": p.kappa,
                   "eps": p.meta.get("eps"), "space": p.space, "dof_per_gpu": p.dof, "precision": "mixed",
                   "newton_tol": NL_NEWTON_TOL, "inner_tol": NL_TOL, "outer_steps": len(sweeps),
                   "inner_sweeps": sweeps, "outer_updates": upds,
                   "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
                   "l2_policy": f"small problem: arrays of {N * M * 8 / 1e6:.1f} MB stay L2-resident between steps (latency figure)",
                   "launch_mode": "per outer step: linearisation kernels + one CUDA graph for the inner WR solve",
                   "parallelism": f"replicas x{world}", "kernels": per_kernel},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": dof_total / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": (v_h.size + f_h.size + fd_h.size) * 8,
                "d2h_bytes_per_step": N * M * 8, "ms_per_step": ms_e2e},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0:
        if isinstance(cpu, dict) and "rel_err_vs_oracle" in cpu:
            line["config"]["rel_err_vs_oracle"] = cpu["rel_err_vs_oracle"]
        print(json.dumps(line), flush=True)
    plan.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


def run_once(precision: str) -> int:
    import torch
    from paper_2007_13125_gb300 import Plan, pint
    pint.set_profiling(True)   # per-sweep launches
    p = problem_for_rank(0)
    dev = torch.device("cuda", 0)
    v = torch.tensor(p.v, device=dev)
    f = torch.tensor(p.f(), device=dev)
    fd = torch.tensor(p.fderiv(), device=dev)
    with Plan.for_problem(p, precision) as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device=dev)
        U = torch.empty_like(F)
        if isinstance(p, workloads.NlProblem):
            plan.nl_form_rhs(p.g, v, f, fd, F)
            plan.initial_guess(v, U)
            st, sweeps, upd = plan.nl_solve(p.g, F, U, newton_tol=NL_NEWTON_TOL, max_steps=20, tol=NL_TOL,
                                            max_sweeps=40)
        else:
            st, sweeps, upd = plan.solve_fv(v, f, fd, U, tol=TOL, max_sweeps=30)
        torch.cuda.synchronize()
    print(json.dumps({"once": precision, "workload": p.name, "sweeps": sweeps, "final_update": upd}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--once", choices=["mixed", "fp64", "fp32"], default=None,
                    help="run one untimed solve of the workload with per-sweep launches (for profiler "
                         "captures: kernels inside graphs with conditional nodes cannot be profiled) and exit")
    ap.add_argument("--per-sweep-launches", action="store_true",
                    help="launch sweeps one by one from the host instead of one graph per solve")
    ap.add_argument("--workload", default="heat2d",
                    choices=["heat2d", "heat1d", "subdiff1d", "fem1d", "periodic2d", "heat3d", "heat3d_small",
                             "allencahn1d", "mix64", "serve"],
                    help="heat2d (default): 2D heat 255x255, N=256, BDF4; heat1d: M=63, N=64, BDF2; "
                         "subdiff1d: alpha=0.5, M=1023, N=1024, CQ-BDF3; fem1d: P1 FEM, Example 1 data, "
                         "1023 nodes, N=128, BDF3; periodic2d: periodic 256x256, N=256, BDF4; "
                         "heat3d: 127^3, N=128, BDF4; heat3d_small: 127x127x63, N=32, BDF4; allencahn1d: Algorithm 3 on Example 4 (P1, 1023 nodes, "
                         "N=128, alpha=0.75, CQ-BDF3); "
                         "mix64: one graph launch over 64 "
                         "mixed problems; serve: Poisson request stream through the serving loop")
    ap.add_argument("--requests", type=int, default=100, help="serve: number of requests")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = args.workload if (args.workload in WORKLOADS or args.workload in NL_WORKLOADS) else "heat2d"
    if args.workload in NL_WORKLOADS and args.impl != "reference" and not args.once:
        return run_nl(args)
    if args.workload == "mix64":
        return run_mix(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.once:
        return run_once(args.once)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    from paper_2007_13125_gb300 import Plan, pint
    from paper_2007_13125_gb300 import build as pbuild
    if not pbuild.up_to_date():
        raise RuntimeError("libpint.so is not built (run __graft_entry__.build())")

    p = problem_for_rank(rank)
    N, M = p.N, p.M
    v_h, f_h, fd_h = p.v, p.f(), p.fderiv()
    v = torch.tensor(v_h, device=dev)
    f = torch.tensor(f_h, device=dev)
    fd = torch.tensor(fd_h, device=dev)
    F = torch.empty((N, M), dtype=torch.float64, device=dev)
    U = torch.empty((N, M), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    # the FP64 diagonalised path exists for finite differences only (P1 FEM runs MIXED)
    has_fp64 = getattr(p, "space", "fd") != "fem"
    plans = {"mixed": Plan.for_problem(p, "mixed")}
    if has_fp64:
        plans["fp64"] = Plan.for_problem(p, "fp64")
    last = {}

    def step(prec):
        # from the problem data to U: pint_solve_fv (MIXED BDF: F_hat never materialised, the
        # residual kernels read f; otherwise F_hat formed in the plan's workspace, then the solve)
        plan = plans[prec]
        st, sweeps, upd = plan.solve_fv(v, f, fd, U, tol=TOL, max_sweeps=30, stream=stream)
        last[prec] = (sweeps, upd)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)

    def timed(prec, steps, warmup, per_step=False):
        for _ in range(warmup):
            step(prec)
        barrier()
        lat = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            if per_step:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            step(prec)
            if per_step:
                b.record(stream)
                lat.append((a, b))
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(pg, ms, dev)
        lats = [a.elapsed_time(b) for a, b in lat]
        return ms / steps, lats

    # ---- main timed region: MIXED path (one graph launch per solve), clocks sampled ----
    if args.per_sweep_launches:
        pint.set_profiling(True)
    clk = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clk.start()
    for _ in range(args.warmup):
        step("mixed")
    barrier()
    t_clk0 = time.monotonic()
    ms_mixed, lat_mixed = timed("mixed", args.steps, 0, per_step=True)
    clocks = clk.stop(t_clk0, time.monotonic())
    # our kernels per solve: form_rhs, control init, the first sweep from v (no history product),
    # the later sweeps (with the CQ history product), each with the device-side convergence check
    # (graph launches), conversion out
    sweeps_main = last["mixed"][0]
    spatial_k = {1: 1, 2: 3, 3: 5}[p.dim]
    per_sweep = 2 + spatial_k + (1 if p.alpha != 1.0 else 0)
    check = 0 if args.per_sweep_launches else 1
    launches = args.steps * (1 + 1 + (2 + spatial_k + check) + (sweeps_main - 1) * (per_sweep + check) + 1)

    # ---- per-kernel CUDA-event times: the same kernels launched sweep by sweep ----
    pint.set_profiling(True)
    pint.kernel_stats(reset=True)
    timed("mixed", max(3, args.steps // 2), 1)
    kstats = pint.kernel_stats(reset=True)
    pint.set_profiling(False)

    # ---- FP64 diagonalised path, same workload ----
    ms_fp64, lat_fp64 = timed("fp64", max(2, args.steps // 2), 1, per_step=True) if has_fp64 else (None, [])

    # ---- end to end: host buffers, H2D + solve + D2H per step, through pint_solve_host ----
    # Every step hands the library its inputs (v, f, d^l f(0)) in pinned host memory and gets its
    # solution U back in pinned host memory; the copies are inside the timed region. The library
    # stages them through two buffer sets on its own copy streams, so the inputs of step i + 1 go in
    # and the solution of step i - 1 comes out while step i solves; pint_solve_host_join makes the
    # timing stream wait for the last copy-out.
    v_pin = torch.tensor(v_h).pin_memory()
    f_pin = torch.tensor(f_h).pin_memory()
    fd_pin = torch.tensor(fd_h).pin_memory()
    U_pin = [torch.empty((N, M), dtype=torch.float64).pin_memory() for _ in range(2)]
    plan_m = plans["mixed"]

    def run_e2e(k):
        for i in range(k):
            plan_m.solve_host(v_pin, f_pin, fd_pin if p.k > 1 else None, U_pin[i % 2], tol=TOL, max_sweeps=30,
                              stream=stream)
        plan_m.solve_host_join(stream)

    run_e2e(2)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ke = max(10, args.steps)
    e0.record(stream)
    run_e2e(ke)
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1) / ke
    ms_e2e = max_over_ranks(pg, ms_e2e, dev)
    h2d = (v_h.size + f_h.size + fd_h.size) * 8
    d2h = N * M * 8
    # the last solution that came back agrees with the device result of the same step, and that
    # solve converged
    plan_m.solve_result()
    step("mixed")
    torch.cuda.synchronize(dev)
    e2e_check = float((U_pin[(ke - 1) % 2] - U.cpu()).abs().max())

    # ---- roofline of the dominant kernel ----
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    top = max(kstats.items(), key=lambda kv: kv[1][1]) if kstats else None
    roofline = None
    per_kernel = {}
    for name, (n, tot) in kstats.items():
        avg_ms = tot / max(n, 1)
        b = algo_bytes(name, N, M, p.k)
        per_kernel[name] = {"launches": n, "avg_us": round(1e3 * avg_ms, 2),
                            "share": round(tot / sum(t for _, t in kstats.values()), 3),
                            "algo_GBps": round(b / (avg_ms * 1e-3) / 1e9, 1) if b else None}
    if top:
        name, (n, tot) = top
        avg_s = tot / n * 1e-3
        ach = algo_bytes(name, N, M, p.k) / avg_s / 1e9
        roofline = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1), "peak": hbm_peak,
                    "unit": "GB/s", "frac": round(ach / hbm_peak, 3), "traffic": traffic_for(name, p.name),
                    "peak_source": peak_src + " hbm_gbs (STREAM-style copy)",
                    "algo_bytes_per_launch": algo_bytes(name, N, M, p.k)}

    dof_total = job_units(pg, p.dof, dev)
    value = dof_total / (ms_mixed * 1e-3)
    lat_sorted = sorted(lat_mixed)
    p50 = float(np.percentile(lat_sorted, 50)) if lat_sorted else None
    p99 = float(np.percentile(lat_sorted, 99)) if lat_sorted else None

    cpu = None
    cpu_diag = None
    fp32_info = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            # (after the timed regions) the solutions of both paths, compared with the oracle's
            results = {}
            for prec in plans:
                step(prec)
                torch.cuda.synchronize(dev)
                results[prec] = U.cpu().numpy()
            if has_fp64:
                # the pure-FP32 floor (Algorithm 1 entirely in single precision): sweeps until the
                # update stalls at its rounding floor (at most 8), reported beside the MIXED error
                with Plan.for_problem(p, "fp32") as p32:
                    p32.form_rhs(v, f, fd, F, stream)
                    st32, sw32, up32 = p32.solve_v(F, v, U, tol=1e-14, max_sweeps=8, stream=stream,
                                                   raise_on_notconv=False)
                    torch.cuda.synchronize(dev)
                    results["fp32"] = U.cpu().numpy()
                    fp32_info = {"sweeps": sw32, "final_update": up32}
            try:
                dw = diag_wr_sample(p, last["mixed"][0])
            except Exception as e:
                dw = ({"error": str(e)}, None)
            if dw is not None and dw[1] is not None:
                results["cpu_diag_wr"] = dw[1]
            cpu = oracle_sample(p, results=results)
            if dw is not None:
                cpu_diag = dw[0]
        except Exception as e:  # never let the baseline break the bench line
            cpu = {"error": str(e)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
        "config": {
            "workload": p.name, "dim": p.dim, "mx": p.mx, "my": p.my, "N": N, "k": p.k,
            "kappa": p.kappa, "dof_per_gpu": p.dof, "precision": "mixed", "tol": TOL,
            "sweeps": last["mixed"][0], "final_update": last["mixed"][1],
            "latency_ms_p50": p50, "latency_ms_p99": p99,
            "fp64_diag": ({"dof_per_s": dof_total / (ms_fp64 * 1e-3), "ms_per_solve": ms_fp64,
                           "sweeps": last["fp64"][0],
                           "latency_ms_p50": float(np.percentile(lat_fp64, 50)),
                           "latency_ms_p99": float(np.percentile(lat_fp64, 99))}
                          if has_fp64 else "not available for P1 FEM (MIXED only)"),
            "mixed_over_fp64": ms_fp64 / ms_mixed if has_fp64 else None,
            "l2_policy": (f"inputs larger than L2 (U, F_hat, f: {N * M * 8 / 1e6:.0f} MB each in FP64)"
                          if N * M * 8 > 129e6 else
                          f"small problem: arrays of {N * M * 8 / 1e6:.1f} MB stay L2-resident between steps (latency figure)"),
            "launch_mode": "per-sweep launches" if args.per_sweep_launches else "one CUDA graph per solve (device-side convergence loop)",
            "parallelism": f"replicas x{world}",
            "kernels": per_kernel,
            "tuning": plans["mixed"].tuning(),
        },
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_diag_wr": cpu_diag,
        "e2e": {"value": dof_total / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                "api": "pint_solve_host (host arrays in and out; the library's two staging sets and copy streams overlap the copies of steps i-1 / i+1 with solve i)",
                "host_copy_max_abs_diff": e2e_check},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0:
        if isinstance(cpu, dict) and "rel_err_vs_oracle" in cpu:
            line["config"]["rel_err_vs_oracle"] = cpu["rel_err_vs_oracle"]
            if "fp32" in cpu["rel_err_vs_oracle"]:
                line["config"]["fp32_floor_rel_err"] = cpu["rel_err_vs_oracle"]["fp32"]
                line["config"]["fp32_floor"] = dict(fp32_info or {}, note="PINT_FP32: Algorithm 1 in single "
                                                    "precision, stalled at its rounding floor (reported, not a target)")
        print(json.dumps(line), flush=True)
    for pl in plans.values():
        pl.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
