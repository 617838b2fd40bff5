"""The one-CTA MIXED solve of small 1D problems (finite differences, Dirichlet, BDF-k; up to 4096
space-time unknowns): the CUDA path against the FP64 oracle through the C ABI, starting from v
or from a materialised guess, alone, batched and repeated."""
import numpy as np
import pytest

import workloads
from gpu_helpers import device_inputs, oracle_solution, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

# (mx, N, k, kappa): every line length 8..256 of the odd extension, N from 8 to 256 (one, two and
# three batches of the spatial step), k = 1..6
CASES = [(3, 8, 1, 0.1), (3, 8, 6, 0.1), (7, 16, 2, 0.1), (15, 32, 3, 0.05), (31, 64, 4, 0.1),
         (63, 64, 5, 0.1), (31, 128, 6, 0.1), (127, 32, 2, 0.05), (15, 256, 3, 0.1), (15, 8, 4, 0.3)]


def _solve(p, torch, tol, from_v=True, max_sweeps=50, raise_on_notconv=True):
    from paper_2007_13125_gb300 import Plan
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, "mixed") as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        U = torch.empty_like(F)
        if from_v:
            st, sweeps, upd = plan.solve_v(F, v, U, tol=tol, max_sweeps=max_sweeps,
                                           raise_on_notconv=raise_on_notconv)
        else:
            plan.initial_guess(v, U)
            st, sweeps, upd = plan.solve(F, U, tol=tol, max_sweeps=max_sweeps, raise_on_notconv=raise_on_notconv)
        torch.cuda.synchronize()
    return U.cpu().numpy(), st, sweeps, upd


@pytest.mark.parametrize("case", CASES)
def test_small_solve_matches_the_oracle(case):
    torch = torch_cuda()
    mx, N, k, kappa = case
    p = workloads.small_problem(dim=1, mx=mx, N=N, k=k, alpha=1.0, kappa=kappa, seed=mx + N + k)
    ref = oracle_solution(p)
    for from_v in (True, False):
        U, st, sweeps, upd = _solve(p, torch, 1e-10, from_v=from_v)
        assert st == 0
        assert rel_l2(U, ref) <= 1e-8, (case, from_v, sweeps, upd)


def test_c1_heat1d_is_one_kernel_and_starts_agree():
    # the configuration of 63 points and 64 levels runs as a single launch; starting from v and
    # from U_0 = v written out are the same computation (bitwise)
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    p = workloads.c1_heat1d()
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, "mixed") as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        torch.cuda.synchronize()
        U1 = torch.empty_like(F)
        pint.set_profiling(True)
        try:
            pint.kernel_stats(reset=True)
            plan.solve_v(F, v, U1, tol=1e-12)
            torch.cuda.synchronize()
            stats = pint.kernel_stats(reset=True)
        finally:
            pint.set_profiling(False)
        assert set(stats) == {"small_solve_ff"} and stats["small_solve_ff"][0] == 1, stats
        U2 = torch.empty_like(F)
        plan.initial_guess(v, U2)
        plan.solve(F, U2, tol=1e-12)
        U3 = torch.empty_like(F)
        plan.solve_v(F, v, U3, tol=1e-12)            # graph launch
        torch.cuda.synchronize()
    assert torch.equal(U1, U2) and torch.equal(U1, U3)
    assert rel_l2(U1.cpu().numpy(), oracle_solution(p)) <= 1e-8


def test_small_solve_reports_max_sweeps():
    torch = torch_cuda()
    p = workloads.small_problem(dim=1, mx=31, N=32, k=3, alpha=1.0, kappa=0.1)
    U, st, sweeps, upd = _solve(p, torch, 1e-14, max_sweeps=1, raise_on_notconv=False)
    from paper_2007_13125_gb300.pint import PINT_ENOTCONV
    assert st == PINT_ENOTCONV and sweeps == 1 and upd > 1e-14


def test_small_problems_batched():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    probs = [workloads.small_problem(dim=1, mx=mx, N=N, k=k, alpha=1.0, kappa=0.1, seed=i)
             for i, (mx, N, k) in enumerate([(15, 16, 2), (63, 64, 3), (31, 128, 4), (127, 32, 1)])]
    plans, Fs, vs, Us = [], [], [], []
    for p in probs:
        v, f, fd = device_inputs(p, torch)
        pl = Plan.for_problem(p, "mixed")
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        pl.form_rhs(v, f, fd, F)
        plans.append(pl); Fs.append(F); vs.append(v); Us.append(torch.empty_like(F))
    try:
        st, sweeps, upds = pint.batch_solve_v(plans, Fs, vs, Us, tol=1e-10)
        torch.cuda.synchronize()
        assert st == 0
        for p, U in zip(probs, Us):
            assert rel_l2(U.cpu().numpy(), oracle_solution(p)) <= 1e-8
    finally:
        for pl in plans:
            pl.close()


@pytest.mark.parametrize("case", CASES)
def test_small_cases_take_the_one_cta_solve(case):
    # every case above runs as the single small-solve launch (and nothing else)
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    mx, N, k, kappa = case
    p = workloads.small_problem(dim=1, mx=mx, N=N, k=k, alpha=1.0, kappa=kappa)
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, "mixed") as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        torch.cuda.synchronize()
        U = torch.empty_like(F)
        pint.set_profiling(True)
        try:
            pint.kernel_stats(reset=True)
            plan.solve_v(F, v, U, tol=1e-10)
            torch.cuda.synchronize()
            stats = pint.kernel_stats(reset=True)
        finally:
            pint.set_profiling(False)
    assert set(stats) == {"small_solve_ff"}, (case, stats)


def test_batch_mixing_one_cta_and_multi_kernel_solves():
    # one graph holding both kinds of solve: the small problems' single kernels and the larger
    # problems' while-loops of sweeps
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    probs = [workloads.small_problem(dim=1, mx=31, N=32, k=2, alpha=1.0, kappa=0.1, seed=1),
             workloads.small_problem(dim=2, mx=31, N=32, k=3, alpha=1.0, kappa=0.1, seed=2),
             workloads.small_problem(dim=1, mx=63, N=64, k=4, alpha=1.0, kappa=0.1, seed=3),
             workloads.small_problem(dim=1, mx=127, N=64, k=2, alpha=0.5, kappa=0.1, seed=4)]
    plans, Fs, vs, Us = [], [], [], []
    for p in probs:
        v, f, fd = device_inputs(p, torch)
        pl = Plan.for_problem(p, "mixed")
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        pl.form_rhs(v, f, fd, F)
        plans.append(pl); Fs.append(F); vs.append(v); Us.append(torch.empty_like(F))
    try:
        st, sweeps, upds = pint.batch_solve_v(plans, Fs, vs, Us, tol=1e-10)
        torch.cuda.synchronize()
        assert st == 0
        for p, U in zip(probs, Us):
            assert rel_l2(U.cpu().numpy(), oracle_solution(p)) <= 1e-8
    finally:
        for pl in plans:
            pl.close()
