"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and the
oracle on the same seeded inputs."""
import numpy as np

import workloads
from oracle import allatonce, grid, sequential


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def oracle_solution(p, corrected=True):
    A = grid.operator(p)
    return sequential.solve_sequential(p.k, p.alpha, p.tau, A, p.v, p.f(), p.fderiv(), corrected)


def oracle_rhs(p):
    A = grid.operator(p)
    return sequential.all_at_once_rhs(p.k, p.alpha, p.tau, A, p.v, p.f(), p.fderiv())


def device_inputs(p, torch):
    dev = torch.device("cuda:0")
    v = torch.tensor(p.v, dtype=torch.float64, device=dev)
    f = torch.tensor(p.f(), dtype=torch.float64, device=dev)
    fd = torch.tensor(p.fderiv(), dtype=torch.float64, device=dev)
    return v, f, fd


def gpu_rhs(p, torch, precision="fp64"):
    from paper_2007_13125_gb300 import Plan
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, precision) as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        torch.cuda.synchronize()
    return F.cpu().numpy()


def gpu_solve(p, torch, precision="mixed", tol=1e-10, max_sweeps=50, eig=0, raise_on_notconv=True):
    from paper_2007_13125_gb300 import Plan
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, precision, eig) as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        U = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.initial_guess(v, U)                           # U_0^n = v (Theorem 2.7)
        st, sweeps, upd = plan.solve(F, U, tol=tol, max_sweeps=max_sweeps,
                                     raise_on_notconv=raise_on_notconv)
        torch.cuda.synchronize()
    return U.cpu().numpy(), st, sweeps, upd


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
