"""P1 finite elements (the paper's 1D tests, Sec. 4): the MIXED solve against the FEM oracle, and
the iteration errors of Example 1's data against the oracle's WR iterates."""
import numpy as np
import pytest

import workloads
from gpu_helpers import device_inputs, rel_l2, torch_cuda
from oracle import fem

pytestmark = pytest.mark.gpu


def oracle_fem_solution(p):
    h, Mh, Kh = fem.fem_matrices(p.mx)
    return fem.solve_sequential_fem(p.k, p.alpha, p.tau, Mh, Kh, p.v, p.f(), p.fderiv())


CASES = [
    dict(mx=63, N=32, k=1, alpha=1.0, kappa=0.1),
    dict(mx=63, N=64, k=2, alpha=1.0, kappa=0.1),
    dict(mx=255, N=64, k=3, alpha=1.0, kappa=0.5),
    dict(mx=127, N=128, k=4, alpha=1.0, kappa=0.05),
    dict(mx=31, N=32, k=5, alpha=1.0, kappa=0.1),
    dict(mx=1023, N=32, k=6, alpha=1.0, kappa=0.1),
    dict(mx=255, N=64, k=3, alpha=0.5, kappa=0.1),
    dict(mx=63, N=128, k=2, alpha=0.3, kappa=0.01),
]


@pytest.mark.parametrize("kw", CASES, ids=lambda kw: "M{mx}_N{N}_k{k}_a{alpha}".format(**kw))
def test_fem_mixed_solve_matches_oracle(kw):
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.fem_problem(seed=11, **kw)
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, "mixed") as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        U = torch.zeros_like(F)
        st, sweeps, upd = plan.solve(F, U, tol=1e-10, max_sweeps=40)
        torch.cuda.synchronize()
    ref = oracle_fem_solution(p)
    assert rel_l2(U.cpu().numpy(), ref) <= 1e-8, (sweeps, upd)


def test_fem_rhs_matches_oracle():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.fem_problem(mx=63, N=32, k=4, alpha=1.0, kappa=0.1, seed=3)
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, "mixed") as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        torch.cuda.synchronize()
    h, Mh, Kh = fem.fem_matrices(p.mx)
    ref = fem.all_at_once_rhs_fem(p.k, p.alpha, p.tau, Mh, Kh, p.v, p.f(), p.fderiv())
    assert rel_l2(F.cpu().numpy(), ref) <= 1e-13


@pytest.mark.parametrize("k", [1, 3, 6])
def test_example1_iteration_errors_follow_oracle(k):
    # Example 1's data (Sec. 4) on a power-of-two mesh and step count, kappa = 0.5, U_0 = 0: the
    # L2 errors of the WR iterates at t_N (the quantity of Table 2) against the oracle's iterates
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.fem_problem(mx=1023, N=128, k=k, alpha=1.0, kappa=0.5, T=0.5, data="example1")
    v, f, fd = device_inputs(p, torch)
    h, Mh, Kh = fem.fem_matrices(p.mx)
    Useq = fem.solve_sequential_fem(p.k, p.alpha, p.tau, Mh, Kh, p.v, p.f(), p.fderiv())
    Fo = fem.all_at_once_rhs_fem(p.k, p.alpha, p.tau, Mh, Kh, p.v, p.f(), p.fderiv())
    Uo = np.zeros((p.N, p.M))
    with Plan.for_problem(p, "mixed") as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        U = torch.zeros_like(F)
        U2 = torch.empty_like(F)
        for m in range(4):
            plan.wr_sweep(F, U, U2)
            U, U2 = U2, U
            Uo = fem.wr_sweep_fem(p.k, p.alpha, p.kappa, p.tau, Mh, Kh, Fo, Uo)
            e_gpu = fem.l2_norm(Mh, U[-1].cpu().numpy() - Useq[-1])
            e_orc = fem.l2_norm(Mh, Uo[-1] - Useq[-1])
            # the oracle's m-th error is the exact-arithmetic iterate's; the GPU preconditioner
            # runs in FP32, which perturbs each sweep's correction by ~1e-6 of itself
            assert abs(e_gpu - e_orc) <= 0.02 * e_orc + 1e-9 * fem.l2_norm(Mh, Useq[-1]), (m, e_gpu, e_orc)
