"""Time windows (BDF-k, the remark closing Sec. 4.3) through the C ABI: window by window with one
plan of N_w levels, against the oracle's sequential solution of the whole horizon."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from gpu_helpers import rel_l2, torch_cuda
from oracle import grid, nonlinear as nl

pytestmark = pytest.mark.gpu

BAR = {"mixed": 1e-8, "fp64": 1e-10}
ZERO = (0.0, 0.0, 0.0, 0.0)


def dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def windowed(p, prec, Nw, torch, g=None, newton_tol=None, tol=None, max_steps=20, max_sweeps=60):
    """Solve p's N levels as windows of Nw levels with one plan; returns ([N, M] solution, statuses)."""
    from paper_2007_13125_gb300 import Plan
    N, M = p.N, p.M
    F_all, fd = p.f(), p.fderiv()
    sub = type(p).__new__(type(p))
    sub.__dict__.update(p.__dict__)
    sub.N, sub.T = Nw, p.T * Nw / N
    out, stats = [], []
    with Plan.for_problem(sub, prec) as plan:
        F = torch.empty((Nw, M), dtype=torch.float64, device="cuda:0")
        prev = None
        for s in range(0, N, Nw):
            f = dev(torch, F_all[s:s + Nw])
            U = torch.empty((Nw, M), dtype=torch.float64, device="cuda:0")
            if prev is None:
                v = dev(torch, p.v)
                fdd = dev(torch, fd)
                if g is None:
                    plan.form_rhs(v, f, fdd, F)
                else:
                    plan.nl_form_rhs(g, v, f, fdd, F)
                plan.initial_guess(v, U)
            else:
                plan.form_rhs_window(f, prev, F)
                plan.initial_guess(prev[Nw - 1], U)
            if g is None:
                st = plan.solve(F, U, tol=tol, max_sweeps=max_sweeps)[0]
            else:
                st = plan.nl_solve(g, F, U, newton_tol=newton_tol, max_steps=max_steps, tol=tol,
                                   max_sweeps=max_sweeps, raise_on_notconv=False)[0]
            stats.append(st)
            prev = U
            out.append(U)
        torch.cuda.synchronize()
        return torch.cat(out).cpu().numpy(), stats


@pytest.mark.parametrize("prec,space,dim,k", [("mixed", "fd", 2, 4), ("fp64", "fd", 2, 4), ("mixed", "fd", 1, 6),
                                              ("fp64", "fd", 1, 2), ("mixed", "fem", 1, 3)])
def test_linear_windows_match_the_whole_horizon(prec, space, dim, k):
    torch = torch_cuda()
    N, Nw = 128, 32
    if dim == 2:
        p = workloads.small_problem(dim=2, mx=63, my=63, N=N, k=k, kappa=0.05, T=1.0, seed=3)
        A = sp.csc_matrix(grid.laplacian(63, 63, 2))
        Mass, w = sp.identity(p.M, format="csc"), 1.0
    elif space == "fd":
        p = workloads.small_problem(dim=1, mx=255, N=N, k=k, kappa=0.1, T=1.0, seed=3)
        Mass, A, w = nl.space_ops("fd", 255)
    else:
        p = workloads.fem_problem(mx=255, N=N, k=k, kappa=0.1, T=1.0, seed=3)
        Mass, A, w = nl.space_ops("fem", 255)
    Fh = nl.nl_rhs(k, 1.0, p.tau, Mass, A, w, ZERO, p.v, p.f(), p.fderiv())
    ref = nl.solve_sequential_nl(k, 1.0, p.tau, Mass, A, w, ZERO, Fh)
    U, stats = windowed(p, prec, Nw, torch, tol=0.1 * BAR[prec])
    assert all(s == 0 for s in stats)
    assert rel_l2(U, ref) <= BAR[prec]


@pytest.mark.parametrize("prec,space", [("mixed", "fd"), ("fp64", "fd"), ("mixed", "fem")])
def test_windowed_algorithm3_matches_the_sequential_solution(prec, space):
    torch = torch_cuda()
    p = workloads.allen_cahn_problem(space, mx=127, N=128, k=3, alpha=1.0, kappa=0.1, T=0.4, eps=0.5, data="modes")
    Mass, A, w = nl.space_ops(space, 127)
    Fh = nl.nl_rhs(p.k, 1.0, p.tau, Mass, A, w, p.g, p.v, p.f(), p.fderiv())
    ref = nl.solve_sequential_nl(p.k, 1.0, p.tau, Mass, A, w, p.g, Fh)
    U, stats = windowed(p, prec, 32, torch, g=p.g, newton_tol=0.1 * BAR[prec], tol=0.01 * BAR[prec])
    assert all(s == 0 for s in stats)
    assert rel_l2(U, ref) <= BAR[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_windows_converge_where_the_whole_horizon_diverges(prec):
    # Allen-Cahn with eps = 0.1 on Example 4's solution: over the whole horizon (N = 128) the forced
    # mode grows too fast for the WR contraction and Algorithm 3 fails; windows of 16 levels
    # converge to the sequential solution
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.allen_cahn_problem("fd", mx=63, N=128, k=2, alpha=1.0, kappa=0.01, T=0.1, eps=0.1)
    Mass, A, w = nl.space_ops("fd", 63)
    Fh = nl.nl_rhs(p.k, 1.0, p.tau, Mass, A, w, p.g, p.v, p.f(), p.fderiv())
    ref = nl.solve_sequential_nl(p.k, 1.0, p.tau, Mass, A, w, p.g, Fh)
    with Plan.for_problem(p, prec) as plan:
        v, f, fd = dev(torch, p.v), dev(torch, p.f()), dev(torch, p.fderiv())
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.nl_form_rhs(p.g, v, f, fd, F)
        U = torch.empty_like(F)
        plan.initial_guess(v, U)
        st, sweeps, upds = plan.nl_solve(p.g, F, U, newton_tol=1e-8, max_steps=3, tol=1e-9, max_sweeps=20,
                                         raise_on_notconv=False)
        torch.cuda.synchronize()
        full = U.cpu().numpy()
    assert st != 0
    assert not np.isfinite(full).all() or rel_l2(full, ref) > 1.0
    U, stats = windowed(p, prec, 16, torch, g=p.g, newton_tol=0.1 * BAR[prec], tol=0.01 * BAR[prec])
    assert all(s == 0 for s in stats)
    assert rel_l2(U, ref) <= BAR[prec]


def test_window_rhs_rejects_cq_plans():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    from paper_2007_13125_gb300.pint import PintError, PINT_EINVAL
    p = workloads.small_problem(dim=1, mx=31, N=16, k=2, alpha=0.5)
    with Plan.for_problem(p, "mixed") as plan:
        z = torch.zeros((p.N, p.M), dtype=torch.float64, device="cuda:0")
        with pytest.raises(PintError) as e:
            plan.form_rhs_window(z, z, z)
        assert e.value.status == PINT_EINVAL
