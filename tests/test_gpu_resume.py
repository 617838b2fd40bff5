"""Checkpoint / restart of a solve (pint_solve_resume). A solve stopped after m sweeps (PINT_ENOTCONV
at max_sweeps = m), its iterate saved to host memory and written into a fresh plan's buffers, resumes
with the sweep count and the last update: it takes the same total sweeps, the same stopping decision
and (FP64) bit-identical iterates as the uninterrupted solve; MIXED within the last bits."""
import numpy as np
import pytest

import workloads
from gpu_helpers import device_inputs, oracle_solution, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
@pytest.mark.parametrize("kw", [dict(dim=2, mx=31, N=32, k=3, alpha=1.0, kappa=0.1),
                                dict(dim=1, mx=255, N=64, k=2, alpha=0.5, kappa=0.01)])
def test_resume_matches_the_uninterrupted_solve(kw, prec, tol):
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    p = workloads.small_problem(**kw)
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, prec) as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        U_full = torch.empty_like(F)
        st, n_full, upd_full = plan.solve_v(F, v, U_full, tol=tol)
        assert st == 0 and n_full >= 3
        # preempt after 2 sweeps: the checkpoint is the iterate (to host) and the two numbers
        U = torch.empty_like(F)
        st, m, upd_m = plan.solve_v(F, v, U, tol=tol, max_sweeps=2, raise_on_notconv=False)
        assert st == pint.PINT_ENOTCONV and m == 2
        saved = U.cpu().numpy().copy()
        F_h = F.cpu().numpy()
    # restart in a fresh plan with the same description
    with Plan.for_problem(p, prec) as plan2:
        F2 = torch.tensor(F_h, device="cuda:0")
        U2 = torch.tensor(saved, device="cuda:0")
        st, n_res, upd_res = plan2.solve_resume(F2, U2, m, upd_m, tol=tol)
        torch.cuda.synchronize()
    assert st == 0 and n_res == n_full
    got, want = U2.cpu().numpy(), U_full.cpu().numpy()
    if prec == "fp64":
        assert np.array_equal(got, want)
        # (the update norm is formed on the device in the graph and on the host here: last bit)
        assert upd_res == pytest.approx(upd_full, rel=1e-12)
    else:
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    assert rel_l2(got, oracle_solution(p)) <= (1e-10 if prec == "fp64" else 1e-8)


def test_resume_rejects_inconsistent_history():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, PintError
    p = workloads.small_problem(dim=1, mx=31, N=32, k=2)
    with Plan.for_problem(p, "fp64") as plan:
        F = torch.zeros((p.N, p.M), dtype=torch.float64, device="cuda:0")
        U = torch.zeros_like(F)
        for args in [(5, 1e-3, 1e-10, 4), (-1, 1e-3, 1e-10, 10), (1, -1.0, 1e-10, 10)]:
            with pytest.raises(PintError):
                plan.solve_resume(F, U, args[0], args[1], tol=args[2], max_sweeps=args[3])
