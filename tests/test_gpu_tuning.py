"""The project's autotuner: tile widths, the radix schedule of time FFTs without a compiled shape,
and the y-direction solver, as reported by pint_plan_tuning; tuned plans keep the parity bars."""
import pytest

import workloads
from gpu_helpers import gpu_solve, oracle_solution, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw", [dict(dim=1, mx=1023, N=2048, k=2, alpha=1.0, kappa=0.1),   # runtime shape
                                dict(dim=1, mx=511, N=1000, k=3, alpha=0.5, kappa=0.1),    # 2^a 5^b, CQ
                                dict(dim=2, mx=127, N=64, k=4, alpha=1.0, kappa=0.1)])
def test_tuned_plans_report_their_choices_and_keep_parity(kw):
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.small_problem(**kw)
    with Plan.for_problem(p, "mixed") as plan:
        t = plan.tuning()
    assert t["resid_max_radix"] in (8, 16) and t["update_max_radix"] in (8, 16)
    assert t["resid_width"] >= 1 and t["update_width"] >= 1 and t["ysolve"] in (1, 2, 4)
    U, st, sweeps, upd = gpu_solve(p, torch, "mixed", tol=1e-10)
    assert st == 0 and rel_l2(U, oracle_solution(p)) <= 1e-8


def test_compiled_shape_reports_radix_16():
    torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.c2_heat2d()
    with Plan.for_problem(p, "mixed", ysolve=3) as plan:
        t = plan.tuning()
    assert t["resid_max_radix"] == 16 and t["update_max_radix"] == 16
    assert t["ysolve"] in (1, 2, 4)
