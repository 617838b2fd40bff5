"""pint_solve_fv: from the problem data (v, f, the derivatives of f at 0) to U without a separate
F_hat, against pint_form_rhs + pint_solve_v and the oracle.

For BDF-k the right-hand side of eq. (2.1) with the starting corrections of eq. (2.7) differs from
f(t_n) only on the first k levels (the corrections act on n <= k - 1, the beta_n v term vanishes
from n = k + 1 on), so PINT_MIXED BDF plans read those levels of F_hat from a block of the plan and
f elsewhere; every other plan forms F_hat into a workspace first. Either way the kernels see the
same F_hat values as pint_form_rhs writes, so the solutions are the same to the last bit."""
import numpy as np
import pytest

import workloads
from gpu_helpers import device_inputs, oracle_solution, rel_l2, torch_cuda
from oracle import fem


def oracle(p):
    if getattr(p, "space", "fd") == "fem":
        h, Mh, Kh = fem.fem_matrices(p.mx)
        return fem.solve_sequential_fem(p.k, p.alpha, p.tau, Mh, Kh, p.v, p.f(), p.fderiv())
    return oracle_solution(p)

pytestmark = pytest.mark.gpu

CASES = [
    ("2d_255x255_N32_bdf4_tc", lambda: workloads.small_problem(dim=2, mx=255, my=255, N=32, k=4, kappa=0.05), "mixed"),
    ("2d_63_N64_bdf6", lambda: workloads.small_problem(dim=2, mx=63, N=64, k=6, kappa=0.1), "mixed"),
    ("1d_255_N128_bdf3", lambda: workloads.small_problem(dim=1, mx=255, N=128, k=3), "mixed"),
    ("fem1d_127_N64_bdf2", lambda: workloads.fem_problem(mx=127, N=64, k=2), "mixed"),
    ("periodic2d_64_N32_bdf3", lambda: workloads.periodic_problem(dim=2, mx=64, N=32, k=3), "mixed"),
    ("3d_31_N16_bdf2", lambda: workloads.heat3d_problem(m=31, N=16, k=2), "mixed"),
    ("cq1d_255_N128_a0.5", lambda: workloads.small_problem(dim=1, mx=255, N=128, k=3, alpha=0.5), "mixed"),
    ("2d_63_N64_bdf4_fp64", lambda: workloads.small_problem(dim=2, mx=63, N=64, k=4), "fp64"),
    ("1d_31_N32_small", lambda: workloads.small_problem(dim=1, mx=31, N=32, k=2), "mixed"),
    ("1d_127_N64_bdf1", lambda: workloads.small_problem(dim=1, mx=127, N=64, k=1), "mixed"),   # one head level, no d^l f(0)
    ("2d_63_N32_bdf3_fp32", lambda: workloads.small_problem(dim=2, mx=63, N=32, k=3), "fp32"),
]


@pytest.mark.parametrize("name,make,precision", CASES)
def test_solve_fv_matches_form_rhs_and_solve_v(name, make, precision):
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = make()
    v, f, fd = device_inputs(p, torch)
    bar = {"mixed": 1e-8, "fp64": 1e-10, "fp32": 1e-4}[precision]
    tol = 1e-5 if precision == "fp32" else 1e-10
    with Plan.for_problem(p, precision) as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        U1 = torch.empty_like(F)
        st1, sw1, _ = plan.solve_v(F, v, U1, tol=tol)
        U2 = torch.empty_like(F)
        st2, sw2, _ = plan.solve_fv(v, f, fd, U2, tol=tol)
        # a second call reuses the plan's state (correction block or F_hat workspace, graphs)
        U3 = torch.empty_like(F)
        st3, sw3, _ = plan.solve_fv(v, f, fd, U3, tol=tol)
        torch.cuda.synchronize()
    a, b, c = U1.cpu().numpy(), U2.cpu().numpy(), U3.cpu().numpy()
    assert st1 == st2 == st3 == 0 and sw1 == sw2 == sw3, (sw1, sw2, sw3)
    assert np.array_equal(b, a), (name, rel_l2(b, a))
    assert np.array_equal(b, c) or rel_l2(c, b) <= 1e-13
    assert rel_l2(b, oracle(p)) <= bar, name


def test_fused_path_allocates_nothing_and_the_other_allocates_once():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    fused = workloads.small_problem(dim=2, mx=63, N=64, k=3)
    other = workloads.small_problem(dim=1, mx=127, N=64, k=3, alpha=0.6)     # CQ: F_hat formed
    for p, grows in ((fused, False), (other, True)):
        v, f, fd = device_inputs(p, torch)
        with Plan.for_problem(p, "mixed") as plan:
            U = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
            b0 = pint.device_bytes_held()
            plan.solve_fv(v, f, fd, U, tol=1e-10)
            b1 = pint.device_bytes_held()
            plan.solve_fv(v, f, fd, U, tol=1e-10)
            b2 = pint.device_bytes_held()
            torch.cuda.synchronize()
        assert b2 == b1
        assert (b1 - b0 == 8 * p.N * p.M) if grows else (b1 == b0), (p.name, b0, b1)
