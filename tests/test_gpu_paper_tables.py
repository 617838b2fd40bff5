"""Tables 2 and 3 of the paper computed on the GPU at the paper's own sizes.

Sec. 4, Example 1 (Table 2): 1D heat with P1 elements, h = 1/1000 (999 interior nodes), N = 100,
T = 0.5, kappa = 0.5, BDF-k for k = 1..6. Example 2 (Table 3): subdiffusion alpha = 0.5, T = 0.1,
kappa = 0.1, CQ-BDF-k. The time FFTs have length 100 = 2^2 5^2 (2N = 200 for the CQ history) and
the sine transforms length 2000 = 2^4 5^3, so these runs go through the radix-5 passes.

Each WR iterate U_m (m = 1..5, from U_0 = 0, the reading under which the oracle reproduces the
printed m = 0 row) comes from pint_wr_sweep; e_m = ||U_m^N - U^N||_{L2} with U^N the oracle's
sequential solution at t_N. Rows m = 0..3 must match the printed values to the printed digits
(within one unit of the third significant digit), rows m = 4, 5 must be at the rounding floor as
printed. FP64 runs the paper-literal direct form (Algorithm 1 / 2 in FP64), so its iterates are the
paper's.

MIXED runs the same iteration in residual-correction form with FP32 inner solves: its fixed point is
the sequential solution (the residual is double-float), but each correction carries the FP32 inner
solve's rounding, spread over all levels by the time DFT. Its iterates therefore follow the printed
ones to within that rounding: Table 2's rows m = 1, 2 within 2% (k = 6, m = 1 gives 4.453e-04
against the printed 4.44e-04; at m = 3, k = 5 gives 5.75e-09 against 5.79e-09); in Table 3 the
starting correction
a_1 (f(0) - K_h v) of the projected Dirac delta puts ~1e6 into F_hat's first level, and the FP32
rounding of that spike changes the first iterate beyond the printed digits for k >= 2 (row m = 0 is
U_0 = 0 itself). For MIXED the test checks those printed rows and that further sweeps reach the
rounding floor of the printed tables (the fixed point) within 12 sweeps.
"""
import math
import os

import numpy as np
import pytest

import workloads
from gpu_helpers import device_inputs, torch_cuda
from oracle import fem

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([float(x) for x in line.split()])
    return np.array(rows)


def same_to_printed_digits(ours, printed):
    unit = 10.0 ** (math.floor(math.log10(printed)) - 2)
    return abs(ours - printed) <= unit


def gpu_iteration_errors(p, prec, torch, m_max=5):
    from paper_2007_13125_gb300 import Plan
    h, Mh, Kh = fem.fem_matrices(p.mx)
    ref = fem.solve_sequential_fem(p.k, p.alpha, p.tau, Mh, Kh, p.v, p.f(), p.fderiv())
    v, f, fd = device_inputs(p, torch)
    errs = []
    with Plan.for_problem(p, prec) as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        U = torch.zeros_like(F)                          # U_0 = 0
        errs.append(fem.l2_norm(Mh, U[-1].cpu().numpy() - ref[-1]))
        Un = torch.empty_like(U)
        for _ in range(m_max):
            plan.wr_sweep(F, U, Un, want_update=False)
            U, Un = Un, U
            errs.append(fem.l2_norm(Mh, U[-1].cpu().numpy() - ref[-1]))
    return errs


@pytest.mark.parametrize("example,table,floor", [(1, "table2.txt", 1e-10), (2, "table3.txt", 1e-9)])
def test_paper_table_on_the_gpu_fp64(example, table, floor):
    torch = torch_cuda()
    printed = load_table(table)
    for k in range(1, 7):
        p = workloads.paper_fem_example(example, k)
        e = gpu_iteration_errors(p, "fp64", torch)
        for m in range(4):
            assert same_to_printed_digits(e[m], printed[m, k - 1]), (k, m, e[m], printed[m, k - 1])
        for m in (4, 5):
            assert e[m] < floor and printed[m, k - 1] < floor, (k, m, e[m])


@pytest.mark.parametrize("example,table,floor,rows", [(1, "table2.txt", 1e-10, 3), (2, "table3.txt", 1e-9, 1)])
def test_paper_table_on_the_gpu_mixed(example, table, floor, rows):
    torch = torch_cuda()
    printed = load_table(table)
    for k in range(1, 7):
        p = workloads.paper_fem_example(example, k)
        e = gpu_iteration_errors(p, "mixed", torch, m_max=12)
        assert same_to_printed_digits(e[0], printed[0, k - 1]), (k, e[0])
        for m in range(1, rows):
            # within the FP32 inner solve's effect on the iterate (~1%)
            assert abs(e[m] - printed[m, k - 1]) <= 0.02 * printed[m, k - 1], (k, m, e[m], printed[m, k - 1])
        assert min(e[4:]) < floor, (k, e)
