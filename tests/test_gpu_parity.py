"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (space-time relative l2 against the sequential FP64 solution):
  PINT_FP64  <= 1e-10,  PINT_MIXED <= 1e-8   (the bars of the method's accuracy targets);
  F_hat (pure FP64 formula) <= 1e-13; one FP64 sweep vs the dense WR sweep <= 1e-11.
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import (device_inputs, gpu_rhs, gpu_solve, oracle_rhs, oracle_solution, rel_l2,
                         torch_cuda)
from oracle import allatonce, grid, sequential

pytestmark = pytest.mark.gpu

CASES = [
    # dim, mx, N, k, alpha, kappa
    (1, 15, 16, 1, 1.0, 0.1),
    (1, 31, 32, 2, 1.0, 0.1),
    (1, 63, 64, 3, 1.0, 0.05),
    (1, 127, 128, 4, 1.0, 0.1),
    (1, 63, 64, 5, 1.0, 0.1),
    (1, 31, 64, 6, 1.0, 0.1),
    (2, 15, 16, 2, 1.0, 0.1),
    (2, 31, 32, 4, 1.0, 0.05),
    (2, 63, 64, 3, 1.0, 0.1),
    (1, 63, 64, 1, 0.5, 0.1),
    (1, 63, 128, 3, 0.3, 0.05),
    (1, 127, 64, 2, 0.7, 0.1),
    (2, 15, 32, 3, 0.5, 0.1),
    (2, 31, 16, 4, 0.7, 0.1),
]


def _p(dim, mx, N, k, alpha, kappa, **kw):
    return workloads.small_problem(dim=dim, mx=mx, N=N, k=k, alpha=alpha, kappa=kappa, **kw)


@pytest.mark.parametrize("case", CASES[:9] + CASES[10:11])
def test_rhs_parity(case):
    torch = torch_cuda()
    p = _p(*case)
    got = gpu_rhs(p, torch)
    ref = oracle_rhs(p)
    assert rel_l2(got, ref) <= 1e-13


@pytest.mark.parametrize("case", CASES)
def test_solve_fp64_parity(case):
    torch = torch_cuda()
    p = _p(*case)
    ref = oracle_solution(p)
    U, st, sweeps, upd = gpu_solve(p, torch, "fp64", tol=1e-12)
    assert st == 0
    assert rel_l2(U, ref) <= 1e-10, (sweeps, upd)


@pytest.mark.parametrize("case", CASES)
def test_solve_mixed_parity(case):
    torch = torch_cuda()
    p = _p(*case)
    ref = oracle_solution(p)
    U, st, sweeps, upd = gpu_solve(p, torch, "mixed", tol=1e-10)
    assert st == 0
    assert rel_l2(U, ref) <= 1e-8, (sweeps, upd)


@pytest.mark.parametrize("case", [(1, 15, 16, 3, 1.0, 0.1), (1, 15, 16, 2, 0.5, 0.1),
                                  (2, 7, 8, 2, 1.0, 0.2), (2, 7, 16, 4, 0.7, 0.1)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_sweep_matches_dense_wr(case, precision):
    """One sweep from U_0 = v equals the dense paper-literal WR sweep (eq. (2.5)/(3.10))."""
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = _p(*case)
    A = grid.laplacian(p.mx, p.my, p.dim).toarray()
    Fhat = oracle_rhs(p)
    U0 = np.tile(p.v, (p.N, 1))
    ref = allatonce.wr_sweep_dense(p.k, p.alpha, p.kappa, p.tau, A, Fhat, U0)
    with Plan.for_problem(p, precision) as plan:
        Fd = torch.tensor(Fhat, device="cuda:0")
        Ud = torch.tensor(U0, device="cuda:0")
        Un = torch.empty_like(Ud)
        upd = plan.wr_sweep(Fd, Ud, Un)
        got = Un.cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 2e-5
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref - U0)
    assert abs(upd - np.linalg.norm(ref - U0) / np.linalg.norm(ref)) <= 1e-4 * upd + 1e-14


def test_config_c1_heat1d():
    """1D heat, M=63, N=64, BDF2, kappa=0.1: iterate until the update is < 1e-12 and compare
    with sequential FP64 BDF2."""
    torch = torch_cuda()
    p = workloads.c1_heat1d()
    ref = oracle_solution(p)
    for prec, bar in (("fp64", 1e-10), ("mixed", 1e-8)):
        U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=1e-12)
        assert st == 0
        assert rel_l2(U, ref) <= bar, (prec, sweeps, upd)


def per_level_rel(U, ref):
    """l2 error of each time level (row n-1 = level t_n) relative to max(||U_ref^n||, the RMS level
    norm ||U_ref|| / sqrt(N)). The diagonalised solve spreads its rounding evenly over the levels
    (the DFT along time mixes them; the paper's roundoff estimates are norm-wise), so a level far
    smaller than the typical one -- the first levels of a problem started from v = 0 -- carries a
    large error relative to itself while its absolute error is that of every other level; an error
    confined to a few levels of ordinary size still shows."""
    rms = np.linalg.norm(ref) / np.sqrt(ref.shape[0])
    return np.linalg.norm(U - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), rms)


def test_config_c2_heat2d_full():
    """2D heat 255x255, N=256, BDF4 with corrections, kappa=0.05: full comparison."""
    torch = torch_cuda()
    p = workloads.c2_heat2d()
    ref = oracle_solution(p)
    for prec, bar, tol in (("fp64", 1e-10, 1e-10), ("mixed", 1e-8, 1e-8)):
        U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=tol)
        assert st == 0
        assert rel_l2(U, ref) <= bar, (prec, sweeps, upd)
        # final-time error (the paper's e_m^N metric)
        assert np.linalg.norm(U[-1] - ref[-1]) <= bar * np.linalg.norm(ref[-1])
        # every level on its own (an error confined to early levels, where the starting
        # corrections act, cannot hide under the norm of all 256 levels)
        lev = per_level_rel(U, ref)
        assert lev.max() <= 10 * bar, (prec, int(lev.argmax()), float(lev.max()))


def test_config_c3_subdiffusion_full():
    """1D subdiffusion alpha=0.5, M=1023, N=1024, CQ-BDF3, kappa=0.01."""
    torch = torch_cuda()
    p = workloads.c3_subdiff1d()
    ref = oracle_solution(p)
    for prec, bar in (("fp64", 1e-10), ("mixed", 1e-8)):
        U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=1e-9)
        assert st == 0
        assert rel_l2(U, ref) <= bar, (prec, sweeps, upd)
        lev = per_level_rel(U, ref)
        assert lev.max() <= 10 * bar, (prec, int(lev.argmax()), float(lev.max()))


def test_fp32_floor_reported():
    """Pure FP32 (Algorithm 1 in single precision) stalls at its roundoff floor; the mixed
    path refines through it."""
    torch = torch_cuda()
    p = _p(2, 31, 64, 3, 1.0, 0.05)
    ref = oracle_solution(p)
    U32, st, sweeps, upd = gpu_solve(p, torch, "fp32", tol=1e-12, max_sweeps=8, raise_on_notconv=False)
    Umx, _, _, _ = gpu_solve(p, torch, "mixed", tol=1e-10)
    e32, emx = rel_l2(U32, ref), rel_l2(Umx, ref)
    assert 1e-9 < e32 < 1e-3
    assert emx < e32 / 100


def test_closed_form_eigenvalues_converge_to_same_solution():
    # residual form: the fixed point is K U = F_hat for either preconditioner
    torch = torch_cuda()
    p = _p(1, 63, 64, 3, 0.5, 0.1)
    ref = oracle_solution(p)
    U, st, sweeps, upd = gpu_solve(p, torch, "mixed", tol=1e-11, eig=1)
    assert st == 0 and rel_l2(U, ref) <= 1e-8
    from paper_2007_13125_gb300 import Plan, PintError
    with pytest.raises(PintError):
        Plan.for_problem(p, "fp64", eig=1)


@pytest.mark.parametrize("ysolve", [1, 2, 3, 4])
@pytest.mark.parametrize("case", [(2, 31, 32, 4, 1.0, 0.05), (2, 63, 16, 2, 0.5, 0.1), (2, 7, 64, 6, 1.0, 0.1),
                                  (2, 15, 8, 3, 1.0, 0.1), (2, 255, 16, 2, 1.0, 0.1), (2, 511, 8, 2, 1.0, 0.1),
                                  (2, 99, 20, 3, 1.0, 0.1)])
def test_ysolve_variants(case, ysolve):
    # 1: sine transform along y; 2: thread-per-line recurrence; 4: parallel cyclic reduction (a warp
    # per line up to 32 rows, the CTA on a line beyond); 3: the fastest of them, timed at plan creation
    torch = torch_cuda()
    p = _p(*case)
    ref = oracle_solution(p)
    from paper_2007_13125_gb300 import Plan
    v, f, fd = device_inputs(p, torch)
    with Plan.for_problem(p, "mixed", ysolve=ysolve) as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        plan.form_rhs(v, f, fd, F)
        U = torch.empty_like(F)
        plan.initial_guess(v, U)
        st, sweeps, upd = plan.solve(F, U, tol=1e-10)
    assert rel_l2(U.cpu().numpy(), ref) <= 1e-8, (sweeps, upd)


def test_edge_sizes():
    torch = torch_cuda()
    for case in [(1, 3, 8, 1, 1.0, 0.1), (1, 3, 8, 6, 1.0, 0.1), (2, 3, 8, 2, 1.0, 0.1),
                 (1, 7, 8, 3, 0.5, 0.1), (1, 2047, 16, 2, 1.0, 0.1)]:
        p = _p(*case)
        ref = oracle_solution(p)
        # tol at the bar: mx = 2047 puts the MIXED floor (double-float residual x cond(A_h) ~ 1e6)
        # near 1e-11
        for prec, bar in (("fp64", 1e-10), ("mixed", 1e-8)):
            U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=bar)
            assert st == 0, (case, prec)
            assert rel_l2(U, ref) <= bar, (case, prec, sweeps)


@pytest.mark.parametrize("dim,mx,my", [(1, 63, 0), (1, 127, 0), (1, 255, 0), (1, 511, 0), (1, 1023, 0), (1, 2047, 0),
                                       (2, 63, 63), (2, 127, 31), (2, 255, 15), (2, 511, 15), (2, 1023, 7),
                                       (2, 15, 511), (2, 7, 1023)])
def test_compiled_line_lengths(dim, mx, my):
    # every compiled sine-transform length (odd sequences of L = 128 .. 4096 points), as the x
    # transform / solve along contiguous lines and as the y solve across rows
    torch = torch_cuda()
    kw = {"my": my} if dim == 2 else {}
    p = workloads.small_problem(dim=dim, mx=mx, N=16, k=3, alpha=1.0, kappa=0.1, **kw)
    ref = oracle_solution(p)
    for prec, bar in (("fp64", 1e-10), ("mixed", 1e-8)):
        U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=bar)
        assert st == 0, prec
        assert rel_l2(U, ref) <= bar, (prec, sweeps)


def test_rectangular_2d_grid():
    torch = torch_cuda()
    p = workloads.small_problem(dim=2, mx=31, my=15, N=32, k=3, alpha=1.0, kappa=0.1)
    ref = oracle_solution(p)
    for prec, bar in (("fp64", 1e-10), ("mixed", 1e-8)):
        U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=1e-11)
        assert rel_l2(U, ref) <= bar, prec


def test_repeat_is_bitwise_identical():
    torch = torch_cuda()
    p = _p(2, 31, 32, 4, 1.0, 0.05)
    U1 = gpu_solve(p, torch, "mixed", tol=1e-10)[0]
    U2 = gpu_solve(p, torch, "mixed", tol=1e-10)[0]
    assert np.array_equal(U1, U2)


def test_invalid_arguments_rejected():
    torch_cuda()
    from paper_2007_13125_gb300 import Plan, PintError
    for args in [(0, 1.0, 0.1, 0.01, 64, 1, 63), (2, 1.5, 0.1, 0.01, 64, 1, 63),
                 (2, 1.0, 1.0, 0.01, 64, 1, 63), (2, 1.0, 0.1, -1.0, 64, 1, 63),
                 (2, 1.0, 0.1, 0.01, 96, 1, 63), (2, 1.0, 0.1, 0.01, 64, 1, 64),
                 (2, 0.5, 0.1, 0.01, 4096, 1, 63)]:
        with pytest.raises(PintError):
            Plan(*args)


@pytest.mark.parametrize("case", [
    # lengths 2^a 5^b: the time FFT (N) and / or the sine transforms (2 (m + 1)) take radix-5 passes
    (1, 99, 100, 3, 1.0, 0.1),      # N = 100, L = 200
    (1, 999, 100, 2, 0.5, 0.1),     # CQ: 2N = 200, L = 2000
    (1, 127, 40, 4, 1.0, 0.05),     # N = 40 only
    (1, 49, 64, 6, 1.0, 0.1),       # L = 100 only
    (2, 49, 20, 3, 1.0, 0.1),       # 2D, both
    (2, 39, 80, 2, 0.7, 0.1),       # 2D CQ, L = 80, N = 80
])
def test_radix5_sizes(case):
    torch = torch_cuda()
    p = _p(*case)
    ref = oracle_solution(p)
    # tolerances as in test_solve_*_parity (the stopping rule's estimate against the bar)
    for prec, bar, tol in (("fp64", 1e-10, 1e-12), ("mixed", 1e-8, 1e-10)):
        U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=tol)
        assert st == 0, (case, prec)
        assert rel_l2(U, ref) <= bar, (case, prec, sweeps)
