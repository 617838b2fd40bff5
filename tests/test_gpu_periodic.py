"""Periodic boundary conditions (the remark of Sec. 2.2: FFT diagonalisation in space): FP64 and
MIXED solves against the oracle's sequential solution with the periodic Laplacian."""
import numpy as np
import pytest

import workloads
from gpu_helpers import gpu_rhs, gpu_solve, oracle_rhs, oracle_solution, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    dict(dim=1, mx=64, N=32, k=2, alpha=1.0, kappa=0.1),
    dict(dim=1, mx=8, N=16, k=3, alpha=1.0, kappa=0.1),              # rows narrower than a warp
    dict(dim=2, mx=16, my=16, N=32, k=4, alpha=1.0, kappa=0.05),     # 2D, rows narrower than a warp
    dict(dim=2, mx=64, my=32, N=64, k=3, alpha=1.0, kappa=0.05),     # rectangular
    dict(dim=1, mx=256, N=64, k=3, alpha=0.5, kappa=0.1),            # CQ
    dict(dim=2, mx=32, my=32, N=32, k=2, alpha=0.7, kappa=0.1),      # CQ, 2D
    dict(dim=1, mx=4096, N=16, k=2, alpha=1.0, kappa=0.1),           # largest axis
    dict(dim=2, mx=256, my=256, N=32, k=6, alpha=1.0, kappa=0.05),
]


@pytest.mark.parametrize("kw", CASES, ids=lambda kw: "{dim}d_{mx}_N{N}_k{k}_a{alpha}".format(**kw))
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_periodic_solve_matches_oracle(kw, precision, bar):
    torch = torch_cuda()
    p = workloads.periodic_problem(seed=13, **kw)
    # the solver stops on an a-posteriori estimate of the error: ask for a tenth of the bar
    U, st, sweeps, upd = gpu_solve(p, torch, precision, tol=0.1 * bar)
    assert rel_l2(U, oracle_solution(p)) <= bar, (sweeps, upd)


def test_periodic_rhs_matches_oracle():
    torch = torch_cuda()
    p = workloads.periodic_problem(dim=2, mx=16, my=8, N=16, k=5, alpha=1.0, kappa=0.1, seed=2)
    assert rel_l2(gpu_rhs(p, torch, "fp64"), oracle_rhs(p)) <= 1e-13


def test_periodic_fp64_wide_inverse_axis():
    # FP64 2D with 4096 points along x: the inverse x transform's tile is too large for the
    # in-register reordering and loads straight into the transform's digit-reversed rows.
    # The FP64 direct form recomputes U from F every sweep, so its accuracy is bounded by
    # eps * cond(P_kappa), cond = (lambda_max + max|sigma_j|) / min_j |sigma_j + lambda_min|: with
    # lambda_min = 0 (periodic) and lambda_max = 4 (mx^2 + my^2) that bound, ~3e-9 here, is the bar.
    torch = torch_cuda()
    from oracle import bdf
    p = workloads.periodic_problem(dim=2, mx=4096, my=8, N=8, k=2, alpha=1.0, kappa=0.1, seed=4)
    g = bdf.circulant_eigenvalues(bdf.cq_weights(p.k, p.alpha, p.N), p.kappa, p.N) / p.tau
    cond = (4.0 * (p.mx ** 2 + p.my ** 2) + np.abs(g).max()) / np.abs(g).min()
    bar = 2.0 ** -52 * cond
    U, st, sweeps, upd = gpu_solve(p, torch, "fp64", tol=1e-10, raise_on_notconv=False)
    assert rel_l2(U, oracle_solution(p)) <= bar, bar
