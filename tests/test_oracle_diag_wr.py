"""Pins of oracle/diag_wr.py (the diagonalised WR solve in NumPy/SciPy, the second CPU reference):
one sweep equals the dense WR sweep of Algorithm 1 / 2 in exact linear algebra, and the iteration
converges to the sequential time-stepping solution (its fixed point, Theorem 2.7)."""
import numpy as np
import pytest

import workloads
from oracle import allatonce, diag_wr, grid, sequential


def _setup(dim, mx, my, N, k, alpha, kappa):
    kw = {"my": my} if dim == 2 else {}
    p = workloads.small_problem(dim=dim, mx=mx, N=N, k=k, alpha=alpha, kappa=kappa, seed=mx + N + k, **kw)
    A = grid.laplacian(p.mx, p.my, p.dim)
    Fh = sequential.all_at_once_rhs(p.k, p.alpha, p.tau, A, p.v, p.f(), p.fderiv())
    return p, A, Fh


@pytest.mark.parametrize("case", [(1, 7, 1, 8, 2, 1.0, 0.1), (1, 15, 1, 16, 4, 1.0, 0.3),
                                  (2, 7, 3, 8, 3, 1.0, 0.1), (1, 7, 1, 16, 3, 0.5, 0.1),
                                  (2, 3, 7, 8, 2, 0.7, 0.2)])
def test_one_sweep_equals_the_dense_wr_sweep(case):
    p, A, Fh = _setup(*case)
    rng = np.random.default_rng(1)
    U0 = rng.standard_normal((p.N, p.M))
    U1, _ = diag_wr.sweep(p.k, p.alpha, p.kappa, p.tau, p.mx, p.my, p.dim, Fh, U0, A)
    Ud = allatonce.wr_sweep_dense(p.k, p.alpha, p.kappa, p.tau, A.toarray(), Fh, U0)
    assert np.linalg.norm(U1 - Ud) <= 1e-11 * np.linalg.norm(Ud)


@pytest.mark.parametrize("case", [(1, 63, 1, 64, 2, 1.0, 0.1), (2, 31, 15, 32, 4, 1.0, 0.05),
                                  (1, 63, 1, 128, 3, 0.5, 0.05)])
def test_iteration_converges_to_the_sequential_solution(case):
    p, A, Fh = _setup(*case)
    ref = sequential.solve_sequential(p.k, p.alpha, p.tau, A, p.v, p.f(), p.fderiv())
    U0 = np.tile(p.v, (p.N, 1))
    U, sweeps, upd = diag_wr.solve(p.k, p.alpha, p.kappa, p.tau, p.mx, p.my, p.dim, Fh, U0, tol=1e-13)
    assert upd <= 1e-13 and sweeps < 50
    assert np.linalg.norm(U - ref) <= 1e-11 * np.linalg.norm(ref)
