"""Pins of oracle/windows.py: windowed solves against the whole-horizon sequential solution, and
the strongly nonlinear case of Sec. 4.3's closing remark."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import grid, nonlinear as nl, windows

ZERO = (0.0, 0.0, 0.0, 0.0)


@pytest.mark.parametrize("space,dim,k", [("fd", 1, 1), ("fd", 1, 3), ("fd", 2, 4), ("fem", 1, 2), ("fem", 1, 6),
                                         ("fd", 2, 6)])
def test_linear_windows_reproduce_the_sequential_solution(space, dim, k):
    # linear BDF-k: window by window (each window's all-at-once system solved directly) equals the
    # sequential solution of the whole horizon, starting corrections included in the first window
    N, Nw, T = 32, 8, 0.5
    if dim == 1:
        p = workloads.small_problem(dim=1, mx=15, N=N, k=k, T=T, seed=k) if space == "fd" else \
            workloads.fem_problem(mx=15, N=N, k=k, T=T, seed=k)
        Mass, A, w = nl.space_ops(space, 15)
    else:
        p = workloads.small_problem(dim=2, mx=7, my=7, N=N, k=k, T=T, seed=k)
        A = sp.csc_matrix(grid.laplacian(7, 7, 2))
        Mass, w = sp.identity(49, format="csc"), 1.0
    F_t, F_der = p.f(), p.fderiv()
    Fh = nl.nl_rhs(k, 1.0, p.tau, Mass, A, w, ZERO, p.v, F_t, F_der)
    U = nl.solve_sequential_nl(k, 1.0, p.tau, Mass, A, w, ZERO, Fh)
    parts, prev = [], None
    for s in range(0, N, Nw):
        Fw = (nl.nl_rhs(k, 1.0, p.tau, Mass, A, w, ZERO, p.v, F_t[s:s + Nw], F_der) if prev is None
              else windows.window_rhs(k, p.tau, Mass, F_t[s:s + Nw], prev))
        prev = nl.solve_sequential_nl(k, 1.0, p.tau, Mass, A, w, ZERO, Fw)
        parts.append(prev)
    assert np.linalg.norm(np.vstack(parts) - U) <= 1e-12 * np.linalg.norm(U)


@pytest.mark.parametrize("space", ["fd", "fem"])
def test_windowed_algorithm3_reproduces_the_sequential_solution(space):
    p = workloads.allen_cahn_problem(space, mx=31, N=64, k=3, alpha=1.0, kappa=0.1, T=0.4, eps=0.5,
                                     data="modes")
    Mass, A, w = nl.space_ops(space, 31)
    Fh = nl.nl_rhs(p.k, 1.0, p.tau, Mass, A, w, p.g, p.v, p.f(), p.fderiv())
    U = nl.solve_sequential_nl(p.k, 1.0, p.tau, Mass, A, w, p.g, Fh)
    Uw, counts = windows.solve_windows_nl(p.k, p.kappa, p.tau, Mass, A, w, p.g, p.v, p.f(), p.fderiv(), 16,
                                          L=12, tol_inf=1e-14)
    assert np.linalg.norm(Uw - U) <= 1e-12 * np.linalg.norm(U)


@pytest.mark.parametrize("space", ["fd", "fem"])
def test_windows_converge_where_the_whole_horizon_diverges(space):
    # Allen-Cahn with eps = 0.1 (Example 4's solution): g'(0) = -100 exceeds the eigenvalue 4 pi^2 of
    # the forced mode, which grows, and the WR contraction kappa r^N / (1 - kappa r^N) of that mode
    # (r^N ~ e^{60 T}) exceeds one over the whole horizon: Algorithm 3 diverges, as the paper reports
    # for strong nonlinearity. Over windows of 8 or 16 levels r^{N_w} is small and each window
    # converges; together they reproduce the sequential solution.
    p = workloads.allen_cahn_problem(space, mx=63, N=128, k=2, alpha=1.0, kappa=0.01, T=0.1, eps=0.1)
    Mass, A, w = nl.space_ops(space, 63)
    Fh = nl.nl_rhs(p.k, 1.0, p.tau, Mass, A, w, p.g, p.v, p.f(), p.fderiv())
    U = nl.solve_sequential_nl(p.k, 1.0, p.tau, Mass, A, w, p.g, Fh)
    its, _ = nl.algorithm3(p.k, 1.0, p.kappa, p.tau, Mass, A, w, p.g, Fh, p.v, 3, max_sweeps=40)
    assert np.linalg.norm(its[-1] - U) > 10.0 * np.linalg.norm(U)
    for Nw in (8, 16):
        Uw, counts = windows.solve_windows_nl(p.k, p.kappa, p.tau, Mass, A, w, p.g, p.v, p.f(), p.fderiv(), Nw,
                                              L=6, max_sweeps=40)
        assert np.linalg.norm(Uw - U) <= 1e-12 * np.linalg.norm(U), Nw
        assert max(max(c) for c in counts) < 40
