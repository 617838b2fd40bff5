"""Pins of the periodic-boundary operator (oracle/grid.py, the remark of Sec. 2.2) and of the
sequential scheme built on it."""
import numpy as np
import pytest

from oracle import allatonce, bdf, grid, sequential
import workloads


@pytest.mark.parametrize("m", [8, 32])
def test_fourier_modes_are_eigenvectors(m):
    A = grid.laplacian_periodic(m)
    x = np.arange(m) / m
    for q in range(m):
        lam = 4.0 * m * m * np.sin(np.pi * q / m) ** 2
        for mode in (np.cos(2 * np.pi * q * x), np.sin(2 * np.pi * q * x)):
            assert np.allclose(A @ mode, lam * mode, rtol=0, atol=1e-9 * max(lam, 1.0))
    assert np.allclose(A @ np.ones(m), 0.0)        # the constant mode is the kernel


def test_periodic_2d_is_kronecker_sum():
    mx, my = 8, 16
    A = grid.laplacian_periodic(mx, my, 2)
    x, y = np.arange(mx) / mx, np.arange(my) / my
    mode = np.outer(np.cos(2 * np.pi * 3 * y), np.sin(2 * np.pi * 2 * x)).reshape(-1)
    lam = 4 * mx * mx * np.sin(np.pi * 2 / mx) ** 2 + 4 * my * my * np.sin(np.pi * 3 / my) ** 2
    assert np.allclose(A @ mode, lam * mode, rtol=0, atol=1e-9 * lam)


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_single_mode_follows_scalar_bdf(k):
    # v = cos(2 pi q x), f = 0: every level is c_n cos(2 pi q x) with c_n the scalar corrected
    # BDF-k recurrence sum_j omega_j (c_{n-j} - 1)/tau + lambda c_n = a_n (0 - lambda) for
    # n <= k-1, = 0 beyond (eq. (2.1); c_{<=0} = 1)
    m, N, tau, q = 16, 24, 0.01, 3
    x = np.arange(m) / m
    v = np.cos(2 * np.pi * q * x)
    A = grid.laplacian_periodic(m)
    lam = 4.0 * m * m * np.sin(np.pi * q / m) ** 2
    U = sequential.solve_sequential(k, 1.0, tau, A, v, np.zeros((N, m)), np.zeros((max(k - 1, 0), m)))
    w = bdf.bdf_weights(k)
    a = bdf.correction_a(k) if k >= 2 else []
    c = []
    for n in range(1, N + 1):
        hist = sum(w[j] * ((c[n - 1 - j] if n - j >= 1 else 1.0) - 1.0) for j in range(1, k + 1))
        fbar = -a[n - 1] * lam if n <= k - 1 else 0.0
        c.append((fbar + w[0] / tau - hist / tau) / (w[0] / tau + lam))
    assert np.allclose(U, np.outer(c, v), rtol=0, atol=1e-13)


@pytest.mark.parametrize("k,alpha,dim", [(2, 1.0, 1), (4, 1.0, 2), (3, 0.5, 1)])
def test_dense_wr_converges_to_periodic_sequential(k, alpha, dim):
    p = workloads.periodic_problem(dim=dim, mx=8, N=12, k=k, alpha=alpha, kappa=0.1)
    A = grid.operator(p)
    U = sequential.solve_sequential(k, alpha, p.tau, A, p.v, p.f(), p.fderiv())
    Fhat = sequential.all_at_once_rhs(k, alpha, p.tau, A, p.v, p.f(), p.fderiv())
    Um = np.tile(p.v, (p.N, 1))
    for _ in range(8):
        Um = allatonce.wr_sweep_dense(k, alpha, p.kappa, p.tau, A.toarray(), Fhat, Um)
    assert np.linalg.norm(Um - U) <= 1e-12 * np.linalg.norm(U)
