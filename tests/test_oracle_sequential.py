"""Pins of oracle/sequential.py and oracle/grid.py."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import allatonce, bdf, grid, sequential
import workloads


def scalar_run(k, N, alpha=1.0, lam=2.0, mu=1.0, v0=1.0, T=1.0, corrected=True):
    """Scalar problem D u + lam u = e^{mu t}, u(0) = v0 (one sine mode of the FD problem)."""
    tau = T / N
    t = np.arange(1, N + 1) * tau
    A = sp.csr_matrix([[lam]])
    dfs = np.array([[mu ** l] for l in range(k - 1)]).reshape(k - 1, 1)
    U = sequential.solve_sequential(k, alpha, tau, A, np.array([v0]), np.exp(mu * t)[:, None],
                                    dfs, corrected)
    return U[-1, 0]


def heat_exact(lam=2.0, mu=1.0, v0=1.0, T=1.0):
    return np.exp(-lam * T) * v0 + (np.exp(mu * T) - np.exp(-lam * T)) / (mu + lam)


@pytest.mark.parametrize("k", range(1, 6))
def test_heat_order_k_with_corrections(k):
    # Lemma 2.2: error O(tau^k) for the corrected BDF-k scheme (incompatible data:
    # f(0) - A v = 1 - 2 != 0, all time derivatives of f nonzero)
    ex = heat_exact()
    Ns = [40, 80, 160]
    e = [abs(scalar_run(k, N) - ex) for N in Ns]
    slope = np.log2(e[-2] / e[-1])
    assert abs(slope - k) < 0.3, (k, e)


def test_heat_order_6():
    ex = heat_exact()
    e = [abs(scalar_run(6, N) - ex) for N in (80, 160)]
    assert e[1] < 1e-12 and e[0] / e[1] > 2 ** 5.7


@pytest.mark.parametrize("k", range(2, 7))
def test_heat_first_order_without_corrections(k):
    ex = heat_exact()
    e = [abs(scalar_run(k, N, corrected=False) - ex) for N in (80, 160)]
    assert abs(np.log2(e[0] / e[1]) - 1.0) < 0.1


def test_table1_b31_k5_sign_decided_by_order():
    # With b_{3,1}^(5) = -1/720 BDF5 is fifth order; the printed +1/720 leaves an O(tau^4)
    # error from the tau^3 d_t^3 f(0) term (lam = mu = v0 = 1, so f(0) - A v = 0 and the
    # a_n terms vanish; d_t^3 f(0) = 1).
    ex = heat_exact(lam=1.0, mu=1.0, v0=1.0)
    run = lambda N: abs(scalar_run(5, N, lam=1.0, mu=1.0, v0=1.0) - ex)
    e_good = [run(N) for N in (80, 160)]
    row = bdf.TABLE1[5][1][3]
    row[0] = -row[0]
    try:
        e_bad = [run(N) for N in (80, 160)]
    finally:
        row[0] = -row[0]
    assert np.log2(e_good[0] / e_good[1]) > 4.6
    assert np.log2(e_bad[0] / e_bad[1]) < 4.4
    assert e_good[1] < e_bad[1] / 4


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
@pytest.mark.parametrize("k", range(1, 6))
def test_cq_self_convergence_order_k(alpha, k):
    # Lemma 3.2: the corrected CQ-BDF-k solution converges like tau^k at t = T
    Ns = [64, 128, 256, 512]
    u = [scalar_run(k, N, alpha=alpha) for N in Ns]
    d = [abs(u[i] - u[i + 1]) for i in range(len(u) - 1)]
    slope = np.log2(d[-2] / d[-1])
    # a secondary tau^{1+2 alpha} term (alpha = 0.7, k = 2) approaches from above
    assert k - 0.3 < slope < k + 0.65, (alpha, k, d)


@pytest.mark.parametrize("alpha", [0.3, 0.7])
def test_cq_without_corrections_loses_order(alpha):
    Ns = [64, 128, 256, 512]
    u = [scalar_run(3, N, alpha=alpha, corrected=False) for N in Ns]
    d = [abs(u[i] - u[i + 1]) for i in range(len(u) - 1)]
    assert np.log2(d[-2] / d[-1]) < 2.2


def test_sine_modes_are_eigenvectors():
    for m in (7, 31):
        A = grid.lap1d(m)
        lam = grid.sine_eigenvalues(m)
        for p in (1, 3, m):
            s = grid.sine_mode(m, p)
            assert np.allclose(A @ s, lam[p - 1] * s, rtol=0, atol=1e-9 * lam[-1])


@pytest.mark.parametrize("dim,alpha,k", [(1, 1.0, 3), (2, 1.0, 4), (1, 0.5, 2), (2, 0.7, 5)])
def test_full_grid_equals_modal_sum(dim, alpha, k):
    """v and f in a few sine modes: each mode evolves by its scalar recurrence with
    lambda_p (Remark 2.1's decoupling); the sparse-LU full-grid solve must match."""
    mx, my, N, T = (15, 1, 24, 1.0) if dim == 1 else (9, 7, 16, 1.0)
    tau = T / N
    t = np.arange(1, N + 1) * tau
    modes = [(1, 1, 0.7), (3, 2, -0.4), (2, 5, 0.25)] if dim == 2 else [(1, 1, 0.7), (4, 1, -0.4), (9, 1, 0.25)]
    A = grid.laplacian(mx, my, dim)
    lx, ly = grid.sine_eigenvalues(mx), grid.sine_eigenvalues(my)
    v = np.zeros(mx * my)
    g = np.exp(-t) * 1.5
    phi = workloads.mode_field(dim, mx, my, 2, 1)
    f = np.outer(g, phi)
    dfs = np.array([(-1.0) ** l * 1.5 * phi for l in range(k - 1)]).reshape(k - 1, -1)
    # v = sum of modes; each mode (and the source mode) solved as a scalar problem
    Umod = np.zeros((N, mx * my))
    for (px, py, c) in modes:
        field = workloads.mode_field(dim, mx, my, px, py)
        lam = lx[px - 1] + (ly[py - 1] if dim == 2 else 0.0)
        u = sequential.solve_sequential(k, alpha, tau, sp.csr_matrix([[lam]]), np.array([c]),
                                        np.zeros((N, 1)), np.zeros((k - 1, 1)))
        Umod += np.outer(u[:, 0], field)
        v += c * field
    U = sequential.solve_sequential(k, alpha, tau, A, v, f, dfs)
    lam_f = lx[1] + (ly[0] if dim == 2 else 0.0)
    dfs_s = np.array([[(-1.0) ** l * 1.5] for l in range(k - 1)]).reshape(k - 1, 1)
    uf = sequential.solve_sequential(k, alpha, tau, sp.csr_matrix([[lam_f]]), np.array([0.0]),
                                     g[:, None], dfs_s)
    Umod += np.outer(uf[:, 0], phi)
    assert np.linalg.norm(U - Umod) <= 1e-13 * np.linalg.norm(U)


@pytest.mark.parametrize("k,alpha", [(1, 1.0), (2, 1.0), (4, 1.0), (6, 1.0), (3, 0.5), (2, 0.3)])
def test_dense_all_at_once_equals_sequential(k, alpha):
    p = workloads.small_problem(dim=1, mx=7, N=12, k=k, alpha=alpha)
    A = grid.laplacian(p.mx, 1, 1)
    U = sequential.solve_sequential(k, alpha, p.tau, A, p.v, p.f(), p.fderiv())
    Fhat = sequential.all_at_once_rhs(k, alpha, p.tau, A, p.v, p.f(), p.fderiv())
    K = allatonce.K_matrix(k, alpha, p.tau, A.toarray(), p.N)
    U2 = np.linalg.solve(K, Fhat.reshape(-1)).reshape(p.N, p.M)
    assert np.linalg.norm(U - U2) <= 1e-12 * np.linalg.norm(U)
