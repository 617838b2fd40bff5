"""Pins of oracle/allatonce.py: WR fixed point, convergence, contraction vs Tables 2/3."""
import os

import numpy as np
import pytest

from oracle import allatonce, grid, sequential
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([float(x) for x in line.split()])
    return np.array(rows)  # [m, k-1]


def setup(k, alpha, dim=1, mx=7, N=12, kappa=0.1, time_kind="exp"):
    p = workloads.small_problem(dim=dim, mx=mx, N=N, k=k, alpha=alpha, kappa=kappa,
                                time_kind=time_kind, my=5 if dim == 2 else None)
    A = grid.laplacian(p.mx, p.my, dim)
    U = sequential.solve_sequential(k, alpha, p.tau, A, p.v, p.f(), p.fderiv())
    Fhat = sequential.all_at_once_rhs(k, alpha, p.tau, A, p.v, p.f(), p.fderiv())
    return p, A, U, Fhat


@pytest.mark.parametrize("k,alpha", [(1, 1.0), (2, 1.0), (3, 1.0), (6, 1.0), (2, 0.5), (4, 0.3)])
def test_sequential_solution_is_wr_fixed_point(k, alpha):
    # remark after eq. (2.5) / eq. (3.10): the time-stepping solution is a fixed point
    p, A, U, Fhat = setup(k, alpha)
    U1 = allatonce.wr_sweep_dense(k, alpha, p.kappa, p.tau, A.toarray(), Fhat, U)
    assert np.linalg.norm(U1 - U) <= 1e-13 * np.linalg.norm(U)


@pytest.mark.parametrize("k,alpha,dim", [(1, 1.0, 1), (2, 1.0, 2), (4, 1.0, 1), (3, 0.5, 1), (5, 0.7, 2)])
def test_dense_wr_converges_to_sequential(k, alpha, dim):
    p, A, U, Fhat = setup(k, alpha, dim=dim)
    Um = np.tile(p.v, (p.N, 1))  # U_0^n = v (Theorem 2.7)
    errs = []
    for m in range(8):
        Um = allatonce.wr_sweep_dense(k, alpha, p.kappa, p.tau, A.toarray(), Fhat, Um)
        errs.append(np.linalg.norm(Um - U) / np.linalg.norm(U))
    assert errs[-1] < 1e-13
    assert errs[1] < errs[0] < 1e-1


def test_printed_bdf_rhs_index_has_wrong_fixed_point():
    # eq. (2.7) as printed, sum_{j=1}^{n} omega_j U^{N-j+1}, does not reproduce the BDF
    # solution; the reading sum_{j=n}^{k} omega_j U^{N+n-j} (matching B_k(kappa)) does.
    k = 3
    p, A, U, Fhat = setup(k, 1.0, N=16)
    Um = np.tile(p.v, (p.N, 1))
    Up = Um.copy()
    for _ in range(12):
        Um = allatonce.wr_sweep_dense(k, 1.0, p.kappa, p.tau, A.toarray(), Fhat, Um)
        Up = allatonce.wr_sweep_dense(k, 1.0, p.kappa, p.tau, A.toarray(), Fhat, Up,
                                      printed_bdf_index=True)
    assert np.linalg.norm(Um - U) < 1e-13 * np.linalg.norm(U)
    assert np.linalg.norm(Up - U) > 1e-7 * np.linalg.norm(U)


@pytest.mark.parametrize("lam,N,tau,kappa", [(np.pi ** 2, 100, 0.005, 0.5), (30.0, 40, 0.02, 0.1),
                                              (2.0, 64, 1 / 64, 0.2)])
def test_bdf1_contraction_closed_form(lam, N, tau, kappa):
    # Remark 2.2: for backward Euler the factor is kappa r^N / (1 - kappa r^N)
    got = allatonce.contraction(1, 1.0, kappa, tau, lam, N)
    # (eigenvalues of size ~1e-9 carry a relative rounding error ~1e-8)
    assert abs(got / allatonce.contraction_bdf1_closed_form(kappa, tau, lam, N) - 1) < 1e-6


def test_contraction_matches_table2_ratios():
    # Table 2 (Example 1: T = 0.5, tau = T/100, kappa = 0.5): e_{m+1}/e_m for m = 0..2 is the
    # contraction of the slowest mode (lambda_1 ~ pi^2 for h = 1/1000).
    t2 = load_table("table2.txt")
    for k in range(1, 7):
        rho = allatonce.contraction(k, 1.0, 0.5, 0.005, np.pi ** 2, 100)
        ratios = t2[1:4, k - 1] / t2[0:3, k - 1]
        # the first ratio mixes in the initial error's mode content; later ones are asymptotic
        assert np.all(np.abs(ratios[1:] / rho - 1) < 0.02), (k, rho, ratios)
        assert abs(ratios[0] / rho - 1) < 0.04


def test_contraction_matches_table3_ratios():
    # Table 3 (Example 2: alpha = 0.5, T = 0.1, tau = T/100, kappa = 0.1)
    t3 = load_table("table3.txt")
    for k in range(1, 7):
        rho = allatonce.contraction(k, 0.5, 0.1, 0.001, np.pi ** 2, 100)
        ratios = t3[2:4, k - 1] / t3[1:3, k - 1]
        assert np.all(np.abs(ratios / rho - 1) < 0.06), (k, rho, ratios)


@pytest.mark.parametrize("k,alpha", [(1, 1.0), (2, 1.0), (4, 1.0), (6, 1.0), (3, 0.5)])
def test_observed_contraction_within_modal_bound(k, alpha):
    # Lemma 2.5 / Lemma 3.5: per-sweep contraction of the last k levels is bounded by the
    # generating-function factor; here that factor is computed exactly per sine mode.
    p, A, U, Fhat = setup(k, alpha, N=16, kappa=0.3)
    lam = grid.sine_eigenvalues(p.mx)
    bound = max(allatonce.contraction(k, alpha, p.kappa, p.tau, l, p.N) for l in lam)
    Um = np.tile(p.v, (p.N, 1))
    errs = []
    for _ in range(5):
        Um = allatonce.wr_sweep_dense(k, alpha, p.kappa, p.tau, A.toarray(), Fhat, Um)
        e = Um - U
        if np.linalg.norm(e) < 1e-12 * np.linalg.norm(U):
            break  # roundoff floor
        errs.append(sum(np.linalg.norm(e[-1 - j]) for j in range(k)))
    ratios = [errs[i + 1] / errs[i] for i in range(len(errs) - 1)]
    assert ratios and max(ratios) < 4 * bound
