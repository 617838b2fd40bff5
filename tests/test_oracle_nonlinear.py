"""Pins of oracle/nonlinear.py (Algorithm 3, the semilinear extension of Sec. 4.3) against
Table 4, an exact semi-discrete solution, the linear oracle and brute force."""
import math
import os

import numpy as np
import numpy.polynomial.polynomial as P
import pytest
import scipy.sparse as sp

import workloads
from oracle import bdf, fem, nonlinear as nl, sequential

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def table4():
    rows = {}
    with open(os.path.join(GOLDEN, "table4.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            a, k, l, e, s = line.split()
            rows.setdefault((float(a), int(k)), []).append((float(e), int(s)))
    return rows


@pytest.fixture(scope="module")
def table4_ours():
    out = {}
    for alpha, ks in ((0.25, (1, 2)), (0.75, (1, 2, 3))):
        Mass, A, w = nl.space_ops("fem", 999)
        for k in ks:
            # Example 4: T = 0.4, tau = T/100, h = 1/1000, kappa = 0.1, eps = 1
            p = workloads.allen_cahn_problem("fem", mx=999, N=100, k=k, alpha=alpha, kappa=0.1, T=0.4)
            tau, v, c = p.tau, p.v, p.g
            Fh = nl.nl_rhs(k, alpha, tau, Mass, A, w, c, v, p.f(), p.fderiv())
            U = nl.solve_sequential_nl(k, alpha, tau, Mass, A, w, c, Fh)
            its, counts = nl.algorithm3(k, alpha, 0.1, tau, Mass, A, w, c, Fh, v, 3)
            errs = [nl.l2_norm("fem", Mass, X[-1] - U[-1], 999) for X in its]
            out[(alpha, k)] = (errs, counts)
    return out


def test_table4_inner_sweeps_and_rescaled_errors(table4_ours):
    # Table 4 (Example 4, Sec. 4.3): the inner WR counts (5, 4, 3) are reproduced exactly. The
    # printed m = 0 errors, ||U^N|| since U_0 = v = 0, are 11% (alpha = 0.25) and 5% (alpha =
    # 0.75) above the norm of the stated manufactured solution t^2/2 sin(2 pi x) (which ours
    # matches); the modified-Newton error after l steps scales with the solution amplitude r as
    # r^{2l+1} (e_0 ~ r, g'(U) - g'(Ubar) ~ r^2 per step), and with r taken from the m = 0 row
    # every later printed error is reproduced within 1.5%.
    printed = table4()
    for key, rows in printed.items():
        errs, counts = table4_ours[key]
        assert counts == [s for _, s in rows[1:]], (key, counts)
        r = rows[0][0] / errs[0]
        assert 1.0 < r < 1.12, (key, r)
        for l in range(1, 4):
            assert abs(errs[l] * r ** (2 * l + 1) / rows[l][0] - 1.0) < 0.015, (key, l, errs[l], rows[l][0])
        # the norm of the manufactured solution at T = 0.4: 0.08 / sqrt(2)
        assert abs(errs[0] - 0.08 / math.sqrt(2)) < 1e-3 * errs[0]


def test_printed_sign_does_not_reproduce_table4():
    # eqs. (4.6)-(4.7) print -g'(Ubar) W; with that sign the first outer step reduces the error by
    # ~5e-2 instead of the ~1.5e-4 of Table 4, so the Newton sign +g'(Ubar) is the reading
    alpha, k = 0.25, 1
    p = workloads.allen_cahn_problem("fem", mx=255, N=100, k=k, alpha=alpha, kappa=0.1, T=0.4)
    tau, v, c = p.tau, p.v, p.g
    Mass, A, w = nl.space_ops("fem", 255)
    Fh = nl.nl_rhs(k, alpha, tau, Mass, A, w, c, v, p.f(), p.fderiv())
    U = nl.solve_sequential_nl(k, alpha, tau, Mass, A, w, c, Fh)
    ratio = {}
    for sign in (1.0, -1.0):
        its, _ = nl.algorithm3(k, alpha, 0.1, tau, Mass, A, w, c, Fh, v, 1, sign=sign)
        e = [nl.l2_norm("fem", Mass, X[-1] - U[-1], 255) for X in its]
        ratio[sign] = e[1] / e[0]
    assert ratio[1.0] < 3e-4
    assert ratio[-1.0] > 1e-2


def _poly_data(m, N, T, coeffs, c):
    """Finite differences, alpha = 1: u(t, x_i) = p(t) sin(2 pi x_i) solves the semi-discrete
    problem exactly when f = (p' + lambda_h p) s + g(p s), lambda_h the discrete eigenvalue of
    sin(2 pi x). Returns (tau, v, F_t, F_der, exact U^n [N, m])."""
    h = 1.0 / (m + 1)
    x = h * np.arange(1, m + 1)
    s = np.sin(2 * np.pi * x)
    lam = 4.0 / h ** 2 * np.sin(np.pi * h) ** 2
    p = np.asarray(coeffs, dtype=float)
    c0, c1, c2, c3 = c
    # f(t, x) = sum_q F_q(t) s^q, q = 0..3: polynomial coefficient series in t
    F1 = P.polyadd(P.polyder(p), (lam + c1) * p)
    F2 = c2 * P.polypow(p, 2)
    F3 = c3 * P.polypow(p, 3)

    def f_at(t):
        return (c0 + P.polyval(t, F1) * s + P.polyval(t, F2) * s ** 2 + P.polyval(t, F3) * s ** 3)

    tau = T / N
    t = tau * np.arange(1, N + 1)
    F_t = np.stack([f_at(tn) for tn in t])
    F_der = []
    for l in range(6):
        d1, d2, d3 = (P.polyder(F, l) if l else F for F in (F1, F2, F3))
        F_der.append((c0 if l == 0 else 0.0) + P.polyval(0.0, d1) * s + P.polyval(0.0, d2) * s ** 2
                     + P.polyval(0.0, d3) * s ** 3)
    exact = np.stack([P.polyval(tn, p) * s for tn in t])
    return tau, P.polyval(0.0, p) * s, F_t, np.array(F_der), exact


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_sequential_nl_converges_at_the_order_of_eq_4_5(k):
    # alpha = 1, a cubic g (Allen-Cahn with eps = 1/2 plus a quadratic term), v != 0 and
    # d_t u(0) != 0: the error at T decays as tau^min(k, 1 + 2 alpha), the rate of eq. (4.5)
    # (3 for k >= 3 at alpha = 1, where the linear scheme keeps k). A dropped or mis-signed
    # -g(v) in the corrected source leaves first order.
    m, T = 31, 0.5
    c = (0.3, -4.0, 1.0, 4.0)
    coeffs = [0.5, 1.0, -0.7, 0.4, 0.2]
    Mass, A, w = nl.space_ops("fd", m)
    errs = []
    for N in (32, 64, 128):
        tau, v, F_t, F_der, ex = _poly_data(m, N, T, coeffs, c)
        Fh = nl.nl_rhs(k, 1.0, tau, Mass, A, w, c, v, F_t, F_der)
        U = nl.solve_sequential_nl(k, 1.0, tau, Mass, A, w, c, Fh)
        errs.append(np.linalg.norm(U[-1] - ex[-1]))
    order = math.log2(errs[1] / errs[2])
    assert abs(order - min(k, 3)) < 0.15, (k, errs, order)


@pytest.mark.parametrize("space", ["fd", "fem"])
@pytest.mark.parametrize("k,alpha", [(2, 1.0), (3, 0.6)])
def test_linear_g_is_the_linear_method_with_a_shifted_operator(space, k, alpha):
    # g(u) = c0 + c1 u: the scheme is the linear one for A + w c1 I and f - w c0 (solved by the
    # linear oracles), and the modified Newton Jacobian is exact: one outer step converges
    m, N, tau, kappa = 15, 16, 0.02, 0.1
    rng = np.random.default_rng(7 + k)
    Mass, A, w = nl.space_ops(space, m)
    c = (0.8, 2.5, 0.0, 0.0)
    v = rng.standard_normal(m)
    F_t = rng.standard_normal((N, m))
    F_der = rng.standard_normal((4, m))
    Fh = nl.nl_rhs(k, alpha, tau, Mass, A, w, c, v, F_t, F_der)
    U = nl.solve_sequential_nl(k, alpha, tau, Mass, A, w, c, Fh)
    As = sp.csc_matrix(A + w * c[1] * sp.identity(m))
    F_t0 = F_t - w * c[0]
    F_d0 = F_der.copy()
    F_d0[0] -= w * c[0]
    if space == "fd":
        ref = sequential.solve_sequential(k, alpha, tau, As, v, F_t0, F_d0)
    else:
        h, Mh, _ = fem.fem_matrices(m)
        ref = fem.solve_sequential_fem(k, alpha, tau, Mh, As, v, F_t0, F_d0)
    assert np.linalg.norm(U - ref) <= 1e-12 * np.linalg.norm(ref)
    its, counts = nl.algorithm3(k, alpha, kappa, tau, Mass, A, w, c, Fh, v, 1, tol_inf=1e-14)
    assert np.linalg.norm(its[1] - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("space", ["fd", "fem"])
@pytest.mark.parametrize("k,alpha", [(1, 1.0), (3, 1.0), (2, 0.4)])
def test_sequential_nl_solves_the_all_at_once_system(space, k, alpha):
    # brute force: Newton's method on the whole space-time system K U + w g(U) = F_hat with the
    # dense Jacobian (no time stepping) reaches the sequential solution
    m, N, tau = 7, 8, 0.05
    rng = np.random.default_rng(20 + k)
    Mass, A, w = nl.space_ops(space, m)
    c = (0.1, -2.0, 0.5, 3.0)
    v = 0.5 * rng.standard_normal(m)
    F_t = rng.standard_normal((N, m))
    F_der = rng.standard_normal((4, m))
    Fh = nl.nl_rhs(k, alpha, tau, Mass, A, w, c, v, F_t, F_der)
    U = nl.solve_sequential_nl(k, alpha, tau, Mass, A, w, c, Fh)
    om = bdf.cq_weights(k, alpha, N)
    L = np.zeros((N, N))
    for n in range(N):
        L[n, :n + 1] = om[n::-1]
    K = tau ** -alpha * np.kron(L, Mass.toarray()) + np.kron(np.eye(N), A.toarray())
    X = np.zeros(N * m)
    for _ in range(40):
        G = K @ X + w * nl.g_of(c, X) - Fh.ravel()
        J = K + w * np.diag(nl.dg_of(c, X))
        dX = np.linalg.solve(J, -G)
        X += dX
        if np.linalg.norm(dX) < 1e-15 * np.linalg.norm(X):
            break
    assert np.linalg.norm(X.reshape(N, m) - U) <= 1e-12 * np.linalg.norm(U)
    assert np.linalg.norm(nl.nl_residual(k, alpha, tau, Mass, A, w, c, Fh, U)) <= 1e-10 * np.linalg.norm(Fh)


@pytest.mark.parametrize("space", ["fd", "fem"])
@pytest.mark.parametrize("k,alpha,kappa", [(2, 1.0, 0.1), (4, 1.0, 0.05), (3, 0.5, 0.1)])
def test_algorithm3_converges_to_the_sequential_solution(space, k, alpha, kappa):
    m, N, tau = 15, 16, 0.02
    rng = np.random.default_rng(40 + k)
    Mass, A, w = nl.space_ops(space, m)
    c = nl.allen_cahn(0.5)
    v = 0.6 * np.sin(np.pi * np.arange(1, m + 1) / (m + 1)) + 0.05 * rng.standard_normal(m)
    F_t = rng.standard_normal((N, m))
    F_der = rng.standard_normal((4, m))
    Fh = nl.nl_rhs(k, alpha, tau, Mass, A, w, c, v, F_t, F_der)
    U = nl.solve_sequential_nl(k, alpha, tau, Mass, A, w, c, Fh)
    # modified Newton converges linearly (rate ~0.2 in the slowest of these cases)
    its, counts = nl.algorithm3(k, alpha, kappa, tau, Mass, A, w, c, Fh, v, 24, tol_inf=1e-14)
    assert np.linalg.norm(its[-1] - U) <= 1e-11 * np.linalg.norm(U)
    # the limit solves the scheme
    R = nl.nl_residual(k, alpha, tau, Mass, A, w, c, Fh, U)
    assert np.linalg.norm(R) <= 1e-10 * np.linalg.norm(Fh)


@pytest.mark.parametrize("space", ["fd", "fem"])
def test_inner_wr_limit_solves_the_linearised_system(space):
    # the WR of eq. (4.7) with the shifted kappa-circulant preconditioner converges to the
    # solution of (K + I (x) diag(w D)) W = R (dense solve)
    m, N, tau, k, alpha = 11, 12, 0.03, 3, 0.7
    rng = np.random.default_rng(3)
    Mass, A, w = nl.space_ops(space, m)
    wD = w * (rng.uniform(-1.0, 4.0, m))
    R = rng.standard_normal((N, m))
    W, n_in = nl.linearised_wr(k, alpha, 0.1, tau, Mass, A, wD, R, tol_inf=1e-15, max_sweeps=60)
    om = bdf.cq_weights(k, alpha, N)
    L = np.zeros((N, N))
    for n in range(N):
        L[n, :n + 1] = om[n::-1]
    K = tau ** -alpha * np.kron(L, Mass.toarray()) + np.kron(np.eye(N), A.toarray() + np.diag(wD))
    Wd = np.linalg.solve(K, R.ravel()).reshape(N, m)
    assert n_in < 60
    assert np.linalg.norm(W - Wd) <= 1e-12 * np.linalg.norm(Wd)
