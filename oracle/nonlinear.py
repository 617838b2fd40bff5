"""Semilinear (sub)diffusion and the modified Newton iteration of Algorithm 3 (Sec. 4.3).

Test infrastructure only (see ``oracle/__init__``).

Problem, eq. (4.3): D_t^alpha u + A u + g(u) = f, u(0) = v, here with a cubic
g(u) = c_0 + c_1 u + c_2 u^2 + c_3 u^3 (the Allen-Cahn term of Example 4 is
g(u) = (u^3 - u) / eps^2). In space, 1D on (0, 1) with homogeneous Dirichlet conditions:

* finite differences -- mass I, stiffness A_h, reaction weight w = 1;
* P1 elements        -- mass M_h, stiffness K_h, reaction weight w = h: (g(U_h), phi_i) is
                        taken by nodal quadrature, h g(U_i) (reading: the paper does not say
                        how the nonlinear load is integrated; its Newton errors do not resolve
                        the choice -- consistent and nodal integration agree to the printed
                        digits of Table 4).

Scheme, eq. (4.4): corrected CQ-BDF-k (BDF-k for alpha = 1) with the source
    f_bar_n = f(t_n) + a_n (f(0) - A v - w g(v)) + sum_{l=1}^{k-2} b_{l,n} tau^l d_t^l f(0),
so that in all-at-once form  K U + w g(U) = F_hat  with the K of the linear method
(tau^-alpha (L (x) M) + I (x) A) and F_hat = f_bar + tau^-alpha sum_{j<n} omega_j M v.

Algorithm 3 (modified Newton, eqs. (4.6)-(4.7)): U_0^n = v; for l = 1, 2, ...
    Ubar = (1/N) sum_n U_{l-1}^n,   D = g'(Ubar)   (one spatial field for all levels),
    solve (K + I (x) w D) W = F_hat - K U_{l-1} - w g(U_{l-1})  by WR from W_0 = 0,
    U_l = U_{l-1} + W.
The WR of eq. (4.7) is run in residual-correction form, W_m = W_{m-1} + P^-1 (R - (K + wD) W_{m-1}),
with P the kappa-circulant of the linearised operator: scale by kappa^{n/N}, DFT along time,
solve (sigma_j M + A + w D) q_j = h_j (tridiagonal, banded LU), inverse DFT, unscale; sigma_j
are the circulant eigenvalues of Lemma 2.3 / 3.3 times tau^-alpha.

Reading (sign): eqs. (4.6)-(4.7) print the linearised term as -g'(Ubar) W. Newton's
linearisation of A u + g(u) has +g'(Ubar) W, and only that sign reproduces Table 4: the printed
sign contracts by ~5e-2 per outer step on Example 4, Table 4 shows ~1e-4
(tests/test_oracle_nonlinear.py::test_printed_sign_does_not_reproduce_table4).

Pins (tests/test_oracle_nonlinear.py): Table 4's inner iteration counts exactly and its errors
after the solution-amplitude rescaling that its m = 0 row implies (the printed e_0 are 11% / 5%
above the norm of the stated manufactured solution, and the modified-Newton error after l steps
scales with the amplitude r like r^(2l+1)); order-k
convergence to an exact semi-discrete solution (alpha = 1, finite differences, the discrete
eigenvalue in f); a linear g reduces Algorithm 3 to one step of the linear method with a shifted
operator; the sequential solution solves the all-at-once nonlinear system (global Newton on the
dense system, tiny sizes) and is the fixed point of Algorithm 3.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import bdf, fem, grid


# ---------------------------------------------------------------------------
# the nonlinearity and the spatial operators
# ---------------------------------------------------------------------------

def g_of(c, u):
    """g(u) = c_0 + c_1 u + c_2 u^2 + c_3 u^3."""
    return c[0] + u * (c[1] + u * (c[2] + u * c[3]))


def dg_of(c, u):
    """g'(u) = c_1 + 2 c_2 u + 3 c_3 u^2."""
    return c[1] + u * (2.0 * c[2] + u * 3.0 * c[3])


def allen_cahn(eps: float):
    """Example 4: g(u) = (u^3 - u) / eps^2."""
    return (0.0, -1.0 / eps ** 2, 0.0, 1.0 / eps ** 2)


def space_ops(space: str, m: int):
    """(mass, stiffness, reaction weight w) for m interior points of (0, 1)."""
    if space == "fd":
        return sp.identity(m, format="csc"), sp.csc_matrix(grid.lap1d(m)), 1.0
    if space == "fem":
        h, Mh, Kh = fem.fem_matrices(m)
        return Mh, Kh, h
    raise ValueError(space)


# ---------------------------------------------------------------------------
# the scheme (eq. (4.4)) and its all-at-once form
# ---------------------------------------------------------------------------

def nl_rhs(k, alpha, tau, Mass, A, w, c, v, F_t, F_der):
    """F_hat [N, m] = f_bar_n + tau^-alpha (sum_{j<n} omega_j) M v, with the a_n term of f_bar
    taking f(0) - A v - w g(v). F_der[l] = d_t^l f(0) (load vectors), l = 0..k-2."""
    N = F_t.shape[0]
    om = bdf.cq_weights(k, alpha, N)
    Fbar = np.array(F_t, dtype=float, copy=True)
    if k >= 2:
        a = bdf.correction_a(k)
        b = bdf.correction_b(k)
        vt = F_der[0] - A @ v - w * g_of(c, v)
        for n in range(1, min(k - 1, N) + 1):
            Fbar[n - 1] += a[n - 1] * vt
            for l in range(1, k - 1):
                Fbar[n - 1] += b[l - 1, n - 1] * tau ** l * F_der[l]
    return Fbar + tau ** -alpha * np.cumsum(om)[:, None] * (Mass @ v)[None, :]


def apply_K(k, alpha, tau, Mass, A, X):
    """K X = tau^-alpha sum_{j=0}^{n-1} omega_j M X^{n-j} + A X^n (the linear all-at-once operator)."""
    return fem.apply_K_fem(k, alpha, tau, Mass, A, X)


def nl_residual(k, alpha, tau, Mass, A, w, c, Fhat, U):
    """F_hat - K U - w g(U): zero at the solution of the scheme."""
    return Fhat - apply_K(k, alpha, tau, Mass, A, U) - w * g_of(c, U)


def solve_sequential_nl(k, alpha, tau, Mass, A, w, c, Fhat, newton_tol=1e-15, max_newton=50):
    """U [N, m] of eq. (4.4) stepping n = 1..N; each step solves
    omega_0 tau^-alpha M U^n + A U^n + w g(U^n) = F_hat_n - tau^-alpha sum_{j=1}^{n-1} omega_j M U^{n-j}
    by Newton's method with the exact Jacobian, from U^{n-1}."""
    N, m = Fhat.shape
    om = bdf.cq_weights(k, alpha, N)
    ta = tau ** -alpha
    U = np.zeros((N, m))
    MU = np.zeros((N, m))
    u = np.zeros(m)
    for n in range(1, N + 1):
        rhs = Fhat[n - 1].copy()
        for j in range(1, n):
            if om[j] != 0.0:
                rhs -= ta * om[j] * MU[n - 1 - j]
        for _ in range(max_newton):
            res = rhs - (ta * om[0] * (Mass @ u) + A @ u + w * g_of(c, u))
            J = sp.csc_matrix(ta * om[0] * Mass + A + w * sp.diags(dg_of(c, u)))
            du = spla.spsolve(J, res)
            u = u + du
            if np.linalg.norm(du) <= newton_tol * max(1.0, np.linalg.norm(u)):
                break
        U[n - 1] = u
        MU[n - 1] = Mass @ u
    return U


# ---------------------------------------------------------------------------
# Algorithm 3
# ---------------------------------------------------------------------------

def apply_P_inverse_shift(k, alpha, kappa, tau, Mass, A, wD, R):
    """P^-1 R for the kappa-circulant of K + I (x) diag(wD): scale by kappa^{i/N}, DFT along time,
    solve (sigma_j M + A + diag(wD)) q_j = h_j for every j (banded LU), inverse DFT, unscale."""
    N, m = R.shape
    om = bdf.cq_weights(k, alpha, N)
    g = bdf.circulant_eigenvalues(om, kappa, N)
    s = kappa ** (np.arange(N) / N)
    H = np.fft.fft(s[:, None] * R, axis=0)
    Md = sp.csc_matrix(Mass)
    Ad = sp.csc_matrix(A)
    md, mu, ml = Md.diagonal(0), Md.diagonal(1), Md.diagonal(-1)
    ad, au, al = Ad.diagonal(0), Ad.diagonal(1), Ad.diagonal(-1)
    Q = np.empty_like(H)
    for j in range(N):
        sig = g[j] * tau ** -alpha
        ab = np.zeros((3, m), dtype=complex)
        ab[0, 1:] = sig * mu + au
        ab[1, :] = sig * md + ad + wD
        ab[2, :-1] = sig * ml + al
        Q[j] = sla.solve_banded((1, 1), ab, H[j])
    return np.fft.ifft(Q, axis=0).real / s[:, None]


def linearised_wr(k, alpha, kappa, tau, Mass, A, wD, R, tol_inf=1e-12, max_sweeps=100, sweeps=None):
    """W solving (K + I (x) diag(wD)) W = R by the WR of eq. (4.7) from W_0 = 0. Stops when
    ||W_m - W_{m-1}||_inf < tol_inf (the inner criterion of Example 4) or after `sweeps` sweeps
    when given. Returns (W, sweeps taken)."""
    W = np.zeros_like(R)
    limit = sweeps if sweeps is not None else max_sweeps
    for m_ in range(1, limit + 1):
        r = R - apply_K(k, alpha, tau, Mass, A, W) - wD[None, :] * W
        dW = apply_P_inverse_shift(k, alpha, kappa, tau, Mass, A, wD, r)
        W = W + dW
        if sweeps is None and np.abs(dW).max() < tol_inf:
            return W, m_
    return W, limit


def algorithm3(k, alpha, kappa, tau, Mass, A, w, c, Fhat, v, L, tol_inf=1e-12, max_sweeps=100,
               sweeps=None, sign=1.0):
    """Iterates [U_0, U_1, ..., U_L] of Algorithm 3 and the inner sweep counts per outer step.
    sign = -1 takes the linearised term with the sign printed in eqs. (4.6)-(4.7) (for the test
    that rejects that reading)."""
    N, m = Fhat.shape
    U = np.tile(np.asarray(v, dtype=float), (N, 1))
    its = [U.copy()]
    counts = []
    for _ in range(L):
        D = dg_of(c, U.mean(axis=0))
        R = nl_residual(k, alpha, tau, Mass, A, w, c, Fhat, U)
        W, n_in = linearised_wr(k, alpha, kappa, tau, Mass, A, sign * w * D, R, tol_inf, max_sweeps, sweeps)
        U = U + W
        its.append(U.copy())
        counts.append(n_in)
    return its, counts


def l2_norm(space, Mass, x, m):
    """||x||_{L2(0,1)}: x^T M x for P1 elements, h sum x_i^2 for grid functions."""
    if space == "fem":
        return float(math.sqrt(x @ (Mass @ x)))
    return float(math.sqrt(x @ x / (m + 1)))
