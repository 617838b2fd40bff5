"""1D piecewise-linear finite elements: the spatial discretisation of the paper's 1D tests.

Test infrastructure only (see ``oracle/__init__``).

Sec. 4 discretises the 1D examples in space with the P1 Galerkin finite element method on a
uniform mesh of (0, 1). With m interior nodes x_i = i h, h = 1/(m+1), and hat functions phi_i,
the semi-discrete problem is  M_h u' + K_h u = F(t)  (alpha = 1) or its CQ analogue, with the
mass matrix M_h = (phi_j, phi_i) = (h/6) tridiag(1, 4, 1), the stiffness matrix
K_h = (phi_j', phi_i') = (1/h) tridiag(-1, 2, -1), and the load vector F_i(t) = (f(t), phi_i).
The time discretisation and the WR iteration are those of the FD oracle with the identity
acting on the unknowns replaced by M_h and A_h replaced by K_h:

* ``solve_sequential_fem`` -- corrected BDF-k / CQ-BDF-k (eq. (2.1) / eq. (3.7)) in weak form:
      (omega_0 tau^-alpha M_h + K_h) U^n
          = Fbar_n + tau^-alpha M_h [omega_0 v + sum_{j=1}^{n-1} omega_j (v - U^{n-j})],
      Fbar_n = F(t_n) + a_n (F(0) - K_h v) + sum_l b_{l,n} tau^l d_t^l F(0).
* ``all_at_once_rhs_fem`` / ``apply_K_fem`` -- K U = F_hat with
      K = tau^-alpha (L (x) M_h) + I (x) K_h,  F_hat_n = Fbar_n + tau^-alpha sum_{j<n} omega_j M_h v.
* ``wr_sweep_fem`` -- one sweep of eq. (2.5) / eq. (3.10) in residual-correction form,
      U_m = U_{m-1} + P_kappa^-1 (F_hat - K U_{m-1}),
  with P_kappa^-1 applied as Algorithm 1 / 2 prescribe: kappa^{n/N} scaling, DFT along time,
  the shifted systems (g_j tau^-alpha M_h + K_h) q_j = h_j (tridiagonal, solved banded),
  inverse DFT and unscaling. g_j are the circulant eigenvalues of Lemma 2.3 / 3.3
  (``bdf.circulant_eigenvalues``).
* ``example1_data`` / ``example2_data`` -- the data of Examples 1 and 2 (Sec. 4):
  v = indicator of (0, 1/2) and f = e^t cos x; v = Dirac delta at 1/2 (its L2 projection), f = 0.
* ``iteration_errors`` -- e_m^N = ||U_m^N - U^N||_{L2(Omega)} (Sec. 4), m = 0..m_max, from the
  initial guess U_0 = 0, the reading under which Tables 2 and 3 are reproduced.

Pins (tests/test_oracle_fem.py): Tables 2 and 3 reproduced to their printed three digits for
m = 0..3 and every k; sine vectors are exact eigenvectors of M_h and K_h with closed-form
eigenvalues; the sequential solution solves the dense all-at-once system and is a WR fixed point.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import bdf


def fem_matrices(m: int):
    """(h, M_h, K_h) for m interior nodes of a uniform mesh of (0, 1)."""
    h = 1.0 / (m + 1)
    e = np.ones(m)
    Mh = sp.diags([h / 6 * e[:-1], 4 * h / 6 * e, h / 6 * e[:-1]], [-1, 0, 1], format="csc")
    Kh = sp.diags([-e[:-1] / h, 2 * e / h, -e[:-1] / h], [-1, 0, 1], format="csc")
    return h, Mh, Kh


def l2_norm(Mh, x) -> float:
    """||x||_{L2(Omega)} of the P1 function with nodal values x."""
    return float(np.sqrt(x @ (Mh @ x)))


def corrected_load(k, tau, F_t, v, F_der, Kh):
    """Fbar [N, m]: F(t_n) + a_n (F(0) - K_h v) + sum_{l=1}^{k-2} b_{l,n} tau^l d_t^l F(0)."""
    Fbar = np.array(F_t, dtype=float, copy=True)
    if k < 2:
        return Fbar
    a = bdf.correction_a(k)
    b = bdf.correction_b(k)
    vt = F_der[0] - Kh @ v
    for n in range(1, min(k - 1, Fbar.shape[0]) + 1):
        Fbar[n - 1] += a[n - 1] * vt
        for l in range(1, k - 1):
            Fbar[n - 1] += b[l - 1, n - 1] * tau ** l * F_der[l]
    return Fbar


def all_at_once_rhs_fem(k, alpha, tau, Mh, Kh, v, F_t, F_der):
    N = F_t.shape[0]
    w = bdf.cq_weights(k, alpha, N)
    Fbar = corrected_load(k, tau, F_t, v, F_der, Kh)
    return Fbar + tau ** -alpha * np.cumsum(w)[:, None] * (Mh @ v)[None, :]


def apply_K_fem(k, alpha, tau, Mh, Kh, X):
    """K X for X [N, m]: tau^-alpha sum_{j=0}^{n-1} omega_j M_h X^{n-j} + K_h X^n."""
    N = X.shape[0]
    w = bdf.cq_weights(k, alpha, N)
    MX = (Mh @ X.T).T
    conv = np.zeros_like(MX)
    for j in range(N):
        if w[j] != 0.0:
            conv[j:] += w[j] * MX[:N - j]
    return tau ** -alpha * conv + (Kh @ X.T).T


def solve_sequential_fem(k, alpha, tau, Mh, Kh, v, F_t, F_der):
    """U [N, m], U[n-1] = U^n, stepping n = 1..N."""
    N, m = F_t.shape
    w = bdf.cq_weights(k, alpha, N)
    ta = tau ** -alpha
    Fbar = corrected_load(k, tau, F_t, v, F_der, Kh)
    lu = spla.splu(sp.csc_matrix(w[0] * ta * Mh + Kh))
    Mv = Mh @ v
    U = np.zeros((N, m))
    MU = np.zeros((N, m))
    for n in range(1, N + 1):
        rhs = Fbar[n - 1] + ta * w[0] * Mv
        for j in range(1, n):
            if w[j] != 0.0:
                rhs += ta * w[j] * (Mv - MU[n - 1 - j])
        U[n - 1] = lu.solve(rhs)
        MU[n - 1] = Mh @ U[n - 1]
    return U


def apply_P_inverse_fem(k, alpha, kappa, tau, Mh, Kh, R):
    """P_kappa^-1 R along Algorithm 1 / 2: scale by kappa^{i/N} (i = 0..N-1), DFT along time,
    solve (g_j tau^-alpha M_h + K_h) q_j = h_j for every j, inverse DFT, unscale."""
    N, m = R.shape
    w = bdf.cq_weights(k, alpha, N)
    g = bdf.circulant_eigenvalues(w, kappa, N)
    s = kappa ** (np.arange(N) / N)
    H = np.fft.fft(s[:, None] * R, axis=0)
    md = Mh.diagonal(0)
    mo = Mh.diagonal(1)
    kd = Kh.diagonal(0)
    ko = Kh.diagonal(1)
    Q = np.empty_like(H)
    for j in range(N):
        sig = g[j] * tau ** -alpha
        ab = np.zeros((3, m), dtype=complex)
        ab[0, 1:] = sig * mo + ko
        ab[1, :] = sig * md + kd
        ab[2, :-1] = sig * mo + ko
        Q[j] = sla.solve_banded((1, 1), ab, H[j])
    return np.fft.ifft(Q, axis=0).real / s[:, None]


def wr_sweep_fem(k, alpha, kappa, tau, Mh, Kh, Fhat, U_prev):
    R = Fhat - apply_K_fem(k, alpha, tau, Mh, Kh, U_prev)
    return U_prev + apply_P_inverse_fem(k, alpha, kappa, tau, Mh, Kh, R)


def l2_projection(Mh, b):
    """Nodal values of the L2 projection onto P1, given b_i = (g, phi_i)."""
    return spla.spsolve(sp.csc_matrix(Mh), b)


def example1_data(N: int = 100, m: int = 999, T: float = 0.5):
    """Example 1 (Sec. 4): v = indicator of (0, 1/2) (L2 projection), f = e^t cos x.
    Returns (tau, v_h, F_t [N, m], F_der [5, m]); d_t^l F(0) = F(0) for every l."""
    h, Mh, Kh = fem_matrices(m)
    x = h * np.arange(1, m + 1)
    tau = T / N
    # (cos, phi_i) = (2 cos x_i - cos x_{i-1} - cos x_{i+1}) / h = 2 cos x_i (1 - cos h) / h
    load_cos = 2.0 * np.cos(x) * (1.0 - np.cos(h)) / h
    F_t = np.exp(tau * np.arange(1, N + 1))[:, None] * load_cos[None, :]
    F_der = np.tile(load_cos, (5, 1))
    # (indicator of (0, 1/2), phi_i): h for x_i < 1/2, h/2 at x_i = 1/2, 0 beyond
    b = np.where(x < 0.5 - 0.25 * h, h, np.where(np.abs(x - 0.5) <= 0.25 * h, h / 2, 0.0))
    return tau, l2_projection(Mh, b), F_t, F_der


def example2_data(N: int = 100, m: int = 999, T: float = 0.1):
    """Example 2 (Sec. 4): v = Dirac delta at 1/2 (its L2 projection: (delta, phi_i) = phi_i(1/2)),
    f = 0. Returns (tau, v_h, F_t, F_der)."""
    h, Mh, Kh = fem_matrices(m)
    x = h * np.arange(1, m + 1)
    b = np.maximum(0.0, 1.0 - np.abs(x - 0.5) / h)
    return T / N, l2_projection(Mh, b), np.zeros((N, m)), np.zeros((5, m))


def iteration_errors(k, alpha, kappa, tau, m, v, F_t, F_der, m_max=5, U0=None):
    """[e_0, ..., e_{m_max}], e_j = ||U_j^N - U^N||_{L2}, U^N the sequential solution at t_N."""
    h, Mh, Kh = fem_matrices(m)
    N = F_t.shape[0]
    U = solve_sequential_fem(k, alpha, tau, Mh, Kh, v, F_t, F_der)
    Fhat = all_at_once_rhs_fem(k, alpha, tau, Mh, Kh, v, F_t, F_der)
    Um = np.zeros((N, m)) if U0 is None else np.array(U0, dtype=float, copy=True)
    errs = [l2_norm(Mh, Um[-1] - U[-1])]
    for _ in range(m_max):
        Um = wr_sweep_fem(k, alpha, kappa, tau, Mh, Kh, Fhat, Um)
        errs.append(l2_norm(Mh, Um[-1] - U[-1]))
    return errs
