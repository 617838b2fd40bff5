"""Dense all-at-once matrices and the dense WR iteration (tiny sizes only).

Test infrastructure only (see ``oracle/__init__``).

* ``K_matrix``      -- K = tau^{-alpha} (L (x) I_x) + I_t (x) A, L the lower triangular
                       Toeplitz matrix of omega_0..omega_{N-1}: the sequential scheme
                       eq. (2.1) / eq. (3.7) written all at once (K U = F_hat).
* ``P_matrix``      -- P_kappa = tau^{-alpha} (B_k(kappa) (x) I_x) + I_t (x) A with
                       B_k(kappa) as printed in eq. (2.6) / eq. (3.11).
* ``wr_rhs``        -- F_{m-1} = F_hat + (P_kappa - K) U_{m-1}. Row n of (P_kappa - K) U is
                       tau^{-alpha} kappa sum_{j=n}^{J} omega_j U^{N+n-j}, J = k for BDF and
                       J = N - 1 for CQ. For CQ this is eq. (3.12). For BDF it is the reading
                       of eq. (2.7) that matches the matrix B_k(kappa) and G_m^n of eq. (2.16):
                       the printed sum_{j=1}^{n} omega_j U^{N-j+1} does not (its fixed point is
                       not the BDF solution; pinned in tests).
* ``wr_sweep_dense``-- one sweep U_m = P_kappa^{-1} F_{m-1} (Algorithm 1 / Algorithm 2 in
                       exact linear algebra rather than through the diagonalisation).
* ``contraction``   -- spectral radius of the WR error map I - P_kappa^{-1} K for the scalar
                       problem A = lambda (one sine mode), and the BDF1 closed form
                       kappa r^N / (1 - kappa r^N), r = 1/(1 + lambda tau) (Remark 2.2).
"""
from __future__ import annotations

import numpy as np

from . import bdf
from .sequential import time_weights


def lower_toeplitz(omega, N):
    L = np.zeros((N, N))
    w = np.zeros(N)
    m = min(N, len(omega))
    w[:m] = omega[:m]
    for n in range(N):
        L[n, : n + 1] = w[n::-1]
    return L


def K_matrix(k, alpha, tau, A_dense, N):
    w = time_weights(k, alpha, N)
    M = A_dense.shape[0]
    return tau ** -alpha * np.kron(lower_toeplitz(w, N), np.eye(M)) + np.kron(np.eye(N), A_dense)


def P_matrix(k, alpha, kappa, tau, A_dense, N):
    w = time_weights(k, alpha, N)
    M = A_dense.shape[0]
    B = bdf.kappa_time_matrix(w, kappa, N)
    return tau ** -alpha * np.kron(B, np.eye(M)) + np.kron(np.eye(N), A_dense)


def wr_rhs(k, alpha, kappa, tau, Fhat, U_prev, printed_bdf_index=False):
    """F_{m-1} [N, M] from F_hat [N, M] and U_{m-1} [N, M] (row n-1 holds level n)."""
    N, M = Fhat.shape
    w = time_weights(k, alpha, N)
    J = k if alpha == 1.0 else N - 1
    F = Fhat.copy()
    for n in range(1, N + 1):
        acc = np.zeros(M)
        if printed_bdf_index:  # eq. (2.7) exactly as printed: sum_{j=1}^n omega_j U^{N-j+1}
            for j in range(1, min(n, k) + 1):
                acc += w[j] * U_prev[N - j]
        else:
            for j in range(n, min(J, N - 1) + 1):
                acc += w[j] * U_prev[N + n - j - 1]
        F[n - 1] += tau ** -alpha * kappa * acc
    return F


def wr_sweep_dense(k, alpha, kappa, tau, A_dense, Fhat, U_prev, printed_bdf_index=False):
    N, M = Fhat.shape
    P = P_matrix(k, alpha, kappa, tau, A_dense, N)
    F = wr_rhs(k, alpha, kappa, tau, Fhat, U_prev, printed_bdf_index)
    return np.linalg.solve(P, F.reshape(-1)).reshape(N, M)


def error_map(k, alpha, kappa, tau, lam, N):
    """I - P_kappa^{-1} K for the scalar operator A = lam."""
    A = np.array([[lam]])
    K = K_matrix(k, alpha, tau, A, N)
    P = P_matrix(k, alpha, kappa, tau, A, N)
    return np.eye(N) - np.linalg.solve(P, K)


def contraction(k, alpha, kappa, tau, lam, N):
    return float(np.max(np.abs(np.linalg.eigvals(error_map(k, alpha, kappa, tau, lam, N)))))


def contraction_bdf1_closed_form(kappa, tau, lam, N):
    r = (1.0 / (1.0 + lam * tau)) ** N
    return kappa * r / (1.0 - kappa * r)
