"""The diagonalised WR solve of Algorithms 1 / 2 in FP64 with NumPy/SciPy FFTs: a second CPU
reference, timed beside the sequential oracle (the same algorithm as the GPU path, on the host's
cores). Finite differences, Dirichlet, 1D/2D, BDF-k and CQ-BDF-k.

Test infrastructure only (see ``oracle/__init__``).

One sweep, in the residual-correction form (algebraically eq. (2.5) / eq. (3.10)):

    r   = F_hat - K U,   (K U)^n = tau^-alpha sum_{j=0}^{n-1} omega_j U^{n-j} + A U^n
                         (the sum by a zero-padded FFT convolution along time)
    h   = DFT_t(kappa^{n/N} r)                     (frequencies j = 0..N/2 of real data)
    q_j = (g_j tau^-alpha + A)^-1 h_j              (DST-I along each axis: A is diagonal on the
                                                    sine modes, eigenvalues (4/h^2) sin^2(p pi h/2))
    U  += kappa^{-n/N} IDFT_t(q)

with g_j the eigenvalues of B_k(kappa) (Lemma 2.3 / 3.3), taken from ``bdf.circulant_eigenvalues``
(the plain definition). Iterates until ||c|| / ||U|| <= tol.

Pins (``tests/test_oracle_diag_wr.py``): one sweep equals the dense WR sweep of ``allatonce``
(exact linear algebra, no diagonalisation); the iteration converges to the sequential solution.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import bdf, grid
from .sequential import time_weights


def _history(w, U, workers):
    """sum_{j=0}^{n} w_j U^{n-j} for every level n (lower triangular Toeplitz times U)."""
    N = U.shape[0]
    L = 2 * N
    W = sfft.rfft(w[:N], n=L, workers=workers)
    V = sfft.rfft(U, n=L, axis=0, workers=workers)
    return sfft.irfft(W[:, None] * V, n=L, axis=0, workers=workers)[:N]


def sweep(k, alpha, kappa, tau, mx, my, dim, Fhat, U, A=None, workers=-1):
    """One diagonalised sweep from U [N, M]; returns (U_next, correction)."""
    N, M = Fhat.shape
    w = time_weights(k, alpha, N)
    ta = tau ** -alpha
    if A is None:
        A = grid.laplacian(mx, my, dim)
    KU = ta * _history(w, U, workers) + (A @ U.T).T
    s = kappa ** (np.arange(N) / N)
    h = sfft.rfft(s[:, None] * (Fhat - KU), axis=0, workers=workers)          # [N/2+1, M]
    J = N // 2 + 1
    sig = bdf.circulant_eigenvalues(w, kappa, N)[:J] * ta
    lam_x = grid.sine_eigenvalues(mx)
    if dim == 1:
        H = sfft.dst(h, type=1, axis=1, workers=workers)
        H /= sig[:, None] + lam_x[None, :]
        H = sfft.dst(H, type=1, axis=1, workers=workers) / (2 * (mx + 1))
    else:
        lam_y = grid.sine_eigenvalues(my)
        H = h.reshape(J, my, mx)
        H = sfft.dst(sfft.dst(H, type=1, axis=2, workers=workers), type=1, axis=1, workers=workers)
        H /= sig[:, None, None] + lam_y[None, :, None] + lam_x[None, None, :]
        H = sfft.dst(sfft.dst(H, type=1, axis=2, workers=workers), type=1, axis=1, workers=workers)
        H = (H / (4.0 * (mx + 1) * (my + 1))).reshape(J, M)
    c = sfft.irfft(H, n=N, axis=0, workers=workers) / s[:, None]
    return U + c, c


def solve(k, alpha, kappa, tau, mx, my, dim, Fhat, U0, tol=1e-12, max_sweeps=50, workers=-1):
    """Sweeps from U0 until ||c|| / ||U|| <= tol: (U, sweeps, last update)."""
    A = grid.laplacian(mx, my, dim)
    U = np.array(U0, dtype=float, copy=True)
    upd = np.inf
    for m in range(1, max_sweeps + 1):
        U, c = sweep(k, alpha, kappa, tau, mx, my, dim, Fhat, U, A, workers)
        upd = float(np.linalg.norm(c) / np.linalg.norm(U))
        if upd <= tol:
            return U, m, upd
    return U, max_sweeps, upd
