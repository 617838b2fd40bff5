"""Sequential corrected BDF-k and CQ-BDF-k time stepping -- the WR fixed point.

Test infrastructure only (see ``oracle/__init__``).

The WR iteration's fixed point is the sequential time-stepping solution (Sec. 2.2,
remark after eq. (2.5); Sec. 3.2, remark after eq. (3.10)), so that solution, computed
step by step as the paper defines it, is what the GPU path is compared with.

* ``corrected_source``  -- f_bar_n = f(t_n) + a_n^(k) (f(0) - A v)
                           + sum_{l=1}^{k-2} b_{l,n}^(k) tau^l d_t^l f(0),  n = 1..N
                           (eq. (2.1) for alpha = 1, eq. (3.7) for alpha < 1).
* ``all_at_once_rhs``   -- F_hat_n = f_bar_n + tau^{-alpha} sum_{j=0}^{n-1} omega_j v, the
                           v-dependent third term of eq. (2.7) / eq. (3.12); with it the
                           sequential scheme is K U = F_hat, K = tau^{-alpha} (L (x) I) + I (x) A.
* ``solve_sequential``  -- steps n = 1..N of
                           (omega_0 I + tau^alpha A) U^n
                              = tau^alpha f_bar_n - sum_{j=1}^{n-1} omega_j U^{n-j}
                                + (sum_{j=0}^{n-1} omega_j) v,
                           the per-step system of Sec. 3.2 (speedup analysis of Algorithm 2,
                           multiplied by tau^alpha; its history sum and its v-sum are printed
                           separately, and so are they computed here), which for alpha = 1
                           (omega_j = 0, j > k) is the BDF-k scheme eq. (2.1) with
                           U^{-(k-1)} = ... = U^0 = v.

Pins (tests/test_oracle_sequential.py): order-k convergence against the exact solution
of a scalar ODE (alpha = 1) and by self-convergence (alpha < 1); first order without the
corrections; the full-grid solve equals the sum of per-mode scalar solves; the dense
all-at-once solve K U = F_hat gives the same U.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import bdf


def time_weights(k: int, alpha: float, N: int) -> np.ndarray:
    """omega_0..omega_{N-1}: BDF-k polynomial weights (alpha = 1, zero past k) or the
    CQ weights of delta_k^alpha (eq. (3.2))."""
    return bdf.cq_weights(k, alpha, N)


def corrected_source(k, tau, f_t, v_term, dfs, corrected=True):
    """f_bar [N, M].

    f_t    : [N, M] samples f(t_n), n = 1..N
    v_term : [M] f(0) - A v
    dfs    : [k-1, M] d_t^l f(0), l = 0..k-2 (row 0 is f(0) itself)
    """
    fbar = np.array(f_t, dtype=float, copy=True)
    if not corrected or k < 2:
        return fbar
    a = bdf.correction_a(k)
    b = bdf.correction_b(k)
    N = fbar.shape[0]
    for n in range(1, min(k - 1, N) + 1):
        fbar[n - 1] += a[n - 1] * v_term
        for l in range(1, k - 1):
            fbar[n - 1] += b[l - 1, n - 1] * tau ** l * dfs[l]
    return fbar


def all_at_once_rhs(k, alpha, tau, A, v, f_t, dfs, corrected=True):
    N = f_t.shape[0]
    w = time_weights(k, alpha, N)
    v_term = dfs[0] - A @ v if len(dfs) else -(A @ v)
    fbar = corrected_source(k, tau, f_t, v_term, dfs, corrected)
    csum = np.cumsum(w)  # sum_{j=0}^{n-1} omega_j at index n-1
    return fbar + (tau ** -alpha) * csum[:, None] * v[None, :]


def solve_sequential(k, alpha, tau, A, v, f_t, dfs, corrected=True, omega=None):
    """U [N, M], U[n-1] = U^n."""
    N, M = f_t.shape
    w = time_weights(k, alpha, N) if omega is None else omega
    v_term = dfs[0] - A @ v if len(dfs) else -(A @ v)
    fbar = corrected_source(k, tau, f_t, v_term, dfs, corrected)
    ta = tau ** alpha
    lu = spla.splu(sp.csc_matrix(w[0] * sp.identity(M) + ta * A))
    U = np.zeros((N, M))
    nz = int(np.max(np.nonzero(w)[0])) if np.any(w) else 0  # last nonzero weight
    csum = np.cumsum(w)                  # csum[j] = sum_{i=0}^{j} omega_i
    Lw = len(w)
    wrev = np.ascontiguousarray(w[::-1])  # wrev[Lw-1-j] = omega_j (a contiguous vector for BLAS)
    for n in range(1, N + 1):
        jmax = min(n - 1, nz)            # omega_j = 0 beyond nz, so the sums stop there
        rhs = ta * fbar[n - 1] + csum[jmax] * v
        if jmax >= 1:
            # sum_{j=1}^{jmax} omega_j U^{n-j}: U^{n-j} is row n-j-1, so rows n-1-jmax .. n-2
            # meet omega_jmax .. omega_1
            rhs = rhs - wrev[Lw - 1 - jmax:Lw - 1] @ U[n - 1 - jmax:n - 1]
        U[n - 1] = lu.solve(rhs)
    return U
