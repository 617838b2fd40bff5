"""Time windows (the remark closing the discussion of Example 4, Sec. 4.3): solve the levels of a
long horizon window by window, each window by the parallel-in-time method, the next window
restarted from the previous one.

Test infrastructure only (see ``oracle/__init__``).

For BDF-k (alpha = 1) the all-at-once operator K is lower triangular with k sub-diagonal blocks
in time, so cutting the levels into windows of N_w levels is exact: window w solves the same
K (of N_w levels) with the previous window's last k levels moved to the right-hand side,

    F_hat_n = f(t_n) - tau^{-1} sum_{j=n}^{k} omega_j M U_prev^{N_w + n - j},  n = 1..k,
    F_hat_n = f(t_n),                                                            n > k,

(U_prev^m the m-th level of the previous window, M the mass matrix: I for finite differences)
and the windows' solutions together are the sequential solution of the whole horizon. The
first window is the ordinary problem (v and the starting corrections of eq. (2.1) / (4.4)).
The semilinear term w g(U) is pointwise in time, so Algorithm 3 runs per window unchanged; its
linearisation point, the time average over the window, then follows the solution. For CQ
(alpha < 1) K is full lower triangular and every earlier window would enter the history, which
is not done here.

Pins (tests/test_oracle_windows.py): windowed solves equal the whole-horizon sequential solution
(linear, 1D/2D finite differences and P1, k = 1..6; semilinear with Algorithm 3); on a strongly
nonlinear Allen-Cahn case where Algorithm 3 over the whole horizon diverges, windows of 8 and 16
levels converge to the sequential solution (the situation the remark describes).
"""
from __future__ import annotations

import numpy as np

from . import bdf, nonlinear as nl


def window_rhs(k, tau, Mass, F_t, U_prev):
    """F_hat [N_w, m] of a window after the first (alpha = 1): f(t_n) minus the BDF terms that
    reach into the previous window's levels U_prev [N_prev, m] (N_prev >= k)."""
    om = bdf.bdf_weights(k)
    Np = U_prev.shape[0]
    F = np.array(F_t, dtype=float, copy=True)
    for n in range(1, min(k, F.shape[0]) + 1):
        for j in range(n, k + 1):
            F[n - 1] -= om[j] / tau * (Mass @ U_prev[Np + n - j - 1])
    return F


def solve_windows_nl(k, kappa, tau, Mass, A, w, c, v, F_t, F_der, Nw, L=8, tol_inf=1e-12, max_sweeps=100):
    """Algorithm 3 window by window over the N = F_t.shape[0] levels (N a multiple of Nw); each
    window starts from its first level's predecessor, U_0^n = U_prev^{N_w} (v for the first).
    Returns (U [N, m], inner sweep counts per window)."""
    N = F_t.shape[0]
    out, counts = [], []
    prev = None
    for s in range(0, N, Nw):
        Ft = F_t[s:s + Nw]
        if prev is None:
            Fw = nl.nl_rhs(k, 1.0, tau, Mass, A, w, c, v, Ft, F_der)
            v0 = v
        else:
            Fw = window_rhs(k, tau, Mass, Ft, prev)
            v0 = prev[-1]
        its, cnt = nl.algorithm3(k, 1.0, kappa, tau, Mass, A, w, c, Fw, v0, L, tol_inf=tol_inf,
                                 max_sweeps=max_sweeps)
        prev = its[-1]
        out.append(prev)
        counts.append(cnt)
    return np.vstack(out), counts
