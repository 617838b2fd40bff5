"""Time-discretisation constants of the method, in exact or FP64 arithmetic.

Test infrastructure only (see ``oracle/__init__``).

* ``bdf_weights``        -- omega_0..omega_k of delta_k(zeta) = sum_{l=1}^k (1-zeta)^l / l,
                            Sec. 2.1 eq. (2.2). Exact rationals.
* ``delta_k``            -- the generating polynomial itself, evaluated through 1-zeta.
* ``cq_weights``         -- omega_j^(alpha), coefficients of delta_k(xi)^alpha, Sec. 3.1
                            eq. (3.2); computed by the Cauchy integral on a circle of radius
                            rho < 1 with an L-point trapezoid rule (an FFT), principal branch.
* ``TABLE1``             -- the starting-step correction constants a_n^(k), b_{l,n}^(k) of
                            Table 1 (Sec. 2.1), as printed, with one reading: b_{3,1}^(5)
                            is taken as -1/720 (the printed +1/720 contradicts the order
                            conditions below and the observed order of BDF5; pinned in tests).
* ``regenerate_table1``  -- the same constants solved from the order conditions
                            delta_k(xi)^{l+1} ( sum_{n>=1} n^l xi^n / l! + sum_n b_{l,n} xi^n )
                              = 1 + O((1-xi)^k),      (l = 0 uses a_n),
                            the conditions under which the corrected source reproduces the
                            generating function of t^l/l! (the paper takes the constants
                            from its refs. JinLiZhou:SISC2017 / LiWangZhou:SINUM2020).
* ``circulant_eigenvalues`` -- eigenvalues of the kappa-circulant time matrix B_k(kappa),
                            Lemma 2.3 / Lemma 3.3: g_j = sum_{l<N} kappa^{l/N} omega_l
                            e^{-2 pi i j l / N}, by the plain O(N^2) sum.

Pins (tests/test_oracle_bdf.py): weights sum to zero and match the BDF formulas of
textbooks for k=1,2; CQ weights reduce to binomials for k=1 and to the BDF polynomial
for alpha=1, and match the exact product series for k=2; Table 1 regenerates from the
order conditions; eigenvalues match a dense eigendecomposition and the closed form
delta_k(kappa^{1/N} e^{-2 pi i j/N}).
"""
from __future__ import annotations

from fractions import Fraction
from math import comb, factorial

import numpy as np

# ---------------------------------------------------------------------------
# BDF-k generating polynomial (Sec. 2.1, eq. (2.2))
# ---------------------------------------------------------------------------


def bdf_weights_exact(k: int) -> list[Fraction]:
    """omega_0..omega_k with delta_k(zeta) = sum_l (1-zeta)^l / l = sum_j omega_j zeta^j."""
    if not 1 <= k <= 6:
        raise ValueError("BDF order k must be in 1..6")
    w = [Fraction(0)] * (k + 1)
    for l in range(1, k + 1):
        # (1 - zeta)^l = sum_j C(l, j) (-zeta)^j
        for j in range(l + 1):
            w[j] += Fraction(comb(l, j) * (-1) ** j, l)
    return w


def bdf_weights(k: int) -> np.ndarray:
    return np.array([float(x) for x in bdf_weights_exact(k)])


def delta_k(k: int, zeta):
    """delta_k(zeta) evaluated as sum_l s^l / l with s = 1 - zeta (no cancellation near 1)."""
    s = 1.0 - np.asarray(zeta, dtype=complex)
    out = np.zeros_like(s)
    p = np.ones_like(s)
    for l in range(1, k + 1):
        p = p * s
        out = out + p / l
    return out


# ---------------------------------------------------------------------------
# CQ weights (Sec. 3.1, eq. (3.2))
# ---------------------------------------------------------------------------


def cq_weights(k: int, alpha: float, n: int) -> np.ndarray:
    """First n coefficients of delta_k(xi)^alpha (principal branch).

    omega_j = (1 / 2 pi i) \\oint_{|xi| = rho} delta_k(xi)^alpha xi^{-j-1} dxi, evaluated
    with the L-point trapezoid rule on the circle |xi| = rho, i.e.
    omega_j ~= rho^{-j} (1/L) sum_m delta_k(rho e^{2 pi i m / L})^alpha e^{-2 pi i j m / L}.
    The rule aliases omega_{j + pL} rho^{pL} into omega_j; with rho^L = 1e-12 and
    L >= 8 n the aliasing is below 1e-12 |omega_{j+L}| and the rounding is amplified by
    at most rho^{-n} <= 1e-12^{-1/8} ~ 32.
    """
    if n <= 0:
        return np.zeros(0)
    if alpha == 1.0:
        w = np.zeros(n)
        b = bdf_weights(k)
        m = min(n, k + 1)
        w[:m] = b[:m]
        return w
    L = 64
    while L < 8 * n:
        L *= 2
    rho = 1e-12 ** (1.0 / L)
    xi = rho * np.exp(2j * np.pi * np.arange(L) / L)
    vals = np.exp(alpha * np.log(delta_k(k, xi)))
    coef = np.fft.fft(vals) / L  # sum_m vals_m e^{-2 pi i j m / L}
    j = np.arange(n)
    return (coef[:n] * rho ** (-j.astype(float))).real


# ---------------------------------------------------------------------------
# Table 1: starting-step correction constants (Sec. 2.1, Table 1)
# ---------------------------------------------------------------------------

F = Fraction
# TABLE1[k] = (a_1..a_{k-1}, {l: (b_{l,1}..b_{l,k-1})})
TABLE1: dict[int, tuple[list[Fraction], dict[int, list[Fraction]]]] = {
    1: ([], {}),
    2: ([F(1, 2)], {}),
    3: ([F(11, 12), F(-5, 12)], {1: [F(1, 12), F(0)]}),
    4: ([F(31, 24), F(-7, 6), F(3, 8)],
        {1: [F(1, 6), F(-1, 12), F(0)],
         2: [F(0), F(0), F(0)]}),
    5: ([F(1181, 720), F(-177, 80), F(341, 240), F(-251, 720)],
        {1: [F(59, 240), F(-29, 120), F(19, 240), F(0)],
         2: [F(1, 240), F(-1, 240), F(0), F(0)],
         3: [F(-1, 720), F(0), F(0), F(0)]}),   # printed +1/720; see module docstring
    6: ([F(2837, 1440), F(-2543, 720), F(17, 5), F(-1201, 720), F(95, 288)],
        {1: [F(77, 240), F(-7, 15), F(73, 240), F(-3, 40), F(0)],
         2: [F(1, 96), F(-1, 60), F(1, 160), F(0), F(0)],
         3: [F(-1, 360), F(1, 720), F(0), F(0), F(0)],
         4: [F(0), F(0), F(0), F(0), F(0)]}),
}


def correction_a(k: int) -> np.ndarray:
    """a_n^(k) for n = 1..k-1 (a_n = 0 for n >= k)."""
    return np.array([float(x) for x in TABLE1[k][0]])


def correction_b(k: int) -> np.ndarray:
    """b_{l,n}^(k) as an array [l-1, n-1] for l = 1..k-2, n = 1..k-1."""
    b = np.zeros((max(k - 2, 0), max(k - 1, 0)))
    for l, row in TABLE1[k][1].items():
        b[l - 1, :] = [float(x) for x in row]
    return b


# ---- regeneration from the order conditions, in exact rational arithmetic ----
# Polynomials in s = 1 - xi are lists of Fractions, index = power of s.


def _pmul(p, q, deg):
    out = [Fraction(0)] * (deg + 1)
    for i, a in enumerate(p[: deg + 1]):
        if a == 0:
            continue
        for j, b in enumerate(q[: deg + 1 - i]):
            out[i + j] += a * b
    return out


def _ppow(p, e, deg):
    out = [Fraction(1)] + [Fraction(0)] * deg
    for _ in range(e):
        out = _pmul(out, p, deg)
    return out


def _xi_poly_to_s(c):
    """Re-express sum_j c_j xi^j as a polynomial in s = 1 - xi."""
    deg = len(c) - 1
    out = [Fraction(0)] * (deg + 1)
    for j, cj in enumerate(c):
        for i in range(j + 1):  # (1 - s)^j
            out[i] += cj * comb(j, i) * (-1) ** i
    return out


def _series_times_pole(l):
    """(1 - xi)^{l+1} * sum_{n>=1} n^l xi^n / l!, which is a polynomial in xi of degree
    <= l+1; computed from the truncated power series (coefficients past degree l+1 cancel)."""
    R = 4 * (l + 2)
    ser = [Fraction(0)] + [Fraction(n ** l, factorial(l)) for n in range(1, R + 1)]
    one_minus = [Fraction(comb(l + 1, i) * (-1) ** i) for i in range(l + 2)]
    prod = [Fraction(0)] * (R + 1)
    for i, a in enumerate(one_minus):
        for j in range(R + 1 - i):
            prod[i + j] += a * ser[j]
    assert all(x == 0 for x in prod[l + 2:R - l - 1]), "series did not terminate"
    return prod[: l + 2]


def _solve_exact(A, b):
    n = len(b)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def regenerate_table1(k: int):
    """Solve the order conditions for a_n^(k) (l = 0) and b_{l,n}^(k) (l >= 1).

    Returns (a, {l: b_l}) in the layout of TABLE1, each list padded to length k-1.
    """
    deg = k  # work modulo s^k (keep s^0..s^{k-1})
    delta_over_s = [Fraction(0)] + [Fraction(0)] * deg
    for l in range(1, k + 1):  # delta_k / s = sum_l s^{l-1} / l
        delta_over_s[l - 1] += Fraction(1, l)
    delta_over_s = delta_over_s[: deg + 1]
    result = {}
    for l in range(0, k - 1):
        nunk = k - 1 - l
        d_pow = _ppow(delta_over_s, l + 1, deg)              # (delta/s)^{l+1}
        base = _pmul(d_pow, _xi_poly_to_s(_series_times_pole(l)), deg)
        # contribution of b_n: (delta/s)^{l+1} * s^{l+1} * xi^n
        cols = []
        for n in range(1, nunk + 1):
            xin = _xi_poly_to_s([Fraction(0)] * n + [Fraction(1)])
            shifted = [Fraction(0)] * (l + 1) + xin
            cols.append(_pmul(d_pow, shifted, deg))
        # conditions: coefficient of s^0 is 1, of s^1..s^{k-1} is 0
        assert base[0] == 1 and all(base[i] == 0 for i in range(1, l + 1))
        rows = list(range(l + 1, k))
        A = [[cols[c][r] for c in range(nunk)] for r in rows]
        rhs = [-base[r] for r in rows]
        sol = _solve_exact(A, rhs) if nunk else []
        result[l] = sol + [Fraction(0)] * (k - 1 - len(sol))
    a = result.pop(0) if k >= 2 else []
    return a, {l: v for l, v in result.items()}


# ---------------------------------------------------------------------------
# kappa-circulant eigenvalues (Lemma 2.3, Lemma 3.3)
# ---------------------------------------------------------------------------


def circulant_eigenvalues(omega: np.ndarray, kappa: float, N: int) -> np.ndarray:
    """g_j, j = 0..N-1, for the circulant with first column c_l = kappa^{l/N} omega_l
    (l < N), by the plain O(N^2) sum g_j = sum_l c_l e^{-2 pi i j l / N}.

    B_k(kappa) = Lambda C Lambda^{-1} with Lambda = diag(kappa^{-(n-1)/N}) (Lemma 2.3),
    so these are also the eigenvalues of B_k(kappa)."""
    w = np.zeros(N)
    m = min(N, len(omega))
    w[:m] = omega[:m]
    l = np.arange(N)
    c = kappa ** (l / N) * w
    jl = np.outer(l, l) % N
    return (np.exp(-2j * np.pi * jl / N) * c[None, :]).sum(axis=1)


def kappa_time_matrix(omega: np.ndarray, kappa: float, N: int) -> np.ndarray:
    """Dense B_k(kappa) of eq. (2.6) / eq. (3.11): lower triangular Toeplitz of
    omega_0..omega_{N-1} plus kappa * omega_{N+n-n'} above the diagonal."""
    w = np.zeros(N)
    m = min(N, len(omega))
    w[:m] = omega[:m]
    B = np.zeros((N, N))
    for n in range(N):
        for n2 in range(N):
            if n2 <= n:
                B[n, n2] = w[n - n2]
            else:
                B[n, n2] = kappa * w[N + n - n2]
    return B
