"""CPU test of the parallel cyclic reduction of the y-direction solve (csrc/kernels_space.cu,
k_pcr): the reduction steps written out in numpy with the kernel's row formulas and padding (rows
outside 0..n-1 are the identity) solve the constant-coefficient complex tridiagonal systems
(sigma + lambda_x + 2 g) q_i - g (q_{i-1} + q_{i+1}) = s_i exactly as a dense solve does."""
import numpy as np
import pytest


def pcr_solve(e, s, pad):
    """Rows divided by g: a = -1, c = -1, b = 2 + e; returns q (the solution of the divided system)."""
    n = len(s)
    NR = max(n, pad)
    a = np.zeros(NR, complex); b = np.ones(NR, complex); c = np.zeros(NR, complex); d = np.zeros(NR, complex)
    a[1:n] = -1; c[:n - 1] = -1; b[:n] = 2 + e; d[:n] = s
    st = 1
    while st < n:
        idx = np.arange(NR)
        m, p = idx - st, idx + st
        mv, pv = m >= 0, p < NR
        am = np.where(mv, a[np.clip(m, 0, NR - 1)], 0); bm = np.where(mv, b[np.clip(m, 0, NR - 1)], 1)
        cm = np.where(mv, c[np.clip(m, 0, NR - 1)], 0); dm = np.where(mv, d[np.clip(m, 0, NR - 1)], 0)
        ap = np.where(pv, a[np.clip(p, 0, NR - 1)], 0); bp = np.where(pv, b[np.clip(p, 0, NR - 1)], 1)
        cp = np.where(pv, c[np.clip(p, 0, NR - 1)], 0); dp = np.where(pv, d[np.clip(p, 0, NR - 1)], 0)
        k1, k2 = a / bm, c / bp
        a, b, c, d = -am * k1, b - cm * k1 - ap * k2, -cp * k2, d - dm * k1 - dp * k2
        st *= 2
    return (d / b)[:n]


@pytest.mark.parametrize("n,pad", [(1, 32), (7, 32), (31, 32), (32, 32), (33, 256), (255, 256), (511, 512),
                                   (1023, 1024)])
def test_pcr_matches_dense_solve(n, pad):
    rng = np.random.default_rng(n)
    s = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    g = 4.0 * (n + 1) ** 2
    for sigma in (3.0 + 40.0j, -20.0 + 200.0j, 1e4 - 5e3j):
        lam_x = 9.87
        e = (sigma + lam_x) / g
        T = np.diag(np.full(n, sigma + lam_x + 2 * g)) - g * (np.eye(n, k=1) + np.eye(n, k=-1))
        ref = np.linalg.solve(T, s)
        got = pcr_solve(e, s, pad) / g
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
