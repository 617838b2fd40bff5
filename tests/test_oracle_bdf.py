"""Pins of oracle/bdf.py against what the paper and the mathematics fix."""
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import binom

from oracle import bdf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_table1():
    """Printed Table 1 (Sec. 2.1) from the golden fixture: {(k, kind, l, n): Fraction}."""
    out = {}
    with open(os.path.join(GOLDEN, "table1.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, kind, l, n, val = line.split()
            out[(int(k), kind, int(l), int(n))] = Fraction(val)
    return out


def test_bdf_weights_textbook():
    # backward Euler, BDF2, BDF3 in their textbook forms
    assert bdf.bdf_weights_exact(1) == [1, -1]
    assert bdf.bdf_weights_exact(2) == [Fraction(3, 2), -2, Fraction(1, 2)]
    assert bdf.bdf_weights_exact(3) == [Fraction(11, 6), -3, Fraction(3, 2), Fraction(-1, 3)]
    for k in range(1, 7):
        w = bdf.bdf_weights_exact(k)
        assert sum(w) == 0                                  # delta_k(1) = 0
        assert sum(j * wj for j, wj in enumerate(w)) == -1  # delta_k'(1) = -1


def test_bdf_order_k():
    # delta_k(e^{-z}) = z + O(z^{k+1}): consistency of order k (Sec. 2.1)
    for k in range(1, 7):
        errs = []
        for z in (1e-1, 5e-2):
            w = bdf.bdf_weights(k)
            val = sum(wj * np.exp(-z * j) for j, wj in enumerate(w))
            errs.append(abs(val - z))
        slope = np.log(errs[0] / errs[1]) / np.log(2.0)
        assert abs(slope - (k + 1)) < 0.35, (k, slope)


def test_delta_matches_polynomial():
    z = np.exp(1j * np.linspace(0, 2 * np.pi, 17)) * 0.93
    for k in range(1, 7):
        w = bdf.bdf_weights(k)
        poly = sum(wj * z ** j for j, wj in enumerate(w))
        assert np.allclose(bdf.delta_k(k, z), poly, rtol=0, atol=1e-13)


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
def test_cq_weights_bdf1_binomial(alpha):
    # k = 1: delta_1(xi)^alpha = (1 - xi)^alpha, coefficients (-1)^n C(alpha, n)
    # (Lemma 3.1; the leading minus sign printed there is a typo).
    n = 300
    w = bdf.cq_weights(1, alpha, n)
    ref = np.array([(-1) ** j * binom(alpha, j) for j in range(n)])
    assert np.max(np.abs(w - ref)) < 1e-14
    # product form omega_n = prod_{j<=n} (1 - (1 + alpha)/j)
    prod = np.cumprod([1 - (1 + alpha) / j for j in range(1, n)])
    assert np.allclose(w[1:], prod, rtol=1e-12)


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
def test_cq_weights_bdf2_product_series(alpha):
    # delta_2(xi) = (1 - xi)(3 - xi)/2 => delta_2^alpha = (3/2)^alpha (1-xi)^alpha (1-xi/3)^alpha
    n = 200
    a = np.array([(-1) ** j * binom(alpha, j) for j in range(n)])
    b = a / 3.0 ** np.arange(n)
    ref = 1.5 ** alpha * np.convolve(a, b)[:n]
    assert np.max(np.abs(bdf.cq_weights(2, alpha, n) - ref)) < 1e-13


@pytest.mark.parametrize("k", range(1, 7))
def test_cq_weights_square_root_squares_to_bdf(k):
    # (delta^{1/2})^2 = delta: convolution of the alpha = 1/2 weights is the BDF polynomial
    n = 120
    h = bdf.cq_weights(k, 0.5, n)
    sq = np.convolve(h, h)[:n]
    ref = np.zeros(n)
    ref[: k + 1] = bdf.bdf_weights(k)
    assert np.max(np.abs(sq - ref)) < 1e-12


@pytest.mark.parametrize("k", range(1, 7))
def test_cq_weights_alpha_one_and_decay(k):
    n = 400
    assert np.allclose(bdf.cq_weights(k, 1.0, n)[: k + 1], bdf.bdf_weights(k))
    for alpha in (0.3, 0.7):
        w = bdf.cq_weights(k, alpha, n)
        # Lemma 3.1: |omega_n| <= c (n+1)^{-alpha-1}; the scaled sequence stays bounded
        scaled = np.abs(w) * (np.arange(n) + 1.0) ** (alpha + 1)
        assert scaled[200:].max() < 2.0 * scaled[50:200].max()
        # partial sums -> 0 (delta_k(1) = 0) like n^{-alpha}
        ps = np.cumsum(w)
        assert abs(ps[-1]) < abs(ps[10])
        assert abs(w[0] - bdf.delta_k(k, 0.0).real ** alpha) < 1e-13


def test_table1_regenerates_from_order_conditions():
    printed = load_table1()
    mismatches = []
    for k in range(2, 7):
        a, b = bdf.regenerate_table1(k)
        for n in range(1, k):
            if printed[(k, "a", 0, n)] != a[n - 1]:
                mismatches.append((k, "a", 0, n))
        for l in range(1, k - 1):
            for n in range(1, k):
                if printed[(k, "b", l, n)] != b[l][n - 1]:
                    mismatches.append((k, "b", l, n))
    # exactly one printed entry contradicts the order conditions: b_{3,1}^(5)
    assert mismatches == [(5, "b", 3, 1)]
    a, b = bdf.regenerate_table1(5)
    assert b[3][0] == Fraction(-1, 720) == -printed[(5, "b", 3, 1)]


def test_oracle_table1_is_printed_table_with_one_reading():
    printed = load_table1()
    for k in range(2, 7):
        a, b = bdf.TABLE1[k]
        for n in range(1, k):
            assert a[n - 1] == printed[(k, "a", 0, n)]
        for l in range(1, k - 1):
            for n in range(1, k):
                want = printed[(k, "b", l, n)]
                if (k, l, n) == (5, 3, 1):
                    want = -want
                assert b[l][n - 1] == want


def test_table1_invariants():
    for k in range(2, 7):
        a, b = bdf.TABLE1[k]
        assert sum(a) == Fraction(1, 2)
        if k >= 3:
            assert sum(b[1]) == Fraction(1, 12)


def _match(eigs, ref):
    ref = list(ref)
    worst = 0.0
    for e in eigs:
        i = int(np.argmin([abs(e - r) for r in ref]))
        worst = max(worst, abs(e - ref[i]))
        ref.pop(i)
    return worst


@pytest.mark.parametrize("k,alpha", [(1, 1.0), (3, 1.0), (6, 1.0), (2, 0.5), (4, 0.3)])
def test_circulant_eigenvalues_vs_dense(k, alpha):
    N, kappa = 24, 0.1
    w = bdf.cq_weights(k, alpha, N)
    g = bdf.circulant_eigenvalues(w, kappa, N)
    dense = np.linalg.eigvals(bdf.kappa_time_matrix(w, kappa, N))
    scale = np.max(np.abs(g))
    assert _match(g, dense) < 1e-9 * scale
    if alpha == 1.0:
        # Lemma 2.3: eigenvalues delta_k(kappa^{1/N} e^{-2 pi i j / N})
        z = kappa ** (1.0 / N) * np.exp(-2j * np.pi * np.arange(N) / N)
        assert np.max(np.abs(g - bdf.delta_k(k, z))) < 1e-13 * scale
    # conjugate symmetry g_{N-j} = conj(g_j) (real first column)
    assert np.allclose(g[1:], np.conj(g[1:][::-1]), atol=1e-13 * scale)
