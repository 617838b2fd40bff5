"""The seeded synthetic inputs against their written recipe (the configurations' data: random
sine-series initial values, separable sources, the mixed batch's draw order), recomputed here
directly from the recipe rather than through the generators' helpers."""
import numpy as np

import workloads


def _x(m):
    return np.arange(1, m + 1) / (m + 1)


def test_c1_heat1d_recipe():
    # M = 63, N = 64, T = 1, BDF2, kappa = 0.1; f = 0; v = sum_{n<=16} z_n / n^2 sin(n pi x), seed 0
    p = workloads.c1_heat1d()
    z = np.random.default_rng(0).standard_normal(16)
    x = _x(63)
    v = np.zeros(63)
    for n in range(1, 17):
        v += z[n - 1] / n ** 2 * np.sin(n * np.pi * x)
    assert (p.dim, p.mx, p.N, p.k, p.alpha, p.kappa, p.T) == (1, 63, 64, 2, 1.0, 0.1, 1.0)
    assert np.abs(p.v - v).max() <= 1e-14 * np.abs(v).max()
    assert not p.f().any() and not p.fderiv().any()


def test_c2_heat2d_recipe():
    # 255 x 255, N = 256, BDF4, kappa = 0.05; v = sum_{m,n<=64} z_mn / (m^2 + n^2) sin(m pi x) sin(n pi y)
    # (m the x-mode, seed 1, points flattened y * mx + x); f = e^{-t} sin(pi x) sin(2 pi y)
    p = workloads.c2_heat2d()
    z = np.random.default_rng(1).standard_normal((64, 64))
    x = y = _x(255)
    m = np.arange(1, 65)
    rng = np.random.default_rng(5)
    for i, j in zip(rng.integers(0, 255, 6), rng.integers(0, 255, 6)):
        val = sum(z[a - 1, b - 1] / (a * a + b * b) * np.sin(a * np.pi * x[i]) * np.sin(b * np.pi * y[j])
                  for a in m for b in m)
        assert abs(p.v[j * 255 + i] - val) <= 1e-13 * np.abs(p.v).max()
    assert (p.dim, p.mx, p.my, p.N, p.k, p.kappa) == (2, 255, 255, 256, 4, 0.05)
    phi = np.outer(np.sin(2 * np.pi * y), np.sin(np.pi * x)).reshape(-1)
    t = np.arange(1, 257) / 256
    assert np.allclose(p.f(), np.exp(-t)[:, None] * phi[None, :], rtol=0, atol=1e-15)
    # d^l f / dt^l (0) = (-1)^l phi, l = 0..k-2
    assert np.allclose(p.fderiv(), np.array([phi, -phi, phi]), rtol=0, atol=1e-15)


def test_c3_subdiff1d_recipe():
    # M = 1023, N = 1024, alpha = 0.5, CQ-BDF3, kappa = 0.01; f = t sin(pi x): f(0) = 0, f'(0) = sin(pi x); v = 0
    p = workloads.c3_subdiff1d()
    x = _x(1023)
    assert (p.mx, p.N, p.k, p.alpha, p.kappa) == (1023, 1024, 3, 0.5, 0.01)
    assert not p.v.any()
    assert np.allclose(p.fderiv(), np.array([0 * x, np.sin(np.pi * x)]), rtol=0, atol=1e-15)
    t = np.arange(1, 1025) / 1024
    assert np.allclose(p.f(), t[:, None] * np.sin(np.pi * x)[None, :], rtol=0, atol=1e-15)


def test_c4_draw_order():
    # the mixed batch draws, per problem and in this order: dim, axis size, N, k, alpha, kappa, v
    rng_a = np.random.default_rng(2)
    rng_b = np.random.default_rng(2)
    for idx in range(3):
        p = workloads.c4_draw(rng_a, idx)
        dim = int(rng_b.integers(1, 3))
        m = (127, 255, 511)[rng_b.integers(0, 3)]
        N = (64, 256, 1024, 2048)[rng_b.integers(0, 4)]
        k = int(rng_b.integers(1, 7))
        alpha = (0.3, 0.7, 1.0)[rng_b.integers(0, 3)]
        kappa = (0.1, 0.01)[rng_b.integers(0, 2)]
        rng_b.standard_normal(16 if dim == 1 else (16, 16))          # v's coefficients
        assert (p.dim, p.mx, p.N, p.k, p.alpha, p.kappa) == (dim, m, N, k, alpha, kappa)


def test_paper_fem_examples_match_the_oracle_data():
    # the inputs of Tables 2 / 3 (Sec. 4, Examples 1 and 2), written here independently of the
    # oracle's own data routines, agree with them
    from oracle import fem
    for ex, data in ((1, fem.example1_data), (2, fem.example2_data)):
        tau, v, F_t, F_der = data()
        for k in (1, 4, 6):
            p = workloads.paper_fem_example(ex, k)
            assert p.tau == tau and p.N == 100 and p.mx == 999
            assert np.max(np.abs(p.v - v)) <= 1e-14 * np.max(np.abs(v))
            assert np.max(np.abs(p.f() - F_t)) <= 1e-15
            assert np.max(np.abs(p.fderiv() - F_der[: k - 1]), initial=0.0) <= 1e-15
