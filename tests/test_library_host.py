"""The C-ABI library without a GPU: it loads, exports every function include/pint.h declares,
and its host-side constant tables agree with the oracle."""
import numpy as np
import pytest

from oracle import bdf


@pytest.fixture(scope="module")
def pint():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2007_13125_gb300 import pint as P
    return P


def test_exports_every_declared_symbol(pint):
    L = pint.lib()
    names = pint.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing


def test_time_weights_match_oracle(pint):
    for k in range(1, 7):
        for alpha in (1.0, 0.3, 0.5, 0.7):
            n = 512
            got = pint.time_weights(k, alpha, n)
            ref = bdf.cq_weights(k, alpha, n)
            assert np.max(np.abs(got - ref)) < 1e-13, (k, alpha)


def test_correction_table_matches_oracle(pint):
    for k in range(1, 7):
        a, b = pint.correction_coefficients(k)
        assert np.allclose(a[: k - 1], bdf.correction_a(k), rtol=0, atol=1e-16)
        assert np.all(a[k - 1:] == 0)
        if k >= 3:
            assert np.allclose(b[: k - 2, : k - 1], bdf.correction_b(k), rtol=0, atol=1e-16)


@pytest.mark.parametrize("k,alpha,N", [(1, 1.0, 16), (4, 1.0, 64), (6, 1.0, 32), (2, 0.5, 64), (3, 0.3, 128)])
def test_eigenvalues_match_oracle_definition(pint, k, alpha, N):
    kappa = 0.05
    got = pint.circulant_eigenvalues(k, alpha, kappa, N)
    ref = bdf.circulant_eigenvalues(bdf.cq_weights(k, alpha, N), kappa, N)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_closed_form_eigenvalues(pint):
    N, kappa = 64, 0.1
    got = pint.circulant_eigenvalues(3, 0.5, kappa, N, pint.PINT_EIG_CLOSED_FORM)
    z = kappa ** (1.0 / N) * np.exp(-2j * np.pi * np.arange(N) / N)
    ref = np.exp(0.5 * np.log(bdf.delta_k(3, z)))
    assert np.max(np.abs(got - ref)) < 1e-13


def test_invalid_plans_rejected_before_device_use(pint):
    # validation runs before any CUDA call, so these fail cleanly without a GPU
    for args in [(0, 1.0, 0.1, 0.01, 64, 1, 63), (7, 1.0, 0.1, 0.01, 64, 1, 63),
                 (2, 0.0, 0.1, 0.01, 64, 1, 63), (2, 1.0, 0.0, 0.01, 64, 1, 63),
                 (2, 1.0, 0.1, 0.0, 64, 1, 63), (2, 1.0, 0.1, 0.01, 48, 1, 63),
                 (2, 1.0, 0.1, 0.01, 64, 1, 62), (2, 1.0, 0.1, 0.01, 64, 3, 63)]:
        with pytest.raises(pint.PintError) as e:
            pint.Plan(*args)
        assert e.value.status == pint.PINT_EINVAL
    assert "status" in pint.status_string(1) or pint.status_string(1) == "PINT_EINVAL"


def test_invalid_x_transform_variant_rejected_before_device_use(pint):
    for xdst in (-1, 4):
        with pytest.raises(pint.PintError) as e:
            pint.Plan(2, 1.0, 0.1, 0.01, 64, 2, 255, 255, xdst=xdst)
        assert e.value.status == pint.PINT_EINVAL


def test_invalid_fem_plans_rejected_before_device_use(pint):
    # P1 finite elements: 1D only (every precision), mx + 1 of the form 2^a 5^b; an unknown
    # space code is rejected too
    for kw in [dict(dim=2, mx=31, my=31, precision="mixed", space="fem"),
               dict(dim=1, mx=30, precision="fp64", space="fem"),
               dict(dim=1, mx=62, precision="mixed", space="fem"),
               dict(dim=1, mx=31, precision="mixed", space=7)]:
        with pytest.raises(pint.PintError) as e:
            pint.Plan(2, 1.0, 0.1, 0.01, 32, **kw)
        assert e.value.status == pint.PINT_EINVAL


def test_fem_load_vectors_are_exact_integrals():
    # the input generator's load vectors (f, phi_i) against adaptive quadrature
    import workloads
    from scipy.integrate import quad
    m = 31
    h = 1.0 / (m + 1)
    x = workloads.grid_points(m)
    ls, lc = workloads.fem_load_sine(m, 3), workloads.fem_load_cos(m)
    for i in (0, 9, 30):
        hat = lambda t, i=i: max(0.0, 1.0 - abs(t - x[i]) / h)
        qs = quad(lambda t: np.sin(3 * np.pi * t) * hat(t), x[i] - h, x[i] + h, points=[x[i]])[0]
        qc = quad(lambda t: np.cos(t) * hat(t), x[i] - h, x[i] + h, points=[x[i]])[0]
        assert abs(qs - ls[i]) < 1e-14 and abs(qc - lc[i]) < 1e-14


def test_invalid_periodic_plans_rejected_before_device_use(pint):
    # periodic axes take m a power of two in [8, 4096]
    for kw in [dict(dim=1, mx=63), dict(dim=1, mx=4), dict(dim=2, mx=32, my=31), dict(dim=1, mx=8192)]:
        with pytest.raises(pint.PintError) as e:
            pint.Plan(2, 1.0, 0.1, 0.01, 32, precision="mixed", space="periodic", **kw)
        assert e.value.status == pint.PINT_EINVAL


def test_invalid_3d_plans_rejected_before_device_use(pint):
    for kw in [dict(dim=3, mx=7, my=7, mz=7, precision="mixed", space="periodic"),
               dict(dim=3, mx=7, my=7, mz=7, precision="mixed", space="fem"),
               dict(dim=3, mx=7, my=7, mz=6, precision="fp64"),
               dict(dim=4, mx=7, my=7, mz=7, precision="fp64")]:
        with pytest.raises(pint.PintError) as e:
            pint.Plan(2, 1.0, 0.1, 0.01, 32, **kw)
        assert e.value.status == pint.PINT_EINVAL


def test_reaction_and_semilinear_entry_points_reject_null_plans(pint):
    # argument checks run before any CUDA call
    import ctypes
    L = pint.lib()
    g = pint._poly((0.0, -1.0, 0.0, 1.0))
    assert L.pint_set_reaction(None, None, None) == pint.PINT_EINVAL
    assert L.pint_form_rhs_window(None, None, None, None, None) == pint.PINT_EINVAL
    assert L.pint_solve_fv(None, None, None, None, None, 1e-8, 10, None, None, None) == pint.PINT_EINVAL
    assert L.pint_nl_form_rhs(None, ctypes.byref(g), None, None, None, None, None) == pint.PINT_EINVAL
    assert L.pint_nl_solve(None, ctypes.byref(g), None, None, 1e-8, 10, 1e-10, 20, None, None) == pint.PINT_EINVAL
    with pytest.raises(ValueError):
        pint._poly((1.0, 2.0))


def test_allen_cahn_inputs_are_the_manufactured_source():
    # Example 4 (Sec. 4.3): f = D_t^alpha u - u_xx + u^3 - u for u = t^2/2 sin(2 pi x); the finite-
    # difference samples against the formula evaluated independently, the P1 loads against
    # 4-point Gauss quadrature of f phi_i on each element
    import math
    import numpy.polynomial.legendre as leg
    import workloads
    alpha, T, N, m = 0.75, 0.4, 10, 31
    p = workloads.allen_cahn_problem("fd", mx=m, N=N, k=2, alpha=alpha, T=T)
    x = np.arange(1, m + 1) / (m + 1)
    t = T * np.arange(1, N + 1) / N

    def f(tt, xx):
        u = tt ** 2 / 2 * np.sin(2 * np.pi * xx)
        return (tt ** (2 - alpha) / math.gamma(3 - alpha) * np.sin(2 * np.pi * xx)
                + 4 * np.pi ** 2 * u + u ** 3 - u)

    assert np.allclose(p.f(), f(t[:, None], x[None, :]), rtol=1e-13, atol=1e-15)
    q = workloads.allen_cahn_problem("fem", mx=m, N=N, k=2, alpha=alpha, T=T)
    h = 1.0 / (m + 1)
    gx, gw = leg.leggauss(4)
    ref = np.zeros((N, m))
    for i in range(m):
        for a, b in ((x[i] - h, x[i]), (x[i], x[i] + h)):
            xs = (a + b) / 2 + (b - a) / 2 * gx
            phi = 1.0 - np.abs(xs - x[i]) / h
            ref[:, i] += (b - a) / 2 * (f(t[:, None], xs[None, :]) * phi * gw).sum(axis=1)
    assert np.allclose(q.f(), ref, rtol=1e-6, atol=1e-9)


def test_noalloc_wrapper_checks_buffer_sizes_without_a_gpu(pint):
    """The binding of pint_kappa_solve_noalloc refuses buffers that do not hold N * mx elements
    before anything reaches the library (the C entry point cannot see the sizes)."""
    torch = pytest.importorskip("torch")
    R = torch.zeros((64, 63), dtype=torch.float64)
    Q = torch.zeros((32, 63), dtype=torch.float64)
    with pytest.raises(ValueError, match="N \\* mx"):
        pint.kappa_solve_noalloc(2, 0.1, 1.0 / 64, 64, 63, R, Q)
    with pytest.raises(ValueError):
        pint.kappa_solve_noalloc(2, 0.1, 1.0 / 64, 64, 63, R, R)


def test_plan_tuning_query_rejects_null(pint):
    assert pint.lib().pint_plan_tuning(None, None, 0) == -1
