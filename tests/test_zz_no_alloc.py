"""The allocation-free kappa-circulant solve (pint_kappa_solve_noalloc).

It serves callers that cannot allocate device memory at run time (fixed memory budgets,
plugins whose host owns all allocations, real-time loops); its scratch is a static device
array inside the library. Checked through the C ABI against the plan-based entry point
(pint_wr_sweep with U_prev = 0 computes the same P_kappa^{-1} R) on two calls in a row, so
the second call also shows that the previous call's scratch contents do not leak into it.
This file is collected last so that a failure here stops a -x run after all other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_sweep_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13125_gb300 import Plan, pint
    dev = torch.device("cuda:0")
    cases = [(4, 0.05, 256, 127, 11), (2, 0.1, 64, 63, 12)]  # larger first, then smaller
    for k, kappa, N, mx, seed in cases:
        tau = 1.0 / N
        rng = np.random.default_rng(seed)
        R = torch.tensor(rng.standard_normal((N, mx)), device=dev)
        Q = torch.full((N, mx), np.nan, dtype=torch.float64, device=dev)
        pint.kappa_solve_noalloc(k, kappa, tau, N, mx, R, Q)
        with Plan(k, 1.0, kappa, tau, N, 1, mx, precision="fp64") as plan:
            U0 = torch.zeros_like(R)
            ref = torch.empty_like(R)
            plan.wr_sweep(R, U0, ref)
        torch.cuda.synchronize()
        got, want = Q.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        # same tolerance as the FP64 single-sweep parity tests
        assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want), (k, N, mx)


def test_noalloc_matches_dense_kappa_circulant_solve():
    """Q = P_kappa^{-1} R against the oracle's dense kappa-circulant matrix P_kappa (B_k(kappa) of
    eq. (2.6) with the finite-difference Laplacian), solved by dense LU, on two calls in a row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import allatonce, grid
    from paper_2007_13125_gb300 import pint
    dev = torch.device("cuda:0")
    for k, kappa, N, mx, seed in [(3, 0.1, 16, 15, 21), (6, 0.05, 32, 7, 22)]:
        tau = 1.0 / N
        rng = np.random.default_rng(seed)
        R_h = rng.standard_normal((N, mx))
        A = grid.laplacian(mx, 1, 1).toarray()
        P = allatonce.P_matrix(k, 1.0, kappa, tau, A, N)
        want = np.linalg.solve(P, R_h.reshape(-1)).reshape(N, mx)
        R = torch.tensor(R_h, device=dev)
        Q = torch.full((N, mx), np.nan, dtype=torch.float64, device=dev)
        pint.kappa_solve_noalloc(k, kappa, tau, N, mx, R, Q)
        torch.cuda.synchronize()
        got = Q.cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want), (k, N, mx)


def test_noalloc_rejects_bad_buffers():
    """Undersized, aliased or host buffers never reach the kernels."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13125_gb300 import pint
    R = torch.zeros((64, 63), dtype=torch.float64, device="cuda:0")
    small = torch.zeros((32, 63), dtype=torch.float64, device="cuda:0")
    with pytest.raises(ValueError):
        pint.kappa_solve_noalloc(2, 0.1, 1.0 / 64, 64, 63, R, small)
    with pytest.raises(ValueError):
        pint.kappa_solve_noalloc(2, 0.1, 1.0 / 64, 64, 63, R, R)
    # the C entry point itself refuses overlapping arrays and host memory
    import ctypes
    L = pint.lib()
    st = L.pint_kappa_solve_noalloc(2, 0.1, 1.0 / 64, 64, 63, ctypes.c_void_p(R.data_ptr()),
                                    ctypes.c_void_p(R.data_ptr() + 8), None)
    assert st == pint.PINT_EINVAL and "overlap" in pint.last_error()
    host = np.zeros((64, 63))
    Q = torch.empty_like(R)
    st = L.pint_kappa_solve_noalloc(2, 0.1, 1.0 / 64, 64, 63, ctypes.c_void_p(host.ctypes.data),
                                    ctypes.c_void_p(Q.data_ptr()), None)
    assert st == pint.PINT_EINVAL and "device arrays" in pint.last_error()


def test_noalloc_rejects_sizes_beyond_capacity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13125_gb300 import pint
    R = torch.zeros((1024, 1023), dtype=torch.float64, device="cuda:0")
    Q = torch.empty_like(R)
    with pytest.raises(pint.PintError) as e:
        pint.kappa_solve_noalloc(2, 0.1, 1.0 / 1024, 1024, 1023, R, Q)
    assert e.value.status == pint.PINT_EINVAL
    assert "capacity" in str(e.value)
