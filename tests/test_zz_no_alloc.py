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
