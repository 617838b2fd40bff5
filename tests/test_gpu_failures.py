"""Failure paths, all made on the host (nothing is faulted on the GPU).

* A divergent problem: BDF1 with kappa = 0.9 on a short horizon, where the WR contraction
  factor kappa r^N / (1 - kappa r^N), r = 1 / (1 + lambda_1 tau) (the BDF1 closed form of
  Remark 2.2), exceeds one. The solve's device-side stopping rule never fires and the call
  returns PINT_ENOTCONV after max_sweeps, through the graph path of pint_solve and of
  pint_batch_solve (where the other problems of the batch still converge).
* pint_poll on a request that is still queued: PINT_EAGAIN with timeout 0, PINT_ETIMEOUT with a
  short timeout, and the request stays live and completes.
* Allocation failures injected at every allocation the library makes while building a plan or a
  server, and at a request's admission: PINT_ENOMEM / PINT_EBUDGET, with every byte given back.
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import device_inputs, gpu_solve, oracle_solution, rel_l2, torch_cuda
from oracle import allatonce, grid

pytestmark = pytest.mark.gpu


def divergent_problem(mx=127, N=64):
    # lambda_1 ~ pi^2, T = 0.05: kappa r^N ~ 0.9 e^{-0.49} = 0.55 > 1/2, so gamma > 1
    return workloads.small_problem(dim=1, mx=mx, N=N, k=1, alpha=1.0, kappa=0.9, T=0.05)


def test_divergent_problem_is_predicted_to_diverge():
    p = divergent_problem()
    lam1 = grid.sine_eigenvalues(p.mx)[0]
    assert allatonce.contraction_bdf1_closed_form(p.kappa, p.tau, lam1, p.N) > 1.0
    # and the dense error map of the scalar mode agrees (spectral radius above one)
    assert allatonce.contraction(1, 1.0, p.kappa, p.tau, lam1, p.N) > 1.0


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_divergent_problem_returns_notconv_from_the_graph(prec):
    torch = torch_cuda()
    from paper_2007_13125_gb300 import pint
    p = divergent_problem()            # N * M = 8128 points: the multi-kernel graph path
    U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=1e-8, max_sweeps=12, raise_on_notconv=False)
    assert st == pint.PINT_ENOTCONV
    assert sweeps == 12
    assert upd > 1e-3                  # the update does not shrink


def test_batch_with_a_divergent_problem():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    probs = [divergent_problem(), workloads.small_problem(dim=2, mx=31, N=32, k=3, alpha=1.0, kappa=0.1),
             workloads.small_problem(dim=1, mx=255, N=64, k=2, alpha=0.5, kappa=0.1)]
    plans, Fs, Us, vs = [], [], [], []
    for p in probs:
        pl = Plan.for_problem(p, "mixed")
        v, f, fd = device_inputs(p, torch)
        F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
        pl.form_rhs(v, f, fd, F)
        plans.append(pl); Fs.append(F); Us.append(torch.empty_like(F)); vs.append(v)
    st, sweeps, upd = pint.batch_solve_v(plans, Fs, vs, Us, tol=1e-10, max_sweeps=15, raise_on_notconv=False)
    torch.cuda.synchronize()
    assert st == pint.PINT_ENOTCONV
    assert sweeps[0] == 15 and sweeps[1] < 15 and sweeps[2] < 15
    for p, U in zip(probs[1:], Us[1:]):
        assert rel_l2(U.cpu().numpy(), oracle_solution(p)) <= 1e-8
    for pl in plans:
        pl.close()


def test_poll_times_out_on_a_queued_request_which_then_completes():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import pint
    big = workloads.c2_heat2d(mx=255, N=1024)     # 67 M unknowns, host inputs: several ms to admit and run
    small = workloads.small_problem(dim=1, mx=63, N=64, k=2, alpha=1.0, kappa=0.1)
    with pint.Server(24 << 30, max_active=1) as srv:
        t_big = srv.submit(big, big.v, big.f(), big.fderiv(), tol=1e-8)
        t_small = srv.submit(small, small.v, small.f(), small.fderiv(), tol=1e-10)
        st0, _ = srv.poll(t_small, None, timeout_us=0)
        st1, _ = srv.poll(t_small, None, timeout_us=200)
        assert st0 == pint.PINT_EAGAIN
        assert st1 == pint.PINT_ETIMEOUT
        out = np.empty((small.N, small.M))
        st2, info = srv.poll(t_small, out, timeout_us=60_000_000)
        assert st2 == pint.PINT_OK
        assert info.t_start >= info.t_submit
        assert rel_l2(out, oracle_solution(small)) <= 1e-8
        st3, _ = srv.poll(t_big, None, timeout_us=60_000_000)
        assert st3 == pint.PINT_OK
        assert srv.poll(t_small, None, timeout_us=0)[0] == pint.PINT_ENOTFOUND   # retired


def _plan_attempts(make, max_n=64):
    """Arm the hook at n = 0, 1, ... until creation succeeds; every failure must be ENOMEM and give
    back every byte. Returns the number of injected failures."""
    from paper_2007_13125_gb300 import pint
    base = pint.device_bytes_held()
    failures = 0
    try:
        for n in range(max_n):
            pint.debug_fail_allocation(n)
            try:
                obj = make()
            except pint.PintError as e:
                assert e.status == pint.PINT_ENOMEM, str(e)
                assert pint.device_bytes_held() == base, n
                failures += 1
                continue
            pint.debug_fail_allocation(-1)
            assert pint.device_bytes_held() > base
            obj.close()
            assert pint.device_bytes_held() == base
            return failures
    finally:
        pint.debug_fail_allocation(-1)
    raise AssertionError("creation never succeeded")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_injected_allocation_failures_in_plan_creation(prec):
    torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.small_problem(dim=2, mx=63, N=64, k=3, alpha=0.5, kappa=0.1)
    n = _plan_attempts(lambda: Plan.for_problem(p, prec))
    assert n >= 4   # tables, iterate / spectrum workspaces, norms, pinned read-back buffers


def test_injected_allocation_failures_in_server_creation_and_admission():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import pint
    assert _plan_attempts(lambda: pint.Server(1 << 30, max_active=2)) == 2   # the budget, the pinned blocks
    base = pint.device_bytes_held()
    p = workloads.small_problem(dim=2, mx=31, N=32, k=2, alpha=1.0, kappa=0.1)
    with pint.Server(1 << 30, max_active=2) as srv:
        try:
            pint.debug_fail_allocation(0)            # the first sub-allocation of the next admission
            t = srv.submit(p, p.v, p.f(), p.fderiv(), tol=1e-10)
            st, _ = srv.poll(t, None, timeout_us=30_000_000)
        finally:
            pint.debug_fail_allocation(-1)
        assert st == pint.PINT_EBUDGET
        assert srv.stats()["hbm_in_use"] == 0
        # the server still serves the next request
        t = srv.submit(p, p.v, p.f(), p.fderiv(), tol=1e-10)
        out = np.empty((p.N, p.M))
        st, _ = srv.poll(t, out, timeout_us=30_000_000)
        assert st == pint.PINT_OK and rel_l2(out, oracle_solution(p)) <= 1e-8
        assert srv.stats()["hbm_in_use"] == 0
    assert pint.device_bytes_held() == base
