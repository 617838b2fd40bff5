"""pint_solve_host: end-to-end solves through host buffers (inputs copied in, solution copied out
by the library), several calls in a row on one plan so that the two staging sets and copy streams
are both exercised and reused. Each solution must be bit-identical to the device-buffer paths
(pint_solve_fv, and pint_form_rhs + pint_solve_v, on the same plan: the library reads the same
F_hat values whether it forms the whole of it or only its first levels) and within the MIXED bar of
the oracle."""
import numpy as np
import pytest

import workloads
from gpu_helpers import device_inputs, oracle_solution, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,mx,N,k,alpha", [(2, 31, 32, 3, 1.0), (1, 255, 64, 2, 0.5), (1, 63, 64, 1, 1.0)])
def test_solve_host_matches_device_path_and_oracle(dim, mx, N, k, alpha):
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    probs = [workloads.small_problem(dim=dim, mx=mx, N=N, k=k, alpha=alpha, kappa=0.1, seed=s) for s in (1, 2, 3)]
    p0 = probs[0]
    with Plan.for_problem(p0, "mixed") as plan:
        outs = [torch.empty((p0.N, p0.M), dtype=torch.float64).pin_memory() for _ in probs]
        hin = [(torch.tensor(p.v).pin_memory(), torch.tensor(p.f()).pin_memory(),
                torch.tensor(p.fderiv()).pin_memory() if k > 1 else None) for p in probs]
        for (v, f, fd), out in zip(hin, outs):
            plan.solve_host(v, f, fd, out, tol=1e-10)
        plan.solve_host_join()
        torch.cuda.synchronize()
        assert plan.solve_result()[0] == 0
        for p, out in zip(probs, outs):
            v, f, fd = device_inputs(p, torch)
            F = torch.empty((p.N, p.M), dtype=torch.float64, device="cuda:0")
            plan.form_rhs(v, f, fd if k > 1 else None, F)
            U = torch.empty_like(F)
            plan.solve_v(F, v, U, tol=1e-10)
            Ufv = torch.empty_like(F)
            plan.solve_fv(v, f, fd if k > 1 else None, Ufv, tol=1e-10)
            torch.cuda.synchronize()
            got = out.numpy()
            assert np.array_equal(got, Ufv.cpu().numpy())
            assert np.array_equal(got, U.cpu().numpy())
            assert rel_l2(got, oracle_solution(p)) <= 1e-8


def test_solve_host_rejects_bad_buffers():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.small_problem(dim=1, mx=31, N=32, k=2)
    with Plan.for_problem(p, "mixed") as plan:
        v = np.zeros(p.M)
        f = np.zeros((p.N, p.M))
        with pytest.raises(ValueError):
            plan.solve_host(v, f[:-1], np.zeros((1, p.M)), np.empty((p.N, p.M)))
        with pytest.raises(ValueError):
            plan.solve_host(torch.zeros(p.M, device="cuda:0", dtype=torch.float64), f, np.zeros((1, p.M)),
                            np.empty((p.N, p.M)))
