"""The premise of the fused right-hand side (pint_solve_fv): for BDF-k with the starting
corrections of eq. (2.7), the all-at-once right-hand side F_hat_n (eq. (2.1)) equals f(t_n) from
level k + 1 on (the corrections act on n <= k - 1, and beta_n = tau^-1 sum_{j<n} omega_j vanishes
once the sum covers all k + 1 weights, since delta_k(1) = 0), and differs from it on the first k
levels. Checked on the oracle's right-hand side; no GPU."""
import numpy as np
import pytest

import workloads
from oracle import grid, sequential


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_bdf_rhs_is_f_beyond_the_first_k_levels(k):
    p = workloads.small_problem(dim=1, mx=31, N=32, k=k, seed=5)
    A = grid.operator(p)
    Fh = sequential.all_at_once_rhs(p.k, p.alpha, p.tau, A, p.v, p.f(), p.fderiv())
    f = p.f()
    scale = np.max(np.abs(f)) + np.max(np.abs(p.v)) / p.tau
    beyond = np.abs(Fh[k:] - f[k:]).max()
    assert beyond <= 1e-13 * scale, beyond
    # the first k levels differ: the beta_n v terms (and the corrections for k >= 2)
    first = np.abs(Fh[:k] - f[:k]).max(axis=1)
    assert np.all(first > 1e-6 * scale), first


def test_cq_rhs_differs_from_f_on_every_level():
    """For CQ (alpha < 1) beta_n never vanishes, so the fused form does not apply."""
    p = workloads.small_problem(dim=1, mx=31, N=32, k=2, alpha=0.5, seed=5)
    A = grid.operator(p)
    Fh = sequential.all_at_once_rhs(p.k, p.alpha, p.tau, A, p.v, p.f(), p.fderiv())
    assert np.all(np.abs(Fh - p.f()).max(axis=1) > 0)
