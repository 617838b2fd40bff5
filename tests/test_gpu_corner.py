"""Parity at the hardest corner of the batch / serving distribution (N = 2048, kappa = 0.01).

The method's rounding grows with N and with 1/kappa: the paper bounds the relative error of the
diagonalised solve by about eps kappa^-2 N^2 for BDF-k (Sec. 2.3, the roundoff estimate and the
remark after it) and eps kappa^-2 N^(1 + alpha) for CQ-BDF-k (Sec. 3.3), so N = 2048 with
kappa = 0.01 is where the FP32 inner solves of the MIXED path are weakest as a preconditioner and
where the FP64 direct form loses the most digits. These problems are drawn from the batch recipe
(16-mode random sine series v, f = e^{-t} sin(pi x) [sin(2 pi y)]) with the parameters fixed at that
corner, and compared with the oracle's sequential solution: space-time relative l2 (the bars of
the other parity tests), per-level relative l2 (so an error confined to a few levels cannot hide
under the norm of all N levels), and the final-time error.
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import gpu_solve, oracle_solution, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

CORNER = [
    # dim, m, N, k, alpha, kappa
    (1, 511, 2048, 6, 0.3, 0.01),    # CQ-BDF6, the smallest alpha
    (1, 511, 2048, 6, 1.0, 0.01),    # BDF6
    (2, 127, 2048, 4, 0.7, 0.01),    # 2D CQ-BDF4
]


def per_level_rel(U, ref):
    """l2 error of each time level (row n-1 = level t_n) relative to max(||U_ref^n||, the RMS level
    norm ||U_ref|| / sqrt(N)). The diagonalised solve spreads its rounding evenly over the levels
    (the DFT along time mixes them; the paper's roundoff estimates are norm-wise), so a level far
    smaller than the typical one -- the first levels of a problem started from v = 0 -- carries a
    large error relative to itself while its absolute error is that of every other level; an error
    confined to a few levels of ordinary size still shows."""
    rms = np.linalg.norm(ref) / np.sqrt(ref.shape[0])
    return np.linalg.norm(U - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), rms)


@pytest.fixture(scope="module", params=CORNER, ids=lambda c: "{}d_{}_N{}_k{}_a{}_kap{}".format(*c))
def corner(request):
    p = workloads.c4_problem(*request.param)
    return p, oracle_solution(p)


@pytest.mark.parametrize("prec,bar,level_bar", [("mixed", 1e-8, 1e-7), ("fp64", 1e-10, 1e-9)])
def test_corner_parity(corner, prec, bar, level_bar):
    torch = torch_cuda()
    p, ref = corner
    U, st, sweeps, upd = gpu_solve(p, torch, prec, tol=bar)
    assert st == 0, (prec, sweeps, upd)
    assert np.all(np.isfinite(U))
    err = rel_l2(U, ref)
    lev = per_level_rel(U, ref)
    assert err <= bar, (prec, err, sweeps)
    # every level: a bar one decade above the global one (early levels are small, with the
    # starting corrections acting there, and carry larger relative rounding)
    assert lev.max() <= level_bar, (prec, int(lev.argmax()), float(lev.max()))
    assert np.linalg.norm(U[-1] - ref[-1]) <= bar * np.linalg.norm(ref[-1])
