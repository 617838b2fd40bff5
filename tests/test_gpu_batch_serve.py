"""Graph-launched solves, one-launch batches of mixed problems, and the serving loop."""
import time

import numpy as np
import pytest

import workloads
from gpu_helpers import oracle_solution, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

MIX = [
    dict(dim=1, mx=63, N=64, k=2, alpha=1.0, kappa=0.1),
    dict(dim=2, mx=31, N=32, k=4, alpha=1.0, kappa=0.05),
    dict(dim=1, mx=127, N=128, k=3, alpha=0.5, kappa=0.1),
    dict(dim=2, mx=15, N=64, k=6, alpha=1.0, kappa=0.1),
    dict(dim=1, mx=31, N=256, k=1, alpha=0.3, kappa=0.01),
    dict(dim=2, mx=63, N=16, k=5, alpha=0.7, kappa=0.1),
]


def _problems(seed0=20):
    return [workloads.small_problem(seed=seed0 + i, **kw) for i, kw in enumerate(MIX)]


def test_graph_solve_matches_host_loop():
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    p = workloads.small_problem(dim=2, mx=31, N=64, k=3, alpha=1.0, kappa=0.05)
    dev = torch.device("cuda:0")
    v = torch.tensor(p.v, device=dev); f = torch.tensor(p.f(), device=dev); fd = torch.tensor(p.fderiv(), device=dev)
    out = []
    for profiled in (False, True):   # profiling on -> sweeps launched one by one from the host
        pint.set_profiling(profiled)
        with Plan.for_problem(p, "mixed") as plan:
            F = torch.empty((p.N, p.M), dtype=torch.float64, device=dev)
            U = torch.empty_like(F)
            plan.form_rhs(v, f, fd, F)
            plan.initial_guess(v, U)
            st, sweeps, upd = plan.solve(F, U, tol=1e-10)
            # a second solve reuses the cached graph
            plan.initial_guess(v, U)
            st2, sweeps2, upd2 = plan.solve(F, U, tol=1e-10)
            out.append((U.cpu().numpy(), sweeps, sweeps2, upd, upd2))
        pint.kernel_stats(reset=True)
    pint.set_profiling(False)
    (Ug, sg, sg2, ug, ug2), (Uh, sh, sh2, uh, uh2) = out
    assert sg == sh == sg2 == sh2
    assert np.array_equal(Ug, Uh)
    assert ug == pytest.approx(ug2, rel=1e-6)
    assert rel_l2(Ug, oracle_solution(p)) <= 1e-8


def test_graph_cache_rotating_buffers():
    """Solves over more buffer sets than a plan caches graphs for (least recently used replaced):
    every solve gives the same result as the first, bit for bit."""
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan
    p = workloads.small_problem(dim=2, mx=31, N=32, k=4, alpha=1.0, kappa=0.05, seed=5)
    dev = torch.device("cuda:0")
    v = torch.tensor(p.v, device=dev); f = torch.tensor(p.f(), device=dev); fd = torch.tensor(p.fderiv(), device=dev)
    with Plan.for_problem(p, "mixed") as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device=dev)
        plan.form_rhs(v, f, fd, F)
        Us = [torch.empty_like(F) for _ in range(5)]
        results = []
        for r in range(3):
            for i in (0, 1, 2, 3, 4, 1, 0):
                plan.initial_guess(v, Us[i])
                st, sweeps, upd = plan.solve(F, Us[i], tol=1e-9)
                results.append((Us[i].cpu().numpy(), sweeps))
    U0, s0 = results[0]
    for Ui, si in results[1:]:
        assert si == s0
        assert np.array_equal(Ui, U0)
    assert rel_l2(U0, oracle_solution(p)) <= 1e-8


def test_solve_async_back_to_back():
    """Solves enqueued back to back (pint_solve_async) on two buffer sets, with the copies of the
    results to host memory queued behind them, give the synchronous solve's result."""
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    from paper_2007_13125_gb300.pint import PintError
    p = workloads.small_problem(dim=2, mx=31, N=32, k=3, alpha=1.0, kappa=0.05, seed=7)
    dev = torch.device("cuda:0")
    v = torch.tensor(p.v, device=dev); f = torch.tensor(p.f(), device=dev); fd = torch.tensor(p.fderiv(), device=dev)
    with Plan.for_problem(p, "mixed") as plan:
        F = torch.empty((p.N, p.M), dtype=torch.float64, device=dev)
        plan.form_rhs(v, f, fd, F)
        Uref = torch.empty_like(F)
        plan.initial_guess(v, Uref)
        st, sweeps, upd = plan.solve(F, Uref, tol=1e-9)
        ref = Uref.cpu().numpy()
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        Us = [torch.empty_like(F) for _ in range(2)]
        outs = [torch.empty((p.N, p.M), dtype=torch.float64).pin_memory() for _ in range(4)]
        with torch.cuda.stream(s):
            for i in range(4):
                plan.initial_guess(v, Us[i % 2], s)
                plan.solve_async(F, Us[i % 2], tol=1e-9, stream=s)
                outs[i].copy_(Us[i % 2], non_blocking=True)
        s.synchronize()
        st2, sweeps2, upd2 = plan.solve_result()
        assert sweeps2 == sweeps and upd2 == pytest.approx(upd, rel=1e-9)  # atomically summed norms
        for o in outs:
            assert np.array_equal(o.numpy(), ref)
        pint.set_profiling(True)
        try:
            with pytest.raises(PintError):
                plan.solve_async(F, Us[0], tol=1e-9)
        finally:
            pint.set_profiling(False)
            pint.kernel_stats(reset=True)
    assert rel_l2(ref, oracle_solution(p)) <= 1e-8


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_solve_mixed_problems(precision):
    torch = torch_cuda()
    from paper_2007_13125_gb300 import Plan, pint
    dev = torch.device("cuda:0")
    probs = _problems()
    plans, Fs, Us = [], [], []
    for p in probs:
        pl = Plan.for_problem(p, precision)
        v = torch.tensor(p.v, device=dev); f = torch.tensor(p.f(), device=dev); fd = torch.tensor(p.fderiv(), device=dev)
        F = torch.empty((p.N, p.M), dtype=torch.float64, device=dev)
        U = torch.empty_like(F)
        pl.form_rhs(v, f, fd, F)
        pl.initial_guess(v, U)
        plans.append(pl); Fs.append(F); Us.append(U)
    st, sweeps, upd = pint.batch_solve(plans, Fs, Us, tol=1e-10)
    bar = 1e-8 if precision == "mixed" else 1e-10
    for p, U, s in zip(probs, Us, sweeps):
        assert rel_l2(U.cpu().numpy(), oracle_solution(p)) <= bar, (p.name, s)
    for pl in plans:
        pl.close()


def _host_inputs(p):
    return p.v, p.f(), p.fderiv()


def test_server_solves_a_stream_and_matches_oracle():
    torch_cuda()
    from paper_2007_13125_gb300 import pint
    probs = _problems(40)
    with pint.Server(2 << 30, max_active=4) as srv:
        tickets = []
        for p in probs:
            tickets.append(srv.submit(p, *_host_inputs(p), tol=1e-9))
        for p, t in zip(probs, tickets):
            out = np.empty((p.N, p.M))
            st, info = srv.poll(t, out, timeout_us=30_000_000)
            assert st == 0 and info.status == 0, (p.name, st)
            assert info.t_submit <= info.t_start <= info.t_done
            assert rel_l2(out, oracle_solution(p)) <= 1e-8, p.name
        stats = srv.stats()
        assert stats["completed"] == len(probs)
        assert stats["peak_hbm"] <= 2 << 30
        assert stats["hbm_in_use"] == 0


def test_server_result_same_alone_and_in_mix():
    """Invariance: a request's result does not depend on what else is being served."""
    torch_cuda()
    from paper_2007_13125_gb300 import pint
    target = workloads.small_problem(dim=2, mx=63, N=64, k=4, alpha=1.0, kappa=0.05, seed=99)
    out_alone = np.empty((target.N, target.M))
    with pint.Server(2 << 30, max_active=4) as srv:
        t = srv.submit(target, *_host_inputs(target), tol=1e-9)
        st, info_alone = srv.poll(t, out_alone, timeout_us=30_000_000)
        assert st == 0
    out_mix = np.empty_like(out_alone)
    with pint.Server(2 << 30, max_active=4) as srv:
        others = [(p, srv.submit(p, *_host_inputs(p), tol=1e-9)) for p in _problems(60)[:3]]
        t = srv.submit(target, *_host_inputs(target), tol=1e-9)
        others += [(p, srv.submit(p, *_host_inputs(p), tol=1e-9)) for p in _problems(70)[3:]]
        st, info_mix = srv.poll(t, out_mix, timeout_us=30_000_000)
        assert st == 0
        for p, tk in others:
            o = np.empty((p.N, p.M))
            assert srv.poll(tk, o, timeout_us=30_000_000)[0] == 0
    # per-problem arithmetic is independent of the batch: identical sweeps, identical result
    assert info_alone.sweeps == info_mix.sweeps
    assert rel_l2(out_mix, out_alone) <= 1e-12
    assert rel_l2(out_mix, oracle_solution(target)) <= 1e-8


def test_server_budget_admission_and_errors():
    torch_cuda()
    from paper_2007_13125_gb300 import pint
    big = workloads.small_problem(dim=2, mx=255, N=128, k=2, alpha=1.0, kappa=0.1, seed=5)   # ~8.3e6 DOF
    small = workloads.small_problem(dim=1, mx=63, N=64, k=2, alpha=1.0, kappa=0.1, seed=6)
    budget = 512 << 20            # holds one big request at a time (~0.35 GB each)
    with pint.Server(budget, max_active=8) as srv:
        tk = [srv.submit(big, *_host_inputs(big), tol=1e-8) for _ in range(3)]
        ts = srv.submit(small, *_host_inputs(small), tol=1e-8)
        huge = workloads.small_problem(dim=2, mx=511, N=256, k=2, alpha=1.0, kappa=0.1, seed=7)
        th = srv.submit(huge, huge.v, np.zeros((huge.N, huge.M)), np.zeros((1, huge.M)), tol=1e-8)
        st, info = srv.poll(th, None, timeout_us=30_000_000)
        assert st == pint.PINT_EBUDGET
        ref = oracle_solution(big)
        for t in tk:
            out = np.empty((big.N, big.M))
            st, info = srv.poll(t, out, timeout_us=30_000_000)
            assert st == 0 and rel_l2(out, ref) <= 1e-8
        assert srv.poll(ts, np.empty((small.N, small.M)), timeout_us=30_000_000)[0] == 0
        assert srv.stats()["peak_hbm"] <= budget
        st, _ = srv.poll(123456, None, 0)
        assert st == pint.PINT_ENOTFOUND


def test_server_device_inputs():
    """Requests whose inputs already live on the device are read at admission (no host copy)."""
    torch = torch_cuda()
    from paper_2007_13125_gb300 import pint
    dev = torch.device("cuda:0")
    probs = _problems(80)[:3]
    inputs = [(torch.tensor(p.v, device=dev), torch.tensor(p.f(), device=dev), torch.tensor(p.fderiv(), device=dev))
              for p in probs]
    with pint.Server(1 << 30, max_active=2) as srv:
        tickets = [srv.submit(p, *inp, tol=1e-9) for p, inp in zip(probs, inputs)]
        for p, t in zip(probs, tickets):
            out = np.empty((p.N, p.M))
            st, info = srv.poll(t, out, timeout_us=30_000_000)
            assert st == 0 and rel_l2(out, oracle_solution(p)) <= 1e-8


def test_server_unpolled_results_give_way_to_queued_requests():
    """Finished solutions wait on the device until polled; when they keep a queued request out of
    a tight budget the oldest are moved to host memory, so polling in any order completes."""
    torch_cuda()
    from paper_2007_13125_gb300 import pint
    probs = [workloads.small_problem(dim=2, mx=255, N=128, k=2, alpha=1.0, kappa=0.1, seed=30 + i) for i in range(5)]
    budget = 400 << 20            # one running request (~0.35 GB) plus about one held solution (67 MB)
    with pint.Server(budget, max_active=4) as srv:
        tickets = [srv.submit(p, *_host_inputs(p), tol=1e-8) for p in probs]
        for p, t in reversed(list(zip(probs, tickets))):
            out = np.empty((p.N, p.M))
            st, info = srv.poll(t, out, timeout_us=60_000_000)
            assert st == 0 and rel_l2(out, oracle_solution(p)) <= 1e-8
        stats = srv.stats()
        assert stats["peak_hbm"] <= budget
        assert stats["hbm_in_use"] == 0
