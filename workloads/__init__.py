"""Seeded synthetic inputs for the solver and for its oracle.

This module only draws random numbers and samples the problem data (initial value v,
source f and its time derivatives at t = 0) on the grid. It holds none of the method's
arithmetic; both the CUDA path's tests/benchmark and the CPU oracle take their inputs
from here.

The paper's experiments (Sec. 4) use P1 finite elements with specific analytic data and
publish no timings; these synthetic problems stand in for them at the paper's scale
(h ~ 1e-3 in 1D, N = 100..1000), on the finite-difference Dirichlet grid of the unit
interval / square with interior points x_i = i h, h = 1/(M_x + 1), flattened index
y * M_x + x, and uniform time levels t_n = n T / N, n = 1..N.

Random draws use ``numpy.random.default_rng(seed).standard_normal``:

* 1D sine series: v(x) = sum_{n<=P} c_n sin(n pi x), c_n = z_n / n^2, z drawn with shape (P,).
* 2D sine series: v(x, y) = sum_{m,n<=P} c_mn sin(m pi x) sin(n pi y), c_mn = z_mn/(m^2+n^2),
  z drawn with shape (P, P), first index the x-mode.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    name: str
    dim: int
    mx: int
    my: int
    N: int
    k: int
    alpha: float
    kappa: float
    T: float
    v: np.ndarray                       # [M]
    f_time: np.ndarray                  # [N] g(t_n), n = 1..N   (f = g(t) phi(x))
    f_space: np.ndarray                 # [M] phi(x)
    f_derivs0: np.ndarray               # [k-1] d^l g/dt^l (0), l = 0..k-2
    meta: dict = field(default_factory=dict)
    space: str = "fd"                   # "fd" (grid samples), "fem" (P1: nodal v, load vectors),
                                        # "periodic" (grid samples at x_i = i/m, periodic axes)
    mz: int = 1                         # points along z (3D)

    @property
    def M(self) -> int:
        return self.mx * self.my * self.mz

    @property
    def tau(self) -> float:
        return self.T / self.N

    @property
    def dof(self) -> int:
        return self.M * self.N

    def f(self) -> np.ndarray:
        """[N, M] samples f(t_n, x), n = 1..N."""
        return np.outer(self.f_time, self.f_space)

    def fderiv(self) -> np.ndarray:
        """[k-1, M]: row l is d_t^l f(0, x), l = 0..k-2 (row 0 = f(0))."""
        return np.outer(self.f_derivs0, self.f_space).reshape(max(self.k - 1, 0), self.M)


def grid_points(m: int) -> np.ndarray:
    return np.arange(1, m + 1) / (m + 1)


def sine_series_1d(m: int, coef: np.ndarray) -> np.ndarray:
    x = grid_points(m)
    n = np.arange(1, len(coef) + 1)
    return np.sin(np.pi * np.outer(x, n)) @ coef


def sine_series_2d(mx: int, my: int, coef: np.ndarray) -> np.ndarray:
    """coef[m-1, n-1] multiplies sin(m pi x) sin(n pi y); returns [my * mx] (x fastest)."""
    sx = np.sin(np.pi * np.outer(grid_points(mx), np.arange(1, coef.shape[0] + 1)))  # [mx, P]
    sy = np.sin(np.pi * np.outer(grid_points(my), np.arange(1, coef.shape[1] + 1)))  # [my, P]
    return (sy @ coef.T @ sx.T).reshape(-1)  # [my, mx]


def random_v(dim: int, mx: int, my: int, modes: int, rng) -> np.ndarray:
    if dim == 1:
        z = rng.standard_normal(modes)
        return sine_series_1d(mx, z / np.arange(1, modes + 1) ** 2)
    z = rng.standard_normal((modes, modes))
    m = np.arange(1, modes + 1)
    return sine_series_2d(mx, my, z / (m[:, None] ** 2 + m[None, :] ** 2))


def mode_field(dim: int, mx: int, my: int, px: int = 1, py: int = 2) -> np.ndarray:
    if dim == 1:
        return np.sin(px * np.pi * grid_points(mx))
    return np.outer(np.sin(py * np.pi * grid_points(my)), np.sin(px * np.pi * grid_points(mx))).reshape(-1)


def _exp_decay(N, T, k):
    t = np.arange(1, N + 1) * (T / N)
    return np.exp(-t), np.array([(-1.0) ** l for l in range(max(k - 1, 0))])


def make_problem(name, dim, mx, my, N, k, alpha, kappa, T, v, time_kind, f_space):
    t = np.arange(1, N + 1) * (T / N)
    if time_kind == "zero":
        g, d = np.zeros(N), np.zeros(max(k - 1, 0))
    elif time_kind == "exp":          # g(t) = e^{-t}: d^l g(0) = (-1)^l
        g, d = _exp_decay(N, T, k)
    elif time_kind == "linear":       # g(t) = t: g(0) = 0, g'(0) = 1
        g = t.copy()
        d = np.zeros(max(k - 1, 0))
        if k - 1 >= 2:
            d[1] = 1.0
    elif time_kind == "exp_growth":   # g(t) = e^{t}: d^l g(0) = 1
        g, d = np.exp(t), np.ones(max(k - 1, 0))
    else:
        raise ValueError(time_kind)
    return Problem(name, dim, mx, my if dim >= 2 else 1, N, k, alpha, kappa, T, v,
                   g, f_space, d, meta={"time_kind": time_kind})


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------


def c1_heat1d() -> Problem:
    """1D heat, M = 63, N = 64, T = 1, BDF2, kappa = 0.1, f = 0, v = 16-mode sine series (seed 0)."""
    rng = np.random.default_rng(0)
    mx = 63
    v = random_v(1, mx, 1, 16, rng)
    return make_problem("heat1d_M63_N64_bdf2", 1, mx, 1, 64, 2, 1.0, 0.1, 1.0, v, "zero",
                        np.zeros(mx))


def c2_heat2d(mx: int = 255, N: int = 256) -> Problem:
    """2D heat, 255 x 255, N = 256, T = 1, BDF4 with corrections, kappa = 0.05,
    f = e^{-t} sin(pi x) sin(2 pi y), v = 64 x 64-mode sine series (seed 1)."""
    rng = np.random.default_rng(1)
    v = random_v(2, mx, mx, min(64, mx), rng)
    return make_problem(f"heat2d_{mx}x{mx}_N{N}_bdf4", 2, mx, mx, N, 4, 1.0, 0.05, 1.0, v, "exp",
                        mode_field(2, mx, mx, 1, 2))


def c3_subdiff1d(mx: int = 1023, N: int = 1024) -> Problem:
    """1D subdiffusion alpha = 0.5, M = 1023, N = 1024, T = 1, CQ-BDF3, kappa = 0.01,
    f = t sin(pi x), v = 0."""
    return make_problem(f"subdiff1d_M{mx}_N{N}_cqbdf3_a0.5", 1, mx, 1, N, 3, 0.5, 0.01, 1.0,
                        np.zeros(mx), "linear", mode_field(1, mx, 1, 1))


C4_AXIS = (127, 255, 511)
C4_N = (64, 256, 1024, 2048)
C4_ALPHA = (0.3, 0.7, 1.0)
C4_KAPPA = (0.1, 0.01)


def c4_draw(rng, idx: int, axis=C4_AXIS, Ns=C4_N) -> Problem:
    """One problem of the mixed batch. Field order of the draws: dim, axis size, N, k,
    alpha, kappa, then the sine-series coefficients of v."""
    dim = int(rng.integers(1, 3))
    m = int(axis[rng.integers(0, len(axis))])
    N = int(Ns[rng.integers(0, len(Ns))])
    k = int(rng.integers(1, 7))
    alpha = float(C4_ALPHA[rng.integers(0, len(C4_ALPHA))])
    kappa = float(C4_KAPPA[rng.integers(0, len(C4_KAPPA))])
    v = random_v(dim, m, m, 16, rng)
    return make_problem(f"mix{idx}_{dim}d_{m}_N{N}_k{k}_a{alpha}_kap{kappa}", dim, m, m, N, k,
                        alpha, kappa, 1.0, v, "exp", mode_field(dim, m, m, 1, 2))


def c4_batch(n: int = 64, seed: int = 2, axis=C4_AXIS, Ns=C4_N) -> list[Problem]:
    """Batched mix: n problems, 1D or 2D, per-axis size from {127, 255, 511}, N from
    {64, 256, 1024, 2048}, k uniform in 1..6, alpha from {0.3, 0.7, 1.0}, kappa from
    {0.1, 0.01}; f = e^{-t} sin(pi x) [sin(2 pi y)], v a 16 (x 16)-mode sine series."""
    rng = np.random.default_rng(seed)
    return [c4_draw(rng, i, axis, Ns) for i in range(n)]


def c4_problem(dim: int, m: int, N: int, k: int, alpha: float, kappa: float, seed: int = 2) -> Problem:
    """One problem of the batch distribution with its parameters fixed instead of drawn (for
    parity cases at chosen corners of the distribution): v a 16 (x 16)-mode sine series from
    default_rng(seed), f = e^{-t} sin(pi x) [sin(2 pi y)], T = 1."""
    rng = np.random.default_rng(seed)
    v = random_v(dim, m, m, 16, rng)
    return make_problem(f"c4_{dim}d_{m}_N{N}_k{k}_a{alpha}_kap{kappa}", dim, m, m, N, k, alpha, kappa, 1.0, v,
                        "exp", mode_field(dim, m, m, 1, 2))


def c5_arrivals(n: int, rate: float = 200.0, seed: int = 3, axis=C4_AXIS, Ns=C4_N):
    """Poisson arrival stream: (arrival time in s, Problem) pairs, exponential
    inter-arrival times with mean 1/rate, problems drawn from the batch distribution."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        out.append((t, c4_draw(rng, i, axis, Ns)))
    return out


def small_problem(dim=1, mx=31, N=32, k=2, alpha=1.0, kappa=0.1, T=1.0, seed=7,
                  time_kind="exp", modes=8, my=None) -> Problem:
    """Small problems for parity tests (sizes spanning several tiles and ragged tails)."""
    rng = np.random.default_rng(seed)
    my = mx if my is None else my
    v = random_v(dim, mx, my, min(modes, mx, my), rng)
    if dim == 1:
        fs = mode_field(1, mx, 1, 1) + 0.3 * mode_field(1, mx, 1, 3)
    else:
        fs = mode_field(2, mx, my, 1, 2)
    p = make_problem(f"small_{dim}d_{mx}x{my}_N{N}_k{k}_a{alpha}", dim, mx, my, N, k, alpha, kappa,
                     T, v, time_kind, fs)
    return p


# ---------------------------------------------------------------------------
# 1D P1 finite-element problems (nodal values of v; f given by its load vectors (f, phi_i))
# ---------------------------------------------------------------------------


def fem_load_sine(m: int, p: int) -> np.ndarray:
    """(sin(p pi x), phi_i) for the hat functions of the uniform mesh with m interior nodes:
    sin(p pi x_i) * 2 (1 - cos(p pi h)) / (p^2 pi^2 h), the exact integral."""
    h = 1.0 / (m + 1)
    w = p * np.pi
    return np.sin(w * grid_points(m)) * 2.0 * (1.0 - np.cos(w * h)) / (w * w * h)


def fem_load_cos(m: int) -> np.ndarray:
    """(cos x, phi_i) = 2 cos(x_i) (1 - cos h) / h, the exact integral."""
    h = 1.0 / (m + 1)
    return 2.0 * np.cos(grid_points(m)) * (1.0 - np.cos(h)) / h


def fem_problem(mx=63, N=32, k=2, alpha=1.0, kappa=0.1, T=1.0, seed=7, modes=8, data="modes") -> Problem:
    """1D P1-FEM problems.
    data = "modes":    v_h = random sine series (nodal values, seed), f = e^{-t} (sin(pi x) + 0.3 sin(3 pi x));
    data = "example1": the data of the paper's Example 1 on this mesh: v_h = nodal values of the
                       indicator of (0, 1/2) (1/2 at x = 1/2), f = e^t cos x."""
    if data == "modes":
        rng = np.random.default_rng(seed)
        v = random_v(1, mx, 1, min(modes, mx), rng)
        load = fem_load_sine(mx, 1) + 0.3 * fem_load_sine(mx, 3)
        time_kind = "exp"
    elif data == "example1":
        x = grid_points(mx)
        v = np.where(x < 0.5, 1.0, np.where(x == 0.5, 0.5, 0.0))
        load = fem_load_cos(mx)
        time_kind = "exp_growth"
    else:
        raise ValueError(data)
    p = make_problem(f"fem1d_{data}_M{mx}_N{N}_k{k}_a{alpha}", 1, mx, 1, N, k, alpha, kappa, T, v,
                     time_kind, load)
    p.space = "fem"
    return p


def fem_mass_solve(m: int, b: np.ndarray) -> np.ndarray:
    """The nodal values v_h of the L2 projection of a function whose loads (v, phi_i) are b: the
    P1 mass matrix M_h = (h/6) tridiag(1, 4, 1) solved by a banded LU (scipy)."""
    from scipy.linalg import solve_banded
    h = 1.0 / (m + 1)
    ab = np.zeros((3, m))
    ab[0, 1:] = h / 6.0
    ab[1, :] = 4.0 * h / 6.0
    ab[2, :-1] = h / 6.0
    return solve_banded((1, 1), ab, b)


def paper_fem_example(example: int, k: int, N: int = 100, m: int = 999) -> Problem:
    """The data of the paper's 1D tests (Sec. 4) with P1 elements on the uniform mesh h = 1/(m+1)
    (the paper: h = 1/1000, N = 100):
    example 1 (Table 2): heat, T = 0.5, kappa = 0.5, v_h the L2 projection of the indicator of
      (0, 1/2), f = e^t cos x (loads 2 cos(x_i) (1 - cos h) / h e^t, every d_t^l f(0) = cos x);
    example 2 (Table 3): subdiffusion alpha = 0.5, T = 0.1, kappa = 0.1, v_h the L2 projection of
      the Dirac delta at 1/2 (loads phi_i(1/2)), f = 0."""
    h = 1.0 / (m + 1)
    x = grid_points(m)
    if example == 1:
        b = np.where(x < 0.5 - 0.25 * h, h, np.where(np.abs(x - 0.5) <= 0.25 * h, h / 2, 0.0))
        p = make_problem(f"paper_example1_M{m}_N{N}_k{k}", 1, m, 1, N, k, 1.0, 0.5, 0.5,
                         fem_mass_solve(m, b), "exp_growth", fem_load_cos(m))
    elif example == 2:
        b = np.maximum(0.0, 1.0 - np.abs(x - 0.5) / h)
        p = make_problem(f"paper_example2_M{m}_N{N}_k{k}", 1, m, 1, N, k, 0.5, 0.1, 0.1,
                         fem_mass_solve(m, b), "zero", np.zeros(m))
    else:
        raise ValueError(example)
    p.space = "fem"
    return p


# ---------------------------------------------------------------------------
# Periodic problems: m points per axis at x_i = i/m (periodic boundary conditions)
# ---------------------------------------------------------------------------


def periodic_points(m: int) -> np.ndarray:
    return np.arange(m) / m


def periodic_problem(dim=1, mx=32, N=32, k=2, alpha=1.0, kappa=0.1, T=1.0, seed=7, modes=6, my=None,
                     time_kind="exp") -> Problem:
    """v = random real Fourier series (modes 0..modes-1 per axis, coefficients / (1 + p^2) (seed)),
    f = g(t) (cos 2 pi x + 0.5 sin 4 pi x) [(cos 2 pi y)] with g(t) = e^{-t} by default."""
    rng = np.random.default_rng(seed)
    my = mx if my is None else my
    x = periodic_points(mx)
    modes = min(modes, mx // 2)
    if dim == 1:
        v = np.zeros(mx)
        for q in range(modes):
            a, b = rng.standard_normal(2) / (1 + q * q)
            v += a * np.cos(2 * np.pi * q * x) + b * np.sin(2 * np.pi * q * x)
        fs = np.cos(2 * np.pi * x) + 0.5 * np.sin(4 * np.pi * x)
    else:
        y = periodic_points(my)
        v = np.zeros((my, mx))
        for qy in range(modes):
            for qx in range(modes):
                a, b = rng.standard_normal(2) / (1 + qx * qx + qy * qy)
                v += a * np.outer(np.cos(2 * np.pi * qy * y), np.cos(2 * np.pi * qx * x)) \
                    + b * np.outer(np.sin(2 * np.pi * qy * y), np.sin(2 * np.pi * qx * x))
        v = v.reshape(-1)
        fs = np.outer(np.cos(2 * np.pi * y), np.cos(2 * np.pi * x) + 0.5 * np.sin(4 * np.pi * x)).reshape(-1)
    p = make_problem(f"periodic{dim}d_{mx}_N{N}_k{k}_a{alpha}", dim, mx, my, N, k, alpha, kappa, T, v,
                     time_kind, fs)
    p.space = "periodic"
    return p


# ---------------------------------------------------------------------------
# 3D problems on the unit cube (finite differences, Dirichlet), flattened (z my + y) mx + x
# ---------------------------------------------------------------------------


def heat3d_problem(m=15, N=16, k=2, alpha=1.0, kappa=0.1, T=1.0, seed=7, modes=6, my=None, mz=None,
                   time_kind="exp") -> Problem:
    """v = random sine series (modes^3 terms, coefficients N(0,1)/(p^2 + q^2 + r^2), seed),
    f = g(t) sin(pi x) sin(2 pi y) sin(pi z), g(t) = e^{-t} by default."""
    rng = np.random.default_rng(seed)
    my = m if my is None else my
    mz = m if mz is None else mz
    P = min(modes, m, my, mz)
    sx = np.sin(np.pi * np.outer(grid_points(m), np.arange(1, P + 1)))    # [mx, P]
    sy = np.sin(np.pi * np.outer(grid_points(my), np.arange(1, P + 1)))   # [my, P]
    sz = np.sin(np.pi * np.outer(grid_points(mz), np.arange(1, P + 1)))   # [mz, P]
    q = np.arange(1, P + 1)
    c = rng.standard_normal((P, P, P)) / (q[:, None, None] ** 2 + q[None, :, None] ** 2 + q[None, None, :] ** 2)
    v = np.einsum("zr,yq,xp,pqr->zyx", sz, sy, sx, c).reshape(-1)
    fs = np.einsum("z,y,x->zyx", np.sin(np.pi * grid_points(mz)), np.sin(2 * np.pi * grid_points(my)),
                   np.sin(np.pi * grid_points(m))).reshape(-1)
    p = make_problem(f"heat3d_{m}x{my}x{mz}_N{N}_k{k}_a{alpha}", 3, m, my, N, k, alpha, kappa, T, v,
                     time_kind, fs)
    p.mz = mz
    return p


# ---------------------------------------------------------------------------
# Semilinear problems (Sec. 4.3): D_t^alpha u + A u + g(u) = f, 1D, g a cubic
# ---------------------------------------------------------------------------


@dataclass
class NlProblem(Problem):
    """A semilinear problem: g(u) = g[0] + g[1] u + g[2] u^2 + g[3] u^3, and a source that is
    not a single product g(t) phi(x): F_t [N, M] holds f(t_n) (grid samples, or P1 load
    vectors), F_der [k-1, M] holds d_t^l f(0)."""
    g: tuple = (0.0, 0.0, 0.0, 0.0)
    F_t: np.ndarray | None = None
    F_der: np.ndarray | None = None

    def f(self) -> np.ndarray:
        return self.F_t

    def fderiv(self) -> np.ndarray:
        return self.F_der[: max(self.k - 1, 0)]


def allen_cahn_g(eps: float) -> tuple:
    """Example 4: g(u) = (u^3 - u) / eps^2."""
    return (0.0, -1.0 / eps ** 2, 0.0, 1.0 / eps ** 2)


def allen_cahn_problem(space="fem", mx=255, N=64, k=2, alpha=0.75, kappa=0.1, T=0.4, eps=1.0,
                       data="example4", seed=7, modes=8, amp=0.6) -> NlProblem:
    """1D semilinear problems with the Allen-Cahn term (u^3 - u) / eps^2, finite differences
    ("fd": grid samples) or P1 elements ("fem": nodal v, load vectors (f, phi_i), exact).
    data = "example4": Example 4's manufactured solution u = t^2/2 sin(2 pi x) (v = 0):
        f = [t^{2-alpha}/Gamma(3-alpha) + 2 pi^2 t^2] sin(2 pi x) + ((t^2/2)^3 sin^3(2 pi x)
            - (t^2/2) sin(2 pi x)) / eps^2,
      d_t f(0) = sin(2 pi x) when alpha = 1 and 0 for alpha < 1; higher derivatives of f at 0 do
      not exist for alpha < 1 (f ~ t^{2-alpha}), so k <= 3 there.
    data = "modes": v = amp * (random sine series, seed) normalised to max |v| = 1,
      f = e^{-t} (sin(pi x) + 0.3 sin(3 pi x)) * 4."""
    if alpha < 1.0 and k > 3 and data == "example4":
        raise ValueError("Example 4's source has no second time derivative at t = 0 for alpha < 1")
    h = 1.0 / (mx + 1)
    x = grid_points(mx)
    t = np.arange(1, N + 1) * (T / N)
    g = allen_cahn_g(eps)
    if space == "fem":
        s1 = fem_load_sine(mx, 2)
        s3 = (3.0 * s1 - fem_load_sine(mx, 6)) / 4.0  # sin^3 = (3 sin - sin 3.) / 4
    else:
        s1 = np.sin(2 * np.pi * x)
        s3 = s1 ** 3
    F_der = np.zeros((max(k - 1, 1), mx))
    if data == "example4":
        v = np.zeros(mx)
        a = t ** 2 / 2.0
        lin = t ** (2.0 - alpha) / math.gamma(3.0 - alpha) + (2 * np.pi) ** 2 * a
        F_t = np.outer(lin, s1) + np.outer(a ** 3, s3) / eps ** 2 - np.outer(a, s1) / eps ** 2
        if alpha == 1.0 and k >= 3:
            F_der[1] = s1
    elif data == "modes":
        rng = np.random.default_rng(seed)
        v = random_v(1, mx, 1, min(modes, mx), rng)
        v = amp * v / np.max(np.abs(v))
        if space == "fem":
            load = 4.0 * (fem_load_sine(mx, 1) + 0.3 * fem_load_sine(mx, 3))
        else:
            load = 4.0 * (np.sin(np.pi * x) + 0.3 * np.sin(3 * np.pi * x))
        F_t = np.outer(np.exp(-t), load)
        for l in range(F_der.shape[0]):
            F_der[l] = (-1.0) ** l * load
    else:
        raise ValueError(data)
    p = NlProblem(f"allencahn_{space}_{data}_M{mx}_N{N}_k{k}_a{alpha}", 1, mx, 1, N, k, alpha, kappa, T, v,
                  np.zeros(N), np.zeros(mx), np.zeros(max(k - 1, 0)), g=g, F_t=F_t, F_der=F_der)
    p.space = space
    p.meta.update(dict(eps=eps, data=data, h=h))
    return p
