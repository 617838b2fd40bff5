"""Finite-difference spatial operator A_h (test infrastructure only).

The paper's experiments use P1 finite elements (Sec. 4); the workloads here use the
standard finite-difference Dirichlet Laplacian on the unit interval / unit square,
interior points only, h = 1/(M_x + 1):

* 1D: (A_h u)_i = (2 u_i - u_{i-1} - u_{i+1}) / h^2, u_0 = u_{M+1} = 0.
* 2D: 5-point stencil, A_h = I_y (x) T_x + T_y (x) I_x with the grid flattened as
  index = y * M_x + x (x fastest).
* 3D: 7-point stencil, I_z (x) A_h^{2D} + T_z (x) I_xy, index (z M_y + y) M_x + x.

A_h is symmetric positive definite, i.e. it satisfies the coercivity assumption of
eq. (1.2). Its eigenvectors are the sampled sine modes sin(p pi x_i) with eigenvalues
lambda_p = (4/h^2) sin^2(p pi h / 2) -- the textbook closed form used by the pins.

Periodic boundary conditions (the remark of Sec. 2.2, where the spatial systems become FFT-
diagonalisable): m points per axis, x_i = i/m, h = 1/m, the same stencil wrapping around
(``laplacian_periodic``). A_h is then a symmetric circulant, positive semi-definite (the
constant mode is its kernel), with eigenvectors e^{2 pi i p x} and eigenvalues
(4/h^2) sin^2(pi p / m), p = 0..m-1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def lap1d(m: int) -> sp.csr_matrix:
    h = 1.0 / (m + 1)
    e = np.ones(m)
    return sp.diags([-e[1:], 2 * e, -e[1:]], [-1, 0, 1], format="csr") / (h * h)


def laplacian(mx: int, my: int = 1, dim: int = 1, mz: int = 1) -> sp.csr_matrix:
    if dim == 1:
        return lap1d(mx)
    tx = lap1d(mx)
    ty = lap1d(my)
    if dim == 2:
        return (sp.kron(sp.identity(my), tx) + sp.kron(ty, sp.identity(mx))).tocsr()
    # 3D: 7-point stencil, index (z my + y) mx + x
    tz = lap1d(mz)
    ixy = sp.identity(mx * my)
    return (sp.kron(sp.identity(mz), sp.kron(sp.identity(my), tx) + sp.kron(ty, sp.identity(mx)))
            + sp.kron(tz, ixy)).tocsr()


def sine_eigenvalues(m: int) -> np.ndarray:
    """lambda_p = (4/h^2) sin^2(p pi h / 2), p = 1..m."""
    h = 1.0 / (m + 1)
    p = np.arange(1, m + 1)
    return 4.0 / (h * h) * np.sin(p * np.pi * h / 2) ** 2


def sine_mode(m: int, p: int) -> np.ndarray:
    x = np.arange(1, m + 1) / (m + 1)
    return np.sin(p * np.pi * x)


def lap1d_periodic(m: int) -> sp.csr_matrix:
    h = 1.0 / m
    e = np.ones(m)
    A = sp.diags([-e[1:], 2 * e, -e[1:]], [-1, 0, 1], format="lil")
    A[0, m - 1] = -1.0
    A[m - 1, 0] = -1.0
    return A.tocsr() / (h * h)


def laplacian_periodic(mx: int, my: int = 1, dim: int = 1) -> sp.csr_matrix:
    if dim == 1:
        return lap1d_periodic(mx)
    return (sp.kron(sp.identity(my), lap1d_periodic(mx)) + sp.kron(lap1d_periodic(my), sp.identity(mx))).tocsr()


def operator(p) -> sp.csr_matrix:
    """A_h of a workloads.Problem: Dirichlet FD or periodic FD (by p.space)."""
    if getattr(p, "space", "fd") == "periodic":
        return laplacian_periodic(p.mx, p.my, p.dim)
    return laplacian(p.mx, p.my, p.dim, getattr(p, "mz", 1))
