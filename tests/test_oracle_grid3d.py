"""Pins of the 3D finite-difference operator (oracle/grid.py): sampled sine products are its
eigenvectors with the sum of the three 1D eigenvalues."""
import numpy as np
import pytest

from oracle import grid


@pytest.mark.parametrize("mx,my,mz", [(3, 7, 15), (7, 7, 7)])
def test_sine_products_are_eigenvectors_3d(mx, my, mz):
    A = grid.laplacian(mx, my, 3, mz)
    for (p, q, r) in [(1, 1, 1), (2, 3, 1), (mx, my, mz)]:
        mode = np.einsum("z,y,x->zyx", grid.sine_mode(mz, r), grid.sine_mode(my, q), grid.sine_mode(mx, p)).reshape(-1)
        lam = grid.sine_eigenvalues(mx)[p - 1] + grid.sine_eigenvalues(my)[q - 1] + grid.sine_eigenvalues(mz)[r - 1]
        assert np.allclose(A @ mode, lam * mode, rtol=0, atol=1e-9 * lam)


def test_3d_operator_is_symmetric_7_point():
    A = grid.laplacian(7, 3, 3, 15)
    assert abs(A - A.T).max() == 0.0
    assert A.shape == (7 * 3 * 15,) * 2
    assert max(np.diff(A.indptr)) == 7        # interior rows couple to six neighbours
