"""FP64 CPU oracle for the waveform-relaxation / kappa-circulant method of
Wu & Zhou, "A parallel-in-time algorithm for high-order BDF methods for
diffusion and subdiffusion equations" (arXiv 2007.13125).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (the CUDA library and its Python binding) never imports,
links or executes anything in here, and this package imports nothing from the
product package.

What it computes is the plain definition of the method's fixed point: the
sequential corrected BDF-k scheme (Sec. 2.1, eq. (2.1)) and the sequential
corrected CQ-BDF-k scheme (Sec. 3.1, eq. (3.7)), with the spatial operator a
finite-difference Dirichlet Laplacian, solved step by step with a sparse LU.
Secondary routes, for pinning and for iterate-by-iterate references:

* ``bdf``        -- BDF generating polynomial weights (eq. (2.2)), CQ weights
                    (eq. (3.2)) by a contour-integral FFT, Table 1 constants
                    and their regeneration from order conditions, and the
                    kappa-circulant eigenvalues by their plain definition
                    (Lemma 2.3 / Lemma 3.3).
* ``grid``       -- the FD operator A_h and its sine eigenpairs.
* ``sequential`` -- corrected source f_bar_n (eq. (2.1)), the all-at-once
                    right-hand side F_hat, and the sequential solver.
* ``allatonce``  -- dense all-at-once matrices K and P_kappa (eq. (2.5),
                    eq. (3.9)), the dense paper-literal WR iteration
                    (eq. (2.4), eq. (3.8)) and per-mode contraction factors.
* ``fem``        -- the P1 finite-element form used by the paper's 1D tests
                    (Sec. 4): Tables 2 and 3.
* ``diag_wr``    -- the diagonalised WR solve (Algorithms 1 / 2) in FP64 with NumPy/SciPy
                    FFTs: a second CPU reference for timing, pinned against ``allatonce``
                    and ``sequential``.
* ``nonlinear``  -- the semilinear scheme (eq. (4.4)) stepped with Newton's
                    method, and Algorithm 3 (modified Newton with the
                    Jacobian at the time average, inner WR of eq. (4.7)):
                    Table 4.
* ``windows``    -- time windows for BDF-k (the remark closing Sec. 4.3):
                    the right-hand side of a window after the first, and
                    Algorithm 3 window by window.

Parity status of each function is stated in its docstring; every function
listed above is pinned by ``tests/test_oracle_*.py``.
"""
