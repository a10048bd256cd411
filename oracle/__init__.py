"""Plain, slow FP64 CPU oracle for hierarchical proximal Galerkin (hpG).

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code, constants or helpers with ``paper_2412_13733_gb300`` (the
only shared module is the seeded input generator
``paper_2412_13733_gb300.workloads``, which holds no arithmetic of the method).

What it computes (paper sections / equations):

* ``basis1d``  -- the 1D hierarchical p-FEM bases of Section 3: Legendre
  ``P_n`` (the discontinuous space Psi_{h,p}), hats plus the bubbles ``W_n`` of
  eq. (Wn) (the continuous space U_{h,p}), and the spectral-Galerkin
  ``Y_n = P_n - P_{n+2}``.  Every 1D integral is taken by 64-point
  Gauss--Legendre quadrature of ``scipy.special`` evaluations, *not* from
  closed forms; the closed forms are the tests.
* ``space``    -- tensor-product (Kronecker) assembly of A, M, B on
  quad/hex meshes, the Dirichlet lifting, data loads and the Gauss-point
  quadrature of the latent nonlinearity (Section 5, "Quadrature").
* ``hpg``      -- the LVPP subproblem residual of eq. (pG), the Newton matrix
  G of eq. (pG-matrix) assembled sparse, one sparse direct solve per Newton
  step, the backtracking rule, and the alpha_k proximal loop.
* ``gradient`` -- the gradient-type subproblem of eq. (pG:gradient).
* ``schur``    -- the Schur complement S of eq. (schur4), the block-diagonal
  preconditioner S-hat of eq. (schur-preconditioner), and the sequential
  Schur solve of eq. (schur2), for component-level checks.
* ``pgs``      -- a projected Gauss--Seidel solve of the classical Q1 obstacle
  discretisation (brute-force cross-check on tiny meshes only).

Readings of the paper where it is silent or garbled are stated in the
docstrings where they are used.
"""
