"""Plain FP64 CPU oracle for the sparsifying-preconditioned Lippmann-Schwinger solve.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct restatement of
the method of L. Ying, "Sparsifying Preconditioner for the Lippmann-Schwinger Equation"
(arXiv:1408.4495) that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it.  It shares no code with ``paper_1408_4495_gb300`` and never
imports it; inputs (media, directions) are passed in as arrays.

Every function cites the passage of the paper it follows (section / equation).  Readings
taken where the paper is silent are stated in the docstrings.

Parity status per function (what pins it, see ``tests/test_oracle_*.py``):

* ``kernel_table`` / ``green`` (t != 0): Helmholtz-equation residual of the table away
  from the origin; large-argument asymptotics.                                 pinned
* ``k0_weight``: radial quadrature of the Green's function over the equal-area disk /
  equal-volume ball (scipy.integrate), independent of the closed form.          pinned
* ``apply_K_fft``: direct O(N^2) summation of the definition (Sec. 2.1).       pinned
* ``stencil``: optimality against random unit vectors, Gram-matrix eigenvector route
  at small n, mirror/dihedral symmetry, |alpha| = 1.                            pinned
* ``assemble`` + ``Preconditioner``: m = 0 gives P = I exactly (M = [A;B]); the
  sparse LU equals a dense solve of M; ND order is a permutation whose separators
  disconnect the two halves.                                                    pinned
* ``gmres_right``: dense solve of (I + K omega^2 m) u = g at n <= 32.          pinned
* whole discrete solve: Mie series of a constant-contrast disk (2D) and ball (3D), error
  decreasing with n (``mie.py``; the series checked by their interface conditions and
  the Helmholtz equation on both sides).                                        pinned
* the sparsity claim A K ~ C (Sec. 2.2): reported ratio only, the paper prints
  no magnitude.                                                  parity unpinned
* Laplace variant (Sec. 5, ``omega = 0`` in 3D, ``point_source``, ``laplace_solve``):
  harmonicity and unit flux of 1/(4 pi r); k_0 = a^2/2 by ball quadrature and as the
  omega -> 0 limit of the Helmholtz weight; the point-source right-hand side equals the
  Green's function at the grid offsets; V = 0 gives u = g; dense solve of (I + K V) u = g;
  stencil optimality for the Laplace kernel; convergence to the radial solution of a
  delta source at the centre of a constant ball potential.                    pinned
* ``far_field`` (exterior evaluation): equals the direct exterior sum of the Green's
  function at a distant point (constant and sign), zero for m = 0, reciprocity
  u_inf(theta; d) = u_inf(-d; -theta) of the discrete solution, and convergence to the
  Mie series' far field of a constant-contrast disk (``mie.mie_disk_far_field``, itself
  checked as the limit of the Mie field).                                      pinned
* ``k0_corrected`` (higher-order weight of the singular point, Sec. 2.1): the discrete
  convolution of a smooth field converges with order ~4 (against ~2 for the ball weight),
  checked against an independent radial quadrature; independent of the fitting width. pinned
* general domains (Sec. 4: ``general_support``, ``general_sketch``, ``general_stencils``,
  ``general_assemble``, ``general_solve``): the sketch equals the direct O(N^2) sum of its
  definition, the restricted solution equals the full-grid solution on Omega, the
  support is supp(m) with its buffer, boundary stencils attain sigma_min of T(mu(i), :)
  (recomputed by the direct sum), interior rows equal the rectangular ones, iteration
  counts in the band of the Sec. 4 tables and stable under the random draw.   pinned
"""

from .ls_oracle import *  # noqa: F401,F403
