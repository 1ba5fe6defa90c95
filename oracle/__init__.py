"""FP64 CPU oracle for the exponential-Krylov Maxwell solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
links this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library (no kernels, headers, helpers or
tables); the only common module is ``scenario``, which draws the seeded
inputs and holds none of the method's arithmetic.

Contents (each function cites the passage of Botchev, Hanse & Uppu,
arXiv:1707.00023 it follows):

* ``yee``      -- the semi-discrete operator A of eq. (ode), its assembled
                  sparse matrix, the energy weights and the output plane.
* ``krylov``   -- the Arnoldi process (eqs. (Arn), (Arn1)), the projected
                  problem (eq. (corr2)), Lemma 1's residual (eq. (resid)) and
                  shifted Hessenberg solves.
* ``exact``    -- the exact solution y(T) of eq. (ode) with v = 0 by two
                  routes: the augmented homogeneous system and the
                  asymptotic splitting of eq. (split1); the stationary part
                  z_stat = (A + i Omega I)^{-1} g.
* ``restart``  -- residual-based restarting in Krylov dimension with one
                  basis per restart for every frequency (Sect. 3.4,
                  eq. (rst), Corollary 2, Fig. alg:rst).
* ``periodic`` -- the two uses of the source's periodicity (Sect. 3.5):
                  source splitting, eq. (split2), and the neighbouring-
                  frequency difference, eq. (4diff) in Fig. alg:spl1.
* ``pml``      -- the paper's 2D model with the perfectly matched layer
                  (auxiliary field P, eq. (mxw); block form of eq. (ode)).
* ``adjoint``  -- gradient of the output-plane intensity with respect to
                  per-cell permittivity (no counterpart in the paper).

All floating point is float64.  Library routines used as steps:
``scipy.linalg.expm`` (dense Pade scaling and squaring),
``scipy.sparse.linalg.expm_multiply`` (Al-Mohy & Higham 2011),
``scipy.sparse.linalg.spsolve`` (sparse LU) and ``numpy.linalg.solve``.
"""
