"""Plain, slow FP64 CPU oracle of the HDG implicit shallow-water solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the library (the CUDA path, its C ABI
and its Python binding) imports, links or calls anything in this package.  It
is used by ``tests/``, by ``__graft_entry__.smoke()`` (as the checker) and by
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.

What it computes, and where each piece comes from in the paper:

* ``reference``  - Lagrange bases on the reference triangle and on a facet
  (Eqs. DG_space_def, DG_trace_def); every integral is computed exactly by
  expanding products of monomials.
* ``hdg``        - facet numbering, cell geometry and the cell-local operators
  of the upwind HDG form (Eq. bilinear_HDG_upwind, the ABCM split of
  Eq. ABCMform and App. B) with the implicit Coriolis term; the monolithic
  (u, h, lambda) system; the three-step Schur-complement solve of
  Sec. 4.2 (Eqs. AFinverse, schur_system, reconstruct_solution).
* ``stddg``      - the standard (non-hybridised) upwind DG system obtained by
  eliminating the trace, used only to cross-check the HDG solution
  (the equivalence stated after Eq. linear_hybridized).
* ``imex``       - time stepping around the implicit solve (Sec. 3 "Time
  discretisation", Eqs. theta_method, IMEX_HDG_I, IMEX_HDG_II; the ARS2(2,3,2)
  tableaux of Sec. "Timestepping methods"): the theta method and a general
  IMEX Runge-Kutta stage driver (ARS2(2,3,2), SSP2(3,2,2), ARS3(4,4,3)) with
  the Coriolis term explicit, each implicit stage solved directly or by the
  HDG route (tau = alpha dt, f = 0).
* ``solver``     - right-preconditioned (F)GMRES and the non-nested two-level
  V-cycle of Alg. twolevel_vcycle: damped block-Jacobi facet smoothing,
  P1 restriction/prolongation (Sec. 4.4, upwind coarse space), and the
  coarse problem of Eq. coarse_problem_upwind solved by a geometric P1
  V-cycle or exactly.

Every function is written for clarity, not speed: per-cell Python loops,
dense local algebra and SciPy sparse matrices.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except the iteration *count* at large Courant
numbers, for which the paper gives no value ("parity unpinned" for that
number; the algorithm itself is pinned through its fixed point).
"""
