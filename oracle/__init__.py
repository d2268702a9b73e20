"""Plain, slow, FP64 CPU oracle for the lumped pressure-Helmholtz multigrid solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (``paper_1605_00492_gb300``): it has its own mesh generator,
its own assembly, its own tridiagonal solver, V-cycle and Krylov loops.

What it computes (Mitchell & Mueller, "High level implementation of
geometric multigrid solvers for finite element problems: applications in
atmospheric modelling"):

* ``mesh``      icosahedral sphere meshes refined by edge bisection, the
                nested hierarchy of Sec. 3.1 and the column geometry of the
                radially extruded shell (Sec. 4.1).
* ``helmholtz`` the lumped Helmholtz operator H^ of Eq. (Preconditioner),
                built literally as M3 + w_c^2 (D_h Mh^-1 D_h^T +
                (1+w_N^2)^-1 D_z Mz^-1 D_z^T) from sparse D and diagonal M,
                and its column block H^_z of Eq. (HHgeneralbanded).
* ``multigrid`` the block-Jacobi line smoother of Sec. 4.2.1 / Sec. 5.4,
                DG0 restriction / prolongation of Sec. 3.2 and the recursive
                correction-scheme V-cycle of Algorithm 1.
* ``krylov``    preconditioned CG (and flexible CG) on H^ p = b.
* ``nlo``       the next-to-lowest-order (BDFM1 x DG1 / DG1 x DG1) lumped
                operator, its column block solve, the p-coarsening DG1 ->
                DG0 and its V-cycle over the lowest-order hierarchy.
* ``nlo_mixed`` the next-to-lowest-order velocity-pressure system (full
                BDFM1 x DG1 and DG1 x P2 velocity masses) and its
                Schur-complement preconditioner with the NLO V-cycle.
* ``adjoint``   the gradient of a least-squares loss of the solution with
                respect to the right-hand side and a per-cell coefficient of
                the vertical coupling.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, quadrature, invariants, dense linear algebra or
brute force on small meshes.  The only printed values of the paper that
apply are the grid counts of Table "Grid setup" (tests/golden/).
"""
