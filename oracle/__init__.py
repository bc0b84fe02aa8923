"""CPU oracle for the ghost-FEM multigrid V-cycle (TEST INFRASTRUCTURE ONLY).

A plain, slow, fp64 restatement of what the paper defines, written to check the
CUDA path against.  It is not part of the product: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it.  It shares no code with the CUDA path; the only
common module is ``paper_2505_05105_gb300.workloads`` (seeded problem
definitions, none of the method's arithmetic).

Modules
-------
``ghostfem``   Sec. 2 and Sec. 5.2: snapping, cell classes, cut geometry,
               element matrices (Eq. disc_bil_form, Eq. disc_rhs), the local
               stabilisation constant C(K) and the assembled system.
``multigrid``  Sec. 3, Sec. 4.2-4.3 and Sec. 5.1: bilinear prolongation,
               R = P^T, Galerkin coarse operators, Gauss-Seidel smoothers with
               extra cut-cell sweeps, V/W-cycles, two-grid scheme, convergence
               factor, direct solve.

Every function is pinned by a ``-m "not gpu"`` test in ``tests/`` against
something other than itself (printed values, closed forms, invariants or brute
force); see the module docstrings for which.
"""
