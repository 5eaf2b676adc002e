"""FP64 CPU oracle for the velocity fixed-point iteration (V-FPI) of
Lee, Lee & Lee, "Large-Dimensional Multibody Dynamics Simulation Using Contact
Nodalization and Diagonalization" (arXiv 2201.09212).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the test suite, the smoke check of the build entry
point and the CPU-baseline leg of the benchmark use it.  It shares no code with
the CUDA library (no kernels, headers, helpers or tables); the two meet only in
the seeded input generators, which hold none of the method's arithmetic.

Modules
-------
vfpi       Alg. 1 + Alg. 2 written out step by step (eqs. pgd1, subp, vup,
           operator, diagonal), the choice of W (Sec. IV.C), residual and stop
           test, FP64 position update.
delassus   Projected Gauss-Seidel on the dense Delassus operator (eq. delassus),
           the paper's I-FPI baseline (Sec. V.C) -- an independent solver.
enumerate  Brute-force active-set enumeration for 1-3 contacts: every
           open/stick/slip assignment of the Signorini-Coulomb conditions
           (eq. scc) solved directly.
checks     Dynamics residual (eq. lindyn), Signorini-Coulomb residual (eq. scc),
           open/stick/slip classification.
adjoint    Dense implicit-function adjoint of the converged fixed point
           (the map f(v) of Sec. IV) at a frozen active set.

Every function is pinned by the CPU tests against closed forms, invariants,
brute force or hand-worked values (the residual checkers against contacts
built to break exactly one condition of eq. (scc) each, with the violation
worked out by hand), and planted mistakes in each are caught by those pins.
Functions without such a pin say "parity unpinned" in their docstring; at
present there are none.  Trajectories over many time steps are compared step
by step only: their stick/slip switches make long rollouts sensitive to
rounding, so no rollout-level pin exists.
"""
