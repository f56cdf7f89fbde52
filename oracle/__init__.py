"""Plain FP64 CPU oracle for the shared-LHS batched banded solver.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct reference
against which the CUDA library is checked.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import or
run it.  It shares no code with the CUDA path (``paper_2107_05395_gb300``) and
neither side imports the other; the only common module is ``synth`` (seeded
random inputs, no solver arithmetic).

Contents, each function citing the passage it follows:

* ``banded``    -- tridiagonal factor/solve (section 3.1, Algorithms 1-2),
                   pentadiagonal factor/solve (section 4.1, Algorithms 3-4), and the
                   transposed (adjoint) solves with the same factors.
* ``matrices``  -- finite-difference operators and the workloads' shared matrices
                   (sections 3.2, 4.2, 5.1) with Dirichlet / hinged / truncated /
                   no-flux closures.
* ``steppers``  -- backward-Euler and Crank-Nicolson steps, the semi-implicit
                   Cahn-Hilliard step (section 5.1, no-flux and periodic), the
                   travelling-wave forced CH step (section 6.1), the coarsening
                   length (section 5.3), the convergence-study error (Table 3), the
                   FP64 reference for FP32 right-hand sides.
* ``advection`` -- the fifth-order Hamilton-Jacobi WENO derivative of the forced
                   scheme's advection term (section 6.1).
* ``rollout``   -- discrete adjoint of an implicit rollout (no paper counterpart).

Parity pins (tests/test_oracle_*.py) tie every function to something other than
itself: dense LAPACK solves, exact rational elimination, closed-form eigenmode
decay factors, conservation laws, the adjoint identity and finite differences.
"""
from . import advection, banded, matrices, rollout, steppers  # noqa: F401
