"""Plain FP64 CPU oracle for CLAIRE's Gauss-Newton-Krylov registration path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method in arXiv 2401.17493 that the CUDA library is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import it.  It shares no
code, constants, tables or helpers with the CUDA path under
``paper_2401_17493_b300/``, and it never imports that package.

Everything is NumPy/SciPy in float64.  Each function cites the passage of the
paper it follows (section, equation label, algorithm).  Where the paper is
silent or garbled the oracle takes one reading; the readings are named in the
docstrings by their tag (C-1 ... C-15) and listed together in the design
notes of the repository.

Modules
-------
grid       nodal periodic grid, spacing, wavenumbers      (Sec. 2.5.1)
interp     periodic tricubic Lagrange interpolation        (Sec. 2.5.4)
fd8        8th-order finite-difference gradient/divergence (Sec. 2.5.3)
spectral   regulariser, preconditioner, Leray, restrict    (Sec. 2.5.3, 2.5.5, Appendix)
transport  RK2 departure points and the four SL solves     (Sec. 2.5.2, eqs. transport/adjoint/incstate/incadj)
reduced    objective, reduced gradient, Hessian matvec     (eqs. varopt-claire, rgrad, matvec)
precond    two-level zero-velocity preconditioner          (Sec. 2.5.6)
solver     PCG (Algorithm 2), Armijo, Gauss-Newton (Algorithm 1), continuation (Sec. 2.6)
defgrad    deformation-gradient transport and det F1       (Appendix, eq. def-grad)

Parity pins (tests/test_oracle_*.py) tie every module to something other than
itself: closed forms, the v = 0 special case the paper works out, textbook
library routines, brute force on tiny inputs and invariants.  The
near-incompressible weight c(kappa) of ``spectral.near_incompressible_term``
is pinned to the meaning of the Appendix's printed operator: the gradient it
gives vanishes at the minimiser of the constrained problem that operator
comes from (computed independently); which regulariser of the second control
the paper intended stays reading C-2.
"""

from . import grid, interp, fd8, spectral, transport, reduced, precond, solver, defgrad  # noqa: F401
