"""CPU FP64 oracle for the GKB saddle-point solver.

TEST INFRASTRUCTURE ONLY: ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers. The GPU library never imports, links or executes anything here, and
the two share no code.

* :mod:`oracle.mac` assembles the MAC-staggered blocks W, A, N and
  M = W + gamma A N^-1 A^T as sparse matrices (Sec. 2, Eq. (1)-(2)).
* :mod:`oracle.gkb` runs the augmented-Lagrangian transform (Eq. (3)),
  Algorithm 1 and the lower-bound stopping rule (Eq. (5)) with a CG or
  sparse-direct inner solver.

Pins (tests marked ``not gpu``): the Poiseuille discrete-exact solution,
dense direct solves of the full saddle system, exact termination, the error
identity and lower-bound property of Sec. 2.2, the orthogonality relations of
Eq. (4), closed-form stencil values and operator symmetries.
"""
from . import mac, gkb  # noqa: F401
