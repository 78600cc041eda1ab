"""Writes the stored oracle solutions of the parity tests.

Only the oracle (``oracle/``) and the seeded input generators
(``workloads/``) run here; nothing from the GPU library. Each case is a
reduced member of a benchmark family whose oracle solve takes too long to
repeat inside a test run:

* ``stokes3d_64``: the enclosed 3D Stokes cavity of the precision-form
  benchmark (seeded N(0,1) forcing, r = 0, viscosity 1, N = h^3 I,
  gamma = 100) at 64^3 cells. The oracle runs the augmented-Lagrangian
  transform (Sec. 2, Eq. (3)), Algorithm 1 and the stopping rule of Eq. (5)
  with d = 5 to tau = 1e-12, each inner solve by plain CG to a relative
  residual of 1e-13 (a sparse factorisation of M does not fit at this size:
  the fill of a 3D grid grows too fast). Plain CG on M at 64^3 takes a few
  thousand iterations per solve, so the whole solve runs for tens of minutes.

Usage: ``python tests/golden/make_oracle_solutions.py stokes3d_64``
(writes ``tests/golden/stokes3d_64_gamma100.npz`` next to this script).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import gkb as ogkb  # noqa: E402
from oracle import mac  # noqa: E402

CASES = {
    "stokes3d_64": dict(n=64, gamma=100.0, tol=1e-12, delay=5, tol_inner=1e-13,
                        out="stokes3d_64_gamma100.npz"),
}


def make(name):
    c = CASES[name]
    pr = workloads.stokes3d(c["n"])
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    ops = mac.assemble(grid, 1.0, c["gamma"])
    t0 = time.time()
    res = ogkb.solve(grid, ops, pr["g"], pr["r"], tol=c["tol"], delay=c["delay"], inner="cg",
                     tol_inner=c["tol_inner"], maxit_inner=200000)
    secs = time.time() - t0
    assert res["converged"] and res["inner_converged"], name
    path = os.path.join(HERE, c["out"])
    np.savez_compressed(path, w=res["w"], p=res["p"], n=np.array(pr["n"]), gamma=c["gamma"], tol=c["tol"],
                        tol_inner=c["tol_inner"], delay=c["delay"], outer_iterations=res["iterations"],
                        inner_iterations=np.array(res["inner_iterations"]), seconds=secs)
    print("%s: %d outer steps, %d inner CG iterations, %.0f s -> %s"
          % (name, res["iterations"], sum(res["inner_iterations"]), secs, path))


if __name__ == "__main__":
    for nm in sys.argv[1:] or list(CASES):
        make(nm)
