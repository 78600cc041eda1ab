"""Robustness of the inner solver in gamma: the vertex-patch (2D) /
edge-patch (3D) smoother contains the discrete curls, the kernel of the
grad-div term, so PCG iterations per inner solve stay bounded as gamma grows
while the GKB outer steps fall (Sec. 2: larger gamma clusters the
generalized singular values; Tables 2 and 6). Every solve is checked against
the saddle-point equations the oracle assembles."""
import numpy as np
import pytest

import workloads
from oracle import mac

from gpu_helpers import gpu_solve, make_handle

pytestmark = pytest.mark.gpu

GAMMAS = [1e2, 1e3, 1e4, 1e5, 1e6]


def _sweep(gk, pr, precision=0):
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    ops = mac.assemble(grid, pr["mu"], 0.0)
    rows = []
    for gam in GAMMAS:
        h = make_handle(gk, pr["n"], pr["bc"], pr["mu"], gam, precision=precision, tol_inner=1e-10)
        try:
            rc, w, p = gpu_solve(gk, h, pr["g"], pr["r"], 1e-8, 5)
            assert rc == gk.GKB_OK, gk.gkb_last_error(h)
            st = gk.gkb_stats(h)
        finally:
            gk.gkb_destroy(h)
        r1 = pr["g"] - ops["W"] @ w - ops["A"] @ p
        r2 = pr["r"] - ops["A"].T @ w
        rel = float(np.sqrt(r1 @ r1 + r2 @ r2) / np.linalg.norm(pr["g"]))
        rows.append((gam, st["outer_iterations"], st["inner_iterations"] / st["inner_solves"], rel))
    print(rows)
    return rows


def _check(rows, per_solve_max):
    per = [r[2] for r in rows]
    outer = [r[1] for r in rows]
    assert max(per) <= per_solve_max, rows
    assert max(per) <= 1.35 * min(per), rows            # flat in gamma over four decades
    assert all(b <= a for a, b in zip(outer, outer[1:])), rows
    assert outer[-1] <= 8, rows
    # the inner tolerance 1e-10 relative to M = W + gamma A N^-1 A^T bounds
    # the saddle residual by about gamma * 1e-10
    for gam, _, _, rel in rows:
        assert rel <= max(1e-8, 2e-14 * gam), rows


def test_cavity2d_gamma_robust(lib):
    _check(_sweep(lib, workloads.stokes2d(256)), 26)


def test_varvisc2d_gamma_robust(lib):
    _check(_sweep(lib, workloads.varvisc2d(256)), 30)


def test_cavity3d_gamma_robust(lib):
    _check(_sweep(lib, workloads.stokes3d(32)), 48)
