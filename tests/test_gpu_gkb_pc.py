"""GKB as a preconditioner: FGMRES on the saddle system [W A; A^T 0] with the
GKB solve (to a loose tolerance) as preconditioner reaches the saddle
residual it is asked for and the oracle's solution."""
import numpy as np
import pytest

import workloads
from oracle import mac

from gpu_helpers import energy_rel, make_handle, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D = mac.DIRICHLET


def _saddle_residual(ops, g, r, w, p):
    r1 = g - ops["W"] @ w - ops["A"] @ p
    r2 = r - ops["A"].T @ w
    return np.sqrt(r1 @ r1 + r2 @ r2) / np.sqrt(g @ g + r @ r)


@pytest.mark.parametrize("pc_tol,max_its", [(1e-2, 15), (1e-10, 2)])
def test_fgmres_with_gkb_preconditioner_enclosed(lib, pc_tol, max_its):
    gk = lib
    n = (48, 40)
    mu = np.exp(0.6 * np.random.default_rng(12).standard_normal(n))
    grid, ops = oracle_problem(n, (D,) * 4, mu, 100.0)
    g = np.random.default_rng(13).standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    ref = oracle_truth(grid, ops, g, r)
    h = make_handle(gk, n, (D,) * 4, mu, 100.0, tol_inner=1e-11)
    try:
        w, p = np.empty(grid.m), np.empty(grid.n_cells)
        rc, its = gk.gkb_solve_preconditioned(h, g, r, 1e-10, w, p, restart=20, maxit=100, pc_tol=pc_tol)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
    finally:
        gk.gkb_destroy(h)
    assert 1 <= its <= max_its
    assert _saddle_residual(ops, g, r, w, p) <= 2e-10
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
    assert abs(p.mean()) <= 1e-12 * np.abs(p).max()


def test_fgmres_with_gkb_preconditioner_channel(lib):
    """Poiseuille channel with natural outflow (plain CG inner solves)."""
    gk = lib
    pr = workloads.poiseuille(32, shifted=True, guess=False)
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    ops = mac.assemble(grid, 1.0, 100.0)
    g, r = mac.dirichlet_rhs(grid, ops, {0: pr["inflow"]})
    ref = oracle_truth(grid, ops, g, r)
    h = make_handle(gk, pr["n"], pr["bc"], 1.0, 100.0, inner=gk.GKB_INNER_CG, tol_inner=1e-12, maxit_inner=20000)
    try:
        w, p = np.empty(grid.m), np.empty(grid.n_cells)
        rc, its = gk.gkb_solve_preconditioned(h, g, r, 1e-11, w, p, restart=10, maxit=50, pc_tol=1e-3)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
    finally:
        gk.gkb_destroy(h)
    assert its <= 10
    assert _saddle_residual(ops, g, r, w, p) <= 2e-11
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
    assert np.abs(p - ref["p"]).max() <= 1e-7 * np.abs(ref["p"]).max()


def test_outer_solver_reports_non_convergence(lib):
    gk = lib
    n = (24, 24)
    grid, ops = oracle_problem(n, (D,) * 4, 1.0, 10.0)
    g = np.random.default_rng(14).standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    h = make_handle(gk, n, (D,) * 4, 1.0, 10.0)
    try:
        w, p = np.empty(grid.m), np.empty(grid.n_cells)
        rc, its = gk.gkb_solve_preconditioned(h, g, r, 1e-14, w, p, restart=2, maxit=1, pc_tol=0.5)
        assert rc == gk.GKB_ERR_NOT_CONVERGED and its == 1
        with pytest.raises(gk.GkbError):
            gk.gkb_solve_preconditioned(h, g, r, 1e-8, w, p, restart=0)
    finally:
        gk.gkb_destroy(h)
