"""Parity at the default benchmark's full size (1024 x 1024 cavity, the launch
configuration bench.py times): every operator product against the oracle's
sparse matrices, element by element, and the GKB solutions against the
saddle-point equations the oracle assembles."""
import numpy as np
import pytest

import workloads
from oracle import mac

from gpu_helpers import gpu_solve, make_handle

pytestmark = pytest.mark.gpu

D = mac.DIRICHLET


@pytest.fixture(scope="module")
def cavity():
    pr = workloads.stokes2d(1024)
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    return pr, grid


def test_operators_match_oracle_at_full_size(lib, cavity):
    import torch
    gk = lib
    pr, grid = cavity
    ops = mac.assemble(grid, 1.0, 1000.0)
    h = make_handle(gk, pr["n"], pr["bc"], 1.0, 1000.0)
    try:
        rng = np.random.default_rng(31)
        xv = rng.standard_normal(grid.m)
        xc = rng.standard_normal(grid.n_cells)
        xc -= xc.mean()
        cases = [(gk.GKB_OP_W, ops["W"], xv, grid.m), (gk.GKB_OP_M, ops["M"], xv, grid.m),
                 (gk.GKB_OP_A, ops["A"], xc, grid.m), (gk.GKB_OP_AT, ops["A"].T.tocsr(), xv, grid.n_cells)]
        for op, mat, x, ny in cases:
            y = torch.empty(ny, dtype=torch.float64, device="cuda")
            gk.gkb_apply(h, op, torch.tensor(x, device="cuda"), y)
            ref = mat @ x
            err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
            assert err <= 1e-13, (op, err)
    finally:
        gk.gkb_destroy(h)


@pytest.mark.parametrize("gamma", [10.0, 1000.0])
def test_solution_at_full_size_satisfies_the_saddle_system(lib, cavity, gamma):
    """FP64 GMG-PCG, tau = 1e-8, d = 5, tau_in = 1e-10 (the default bench
    form): the relative residual of [W A; A^T 0][w; p] = [g; r] from the
    oracle's matrices stays at the inner solves' level (1e-10 relative
    residual each; the oracle's direct-solver GKB reaches ~1e-12), the
    discrete divergence vanishes to round-off and the pressure is mean-free."""
    gk = lib
    pr, grid = cavity
    ops = mac.assemble(grid, 1.0, gamma)
    h = make_handle(gk, pr["n"], pr["bc"], 1.0, gamma, tol_inner=1e-10)
    try:
        rc, w, p = gpu_solve(gk, h, pr["g"], pr["r"], 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
        st = gk.gkb_stats(h)
    finally:
        gk.gkb_destroy(h)
    g = pr["g"]
    r1 = g - ops["W"] @ w - ops["A"] @ p
    r2 = pr["r"] - ops["A"].T @ w
    rel = np.sqrt(r1 @ r1 + r2 @ r2) / np.linalg.norm(g)
    assert rel <= 1e-7, rel
    assert np.linalg.norm(r2) <= 1e-7 * np.linalg.norm(g)
    assert abs(p.mean()) <= 1e-12 * np.abs(p).max()
    assert 1 <= st["outer_iterations"] < 100 and st["estimate"] <= 1e-8
