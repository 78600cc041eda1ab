"""A handle stays usable after a solve that met non-finite data: the next
finite solve on the same handle reaches the oracle's answer. (Every vector
a solve reads is rewritten before it is read: the first CG direction and
the zero-coefficient updates never multiply stale values by 0.)"""
import numpy as np
import pytest

from oracle import mac

from gpu_helpers import energy_rel, gpu_solve, make_handle, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D = mac.DIRICHLET


@pytest.mark.parametrize("prec", [0, 1])
def test_handle_recovers_after_non_finite_input(lib, prec):
    gk = lib
    n, bc = (32, 32), (D,) * 4
    grid, ops = oracle_problem(n, bc, 1.0, 10.0)
    rng = np.random.default_rng(12)
    h = make_handle(gk, n, bc, 1.0, 10.0, precision=prec, maxit_inner=300)
    try:
        g = rng.standard_normal(grid.m)
        g[17] = np.nan
        try:
            gpu_solve(gk, h, g, np.zeros(grid.n_cells))
        except gk.GkbError:
            pass
        g = rng.standard_normal(grid.m)
        rc, w, p = gpu_solve(gk, h, g, np.zeros(grid.n_cells))
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
    finally:
        gk.gkb_destroy(h)
    ref = oracle_truth(grid, ops, g, np.zeros(grid.n_cells))
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
