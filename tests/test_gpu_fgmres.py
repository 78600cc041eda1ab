"""The FGMRES(m) inner solver with a V-cycle as right preconditioner: GKB with
it reaches the oracle's solution, with inner-iteration counts comparable to
GMG-PCG, also when short restarts force several cycles."""
import numpy as np
import pytest

from oracle import mac

from gpu_helpers import energy_rel, gpu_solve, make_handle, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D = mac.DIRICHLET


def _fgmres_handle(gk, n, mu, gamma, restart=30, precision=0):
    import torch
    opt = gk.gkb_default_options()
    opt.inner = gk.GKB_INNER_FGMRES
    opt.precision = precision
    opt.tol_inner = 1e-11
    opt.fgmres_restart = restart
    opt.stream = torch.cuda.current_stream().cuda_stream
    h = gk.gkb_create(opt)
    visc = None if np.isscalar(mu) else np.ascontiguousarray(np.asarray(mu, dtype=np.float64).ravel(order="F"))
    gk.gkb_set_problem(h, gk.make_grid(n, 1.0 / n[0], (D,) * (2 * len(n))), visc,
                       float(mu) if visc is None else 1.0, gamma, 0.0)
    return h


@pytest.mark.parametrize("n,var,restart", [((64, 48), 1, 30), ((14, 12, 10), 0, 30), ((40, 40), 0, 4)])
def test_gkb_with_fgmres_matches_oracle(lib, n, var, restart):
    gk = lib
    mu = np.exp(0.6 * np.random.default_rng(2).standard_normal(n)) if var else 1.0
    grid, ops = oracle_problem(n, (D,) * (2 * len(n)), mu, 100.0)
    g = np.random.default_rng(3).standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    ref = oracle_truth(grid, ops, g, r)
    h = _fgmres_handle(gk, n, mu, 100.0, restart)
    try:
        rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
        st = gk.gkb_stats(h)
    finally:
        gk.gkb_destroy(h)
    hp = make_handle(gk, n, (D,) * (2 * len(n)), mu, 100.0, tol_inner=1e-11)
    try:
        rc2, _, _ = gpu_solve(gk, hp, g, r, 1e-8, 5)
        stp = gk.gkb_stats(hp)
    finally:
        gk.gkb_destroy(hp)
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
    assert np.abs(p - ref["p"]).max() <= 1e-6 * np.abs(ref["p"]).max()
    # minimal-residual steps with the same V-cycle: about as many as PCG's
    # (short restarts lose the subspace and need more)
    assert st["inner_iterations"] <= (1.3 if restart >= 30 else 3.0) * stp["inner_iterations"]


def test_fgmres_argument_errors(lib):
    import torch
    gk = lib
    opt = gk.gkb_default_options()
    opt.inner = gk.GKB_INNER_FGMRES
    opt.fgmres_restart = 0
    with pytest.raises(gk.GkbError):
        gk.gkb_create(opt)
    with pytest.raises(gk.GkbError):  # FP64 only
        _fgmres_handle(gk, (16, 16), 1.0, 10.0, precision=1)
