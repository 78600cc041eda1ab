"""The FGMRES(m) inner solver with a V-cycle as right preconditioner: GKB with
it reaches the oracle's solution, with inner-iteration counts comparable to
GMG-PCG, also when short restarts force several cycles; the device-resident
form (inside the whole-solve graph) takes the same iterations as the
host-sequenced one."""
import numpy as np
import pytest

from oracle import mac

from gpu_helpers import energy_rel, gpu_solve, make_handle, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D = mac.DIRICHLET


def _fgmres_handle(gk, n, mu, gamma, restart=30, precision=0, use_graph=1):
    import torch
    opt = gk.gkb_default_options()
    opt.inner = gk.GKB_INNER_FGMRES
    opt.precision = precision
    opt.use_graph = use_graph
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


@pytest.mark.parametrize("restart", [30, 5])
def test_device_resident_fgmres_matches_host_sequenced(lib, restart):
    """The graph form keeps the Hessenberg column, the Givens rotations, the
    back substitution and the restart test on the device; it must take the
    host loop's iterations (outer and inner, restarts included) and reach
    the same solution to rounding."""
    gk = lib
    n = (48, 40)
    mu = np.exp(0.5 * np.random.default_rng(8).standard_normal(n))
    grid, ops = oracle_problem(n, (D,) * 4, mu, 100.0)
    g = np.random.default_rng(9).standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    out = []
    for use_graph in (1, 0):
        h = _fgmres_handle(gk, n, mu, 100.0, restart, use_graph=use_graph)
        try:
            rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5)
            assert rc == gk.GKB_OK, gk.gkb_last_error(h)
            st = gk.gkb_stats(h)
            out.append((w, p, st["outer_iterations"], st["inner_iterations"], st["inner_solves"]))
        finally:
            gk.gkb_destroy(h)
    (w1, p1, o1, i1, s1), (w0, p0, o0, i0, s0) = out
    assert (o1, i1, s1) == (o0, i0, s0)
    assert energy_rel(ops["M"], w1, w0) <= 1e-12
    ref = oracle_truth(grid, ops, g, r)
    assert energy_rel(ops["M"], w1, ref["w"]) <= 1e-8
