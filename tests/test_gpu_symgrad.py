"""The symmetric-gradient viscous operator -div(2 mu eps(u)) on the GPU:
operator products and whole GKB solves against the oracle, the deep-interior
fast path against the general path bit for bit, and the argument checks."""
import numpy as np
import pytest

import workloads
from oracle import gkb as ogkb
from oracle import mac

from gpu_helpers import energy_rel, gpu_solve, make_handle, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D, Nat = mac.DIRICHLET, mac.NATURAL
SYM = 1


def _mu(n, seed, sigma=1.0):
    return np.exp(sigma * np.random.default_rng(seed).standard_normal(n))


def _apply(gk, h, op, x, ny):
    import torch
    y = torch.empty(ny, dtype=torch.float64, device="cuda")
    gk.gkb_apply(h, op, torch.tensor(x, device="cuda"), y)
    return y.cpu().numpy()


@pytest.mark.parametrize("n,const_mu,prec", [((40, 24), False, 0), ((40, 24), True, 0), ((12, 10, 8), False, 0),
                                             ((40, 24), False, 1), ((12, 10, 8), True, 1)])
def test_operators_match_oracle(lib, n, const_mu, prec):
    gk = lib
    bc = (D,) * (2 * len(n))
    mu = 1.7 if const_mu else _mu(n, 1)
    grid, ops = oracle_problem(n, bc, mu, 30.0, sym=True)
    h = make_handle(gk, n, bc, mu, 30.0, precision=prec, viscous_form=SYM)
    try:
        rng = np.random.default_rng(2)
        for op, mat in ((gk.GKB_OP_W, ops["W"]), (gk.GKB_OP_M, ops["M"])):
            x = rng.standard_normal(grid.m)
            ref = mat @ x
            assert np.abs(_apply(gk, h, op, x, grid.m) - ref).max() <= 1e-13 * np.abs(ref).max()
    finally:
        gk.gkb_destroy(h)


@pytest.mark.parametrize("n", [(40, 36), (12, 12, 10)])
def test_fast_path_is_bitwise_the_general_path(lib, n):
    """kernel_variant 2 (deep-interior fast path in FP64) and 1 (general
    link-by-link rows everywhere) give identical bits for M x."""
    gk = lib
    bc = (D,) * (2 * len(n))
    mu = _mu(n, 3)
    grid = mac.MacGrid(n, 1.0 / n[0], bc)
    x = np.random.default_rng(4).standard_normal(grid.m)
    ys = []
    for variant in (1, 2):
        h = make_handle(gk, n, bc, mu, 50.0, kernel_variant=variant, viscous_form=SYM)
        try:
            ys.append(_apply(gk, h, gk.GKB_OP_M, x, grid.m))
        finally:
            gk.gkb_destroy(h)
    assert np.array_equal(ys[0], ys[1])


@pytest.mark.parametrize("prec,weighted", [(0, False), (1, False), (0, True)])
def test_solve_reaches_oracle_2d(lib, prec, weighted):
    """64 x 64 log-normal viscosity (Gaussian random field), gamma = 100,
    GMG-PCG inner solves: the 1e-8 energy bound against the oracle's tightly
    converged solution and the oracle's outer step count within one."""
    gk = lib
    n = (64, 64)
    bc = (D,) * 4
    pr = workloads.varvisc2d(64)
    mu, g = pr["mu"], pr["g"]
    r = np.zeros(64 * 64)
    nd = (1.0 / 64) ** 2 / mu if weighted else None
    grid, ops = oracle_problem(n, bc, mu, 100.0, sym=True, n_diag=nd)
    ref = oracle_truth(grid, ops, g, r)
    ref_its = ogkb.solve(grid, ops, g, r, tol=1e-8, delay=5, inner="direct")["iterations"]
    h = make_handle(gk, n, bc, mu, 100.0, precision=prec, tol_inner=1e-11, viscous_form=SYM, n_diag=nd)
    try:
        rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
        st = gk.gkb_stats(h)
    finally:
        gk.gkb_destroy(h)
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
    assert np.abs(p - ref["p"]).max() <= 1e-6 * np.abs(ref["p"]).max()
    assert abs(st["outer_iterations"] - ref_its) <= 1, (st["outer_iterations"], ref_its)


def test_solve_reaches_oracle_3d(lib):
    gk = lib
    n = (16, 16, 16)
    bc = (D,) * 6
    mu = _mu(n, 5, 0.7)
    grid, ops = oracle_problem(n, bc, mu, 100.0, sym=True)
    g = np.random.default_rng(6).standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    ref = oracle_truth(grid, ops, g, r)
    h = make_handle(gk, n, bc, mu, 100.0, tol_inner=1e-11, viscous_form=SYM)
    try:
        rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
    finally:
        gk.gkb_destroy(h)
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8


def test_recurrence_matches_oracle_step_by_step(lib):
    """Unpreconditioned CG inner solves to 1e-13 (the one-kernel cluster CG
    for this size): alpha, beta, zeta of every outer step match the oracle's
    exact-inner recurrence."""
    gk = lib
    n = (24, 20)
    bc = (D,) * 4
    mu = _mu(n, 7, 0.8)
    grid, ops = oracle_problem(n, bc, mu, 10.0, sym=True)
    rng = np.random.default_rng(8)
    g = rng.standard_normal(grid.m)
    r = rng.standard_normal(grid.n_cells)
    r -= r.mean()
    ref = ogkb.solve(grid, ops, g, r, tol=1e-8, delay=5, inner="direct")
    h = make_handle(gk, n, bc, mu, 10.0, inner=gk.GKB_INNER_CG, tol_inner=1e-13, maxit_inner=20000,
                    viscous_form=SYM)
    try:
        rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
        hist = gk.gkb_history(h)
        st = gk.gkb_stats(h)
    finally:
        gk.gkb_destroy(h)
    assert st["outer_iterations"] == ref["iterations"]
    K = len(ref["zeta"])
    assert np.allclose(hist["alpha"][:K], ref["alpha"], rtol=1e-6, atol=0)
    assert np.allclose(hist["beta"][:K], ref["beta"][:K], rtol=1e-6, atol=0)
    assert np.allclose(hist["zeta"][:K], ref["zeta"], rtol=1e-6, atol=0)
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8


def test_argument_errors(lib):
    gk = lib
    with pytest.raises(gk.GkbError):   # natural sides
        make_handle(gk, (16, 16), (D, Nat, D, D), 1.0, 10.0, inner=gk.GKB_INNER_CG, viscous_form=SYM)
    with pytest.raises(gk.GkbError):   # unknown form
        make_handle(gk, (16, 16), (D,) * 4, 1.0, 10.0, viscous_form=7)
    h = make_handle(gk, (16, 16), (D,) * 4, 1.0, 10.0, viscous_form=SYM)
    try:
        with pytest.raises(gk.GkbError):
            gk.gkb_boundary_rhs(h, 0, np.ones(16), np.zeros(gk.gkb_layout(h)[0]), np.zeros(256))
    finally:
        gk.gkb_destroy(h)
