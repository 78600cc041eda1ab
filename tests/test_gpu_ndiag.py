"""Diagonal N (Sec. 3: any symmetric positive definite N): the augmented
operator, the GKB recurrence in the N inner product and whole solves against
the oracle, for the viscosity-weighted pressure mass matrix h^d / mu and for
arbitrary positive diagonals."""
import numpy as np
import pytest

import workloads
from oracle import gkb as ogkb
from oracle import mac

from gpu_helpers import energy_rel, gpu_solve, make_handle

pytestmark = pytest.mark.gpu

D, Nat = mac.DIRICHLET, mac.NATURAL


def _case(n, bc, seed, sigma=1.0, visc_weighted=True, const_mu=False):
    grid = mac.MacGrid(n, 1.0 / n[0], bc)
    rng = np.random.default_rng(seed)
    mu = 1.0 if const_mu else np.exp(sigma * rng.standard_normal(grid.n))
    if visc_weighted and not const_mu:
        nd = grid.h ** grid.dim / mu
    else:
        nd = grid.h ** grid.dim * np.exp(0.7 * rng.standard_normal(grid.n))
    return grid, mu, nd, rng


@pytest.mark.parametrize("n,bc,const_mu,prec", [((40, 24), (D,) * 4, False, 0), ((40, 24), (D,) * 4, True, 0),
                                               ((24, 16), (D, Nat, D, D), False, 0), ((12, 10, 8), (D,) * 6, False, 0),
                                               ((40, 24), (D,) * 4, False, 1)])
def test_augmented_operator_matches_oracle(lib, n, bc, const_mu, prec):
    """y = M x with M = W + gamma A diag(n)^-1 A^T, element by element."""
    import torch
    gk = lib
    grid, mu, nd, rng = _case(n, bc, 1, const_mu=const_mu, visc_weighted=False)
    ops = mac.assemble(grid, mu, 30.0, n_diag=nd)
    inner = gk.GKB_INNER_GMG_PCG if grid.enclosed else gk.GKB_INNER_CG
    h = make_handle(gk, n, bc, mu, 30.0, precision=prec, inner=inner, n_diag=nd)
    try:
        for _ in range(2):
            x = rng.standard_normal(grid.m)
            y = torch.empty(grid.m, dtype=torch.float64, device="cuda")
            gk.gkb_apply(h, gk.GKB_OP_M, torch.tensor(x, device="cuda"), y)
            ref = ops["M"] @ x
            assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    finally:
        gk.gkb_destroy(h)


@pytest.mark.parametrize("bc", [(D,) * 4, (D, Nat, D, D)])
def test_recurrence_matches_oracle_step_by_step(lib, bc):
    """alpha_k, beta_k, zeta_k and the estimates of Algorithm 1 with
    N = h^2 / mu agree with the oracle's (exact inner solves there, inner
    tolerance 1e-13 here); same number of outer steps."""
    gk = lib
    n = (32, 32)
    grid, mu, nd, rng = _case(n, bc, 2, sigma=1.5)
    ops = mac.assemble(grid, mu, 1.0, n_diag=nd)
    g = rng.standard_normal(grid.m)
    r = rng.standard_normal(grid.n_cells)
    if grid.enclosed:
        r -= r.mean()
    ref = ogkb.solve(grid, ops, g, r, tol=1e-8, delay=5, inner="direct")
    inner = gk.GKB_INNER_GMG_PCG if grid.enclosed else gk.GKB_INNER_CG
    h = make_handle(gk, n, bc, mu, 1.0, inner=inner, tol_inner=1e-13, maxit_inner=20000, n_diag=nd)
    try:
        rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
        hist = gk.gkb_history(h)
        st = gk.gkb_stats(h)
    finally:
        gk.gkb_destroy(h)
    assert st["outer_iterations"] == ref["iterations"]
    K = len(ref["zeta"])
    assert np.allclose(hist["beta"][:K], ref["beta"][:K], rtol=1e-6, atol=0)
    assert np.allclose(hist["alpha"][:K], ref["alpha"], rtol=1e-6, atol=0)
    assert np.allclose(hist["zeta"][:K], ref["zeta"], rtol=1e-6, atol=0)
    assert np.allclose(hist["estimate"], ref["estimate"], rtol=1e-4, atol=1e-14)
    M = ops["M"]
    assert energy_rel(M, w, ref["w"]) <= 1e-8
    assert np.abs(p - ref["p"]).max() <= 1e-6 * np.abs(ref["p"]).max()


@pytest.mark.parametrize("n,prec", [((64, 64), 0), ((64, 64), 1), ((16, 16, 16), 0)])
def test_viscosity_weighted_solve_reaches_oracle(lib, n, prec):
    """GMG-PCG inner solves (FP64 or mixed) with N = h^d / mu and with
    N = h^d I: the 1e-8 energy bound against the oracle's tightly converged
    answer and the oracle's outer step count (within one). On the smooth
    log-normal field (2D) the weighted N needs less than half the steps; on
    a cell-by-cell random field (3D) it is not better, so only parity is
    asserted there."""
    gk = lib
    bc = (D,) * len(n) * 2
    grid = mac.MacGrid(n, 1.0 / n[0], bc)
    if len(n) == 2:
        mu = workloads.varvisc2d(n[0], sigma=1.5)["mu"]
    else:
        mu = np.exp(np.random.default_rng(3).standard_normal(n))
    nd = grid.h ** grid.dim / mu
    rng = np.random.default_rng(9)
    g = rng.standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    its = []
    for weights in (nd, None):
        ops = mac.assemble(grid, mu, 1.0, n_diag=weights)
        ref = ogkb.solve(grid, ops, g, r, tol=1e-13, delay=5, inner="direct")
        ref_its = ogkb.solve(grid, ops, g, r, tol=1e-8, delay=5, inner="direct")["iterations"]
        h = make_handle(gk, n, bc, mu, 1.0, precision=prec, tol_inner=1e-11, n_diag=weights)
        try:
            rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5)
            assert rc == gk.GKB_OK, gk.gkb_last_error(h)
            its.append(gk.gkb_stats(h)["outer_iterations"])
        finally:
            gk.gkb_destroy(h)
        assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
        assert abs(its[-1] - ref_its) <= 1, (its[-1], ref_its)
    if len(n) == 2:
        assert its[0] < 0.5 * its[1], its


def test_uniform_diagonal_equals_scalar_N(lib):
    """n_diag = h^2 everywhere solves the same problem as N = h^2 I."""
    gk = lib
    n = (48, 40)
    grid, mu, _, rng = _case(n, (D,) * 4, 4)
    g = rng.standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    out = []
    for nd in (np.full(n, grid.h ** 2), None):
        h = make_handle(gk, n, (D,) * 4, mu, 10.0, tol_inner=1e-12, n_diag=nd)
        try:
            rc, w, p = gpu_solve(gk, h, g, r, 1e-10, 5)
            assert rc == gk.GKB_OK
            out.append((w, p, gk.gkb_stats(h)["outer_iterations"]))
        finally:
            gk.gkb_destroy(h)
    M = mac.assemble(grid, mu, 10.0)["M"]
    assert out[0][2] == out[1][2]
    assert energy_rel(M, out[0][0], out[1][0]) <= 1e-10


def test_batched_and_preconditioned_forms_take_diagonal_N(lib):
    """The batched graph and GKB-as-preconditioner run the same recurrence."""
    gk = lib
    n = (32, 32)
    grid, mu, nd, rng = _case(n, (D,) * 4, 5)
    g = rng.standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    ops = mac.assemble(grid, mu, 10.0, n_diag=nd)
    ref = ogkb.solve(grid, ops, g, r, tol=1e-13, delay=5, inner="direct")
    hs = [make_handle(gk, n, (D,) * 4, mu, 10.0, tol_inner=1e-11, n_diag=nd) for _ in range(2)]
    try:
        ws = [np.empty(grid.m) for _ in hs]
        ps = [np.empty(grid.n_cells) for _ in hs]
        rc = gk.gkb_solve_batched(hs, [g, g], [r, r], 1e-8, 5, ws, ps)
        assert rc == gk.GKB_OK
        for w in ws:
            assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
        w2, p2 = np.empty(grid.m), np.empty(grid.n_cells)
        rc, its = gk.gkb_solve_preconditioned(hs[0], g, r, 1e-10, w2, p2, pc_tol=1e-2)
        assert rc == gk.GKB_OK and its <= 15
        assert energy_rel(ops["M"], w2, ref["w"]) <= 1e-8
    finally:
        for h in hs:
            gk.gkb_destroy(h)


def test_bad_diagonal_is_rejected(lib):
    gk = lib
    n = (16, 16)
    nd = np.full(n, 1.0 / 256)
    nd[3, 4] = 0.0
    with pytest.raises(gk.GkbError):
        make_handle(gk, n, (D,) * 4, 1.0, 10.0, n_diag=nd)
    nd[3, 4] = np.nan
    with pytest.raises(gk.GkbError):
        make_handle(gk, n, (D,) * 4, 1.0, 10.0, n_diag=nd)
