"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: operators agree with the oracle's CSR products to 1e-12 of the
largest entry (FP64, only the summation order differs); solved velocities
agree with a tightly converged oracle solution within relative energy-norm
error 1e-8 (the stated bound for FP64 and for the mixed form, whose inner
solves are refined in FP64 to the same tolerance); pressures within 1e-6 of
their largest entry.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import gkb as ogkb
from oracle import mac

from gpu_helpers import energy_rel, gpu_solve, make_handle, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D, Nat = mac.DIRICHLET, mac.NATURAL
FP64, MIXED = 0, 1
CG, GMG = 0, 1


def _mu(kind, n, seed=0):
    if kind == "const":
        return 1.0
    rng = np.random.default_rng(seed)
    return np.exp(0.7 * rng.standard_normal(n))


@pytest.mark.parametrize("n,bc,mukind,gamma", [
    ((33, 20), (D, D, D, D), "const", 10.0),
    ((40, 37), (D, Nat, D, D), "var", 5.0),
    ((9, 11, 7), (D,) * 6, "var", 3.0),
    ((16, 16, 16), (D,) * 6, "const", 0.0),
    ((35, 6), (Nat, D, D, Nat), "var", 2.0),
    # 3D levels of at least 16 cells per axis take the box / shell operator
    # kernel: odd sizes with the grad-div coupling, and a natural side
    ((18, 16, 17), (D,) * 6, "const", 50.0),
    ((16, 20, 24), (D, Nat, D, D, D, D), "const", 7.0),
])
def test_operators_match_oracle(lib, n, bc, mukind, gamma):
    gk = lib
    mu = _mu(mukind, n)
    grid, ops = oracle_problem(n, bc, mu, gamma)
    h = make_handle(gk, n, bc, mu, gamma, inner=CG)
    try:
        m, nc = gk.gkb_layout(h)
        assert (m, nc) == (grid.m, grid.n_cells)
        rng = np.random.default_rng(1)
        xv = rng.standard_normal(m)
        xp = rng.standard_normal(nc)
        for op, key, xin in ((gk.GKB_OP_W, "W", xv), (gk.GKB_OP_M, "M", xv)):
            y = np.empty(m)
            gk.gkb_apply(h, op, xin, y)
            ref = ops[key] @ xin
            assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max(), key
        y = np.empty(m)
        gk.gkb_apply(h, gk.GKB_OP_A, xp, y)
        ref = ops["A"] @ xp
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
        y = np.empty(nc)
        gk.gkb_apply(h, gk.GKB_OP_AT, xv, y)
        ref = ops["A"].T @ xv
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        gk.gkb_destroy(h)


def test_boundary_rhs_matches_oracle(lib):
    gk = lib
    wl = workloads.poiseuille(32, shifted=True, guess=False)
    grid, ops = oracle_problem(wl["n"], wl["bc"], 1.0, 100.0)
    g_ref, r_ref = mac.dirichlet_rhs(grid, ops, {0: wl["inflow"]})
    h = make_handle(gk, wl["n"], wl["bc"], 1.0, 100.0, inner=CG)
    try:
        g = np.zeros(grid.m)
        r = np.zeros(grid.n_cells)
        gk.gkb_boundary_rhs(h, 0, wl["inflow"], g, r)
        assert np.abs(g - g_ref).max() <= 1e-14
        assert np.abs(r - r_ref).max() <= 1e-14
    finally:
        gk.gkb_destroy(h)
    # 3D, a random normal velocity on the y-high side, variable viscosity
    n = (6, 5, 4)
    mu = _mu("var", n, 3)
    grid, ops = oracle_problem(n, (D,) * 6, mu, 1.0)
    ub = np.random.default_rng(2).standard_normal((6, 4))  # [x, z] of the y-side
    g_ref, r_ref = mac.dirichlet_rhs(grid, ops, {3: ub})
    h = make_handle(gk, n, (D,) * 6, mu, 1.0, inner=CG)
    try:
        g = np.zeros(grid.m)
        r = np.zeros(grid.n_cells)
        gk.gkb_boundary_rhs(h, 3, np.ascontiguousarray(ub.ravel(order="F")), g, r)
        assert np.abs(g - g_ref).max() <= 1e-13
        assert np.abs(r - r_ref).max() <= 1e-13
    finally:
        gk.gkb_destroy(h)


@pytest.mark.parametrize("n,mukind,gamma,prec,variant", [
    ((64, 64), "const", 10.0, FP64, 0),
    ((48, 40), "var", 100.0, FP64, 0),
    ((16, 16, 16), "const", 5.0, FP64, 0),
    ((64, 64), "const", 1000.0, MIXED, 0),
    # the 3D box / shell smoother and operator (levels of at least 16 cells)
    ((18, 16, 20), "const", 50.0, MIXED, 0),
    ((20, 18, 16), "const", 30.0, FP64, 2),
])
def test_vcycle_is_symmetric_positive(lib, n, mukind, gamma, prec, variant):
    """PCG needs an SPD preconditioner: <B x, y> = <x, B y>, <B x, x> > 0."""
    gk = lib
    bc = (D,) * (2 * len(n))
    h = make_handle(gk, n, bc, _mu(mukind, n), gamma, precision=prec, kernel_variant=variant)
    try:
        m, _ = gk.gkb_layout(h)
        rng = np.random.default_rng(4)
        x, y = rng.standard_normal(m), rng.standard_normal(m)
        bx, by = np.empty(m), np.empty(m)
        gk.gkb_precond(h, x, bx)
        gk.gkb_precond(h, y, by)
        tol = 1e-12 if prec == FP64 else 2e-5
        assert abs(bx @ y - x @ by) <= tol * math.sqrt((bx @ bx) * (y @ y))
        assert bx @ x > 0 and by @ y > 0
    finally:
        gk.gkb_destroy(h)


def test_poiseuille_channel_32(lib):
    """32 x 32 Poiseuille channel: FP64, gamma = 100, N = h^2 I, d = 5,
    tau = 1e-8, inner CG to 1e-12, seeded random initial guess. The GPU
    recurrence matches the oracle step by step and both reach the
    discrete-exact parabola within 1e-8 relative energy norm."""
    gk = lib
    wl = workloads.poiseuille(32, shifted=True, guess=True)
    grid, ops = oracle_problem(wl["n"], wl["bc"], 1.0, 100.0)
    g, r = mac.dirichlet_rhs(grid, ops, {0: wl["inflow"]})
    ref = ogkb.solve(grid, ops, g, r, tol=1e-8, delay=5, inner="cg", tol_inner=1e-12,
                     w0=wl["w0"], p0=wl["p0"])
    h = make_handle(gk, wl["n"], wl["bc"], 1.0, 100.0, inner=CG, tol_inner=1e-12, maxit_inner=20000)
    try:
        gg = np.zeros(grid.m)
        rr = np.zeros(grid.n_cells)
        gk.gkb_boundary_rhs(h, 0, wl["inflow"], gg, rr)
        rc, w, p = gpu_solve(gk, h, gg, rr, 1e-8, 5, wl["w0"], wl["p0"])
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
        hist = gk.gkb_history(h)
        st = gk.gkb_stats(h)
    finally:
        gk.gkb_destroy(h)
    assert st["outer_iterations"] == ref["iterations"]
    K = len(ref["zeta"])
    assert np.allclose(hist["zeta"][:K], ref["zeta"], rtol=1e-6, atol=0)
    assert np.allclose(hist["alpha"][:K], ref["alpha"], rtol=1e-6, atol=0)
    assert np.allclose(hist["beta"][:K], ref["beta"][:K], rtol=1e-6, atol=0)
    assert np.allclose(hist["estimate"], ref["estimate"], rtol=1e-4, atol=1e-14)
    X, Y = grid.face_centres(0)
    hh = grid.h
    w_ex = grid.join_velocity([4 * Y * (1 - Y) + hh * hh, np.zeros(grid.face_shape(1))])
    M = ops["M"]
    assert energy_rel(M, w, w_ex) <= 1e-8
    assert energy_rel(M, w, ref["w"]) <= 1e-8
    p_ex = (8.0 * (1.0 - grid.cell_centres()[0])).ravel(order="F")
    assert np.abs(p - p_ex).max() <= 1e-6


def test_poiseuille_literal_inflow_parity(lib):
    """Literal inflow 4y(1-y): no closed form; GPU against the oracle."""
    gk = lib
    wl = workloads.poiseuille(32, shifted=False, guess=False)
    grid, ops = oracle_problem(wl["n"], wl["bc"], 1.0, 100.0)
    g, r = mac.dirichlet_rhs(grid, ops, {0: wl["inflow"]})
    ref = oracle_truth(grid, ops, g, r)
    h = make_handle(gk, wl["n"], wl["bc"], 1.0, 100.0, inner=CG, tol_inner=1e-12, maxit_inner=20000)
    try:
        rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5, device=False)
        assert rc == gk.GKB_OK
    finally:
        gk.gkb_destroy(h)
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
    assert np.abs(p - ref["p"]).max() <= 1e-6 * np.abs(ref["p"]).max()


CASES = [
    ((80, 80), "const", 10.0),
    ((80, 80), "const", 1000.0),
    ((96, 64), "var", 100.0),
    ((64, 64), "grf", 100.0),
    ((16, 16, 16), "const", 100.0),
    ((24, 16, 20), "var", 10.0),
    ((16, 16, 48), "const", 100.0),
]


def _case_mu(kind, n):
    if kind == "grf":
        return workloads.varvisc2d(n[0], seed_offset=4)["mu"]
    return _mu(kind, n, 7)


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("n,mukind,gamma", CASES)
def test_enclosed_stokes_gmg_matches_oracle(lib, n, mukind, gamma, prec):
    """Enclosed cavity, g ~ N(0,1), r = 0, GMG-PCG inner solves, tau = 1e-8:
    relative energy-norm error <= 1e-8 against the oracle's tightly converged
    solution (ragged tiles: 80 and 20 are not multiples of the 32 x 8 tile)."""
    gk = lib
    bc = (D,) * (2 * len(n))
    mu = _case_mu(mukind, n)
    grid, ops = oracle_problem(n, bc, mu, gamma)
    gvec = np.random.default_rng(11).standard_normal(grid.m)
    rvec = np.zeros(grid.n_cells)
    ref = oracle_truth(grid, ops, gvec, rvec)
    h = make_handle(gk, n, bc, mu, gamma, precision=prec, tol_inner=1e-11)
    try:
        rc, w, p = gpu_solve(gk, h, gvec, rvec, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
        st = gk.gkb_stats(h)
    finally:
        gk.gkb_destroy(h)
    assert st["outer_iterations"] >= 1
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
    assert abs(p.mean()) <= 1e-12 * max(1.0, np.abs(p).max())
    assert np.abs(p - ref["p"]).max() <= 1e-6 * np.abs(ref["p"]).max()


def test_host_and_device_buffers_agree_and_solves_are_deterministic(lib):
    gk = lib
    n, bc = (48, 48), (D,) * 4
    grid, ops = oracle_problem(n, bc, 1.0, 10.0)
    gvec = np.random.default_rng(3).standard_normal(grid.m)
    rvec = np.zeros(grid.n_cells)
    h = make_handle(gk, n, bc, 1.0, 10.0)
    try:
        rc1, w1, p1 = gpu_solve(gk, h, gvec, rvec, device=True)
        rc2, w2, p2 = gpu_solve(gk, h, gvec, rvec, device=False)
        rc3, w3, p3 = gpu_solve(gk, h, gvec, rvec, device=True)
    finally:
        gk.gkb_destroy(h)
    assert rc1 == rc2 == rc3 == gk.GKB_OK
    assert np.array_equal(w1, w2) and np.array_equal(p1, p2)
    assert np.array_equal(w1, w3) and np.array_equal(p1, p3)


def test_edge_cases(lib):
    gk = lib
    n, bc = (32, 32), (D,) * 4
    grid, ops = oracle_problem(n, bc, 1.0, 10.0)
    h = make_handle(gk, n, bc, 1.0, 10.0, maxit=2)
    try:
        # zero right-hand side: zero solution, no iterations
        rc, w, p = gpu_solve(gk, h, np.zeros(grid.m), np.zeros(grid.n_cells))
        assert rc == gk.GKB_OK and not w.any() and not p.any()
        assert gk.gkb_stats(h)["outer_iterations"] == 0
        # maxit exhausted
        gvec = np.random.default_rng(5).standard_normal(grid.m)
        rc, w, p = gpu_solve(gk, h, gvec, np.zeros(grid.n_cells))
        assert rc == gk.GKB_ERR_NOT_CONVERGED
        assert gk.gkb_stats(h)["outer_iterations"] == 2
        # argument errors
        with pytest.raises(gk.GkbError) as ei:
            gpu_solve(gk, h, gvec, np.zeros(grid.n_cells), 1e-8, 99)
        assert ei.value.code == gk.GKB_ERR_INVALID_ARG
        with pytest.raises(gk.GkbError):
            gk.gkb_apply(h, 17, gvec, np.empty(grid.m))
    finally:
        gk.gkb_destroy(h)
    # the multigrid needs Dirichlet sides
    with pytest.raises(gk.GkbError) as ei:
        make_handle(gk, (16, 16), (D, Nat, D, D), 1.0, 1.0, inner=GMG)
    assert ei.value.code == gk.GKB_ERR_INVALID_ARG


@pytest.mark.parametrize("n", [(21, 21), (30, 18)])
def test_sizes_that_do_not_coarsen_far(lib, n):
    """Odd sizes stop the coarsening early (direct solve on a small level)."""
    gk = lib
    bc = (D,) * 4
    grid, ops = oracle_problem(n, bc, 1.0, 50.0)
    gvec = np.random.default_rng(8).standard_normal(grid.m)
    ref = oracle_truth(grid, ops, gvec, np.zeros(grid.n_cells))
    h = make_handle(gk, n, bc, 1.0, 50.0)
    try:
        rc, w, p = gpu_solve(gk, h, gvec, np.zeros(grid.n_cells))
        assert rc == gk.GKB_OK
    finally:
        gk.gkb_destroy(h)
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_graph_and_host_loops_agree_bitwise(lib, prec):
    """The graph form (device-side while loop) launches the same kernels in
    the same order as the host-sequenced loop: identical bits, identical
    iteration counts."""
    gk = lib
    n, bc = (64, 48), (D,) * 4
    grid, ops = oracle_problem(n, bc, 1.0, 100.0)
    gvec = np.random.default_rng(13).standard_normal(grid.m)
    out = []
    for use_graph in (1, 0):
        h = make_handle(gk, n, bc, 1.0, 100.0, precision=prec, use_graph=use_graph)
        try:
            rc, w, p = gpu_solve(gk, h, gvec, np.zeros(grid.n_cells))
            st = gk.gkb_stats(h)
            out.append((rc, w, p, st["outer_iterations"], st["inner_iterations"], st["kernel_launches"]))
        finally:
            gk.gkb_destroy(h)
    (rc1, w1, p1, o1, i1, l1), (rc2, w2, p2, o2, i2, l2) = out
    assert rc1 == rc2 == gk.GKB_OK
    assert (o1, i1) == (o2, i2)
    assert np.array_equal(w1, w2) and np.array_equal(p1, p2)
    # the graph form counts its launches from the captured body times the
    # loop executions: at least as many as the host loop (one extra
    # preconditioner application after convergence per inner solve)
    assert sum(l1.values()) >= sum(l2.values()) > 0


@pytest.mark.parametrize("n,prec,var", [((64, 48), FP64, 0), ((70, 66), MIXED, 0), ((14, 12, 10), FP64, 0),
                                        ((12, 14, 16), MIXED, 0), ((64, 48), FP64, 1), ((70, 66), MIXED, 1),
                                        ((14, 12, 10), MIXED, 1), ((40, 36, 64), MIXED, 0), ((24, 20, 48), FP64, 0)])
def test_fast_paths_match_general_paths_bitwise(lib, n, prec, var):
    """The deep-interior fast paths of the operator and smoother kernels must
    reproduce the general paths bit for bit: one V-cycle and one operator
    product with kernel_variant 2 (fast paths everywhere) and 1 (none), for
    constant and variable viscosity. Exception: with constant viscosity the
    smoother's fast path folds the patches through a face into one stencil
    per position class (13 points in 3D, 7 in 2D), which sums the same terms
    in another order, so the V-cycle agrees to rounding; the operator
    products stay bit for bit."""
    gk = lib
    bc = (D,) * (2 * len(n))
    mu = np.exp(0.7 * np.random.default_rng(5).standard_normal(n)) if var else 1.0
    outs = []
    for variant in (2, 1):
        h = make_handle(gk, n, bc, mu, 50.0, precision=prec, kernel_variant=variant)
        try:
            m, _ = gk.gkb_layout(h)
            x = np.random.default_rng(21).standard_normal(m)
            z, y = np.empty(m), np.empty(m)
            gk.gkb_precond(h, x, z)
            gk.gkb_apply(h, gk.GKB_OP_M, x, y)
            outs.append((z, y))
        finally:
            gk.gkb_destroy(h)
    if not var:
        tol = 1e-12 if prec == FP64 else 1e-5
        assert np.abs(outs[0][0] - outs[1][0]).max() <= tol * np.abs(outs[1][0]).max()
    else:
        assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_profiled_solve_reports_the_finest_level(lib):
    """A profiled solve times every launch; per kernel class it also reports
    the launches at the class's largest work per launch, which for the
    stencil classes is the finest level (work = its velocity unknowns)."""
    gk = lib
    n, bc = (64, 48), (D,) * 4
    grid, _ = oracle_problem(n, bc, 1.0, 100.0)
    h = make_handle(gk, n, bc, 1.0, 100.0, profile=1, use_graph=0)
    try:
        m, _ = gk.gkb_layout(h)
        gvec = np.random.default_rng(17).standard_normal(grid.m)
        rc, _, _ = gpu_solve(gk, h, gvec, np.zeros(grid.n_cells))
        assert rc == gk.GKB_OK
        st = gk.gkb_stats(h)
        for k in ("residual", "smooth"):
            assert st["kernel_top_units"][k] == m, k
            assert 0 < st["kernel_top_launches"][k] < st["kernel_launches"][k], k
            assert 0 < st["kernel_top_ms"][k] <= st["kernel_ms"][k], k
    finally:
        gk.gkb_destroy(h)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_non_finite_inputs_return_a_status(lib, prec):
    """A NaN in g or an Inf in r ends the solve with a status (the norm and
    reduction finalisers test every scalar for finiteness), not a hang or a
    silent result."""
    gk = lib
    n, bc = (32, 32), (D,) * 4
    grid, ops = oracle_problem(n, bc, 1.0, 10.0)
    rng = np.random.default_rng(12)
    for bad in ("g", "r"):
        h = make_handle(gk, n, bc, 1.0, 10.0, precision=prec, maxit_inner=300)
        try:
            g = rng.standard_normal(grid.m)
            r = np.zeros(grid.n_cells)
            if bad == "g":
                g[17] = np.nan
            else:
                r[40] = np.inf
            try:
                rc, _, _ = gpu_solve(gk, h, g, r)
            except gk.GkbError as e:
                rc = e.code
            assert rc in (gk.GKB_ERR_NAN, gk.GKB_ERR_INNER_NOT_CONVERGED), rc
        finally:
            gk.gkb_destroy(h)
