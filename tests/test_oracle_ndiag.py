"""Pins of the oracle with a diagonal N (Sec. 3: N may be any symmetric
positive definite matrix), against a cell-by-cell divergence, a dense LAPACK
solve of the saddle system (whose solution does not depend on N), the
relations of Eq. (4) in the N inner product and the error identity of
Sec. 2.2."""
import math

import numpy as np
import pytest

from oracle import gkb, mac
import workloads

from test_oracle_pins import dense_saddle_solve, m_norm

D, Nat = mac.DIRICHLET, mac.NATURAL


def _problem(n, bc, gamma, seed, visc_weighted=True):
    grid = mac.MacGrid(n, 1.0 / n[0], bc)
    rng = np.random.default_rng(seed)
    mu = np.exp(0.8 * rng.standard_normal(grid.n))
    if visc_weighted:
        nd = grid.h ** grid.dim / mu
    else:
        nd = grid.h ** grid.dim * np.exp(0.5 * rng.standard_normal(grid.n))
    ops = mac.assemble(grid, mu, gamma, n_diag=nd)
    g = rng.standard_normal(grid.m)
    r = rng.standard_normal(grid.n_cells)
    if grid.enclosed:
        r -= r.mean()
    return grid, ops, nd, g, r


def _cell_divergence(grid, x):
    """Integrated divergence of the face field x in every cell, cell by cell
    from the face index tables (h^(d-1) times the sum of outgoing fluxes)."""
    comps = grid.split_velocity(x)
    out = np.zeros(grid.n)
    for cell in np.ndindex(*grid.n):
        s = 0.0
        for c in range(grid.dim):
            hi = list(cell)
            hi[c] += 1
            s += comps[c][tuple(hi)] - comps[c][cell]
        out[cell] = s * grid.h ** (grid.dim - 1)
    return out


@pytest.mark.parametrize("n,bc", [((5, 4), (D, D, D, D)), ((4, 3), (D, Nat, D, D)), ((3, 3, 4), (D,) * 6)])
def test_augmented_block_is_the_weighted_divergence_energy(n, bc):
    """x^T M x = x^T W x + gamma sum_c (div x)_c^2 / N_c for the diagonal N,
    with the divergence summed face by face in each cell."""
    grid, ops, nd, _, _ = _problem(n, bc, 7.0, seed=1, visc_weighted=False)
    rng = np.random.default_rng(2)
    for _ in range(3):
        x = rng.standard_normal(grid.m)
        div = _cell_divergence(grid, x)
        ref = float(x @ (ops["W"] @ x)) + 7.0 * float(np.sum(div ** 2 / nd))
        assert abs(float(x @ (ops["M"] @ x)) - ref) <= 1e-12 * abs(ref)


def test_uniform_diagonal_is_the_scalar_case():
    """n_diag = c (constant) reproduces N = c I: the same M to rounding and
    the same GKB iterates."""
    grid = mac.MacGrid((8, 6), 1.0 / 8)
    rng = np.random.default_rng(3)
    mu = np.exp(rng.standard_normal(grid.n))
    c = 0.37 * grid.h ** 2
    a = mac.assemble(grid, mu, 5.0, n_scale=c)
    b = mac.assemble(grid, mu, 5.0, n_diag=np.full(grid.n, c))
    assert abs(a["M"] - b["M"]).max() <= 1e-13 * abs(a["M"]).max()
    g = rng.standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    ra = gkb.solve(grid, a, g, r, tol=1e-10, delay=3, inner="direct")
    rb = gkb.solve(grid, b, g, r, tol=1e-10, delay=3, inner="direct")
    assert ra["iterations"] == rb["iterations"]
    assert np.allclose(ra["zeta"], rb["zeta"], rtol=1e-9, atol=0)
    assert np.abs(ra["w"] - rb["w"]).max() <= 1e-11 * np.abs(ra["w"]).max()


@pytest.mark.parametrize("bc,visc", [((D, D, D, D), True), ((D, Nat, D, D), True), ((D, D, D, D), False)])
def test_solution_does_not_depend_on_N(bc, visc):
    """Eq. (1) does not contain N: GKB with a diagonal N and gamma > 0 reaches
    the dense LAPACK solution of [W A; A^T 0]."""
    grid, ops, _, g, r = _problem((8, 8), bc, 10.0, seed=4, visc_weighted=visc)
    res = gkb.solve(grid, ops, g, r, tol=1e-12, delay=4, inner="direct")
    w_ex, p_ex = dense_saddle_solve(grid, ops, g, r)
    assert res["converged"]
    assert m_norm(ops["M"], res["w"] - w_ex) <= 1e-9 * m_norm(ops["M"], w_ex)
    assert np.abs(res["p"] - p_ex).max() <= 1e-8 * np.abs(p_ex).max()


@pytest.mark.parametrize("bc", [(D, D, D, D), (D, Nat, D, D)])
def test_generalized_gk_relations_in_the_N_inner_product(bc):
    """Eq. (4) with N = diag(n): V^T M V = I, Q^T N Q = I,
    A q_j = alpha_j M v_j + beta_j M v_{j-1},
    A^T v_j = N (alpha_j q_j + beta_{j+1} q_{j+1})."""
    grid, ops, nd, g, r = _problem((8, 8), bc, 1.0, seed=5)
    M, A, N = ops["M"], ops["A"], ops["N"]
    solver = gkb.InnerSolver(M, "direct")
    y, b = gkb.al_transform(A, N, g, r, 1.0, solver)
    res = gkb.gkb(M, A, N, b, solver, tol=0.0, delay=2, maxit=9, enclosed=grid.enclosed, keep_bases=True)
    V = np.array(res["V"]).T
    Q = np.array(res["Q"]).T
    k = V.shape[1]
    assert np.abs(V.T @ (M @ V) - np.eye(k)).max() < 1e-9
    assert np.abs(Q.T @ (N[:, None] * Q) - np.eye(k)).max() < 1e-9
    al, be = res["alpha"], res["beta"]
    for j in range(k):
        lhs = A @ Q[:, j]
        rhs = al[j] * (M @ V[:, j]) + (be[j] * (M @ V[:, j - 1]) if j > 0 else 0.0)
        assert np.abs(lhs - rhs).max() <= 1e-9 * np.abs(lhs).max()
    for j in range(k - 1):
        lhs = A.T @ V[:, j]
        rhs = N * (al[j] * Q[:, j] + be[j + 1] * Q[:, j + 1])
        assert np.abs(lhs - rhs).max() <= 1e-9 * np.abs(lhs).max()
    if grid.enclosed:
        # the N-step vectors are N-orthogonal to the constants
        assert np.abs(N @ Q).max() <= 1e-12 * np.abs(N[:, None] * Q).sum(axis=0).max()


def test_error_identity_with_diagonal_N():
    """Sec. 2.2: ||u - u_k||_M^2 = sum_{j>k} zeta_j^2 with exact inner solves,
    run to exact termination (at most n - 1 steps for an enclosed box)."""
    grid, ops, _, g, r = _problem((5, 5), (D, D, D, D), 3.0, seed=6)
    M, A, N = ops["M"], ops["A"], ops["N"]
    solver = gkb.InnerSolver(M, "direct")
    y, b = gkb.al_transform(A, N, g, r, 3.0, solver)
    w_ex, _ = dense_saddle_solve(grid, ops, g, r)
    u_ex = w_ex - y
    res = gkb.gkb(M, A, N, b, solver, tol=0.0, delay=2, maxit=grid.n_cells - 2, enclosed=True, keep_bases=True)
    zeta = np.array(res["zeta"])
    unorm2 = m_norm(M, u_ex) ** 2
    assert abs(float(np.sum(zeta ** 2)) - unorm2) <= 1e-9 * unorm2
    uk = np.zeros(grid.m)
    for k in range(1, len(zeta)):
        uk = uk + zeta[k - 1] * res["V"][k - 1]
        assert abs(m_norm(M, u_ex - uk) ** 2 - float(np.sum(zeta[k:] ** 2))) <= 1e-8 * unorm2


def test_viscosity_weighted_N_cuts_outer_iterations():
    """With a strongly varying viscosity, N = h^d / mu approximates the Schur
    complement A^T W^-1 A far better than h^d I, so GKB needs fewer steps (the
    spread of the generalized singular values shrinks)."""
    pr = workloads.varvisc2d(32, sigma=2.0)
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    its = []
    for nd in (None, grid.h ** 2 / pr["mu"]):
        ops = mac.assemble(grid, pr["mu"], 1.0, n_diag=nd)
        its.append(gkb.solve(grid, ops, pr["g"], pr["r"], tol=1e-8, delay=5, inner="direct")["iterations"])
    assert its[1] < 0.6 * its[0], its
