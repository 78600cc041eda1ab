"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a closed form, a library routine (dense
LAPACK solve, sparse LU), or an identity stated in the paper (Sec. 2):
exact termination, the error identity and lower bound of Sec. 2.2, the
orthogonality relations of Eq. (4), and the equivalence of Eq. (1) and (3).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gkb, mac
import workloads

D, Nat = mac.DIRICHLET, mac.NATURAL


def dense_saddle_solve(grid, ops, g, r):
    """Full saddle system [W A; A^T 0] solved by LAPACK (numpy.linalg.solve).
    Enclosed grids get a bordering row/column fixing mean(p) = 0."""
    W, A = ops["W"].toarray(), ops["A"].toarray()
    m, n = A.shape
    if grid.enclosed:
        K = np.zeros((m + n + 1, m + n + 1))
        K[n + m, m:m + n] = 1.0
        K[m:m + n, n + m] = 1.0
        rhs = np.concatenate([g, r, [0.0]])
    else:
        K = np.zeros((m + n, m + n))
        rhs = np.concatenate([g, r])
    K[:m, :m] = W
    K[:m, m:m + n] = A
    K[m:m + n, :m] = A.T
    sol = np.linalg.solve(K, rhs)
    return sol[:m], sol[m:m + n]


def m_norm(M, x):
    return math.sqrt(float(x @ (M @ x)))


# ---------------------------------------------------------------------------
# Discretisation pins
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_poiseuille_discrete_exact(n):
    """Sec. 4.1 Poiseuille flow (u = 4y(1-y), linear pressure) on the unit
    square: with inflow 4y(1-y)+h^2 the MAC solution is exactly u = 4y(1-y)+h^2,
    v = 0, p = 8(1-x) at cell centres (the mirror-wall rows see the parabola's
    constant second difference). LAPACK dense solve, round-off agreement."""
    wl = workloads.poiseuille(n, shifted=True, guess=False)
    grid = mac.MacGrid(wl["n"], wl["h"], wl["bc"])
    ops = mac.assemble(grid, 1.0, 0.0)
    g, r = mac.dirichlet_rhs(grid, ops, {0: wl["inflow"]})
    w, p = dense_saddle_solve(grid, ops, g, r)
    X, Y = grid.face_centres(0)
    h = grid.h
    w_ex = grid.join_velocity([4 * Y * (1 - Y) + h * h, np.zeros(grid.face_shape(1))])
    xc = grid.cell_centres()[0]
    p_ex = (8.0 * (1.0 - xc)).ravel(order="F")
    assert np.abs(w - w_ex).max() < 1e-12
    assert np.abs(p - p_ex).max() < 1e-11


@pytest.mark.parametrize("dim", [2, 3])
def test_viscous_operator_closed_form(dim):
    """W u = -h^d div(mu grad u) holds exactly for quadratic u and linear mu
    (central differences of a quadratic flux are exact), on faces whose
    stencil does not reach a wall. Pins both normal links (cell mu) and
    tangential links (node/edge mean of cell mu)."""
    n = (6, 7, 5)[:dim]
    h = 0.1
    grid = mac.MacGrid(n, h)
    xc = grid.cell_centres()
    for c in range(dim):
        for a in range(dim):
            mu = 1.0 + 0.3 * xc[a]
            ops = mac.assemble(grid, mu, 0.0)
            X = grid.face_centres(c)
            comps = [np.zeros(grid.face_shape(b)) for b in range(dim)]
            comps[c] = X[a] ** 2
            w = grid.join_velocity(comps)
            Wu = grid.split_velocity(ops["W"] @ w)[c]
            expect = -(h ** dim) * (2.0 * (1.0 + 0.3 * X[a]) + 0.3 * 2.0 * X[a])
            # interior: two cells away from every wall along every axis
            sl = tuple(slice(2, s - 2) for s in grid.face_shape(c))
            assert np.allclose(Wu[sl], expect[sl], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_divergence_closed_form(dim):
    """(A p)_f = h^(d-1)(p_plus - p_minus): for linear p this is h^d dp/dx_c.
    A^T is minus the integrated divergence: for w = (a x, b y[, c z]) every
    interior cell gets -h^d (a + b [+ c])."""
    n = (5, 6, 4)[:dim]
    h = 0.25
    grid = mac.MacGrid(n, h)
    ops = mac.assemble(grid, 1.0, 0.0)
    coef = np.array([0.7, -1.3, 2.1])[:dim]
    xc = grid.cell_centres()
    p = sum(coef[a] * xc[a] for a in range(dim)).ravel(order="F")
    Ap = grid.split_velocity(ops["A"] @ p)
    for c in range(dim):
        lo, hi = grid.active_range(c)
        sl = [slice(None)] * dim
        sl[c] = slice(lo, hi + 1)
        assert np.allclose(Ap[c][tuple(sl)], h ** dim * coef[c], rtol=1e-12)
    comps = [grid.face_centres(c)[c] * coef[c] for c in range(dim)]
    # the wall faces are not unknowns; only check cells away from walls
    divw = (ops["A"].T @ grid.join_velocity(comps)).reshape(n, order="F")
    inner = tuple(slice(1, s - 1) for s in n)
    assert np.allclose(divw[inner], -(h ** dim) * coef.sum(), rtol=1e-12)


@pytest.mark.parametrize("bc", [(D, D, D, D), (D, Nat, D, D), (D, D, D, D, D, D)])
def test_operator_structure(bc):
    """W and M symmetric positive definite, A has the constant pressure in its
    kernel exactly when every side is Dirichlet (Eq. (1) with SPD M, Eq. (2))."""
    dim = len(bc) // 2
    n = (5, 4, 3)[:dim]
    grid = mac.MacGrid(n, 1.0 / 5, bc)
    rng = np.random.default_rng(0)
    mu = np.exp(rng.standard_normal(n))
    ops = mac.assemble(grid, mu, 10.0)
    for key in ("W", "M"):
        Mx = ops[key].toarray()
        assert np.abs(Mx - Mx.T).max() < 1e-14
        assert np.linalg.eigvalsh(Mx).min() > 0
    one = np.ones(grid.n_cells)
    if grid.enclosed:
        assert np.abs(ops["A"] @ one).max() < 1e-14
    else:
        assert np.abs(ops["A"] @ one).max() > 1e-3
    M2 = ops["W"] + (10.0 / ops["n_scale"]) * (ops["A"] @ ops["A"].T)
    assert abs(M2 - ops["M"]).max() < 1e-12


def test_compact_ordering_counts():
    """The unknown counts match the input generator's layout counting."""
    for n, bc in (((32, 32), (D, Nat, D, D)), ((9, 7), (D,) * 4), ((4, 5, 6), (D,) * 6)):
        grid = mac.MacGrid(n, 0.1, bc)
        assert grid.m == workloads.velocity_size(n, bc)
    assert mac.MacGrid((32, 32), 1 / 32, (D, Nat, D, D)).m == 2016


# ---------------------------------------------------------------------------
# GKB pins (Sec. 2)
# ---------------------------------------------------------------------------

def _small_problem(n, bc, gamma, seed=0, varmu=False):
    grid = mac.MacGrid(n, 1.0 / n[0], bc)
    rng = np.random.default_rng(seed)
    mu = np.exp(0.5 * rng.standard_normal(n)) if varmu else 1.0
    ops = mac.assemble(grid, mu, gamma)
    g = rng.standard_normal(grid.m)
    r = rng.standard_normal(grid.n_cells)
    if grid.enclosed:
        r -= r.mean()
    return grid, ops, g, r


@pytest.mark.parametrize("n,bc,gamma,varmu", [
    ((6, 6), (D, Nat, D, D), 10.0, False),
    ((6, 5), (D, D, D, D), 0.0, True),
    ((5, 5), (D, D, D, D), 100.0, False),
    ((3, 4, 3), (D,) * 6, 5.0, True),
])
def test_gkb_matches_dense_solve(n, bc, gamma, varmu):
    """GKB with an exact inner solver reproduces LAPACK's solution of the full
    saddle system (Eq. (1)) once the estimator is below 1e-13."""
    grid, ops, g, r = _small_problem(n, bc, gamma, varmu=varmu)
    w_ex, p_ex = dense_saddle_solve(grid, ops, g, r)
    if grid.enclosed:
        p_ex -= p_ex.mean()
    res = gkb.solve(grid, ops, g, r, tol=1e-13, delay=3, inner="direct")
    assert res["converged"]
    M = ops["M"]
    assert m_norm(M, res["w"] - w_ex) <= 1e-10 * m_norm(M, w_ex)
    assert np.abs(res["p"] - p_ex).max() <= 1e-8 * np.abs(p_ex).max()


@pytest.mark.parametrize("bc", [(D, Nat, D, D), (D, D, D, D)])
def test_exact_termination_error_identity_and_lower_bound(bc):
    """Sec. 2.2: ||u - u_k||_M^2 = sum_{j>k} zeta_j^2 (error identity), hence
    xi_{k,d}^2 = sum_{j=k+1}^{k+d+1} zeta_j^2 is a lower bound; after at most
    n steps the iterate is exact. Exact inner solves, no early stop."""
    grid, ops, g, r = _small_problem((5, 5), bc, 10.0, seed=3)
    M, A = ops["M"], ops["A"]
    solver = gkb.InnerSolver(M, "direct")
    y, b = gkb.al_transform(A, ops["n_scale"], g, r, 10.0, solver)
    w_ex, _ = dense_saddle_solve(grid, ops, g, r)
    u_ex = w_ex - y
    nsteps = grid.n_cells - (1 if grid.enclosed else 0)
    res = gkb.gkb(M, A, ops["n_scale"], b, solver, tol=0.0, delay=2,
                  maxit=nsteps - 1, enclosed=grid.enclosed, keep_bases=True)
    zeta = np.array(res["zeta"])
    V = res["V"]
    K = len(zeta)
    assert m_norm(M, res["u"] - u_ex) <= 1e-9 * m_norm(M, u_ex)
    uk = np.zeros(grid.m)
    unorm2 = m_norm(M, u_ex) ** 2
    for k in range(1, K):
        uk = uk + zeta[k - 1] * V[k - 1]
        err2 = m_norm(M, u_ex - uk) ** 2
        tail = float(np.sum(zeta[k:] ** 2))
        assert abs(err2 - tail) <= 1e-8 * unorm2
        for dly in (0, 1, 3):
            xi2 = float(np.sum(zeta[k:k + dly + 1] ** 2))
            assert xi2 <= err2 * (1 + 1e-8) + 1e-14 * unorm2
    assert abs(float(np.sum(zeta ** 2)) - unorm2) <= 1e-9 * unorm2


def test_generalized_gk_relations():
    """Eq. (4): V^T M V = I, Q^T N Q = I, A q_j = alpha_j M v_j + beta_j M v_{j-1}
    and A^T v_j = N (alpha_j q_j + beta_{j+1} q_{j+1}) for the first steps."""
    grid, ops, g, r = _small_problem((8, 8), (D, Nat, D, D), 1.0, seed=5, varmu=True)
    M, A, c = ops["M"], ops["A"], ops["n_scale"]
    solver = gkb.InnerSolver(M, "direct")
    y, b = gkb.al_transform(A, c, g, r, 1.0, solver)
    res = gkb.gkb(M, A, c, b, solver, tol=0.0, delay=2, maxit=9, keep_bases=True)
    V = np.array(res["V"]).T
    Q = np.array(res["Q"]).T
    k = V.shape[1]
    assert np.abs(V.T @ (M @ V) - np.eye(k)).max() < 1e-9
    assert np.abs(c * Q.T @ Q - np.eye(k)).max() < 1e-9
    al, be = res["alpha"], res["beta"]
    for j in range(k):
        lhs = A @ Q[:, j]
        rhs = al[j] * (M @ V[:, j]) + (be[j] * (M @ V[:, j - 1]) if j > 0 else 0.0)
        assert np.abs(lhs - rhs).max() <= 1e-9 * np.abs(lhs).max()
    for j in range(k - 1):
        lhs = A.T @ V[:, j]
        rhs = c * (al[j] * Q[:, j] + be[j + 1] * Q[:, j + 1])
        assert np.abs(lhs - rhs).max() <= 1e-9 * np.abs(lhs).max()


def test_augmented_lagrangian_invariance():
    """Eq. (1) and its transformed form Eq. (3) have the same solution for any
    gamma: gamma = 0 (W SPD, all sides Dirichlet) and gamma = 100 agree."""
    grid, ops0, g, r = _small_problem((8, 8), (D, D, D, D), 0.0, seed=7)
    ops1 = mac.assemble(grid, 1.0, 100.0)
    a = gkb.solve(grid, ops0, g, r, tol=1e-12, delay=4, inner="direct")
    b = gkb.solve(grid, ops1, g, r, tol=1e-12, delay=4, inner="direct")
    M = ops1["M"]
    assert m_norm(M, a["w"] - b["w"]) <= 1e-9 * m_norm(M, a["w"])
    assert np.abs(a["p"] - b["p"]).max() <= 1e-7 * np.abs(a["p"]).max()
    # the augmented form needs fewer outer steps (Sec. 2, Tables 2 and 6)
    assert b["iterations"] < a["iterations"]


def test_cg_matches_sparse_lu():
    """The oracle's CG reaches SuperLU's solution of M x = f to its tolerance."""
    grid, ops, g, r = _small_problem((12, 12), (D, D, D, D), 10.0, seed=9)
    M = ops["M"]
    x, it, ok = gkb.cg(M, g, 1e-12, 10000)
    assert ok and it > 5
    x_ref = sp.linalg.spsolve(M.tocsc(), g)
    assert m_norm(M, x - x_ref) <= 1e-10 * m_norm(M, x_ref)


def test_initial_guess_defect_correction_and_stop_quality():
    """Reading for a seeded initial guess: defect correction gives the same
    solution; the returned iterate's true relative energy error is within a
    small factor of tau."""
    wl = workloads.poiseuille(16, shifted=True, guess=True)
    grid = mac.MacGrid(wl["n"], wl["h"], wl["bc"])
    ops = mac.assemble(grid, 1.0, 100.0)
    g, r = mac.dirichlet_rhs(grid, ops, {0: wl["inflow"]})
    w_ex, p_ex = dense_saddle_solve(grid, ops, g, r)
    M = ops["M"]
    for w0, p0 in ((None, None), (wl["w0"], wl["p0"])):
        res = gkb.solve(grid, ops, g, r, tol=1e-8, delay=5, inner="cg",
                        tol_inner=1e-12, w0=w0, p0=p0)
        assert res["converged"]
        rel = m_norm(M, res["w"] - w_ex) / m_norm(M, w_ex)
        assert rel <= 1e-8
        assert np.abs(res["p"] - p_ex).max() <= 1e-6


def test_poiseuille_gkb_config():
    """32 x 32 Poiseuille channel, gamma = 100, N = h^2 I, d = 5, tau = 1e-8,
    inner CG 1e-12, seeded initial guess: GKB reaches the discrete-exact
    solution within 1e-8 relative energy norm."""
    wl = workloads.poiseuille(32, shifted=True, guess=True)
    grid = mac.MacGrid(wl["n"], wl["h"], wl["bc"])
    ops = mac.assemble(grid, 1.0, 100.0)
    g, r = mac.dirichlet_rhs(grid, ops, {0: wl["inflow"]})
    res = gkb.solve(grid, ops, g, r, tol=1e-8, delay=5, inner="cg",
                    tol_inner=1e-12, w0=wl["w0"], p0=wl["p0"])
    X, Y = grid.face_centres(0)
    h = grid.h
    w_ex = grid.join_velocity([4 * Y * (1 - Y) + h * h, np.zeros(grid.face_shape(1))])
    M = ops["M"]
    assert m_norm(M, res["w"] - w_ex) <= 1e-8 * m_norm(M, w_ex)


def test_estimate_is_iterate_difference():
    """Sec. 2.2: with V M-orthonormal, xi_{k,d}^2 = sum_{j=k+1}^{k+d+1} zeta_j^2
    equals ||u_{k+d+1} - u_k||_M^2 and sum_{j<=K} zeta_j^2 = ||u_K||_M^2. So the
    estimate reported after step K must equal ||u_K - u_{K-d-1}||_M / ||u_K||_M,
    computed here from iterates returned by separate truncated runs."""
    grid, ops, g, r = _small_problem((7, 7), (D, Nat, D, D), 3.0, seed=11)
    M, A, c = ops["M"], ops["A"], ops["n_scale"]
    solver = gkb.InnerSolver(M, "direct")
    y, b = gkb.al_transform(A, c, g, r, 3.0, solver)
    delay = 2
    full = gkb.gkb(M, A, c, b, solver, tol=0.0, delay=delay, maxit=12)
    iterates = [np.zeros(grid.m)]
    for it in range(0, 13):
        iterates.append(gkb.gkb(M, A, c, b, solver, tol=0.0, delay=delay, maxit=it)["u"])
    # iterates[K] = u_K (K zetas known); estimate[i] is reported with K = i + 2
    for i, est in enumerate(full["estimate"]):
        K = i + 2
        k = max(K - delay - 1, 0)
        ref = m_norm(M, iterates[K] - iterates[k]) / m_norm(M, iterates[K])
        assert abs(est - ref) <= 1e-9 * max(ref, 1e-6)
