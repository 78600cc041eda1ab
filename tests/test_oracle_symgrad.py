"""Pins of the oracle's symmetric-gradient viscous operator -div(2 mu eps(u)),
the variable-viscosity Stokes operator in its stress form (the method only
needs W symmetric positive definite, Sec. 2): an exact identity for
constant viscosity, rigid rotations carry no stress, second-order agreement
with the continuous operator on a manufactured field, and GKB on it reaching
the dense LAPACK solution."""
import numpy as np
import pytest
import sympy

from oracle import gkb, mac

from test_oracle_pins import dense_saddle_solve, m_norm

D = mac.DIRICHLET


@pytest.mark.parametrize("n", [(6, 5), (4, 3, 5)])
def test_constant_viscosity_is_laplacian_plus_grad_div(n):
    """For constant mu, div(grad u^T) = grad(div u), and on the MAC grid with
    no-slip walls exactly: W_sym = W + mu A A^T / h^d."""
    grid = mac.MacGrid(n, 1.0 / n[0])
    a = mac.assemble(grid, 2.5, 0.0)
    b = mac.assemble(grid, 2.5, 0.0, sym=True)
    diff = b["W"] - a["W"] - 2.5 * (a["A"] @ a["A"].T) / grid.h ** grid.dim
    assert abs(diff).max() <= 1e-14 * abs(b["W"]).max()


def _away_from_walls(grid, c, k=2):
    """Face positions of component c whose stencil stays k cells off the walls."""
    X = np.indices(grid.face_shape(c))
    ok = np.ones(grid.face_shape(c), bool)
    for a in range(grid.dim):
        hi = grid.n[a] if a == c else grid.n[a] - 1
        ok &= (X[a] >= k) & (X[a] <= hi - k)
    return grid.face_index[c][ok]


@pytest.mark.parametrize("n", [(10, 9), (7, 6, 8)])
def test_rigid_rotation_carries_no_stress(n):
    """eps(u) = 0 for a rigid rotation, so -div(2 mu eps(u)) vanishes for any
    viscosity at the rows that do not reach the walls; the Laplacian form
    -div(mu grad u) does not vanish there when mu varies."""
    grid = mac.MacGrid(n, 1.0 / n[0])
    mu = np.exp(np.random.default_rng(0).standard_normal(grid.n))
    sym = mac.assemble(grid, mu, 0.0, sym=True)["W"]
    lap = mac.assemble(grid, mu, 0.0)["W"]
    rots = []
    if grid.dim == 2:
        X = grid.face_centres(0)
        Y = grid.face_centres(1)
        rots.append(grid.join_velocity([-X[1], Y[0]]))            # (-y, x)
    else:
        F = [grid.face_centres(c) for c in range(3)]
        rots.append(grid.join_velocity([-F[0][1], F[1][0], np.zeros(grid.face_shape(2))]))   # about z
        rots.append(grid.join_velocity([np.zeros(grid.face_shape(0)), -F[1][2], F[2][1]]))   # about x
    rows = np.concatenate([_away_from_walls(grid, c) for c in range(grid.dim)])
    assert rows.size > 0
    for u in rots:
        ys = (sym @ u)[rows]
        yl = (lap @ u)[rows]
        assert np.abs(ys).max() <= 1e-13 * abs(sym).max()
        assert np.abs(yl).max() >= 1e-3 * abs(lap).max() * grid.h


def _manufactured():
    x, y = sympy.symbols("x y")
    mu = 1 + sympy.Rational(1, 2) * sympy.sin(2 * x + 1) * sympy.cos(3 * y)
    u = sympy.sin(3 * x) * sympy.cos(2 * y + 1)
    v = sympy.cos(x + 2) * sympy.sin(y) * sympy.exp(x)
    exx, eyy = sympy.diff(u, x), sympy.diff(v, y)
    exy = (sympy.diff(u, y) + sympy.diff(v, x)) / 2
    fx = -(sympy.diff(2 * mu * exx, x) + sympy.diff(2 * mu * exy, y))
    fy = -(sympy.diff(2 * mu * exy, x) + sympy.diff(2 * mu * eyy, y))
    f = lambda e: sympy.lambdify((x, y), e, "numpy")
    return f(mu), f(u), f(v), f(fx), f(fy)


def test_second_order_against_the_continuous_operator():
    """Interior rows of W_sym / h^2 approach -div(2 mu eps(u)) at the face
    centres with second order (manufactured smooth mu, u, v; cell viscosity
    sampled at cell centres)."""
    mu_f, u_f, v_f, fx, fy = _manufactured()
    errs = []
    for n in (16, 32, 64):
        grid = mac.MacGrid((n, n), 1.0 / n)
        C = grid.cell_centres()
        W = mac.assemble(grid, mu_f(C[0], C[1]), 0.0, sym=True)["W"]
        X, Y = grid.face_centres(0), grid.face_centres(1)
        w = grid.join_velocity([u_f(X[0], X[1]), v_f(Y[0], Y[1])])
        ref = grid.join_velocity([fx(X[0], X[1]), fy(Y[0], Y[1])])
        rows = np.concatenate([_away_from_walls(grid, c, 2) for c in range(2)])
        errs.append(np.abs((W @ w)[rows] / grid.h ** 2 - ref[rows]).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


@pytest.mark.parametrize("n", [(8, 8), (4, 4, 4)])
def test_gkb_on_the_symmetric_form_reaches_the_dense_solution(n):
    grid = mac.MacGrid(n, 1.0 / n[0])
    rng = np.random.default_rng(1)
    mu = np.exp(rng.standard_normal(grid.n))
    ops = mac.assemble(grid, mu, 10.0, sym=True, n_diag=grid.h ** grid.dim / mu)
    assert np.linalg.eigvalsh(ops["W"].toarray()).min() > 0
    g = rng.standard_normal(grid.m)
    r = rng.standard_normal(grid.n_cells)
    r -= r.mean()
    res = gkb.solve(grid, ops, g, r, tol=1e-12, delay=4, inner="direct")
    w_ex, p_ex = dense_saddle_solve(grid, ops, g, r)
    assert m_norm(ops["M"], res["w"] - w_ex) <= 1e-9 * m_norm(ops["M"], w_ex)
    assert np.abs(res["p"] - p_ex).max() <= 1e-8 * np.abs(p_ex).max()


def _manufactured3():
    x, y, z = sympy.symbols("x y z")
    mu = 1 + sympy.Rational(2, 5) * sympy.sin(2 * x + 1) * sympy.cos(y - z)
    u = [sympy.sin(2 * x) * sympy.cos(y + 2 * z), sympy.cos(x + y) * sympy.sin(z + 1), sympy.sin(x * y + z)]
    X = (x, y, z)
    eps = [[(sympy.diff(u[a], X[b]) + sympy.diff(u[b], X[a])) / 2 for b in range(3)] for a in range(3)]
    f = [-sum(sympy.diff(2 * mu * eps[a][b], X[b]) for b in range(3)) for a in range(3)]
    lam = lambda e: sympy.lambdify((x, y, z), e, "numpy")
    return lam(mu), [lam(e) for e in u], [lam(e) for e in f]


def test_second_order_against_the_continuous_operator_3d():
    """The same in 3D: all three cross couplings (edges along x, y and z)."""
    mu_f, u_f, f_f = _manufactured3()
    errs = []
    for n in (16, 32):   # n = 8 is still pre-asymptotic (rate 1.4 to 16)
        grid = mac.MacGrid((n, n, n), 1.0 / n)
        C = grid.cell_centres()
        W = mac.assemble(grid, mu_f(*C), 0.0, sym=True)["W"]
        F = [grid.face_centres(c) for c in range(3)]
        w = grid.join_velocity([u_f[c](*F[c]) for c in range(3)])
        ref = grid.join_velocity([f_f[c](*F[c]) for c in range(3)])
        rows = np.concatenate([_away_from_walls(grid, c, 2) for c in range(3)])
        errs.append(np.abs((W @ w)[rows] / grid.h ** 3 - ref[rows]).max())
    rate = np.log2(errs[0] / errs[1])
    assert rate > 1.75, (errs, rate)
