"""MAC-staggered Stokes operators assembled as sparse matrices (CPU, FP64).

TEST INFRASTRUCTURE. This module is part of the oracle: it may be imported only
by ``tests/``, by ``__graft_entry__.smoke()`` and by the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py``. The GPU library never calls it and
shares no code with it.

What it assembles (the blocks of the saddle-point system, Sec. 2, Eq. (1)):

    [ W   A ] [w]   [g]
    [ A^T 0 ] [p] = [r]

on a uniform MAC grid with spacing ``h``: velocity component ``c`` lives on the
faces normal to axis ``c``, pressure in the cells. The discretisation is the
finite-volume (cell-measure integrated) form:

* ``W`` is the component-wise viscous operator ``-div(mu grad u_c)`` integrated
  over each face's control volume, assembled link by link (a graph Laplacian):
  a link between two neighbouring faces with conductance ``kappa`` adds
  ``kappa`` to both diagonals and ``-kappa`` to both off-diagonals. A link
  across a cell (normal direction) uses that cell's viscosity; a link across a
  node (2D) or edge (3D) uses the mean of the in-domain cells touching it.
  ``kappa = mu_link * h**(d-2)``, halved for the tangential links of a face
  whose control volume is cut in half by a natural (outflow) boundary. A
  tangential link that leaves the domain through a Dirichlet side ends on the
  wall at distance h/2 (mirror ghost, conductance doubled); through a natural
  side it is absent (zero flux).
* ``A`` is the integrated gradient: ``(A p)_f = h**(d-1) (p_plus - p_minus)``
  with the cells on the plus and minus side of face ``f``; a missing cell
  (beyond a natural boundary) contributes pressure 0. ``A^T`` is therefore the
  negative integrated divergence.
* ``N = n_scale * I`` (the restriction of the paper's PETSc implementation,
  Sec. 3), the default ``n_scale = h**d`` being the pressure mass matrix; or,
  since Sec. 3 allows any symmetric positive definite N, a positive diagonal
  ``N = diag(n_diag)`` given per cell (e.g. the viscosity-weighted pressure
  mass matrix ``h**d / mu``).
* ``M = W + gamma * A N^-1 A^T`` (Eq. (2), the augmented (1,1) block).

Unknown ordering (shared convention with the library's documented layout, not
shared code): all active u faces, then all active v faces (then w), each block
in row-major order with x fastest. A face normal to axis ``c`` is active unless
it lies on a Dirichlet side normal to ``c``.
"""
import numpy as np
import scipy.sparse as sp

DIRICHLET = 0
NATURAL = 1


class MacGrid:
    """Uniform MAC grid: ``n`` cells per axis (x, y[, z]), spacing ``h``.

    ``bc`` holds one entry per side in the order x-low, x-high, y-low, y-high,
    z-low, z-high; each is DIRICHLET or NATURAL.
    """

    def __init__(self, n, h, bc=None):
        self.dim = len(n)
        assert self.dim in (2, 3)
        self.n = tuple(int(v) for v in n)
        self.h = float(h)
        if bc is None:
            bc = (DIRICHLET,) * (2 * self.dim)
        self.bc = tuple(int(b) for b in bc)
        assert len(self.bc) == 2 * self.dim
        self.enclosed = all(b == DIRICHLET for b in self.bc)
        # index maps, arrays indexed [x, y(, z)]
        self.face_index = []
        off = 0
        for c in range(self.dim):
            idx = np.full(self.face_shape(c), -1, dtype=np.int64)
            lo, hi = self.active_range(c)
            sl = [slice(None)] * self.dim
            sl[c] = slice(lo, hi + 1)
            cnt = idx[tuple(sl)].size
            # x fastest == Fortran order on [x, y, z] arrays
            idx[tuple(sl)] = off + np.arange(cnt).reshape(idx[tuple(sl)].shape, order="F")
            off += cnt
            self.face_index.append(idx)
        self.m = off
        self.n_cells = int(np.prod(self.n))
        self.cell_index = np.arange(self.n_cells).reshape(self.n, order="F")

    def face_shape(self, c):
        s = list(self.n)
        s[c] += 1
        return tuple(s)

    def active_range(self, c):
        """Inclusive range of active face positions along axis ``c``."""
        lo = 1 if self.bc[2 * c] == DIRICHLET else 0
        hi = self.n[c] - 1 if self.bc[2 * c + 1] == DIRICHLET else self.n[c]
        return lo, hi

    def face_centres(self, c):
        """Coordinates (x, y[, z]) of every face position of component ``c``."""
        grids = []
        for a in range(self.dim):
            k = np.arange(self.face_shape(c)[a], dtype=np.float64)
            grids.append(k * self.h if a == c else (k + 0.5) * self.h)
        return np.meshgrid(*grids, indexing="ij")

    def cell_centres(self):
        grids = [(np.arange(self.n[a]) + 0.5) * self.h for a in range(self.dim)]
        return np.meshgrid(*grids, indexing="ij")

    # -- conversions between the compact vector and per-component arrays -----
    def split_velocity(self, w):
        """Compact m-vector -> list of full face arrays (inactive faces = 0)."""
        out = []
        for c in range(self.dim):
            arr = np.zeros(self.face_shape(c))
            idx = self.face_index[c]
            act = idx >= 0
            arr[act] = w[idx[act]]
            out.append(arr)
        return out

    def join_velocity(self, comps):
        """Full face arrays -> compact m-vector (active faces only)."""
        w = np.zeros(self.m)
        for c in range(self.dim):
            idx = self.face_index[c]
            act = idx >= 0
            w[idx[act]] = comps[c][act]
        return w


def _cell_mu(grid, mu, coords):
    """Viscosity of the cells at integer ``coords`` (list of arrays); returns
    (values, valid) with valid=False where the cell lies outside the domain."""
    valid = np.ones(coords[0].shape, dtype=bool)
    clipped = []
    for a in range(grid.dim):
        valid &= (coords[a] >= 0) & (coords[a] < grid.n[a])
        clipped.append(np.clip(coords[a], 0, grid.n[a] - 1))
    return mu[tuple(clipped)], valid


def _edge_mu(grid, mu, X, c, a, a_face):
    """Mean viscosity of the in-domain cells around the node/edge crossed by a
    tangential link of component ``c`` along axis ``a``: cells at c-coordinate
    X[c]-1 and X[c], a-coordinate a_face-1 and a_face, other axes as in X."""
    total = np.zeros(X[0].shape)
    count = np.zeros(X[0].shape)
    for dc in (-1, 0):
        for da in (-1, 0):
            coords = [x.copy() for x in X]
            coords[c] = X[c] + dc
            coords[a] = a_face + da
            vals, ok = _cell_mu(grid, mu, coords)
            total += np.where(ok, vals, 0.0)
            count += ok
    return total / count


def assemble(grid, mu=1.0, gamma=0.0, n_scale=None, n_diag=None, sym=False):
    """Assemble W, A (CSR), N and M = W + gamma A N^-1 A^T (Eq. (2)).

    ``mu`` is a scalar or an array of cell viscosities indexed [x, y(, z)].
    ``sym`` selects the symmetric-gradient viscous operator
    ``-div(2 mu eps(u))`` (every side Dirichlet): the normal links carry
    ``2 mu``, and every interior node (2D) / edge (3D) between the axes
    ``a`` and ``c`` adds the cross coupling of its energy
    ``mu_e h^(d-2) (d_a u_c + d_c u_a)^2``, whose squares are the tangential
    links already present.
    ``n_diag`` (optional, same indexing, every entry > 0) selects the diagonal
    ``N = diag(n_diag)``; otherwise ``N = n_scale * I``.
    Returns a dict with W, A, M (scipy CSR, FP64), n_scale, ``N`` (the scalar
    n_scale, or the diagonal of N in cell-index order) and the link list
    needed to fold Dirichlet data into the right-hand side.
    """
    d, h = grid.dim, grid.h
    if np.isscalar(mu):
        mu = np.full(grid.n, float(mu))
    mu = np.asarray(mu, dtype=np.float64)
    assert mu.shape == grid.n
    if n_scale is None:
        n_scale = h ** d
    N = float(n_scale)
    if n_diag is not None:
        n_diag = np.asarray(n_diag, dtype=np.float64)
        assert n_diag.shape == grid.n and np.all(n_diag > 0)
        # the diagonal in the order of the pressure unknowns
        N = np.empty(grid.n_cells)
        N[grid.cell_index] = n_diag
    scale = h ** (d - 2)
    rows, cols, vals = [], [], []
    # Dirichlet couplings: (active face index, conductance, component,
    # boundary-face position) for the normal-direction links that end on a
    # boundary face; used to fold boundary data into g.
    bnd_links = []

    def add_links(i1, i2, kappa):
        # both endpoints active: graph-Laplacian contribution of each link
        rows.extend([i1, i2, i1, i2])
        cols.extend([i1, i2, i2, i1])
        vals.extend([kappa, kappa, -kappa, -kappa])

    def add_diag(i, kappa):
        rows.append(np.atleast_1d(i))
        cols.append(np.atleast_1d(i))
        vals.append(np.atleast_1d(kappa))

    for c in range(d):
        idx = grid.face_index[c]
        shape = grid.face_shape(c)
        X = np.indices(shape)  # X[a] = a-coordinate of each face position
        # half control volume: face on a natural side normal to c
        half = np.zeros(shape, dtype=bool)
        if grid.bc[2 * c] == NATURAL:
            half |= X[c] == 0
        if grid.bc[2 * c + 1] == NATURAL:
            half |= X[c] == grid.n[c]
        area = np.where(half, 0.5, 1.0)
        for a in range(d):
            # links between position x and x + e_a, both inside the face grid
            sl1 = [slice(None)] * d
            sl2 = [slice(None)] * d
            sl1[a] = slice(0, shape[a] - 1)
            sl2[a] = slice(1, shape[a])
            i1 = idx[tuple(sl1)]
            i2 = idx[tuple(sl2)]
            Xl = [X[b][tuple(sl1)] for b in range(d)]
            if a == c:
                # normal link across the cell between the two faces
                mu_l, _ = _cell_mu(grid, mu, Xl)
                kap = (2.0 if sym else 1.0) * scale * mu_l
            else:
                mu_l = _edge_mu(grid, mu, Xl, c, a, Xl[a] + 1)
                kap = scale * mu_l * area[tuple(sl1)]
            both = (i1 >= 0) & (i2 >= 0)
            add_links(i1[both], i2[both], kap[both])
            # one endpoint active, the other a Dirichlet boundary face (only
            # possible along the normal direction): diagonal + RHS coupling
            if a == c:
                only1 = (i1 >= 0) & (i2 < 0)
                only2 = (i1 < 0) & (i2 >= 0)
                pos2 = [x[tuple(sl2)] for x in X]
                for sel, act, other in ((only1, i1, pos2), (only2, i2, Xl)):
                    add_diag(act[sel], kap[sel])
                    for fa, k, *bpos in zip(act[sel], kap[sel], *[o[sel] for o in other]):
                        bnd_links.append((int(fa), float(k), c, tuple(int(b) for b in bpos)))
            # tangential links leaving the domain through the low/high side
            if a != c:
                for side, apos, aface in ((0, 0, 0), (1, shape[a] - 1, grid.n[a])):
                    if grid.bc[2 * a + side] != DIRICHLET:
                        continue  # natural side: zero flux, no link
                    sl = [slice(None)] * d
                    sl[a] = slice(apos, apos + 1)
                    ib = idx[tuple(sl)]
                    Xb = [X[b][tuple(sl)] for b in range(d)]
                    mu_l = _edge_mu(grid, mu, Xb, c, a, np.full(ib.shape, aface))
                    kap = 2.0 * scale * mu_l * area[tuple(sl)]
                    act = ib >= 0
                    add_diag(ib[act], kap[act])  # wall (tangential) velocity is 0
    if sym:
        assert grid.enclosed, "the symmetric-gradient form needs Dirichlet velocity on every side"
        for c in range(d):
            for a in range(c):
                # interior edges between axes a and c: node coordinates
                # ka in 1..n_a-1, kc in 1..n_c-1, cell coordinates elsewhere
                shape = list(grid.n)
                shape[a] = grid.n[a] - 1
                shape[c] = grid.n[c] - 1
                E = np.indices(shape)
                E[a] += 1
                E[c] += 1
                # u_c above / below the edge along a; u_a right / left along c
                def faces(comp, axis, shift):
                    X = [e.copy() for e in E]
                    X[axis] = X[axis] + shift
                    return grid.face_index[comp][tuple(X)]
                cp, cm = faces(c, a, 0), faces(c, a, -1)
                ap, am = faces(a, c, 0), faces(a, c, -1)
                mu_e = _edge_mu(grid, mu, [e for e in E], c, a, E[a])
                kap = (scale * mu_e).ravel()
                g1 = ((cp.ravel(), 1.0), (cm.ravel(), -1.0))
                g2 = ((ap.ravel(), 1.0), (am.ravel(), -1.0))
                for i1, s1 in g1:
                    for i2, s2 in g2:
                        rows.extend([i1, i2])
                        cols.extend([i2, i1])
                        vals.extend([s1 * s2 * kap, s1 * s2 * kap])
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = np.concatenate(vals) if vals else np.zeros(0)
    W = sp.csr_matrix((vals, (rows, cols)), shape=(grid.m, grid.m))
    W.sum_duplicates()

    # A: integrated gradient, A[f, plus] = +h^(d-1), A[f, minus] = -h^(d-1)
    arow, acol, aval = [], [], []
    hd1 = h ** (d - 1)
    for c in range(d):
        idx = grid.face_index[c]
        X = np.indices(grid.face_shape(c))
        act = idx >= 0
        for shift, sign in ((0, 1.0), (-1, -1.0)):
            coords = [X[b][act] for b in range(d)]
            coords[c] = coords[c] + shift
            ok = np.ones(coords[0].shape, dtype=bool)
            for b in range(d):
                ok &= (coords[b] >= 0) & (coords[b] < grid.n[b])
            cells = grid.cell_index[tuple(np.clip(coords[b], 0, grid.n[b] - 1) for b in range(d))]
            arow.append(idx[act][ok])
            acol.append(cells[ok])
            aval.append(np.full(int(ok.sum()), sign * hd1))
    A = sp.csr_matrix((np.concatenate(aval), (np.concatenate(arow), np.concatenate(acol))),
                      shape=(grid.m, grid.n_cells))
    if np.isscalar(N):
        M = (W + (gamma / N) * (A @ A.T)).tocsr()
    else:
        M = (W + gamma * (A @ sp.diags(1.0 / N) @ A.T)).tocsr()
    M.sum_duplicates()
    return {"W": W, "A": A, "M": M, "n_scale": float(n_scale), "N": N, "gamma": float(gamma),
            "bnd_links": bnd_links}


def dirichlet_rhs(grid, ops, boundary_normal):
    """Fold Dirichlet normal-velocity data into (g, r).

    ``boundary_normal`` maps a side number (0..2d-1, Dirichlet sides only) to
    an array of the normal velocity on that side's boundary faces, indexed like
    the face grid with the normal axis removed ([y] for x-sides in 2D, etc.).
    Walls are no-slip: tangential wall velocity is 0. Returns (g_bc, r_bc):
    g gets kappa * u_b for every normal link ending on a boundary face, and the
    adjacent cell's continuity row gets -A[b, cell] * u_b.
    """
    d, h = grid.dim, grid.h
    g = np.zeros(grid.m)
    r = np.zeros(grid.n_cells)

    def bvalue(c, pos):
        lo_side, hi_side = 2 * c, 2 * c + 1
        side = lo_side if pos[c] == 0 else hi_side
        arr = boundary_normal.get(side)
        if arr is None:
            return 0.0
        rest = tuple(pos[b] for b in range(d) if b != c)
        return float(np.asarray(arr)[rest])

    for fa, kap, c, bpos in ops["bnd_links"]:
        g[fa] += kap * bvalue(c, bpos)
    hd1 = h ** (d - 1)
    for c in range(d):
        for side, pos_c, cell_c, a_val in ((2 * c, 0, 0, hd1), (2 * c + 1, grid.n[c], grid.n[c] - 1, -hd1)):
            if grid.bc[side] != DIRICHLET or side not in boundary_normal:
                continue
            arr = np.asarray(boundary_normal[side], dtype=np.float64)
            other = [b for b in range(d) if b != c]
            for rest in np.ndindex(*[grid.n[b] for b in other]):
                cell = [0] * d
                cell[c] = cell_c
                for b, v in zip(other, rest):
                    cell[b] = v
                r[grid.cell_index[tuple(cell)]] -= a_val * arr[rest]
    return g, r
