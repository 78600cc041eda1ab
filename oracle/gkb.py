"""Generalized Golub-Kahan bidiagonalization (GKB) for saddle-point systems, CPU FP64.

TEST INFRASTRUCTURE. Part of the oracle: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs may import it. It shares no code with the GPU
library.

The steps follow Sec. 2 of Kruse et al., arXiv 2001.10424, in its notation:

* augmented Lagrangian transform, Eq. (2) and Eq. (3):
  ``M = W + gamma A N^-1 A^T``, ``u = w - M^-1 (g + gamma A N^-1 r)``,
  ``b = r - A^T M^-1 (g + gamma A N^-1 r)``, giving ``[M A; A^T 0][u; p] = [0; b]``;
* Algorithm 1 (Craig-variant GKB recurrence) for that transformed system;
* the lower-bound stopping rule of Sec. 2.2, Eq. (5), with delay ``d``.

Readings taken where the paper is silent or ambiguous (each also listed in
the design notes of the repository):

* ``beta_1 = ||b||_{N^-1}`` as in Algorithm 1 (the text's ``||b||_N`` before it
  is the garbled one: only ``N^-1`` makes ``||q_1||_N = 1``).
* Stopping rule: once ``zeta_1 .. zeta_K`` are known, the estimate of the
  relative energy error of the iterate ``d`` steps back is
  ``sqrt( sum_{j=K-d}^{K} zeta_j^2 / sum_{j=1}^{K} zeta_j^2 )`` (d+1 terms as
  printed); the loop stops when it is ``<= tau`` and returns the latest
  iterate. ``squared=True`` compares the squared ratio with ``tau`` instead.
* ``alpha = ||w||_M`` is computed as ``sqrt(w^T (M w))`` with an explicit
  product by ``M``.
* An initial guess ``(w0, p0)`` is handled by defect correction: the method is
  run on ``(g - W w0 - A p0, r - A^T w0)`` and the correction is added.
* Enclosed flow (all sides Dirichlet): ``A`` annihilates constant pressure.
  The mean is removed from ``b`` (which lies in the range of ``A^T``,
  orthogonal to the constants) and the ``N``-weighted mean
  ``sum(N x) / sum(N)`` from each new ``N``-step vector before its norm is
  taken (the exact ``q_k`` are ``N``-orthogonal to the constants; for
  ``N = n I`` this is the plain mean), and the returned pressure has zero mean.
* ``N`` is ``n_scale * I`` or a positive diagonal (Sec. 3 allows any
  symmetric positive definite ``N``); ``N`` below is the scalar or the
  diagonal, and every product with ``N`` or ``N^-1`` is elementwise.
* A zero ``beta`` or ``alpha`` is a happy breakdown: the current iterate is
  the solution.
"""
import math

import numpy as np
import scipy.sparse.linalg as spla


def cg(M, f, tol, maxit):
    """Plain conjugate gradients for ``M x = f`` (Hestenes-Stiefel), zero start.

    Stops when the recursively updated residual satisfies
    ``||f - M x||_2 <= tol ||f||_2``. Returns (x, iterations, converged).
    """
    x = np.zeros_like(f)
    r = f.copy()
    fnorm = math.sqrt(float(f @ f))
    if fnorm == 0.0:
        return x, 0, True
    p = r.copy()
    rr = float(r @ r)
    for it in range(1, maxit + 1):
        q = M @ p
        a = rr / float(p @ q)
        x += a * p
        r -= a * q
        rr_new = float(r @ r)
        if math.sqrt(rr_new) <= tol * fnorm:
            return x, it, True
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, maxit, False


class InnerSolver:
    """Solver for ``M x = f`` used inside GKB (Sec. 3: any solver may be used).

    ``kind='cg'``: plain CG to relative tolerance ``tol``.
    ``kind='direct'``: a sparse LU factorisation of ``M`` (the paper's GKB with
    a direct inner solver, Sec. 4.1.2), via SciPy's SuperLU. ``M`` is
    symmetric, so the columns are ordered by minimum degree on the pattern of
    ``M + M^T`` with diagonal pivots preferred (SuperLU's symmetric mode); the
    ordering changes the fill and the time of the factorisation, and the
    result only up to rounding.
    """

    def __init__(self, M, kind="cg", tol=1e-12, maxit=100000):
        self.M, self.kind, self.tol, self.maxit = M, kind, tol, maxit
        self.iterations = []
        self.converged = True
        if kind == "direct":
            self.lu = spla.splu(M.tocsc(), permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))
        elif kind != "cg":
            raise ValueError(kind)

    def __call__(self, f):
        if self.kind == "direct":
            self.iterations.append(0)
            return self.lu.solve(f)
        x, it, ok = cg(self.M, f, self.tol, self.maxit)
        self.iterations.append(it)
        self.converged &= ok
        return x


def al_transform(A, N, g, r, gamma, solve_M):
    """Eq. (3): returns (y, b) with y = M^-1 (g + gamma A N^-1 r), b = r - A^T y.

    Then u = w - y solves the transformed system [M A; A^T 0][u; p] = [0; b].
    ``N`` is the scalar of ``N = n I`` or the diagonal of ``N``.
    """
    f = g + gamma * (A @ (r / N))
    if not np.any(f):
        y = np.zeros_like(f)
    else:
        y = solve_M(f)
    b = r - A.T @ y
    return y, b


def gkb(M, A, N, b, solve_M, tol, delay, maxit, enclosed=False,
        squared=False, keep_bases=False):
    """Algorithm 1 with the stopping rule of Eq. (5) (reading in module doc).

    ``N`` is the scalar of ``N = n I`` or the diagonal of ``N``. Returns a dict with the velocity ``u``, pressure ``p``,
    the sequences alpha_k, beta_k, zeta_k, the estimate after each step, the
    number of loop iterations and the convergence flag; with ``keep_bases`` it
    also holds the columns of V and Q.
    """
    def centre(x):
        return x - x.mean() if enclosed else x

    def centre_N(x):     # remove the N-weighted mean
        if not enclosed:
            return x
        Nx = N * np.ones_like(x)
        return x - float(Nx @ x) / float(Nx.sum())

    def norm_N(x):       # ||x||_N
        return math.sqrt(float((N * x) @ x))

    def norm_Ninv(x):    # ||x||_{N^-1}
        return math.sqrt(float(x @ (x / N)))

    def norm_M(x):       # ||x||_M
        return math.sqrt(float(x @ (M @ x)))

    b = centre(b)
    out = {"alpha": [], "beta": [], "zeta": [], "estimate": [], "V": [], "Q": []}
    beta = norm_Ninv(b)
    u = np.zeros(M.shape[0])
    p = np.zeros(A.shape[1])
    out["beta"].append(beta)
    if beta == 0.0:
        out.update(u=u, p=p, iterations=0, converged=True)
        return out
    q = (b / N) / beta
    w = solve_M(A @ q)
    alpha = norm_M(w)
    out["alpha"].append(alpha)
    if alpha == 0.0:
        out.update(u=u, p=p, iterations=0, converged=True)
        return out
    v = w / alpha
    zeta = beta / alpha
    d = q / alpha
    p = -zeta * d
    u = zeta * v
    out["zeta"].append(zeta)
    if keep_bases:
        out["V"].append(v.copy())
        out["Q"].append(q.copy())
    zeta2 = [zeta * zeta]
    k = 0
    converged = False
    while not converged and k < maxit:
        k += 1
        # N-step: g = N^-1 (A^T v_k - alpha_k N q_k), beta_{k+1} = ||g||_N
        gv = centre_N((A.T @ v) / N - alpha * q)
        beta = norm_N(gv)
        out["beta"].append(beta)
        if beta == 0.0:
            converged = True
            break
        q = gv / beta
        # M-step: w = M^-1 (A q_{k+1} - beta_{k+1} M v_k), alpha = ||w||_M
        w = solve_M(A @ q - beta * (M @ v))
        alpha = norm_M(w)
        out["alpha"].append(alpha)
        if alpha == 0.0:
            converged = True
            break
        v = w / alpha
        zeta = -beta / alpha * zeta
        d = (q - beta * d) / alpha
        u = u + zeta * v
        p = p - zeta * d
        out["zeta"].append(zeta)
        if keep_bases:
            out["V"].append(v.copy())
            out["Q"].append(q.copy())
        # check: lower bound of the error with delay d (Eq. (5))
        zeta2.append(zeta * zeta)
        K = len(zeta2)
        tail = sum(zeta2[max(0, K - delay - 1):K])
        total = sum(zeta2)
        ratio = tail / total
        est = ratio if squared else math.sqrt(ratio)
        out["estimate"].append(est)
        converged = est <= tol
    if enclosed:
        p = p - p.mean()
    out.update(u=u, p=p, iterations=k, converged=converged)
    return out


def solve(grid, ops, g, r, tol=1e-8, delay=5, maxit=10000, inner="cg",
          tol_inner=1e-12, maxit_inner=100000, w0=None, p0=None,
          squared=False, keep_bases=False, solver=None):
    """Solve [W A; A^T 0][w; p] = [g; r] with the AL transform and GKB.

    ``ops`` comes from :func:`oracle.mac.assemble`. ``solver`` is an
    :class:`InnerSolver` of ``ops["M"]`` built earlier (its factorisation is
    then reused across solves), else one of kind ``inner`` is built here.
    Returns the GKB dict with ``w`` (velocity), ``p`` (pressure) and
    ``inner_iterations`` (of this solve) added.
    """
    W, A, M = ops["W"], ops["A"], ops["M"]
    N, gamma = ops.get("N", ops["n_scale"]), ops["gamma"]
    if solver is None:
        solver = InnerSolver(M, inner, tol_inner, maxit_inner)
    solver.iterations = []
    solver.converged = True
    g = np.asarray(g, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    if w0 is not None:
        g = g - W @ w0 - (A @ p0 if p0 is not None else 0.0)
        r = r - A.T @ w0
    y, b = al_transform(A, N, g, r, gamma, solver)
    res = gkb(M, A, N, b, solver, tol, delay, maxit,
              enclosed=grid.enclosed, squared=squared, keep_bases=keep_bases)
    w = res["u"] + y
    p = res["p"]
    if w0 is not None:
        w = w + w0
        if p0 is not None:
            p = p + p0
        if grid.enclosed:
            p = p - p.mean()
    res["w"] = w
    res["p"] = p
    res["y"] = y
    res["inner_iterations"] = list(solver.iterations)
    res["inner_converged"] = solver.converged
    return res
