"""Shared helpers of the GPU tests: handle creation and oracle comparisons."""
import math

import numpy as np

from oracle import gkb as ogkb
from oracle import mac


def make_handle(gk, n, bc, mu=1.0, gamma=0.0, precision=0, inner=1, tol_inner=1e-11, maxit=1000,
                maxit_inner=3000, coarse_max=8, degree=2, mixed_rtol=1e-3, use_graph=1, n_scale=0.0,
                profile=0, kernel_variant=0, unet_side=0, net=None, n_diag=None, viscous_form=0,
                batch_lockstep=0, tail_side=0):
    import torch
    opt = gk.gkb_default_options()
    opt.precision = precision
    opt.inner = inner
    opt.tol_inner = tol_inner
    opt.maxit = maxit
    opt.maxit_inner = maxit_inner
    opt.coarse_max = coarse_max
    opt.smoother_degree = degree
    opt.mixed_rtol = mixed_rtol
    opt.use_graph = use_graph
    opt.profile = profile
    opt.kernel_variant = kernel_variant
    opt.unet_side = unet_side
    opt.viscous_form = viscous_form
    opt.batch_lockstep = batch_lockstep
    opt.tail_side = tail_side
    opt.stream = torch.cuda.current_stream().cuda_stream
    h = gk.gkb_create(opt)
    if net is not None:
        gk.gkb_set_unet(h, net)
    h_ = 1.0 / n[0]
    visc = None
    mu0 = 1.0
    if np.isscalar(mu):
        mu0 = float(mu)
    else:
        # compact cell ordering: x fastest == Fortran order of an [x, y, z] array
        visc = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).ravel(order="F"))
    if n_diag is not None:
        nd = np.ascontiguousarray(np.asarray(n_diag, dtype=np.float64).ravel(order="F"))
        gk.gkb_set_problem_n(h, gk.make_grid(n, h_, bc), nd, visc, mu0, gamma)
    else:
        gk.gkb_set_problem(h, gk.make_grid(n, h_, bc), visc, mu0, gamma, n_scale)
    return h


def energy_rel(M, a, ref):
    e = a - ref
    return math.sqrt(max(float(e @ (M @ e)), 0.0)) / math.sqrt(float(ref @ (M @ ref)))


def oracle_problem(n, bc, mu=1.0, gamma=0.0, **kw):
    grid = mac.MacGrid(n, 1.0 / n[0], bc)
    ops = mac.assemble(grid, mu, gamma, **kw)
    return grid, ops


def oracle_truth(grid, ops, g, r, **kw):
    """Tightly converged oracle solution (sparse-LU inner solves)."""
    return ogkb.solve(grid, ops, g, r, tol=kw.get("tol", 1e-13), delay=kw.get("delay", 5), inner="direct")


def gpu_solve(gk, h, g, r, tol=1e-8, delay=5, w0=None, p0=None, device=True):
    import torch
    m, n = gk.gkb_layout(h)
    if device:
        gt = torch.tensor(g, device="cuda")
        rt = torch.tensor(r, device="cuda")
        w = torch.empty(m, dtype=torch.float64, device="cuda")
        p = torch.empty(n, dtype=torch.float64, device="cuda")
        w0t = torch.tensor(w0, device="cuda") if w0 is not None else None
        p0t = torch.tensor(p0, device="cuda") if p0 is not None else None
        rc = gk.gkb_solve(h, gt, rt, tol, delay, w, p, w0t, p0t)
        return rc, w.cpu().numpy(), p.cpu().numpy()
    w = np.empty(m)
    p = np.empty(n)
    rc = gk.gkb_solve(h, np.ascontiguousarray(g), np.ascontiguousarray(r), tol, delay, w, p,
                      None if w0 is None else np.ascontiguousarray(w0),
                      None if p0 is None else np.ascontiguousarray(p0))
    return rc, w, p
