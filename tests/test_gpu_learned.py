"""The learned inner solver: the network as a coarse correction inside
flexible CG, its application against the oracle, training pairs harvested
from GMG-PCG, and GKB solves that reach the oracle's answer whatever the
network's weights."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads
from oracle import mac
from oracle import unet as ou

from gpu_helpers import energy_rel, gpu_solve, make_handle, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D = mac.DIRICHLET
SHAPES = ou.layer_shapes(3, 16, 32, 2)


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _random_params(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(ou.num_params(SHAPES))
    off = 0
    for ci, co in SHAPES:
        p[off:off + 9 * ci * co] = rng.standard_normal(9 * ci * co) * np.sqrt(2.0 / (9 * ci))
        off += 9 * ci * co
        p[off:off + co] = 0.1 * rng.standard_normal(co)
        off += co
    return p.astype(np.float32)


def _net(gk, params=None, scale=1.0, seed=3):
    u = gk.gkb_unet_create(3, 16, 32, 2, seed, _stream())
    if params is not None:
        gk.gkb_unet_set_params(u, params)
    gk.gkb_unet_set_target_scale(u, scale)
    return u


def _varvisc(n):
    prob = workloads.varvisc2d(n)
    return prob["mu"], prob["g"]


@pytest.mark.parametrize("prec", [0, 1])
def test_learned_correction_matches_oracle(lib, prec):
    """unet_side = 0: the preconditioner is the network alone; gkb_precond
    against the oracle network with BF16-rounded operands."""
    gk = lib
    n = (32, 24)
    rng = np.random.default_rng(1)
    logmu = 0.5 * rng.standard_normal(n)
    params = _random_params(2)
    u = _net(gk, params, scale=2.5)
    h = make_handle(gk, n, (D,) * 4, np.exp(logmu), 100.0, precision=prec, inner=gk.GKB_INNER_FCG_UNET,
                    unet_side=0, net=u)
    try:
        grid = mac.MacGrid(n, 1.0 / n[0])
        r = rng.standard_normal(grid.m)
        z = np.empty(grid.m)
        gk.gkb_precond(h, r, z)
        M = mac.assemble(grid, np.exp(logmu), 100.0)["M"]
        ref = ou.apply_preconditioner(params.astype(np.float64), SHAPES, grid, r, logmu, 2.5, quant=ou.bf16_round, M=M)
        assert np.abs(z - ref).max() <= 3e-3 * np.abs(ref).max()
        # scale equivariance holds on the GPU too (the normalisation divides it out)
        z2 = np.empty(grid.m)
        gk.gkb_precond(h, 16.0 * r, z2)
        assert np.abs(z2 - 16.0 * z).max() <= 1e-5 * np.abs(16.0 * z).max()
    finally:
        gk.gkb_destroy(h)
        gk.gkb_unet_destroy(u)


@pytest.mark.parametrize("prec,side,composite", [(0, 16, 0), (1, 16, 0), (1, 32, 0), (0, 32, 1), (1, 16, 1)])
def test_fcg_with_network_reaches_oracle_solution(lib, prec, side, composite):
    """GKB with flexible CG preconditioned by a V-cycle with the network at
    the level of `side` cells (replace or composite form; untrained weights)
    meets the same 1e-8 energy bound against the oracle as the plain GMG-PCG
    form."""
    gk = lib
    n = (64, 64)
    mu, gvec = _varvisc(64)
    grid, ops = oracle_problem(n, (D,) * 4, mu, 100.0)
    rvec = np.zeros(grid.n_cells)
    ref = oracle_truth(grid, ops, gvec, rvec)
    u = _net(gk, scale=1.0, seed=7)
    inner = gk.GKB_INNER_FCG_UNET_MG if composite else gk.GKB_INNER_FCG_UNET
    h = make_handle(gk, n, (D,) * 4, mu, 100.0, precision=prec, inner=inner, tol_inner=1e-11,
                    unet_side=side, net=u, maxit=200, maxit_inner=600)
    try:
        rc, w, p = gpu_solve(gk, h, gvec, rvec, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
        st = gk.gkb_stats(h)
    finally:
        gk.gkb_destroy(h)
        gk.gkb_unet_destroy(u)
    assert st["inner_iterations"] > 0
    print("inner solves %d, iterations %d, fallbacks %d" % (st["inner_solves"], st["inner_iterations"],
                                                            st["inner_fallbacks"]))
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
    assert np.abs(p - ref["p"]).max() <= 1e-6 * np.abs(ref["p"]).max()


def test_harvested_pairs_solve_the_level_system(lib):
    """Every pair satisfies M e^ = r^ (checked with the oracle's sparse
    solve), the input carries log viscosity, and the first residual is f."""
    import torch
    gk = lib
    n = (32, 32)
    mu, _ = _varvisc(32)
    grid, ops = oracle_problem(n, (D,) * 4, mu, 100.0)
    f = np.random.default_rng(4).standard_normal(grid.m)
    h = make_handle(gk, n, (D,) * 4, mu, 100.0, precision=0, inner=gk.GKB_INNER_GMG_PCG, tol_inner=1e-12)
    try:
        cap = 40
        x_img = torch.zeros((cap, 32, 32, 3), dtype=torch.float32, device="cuda")
        t_img = torch.zeros((cap, 32, 32, 2), dtype=torch.float32, device="cuda")
        k = gk.gkb_harvest_pairs(h, f, cap, x_img, t_img)
    finally:
        gk.gkb_destroy(h)
    assert 3 <= k < cap
    xi, ti = x_img.cpu().numpy().astype(np.float64), t_img.cpu().numpy().astype(np.float64)
    assert not np.any(xi[k:]) and not np.any(ti[k:])
    lu = spla.splu(ops["M"].tocsc())
    M = ops["M"]
    for j in range(k):
        assert np.abs(xi[j, :, :, 2] - np.log(mu).T).max() <= 1e-6 * np.abs(np.log(mu)).max()
        rhat = ou.image_to_mac(grid, xi[j])
        assert abs(np.linalg.norm(rhat) - 32.0) < 1e-4 * 32.0   # unit RMS over the 32 x 32 cells
        eref = lu.solve(rhat)
        e = ou.image_to_mac(grid, ti[j])
        # the kept pairs have ||r_k|| >= 1e4 ||r*||, so x* - x_k is exact to
        # about 1e-4 (times a spectral factor); FP32 rounding of r^ adds at
        # most sqrt(cond M) * 6e-8 ~ 1e-5 here
        assert energy_rel(M, e, eref) <= 1e-3, j
    r0 = ou.image_to_mac(grid, xi[0])
    assert np.abs(r0 - f * 32.0 / np.linalg.norm(f)).max() <= 1e-6 * np.abs(r0).max()


def test_training_on_harvested_pairs_lowers_the_loss(lib):
    import torch
    gk = lib
    n = (32, 32)
    xs, ts = [], []
    for s in range(3):
        prob = workloads.varvisc2d(32, seed_offset=40 + 2 * s)
        h = make_handle(gk, n, (D,) * 4, prob["mu"], 100.0, precision=0, inner=gk.GKB_INNER_GMG_PCG,
                        tol_inner=1e-10)
        try:
            x_img = torch.zeros((30, 32, 32, 3), dtype=torch.float32, device="cuda")
            t_img = torch.zeros((30, 32, 32, 2), dtype=torch.float32, device="cuda")
            k = gk.gkb_harvest_pairs(h, prob["g"], 30, x_img, t_img)
            xs.append(x_img[:k])
            ts.append(t_img[:k])
        finally:
            gk.gkb_destroy(h)
    x_all, t_all = torch.cat(xs).contiguous(), torch.cat(ts).contiguous()
    scale = float(1.0 / t_all.pow(2).mean().sqrt())
    u = _net(gk, scale=scale, seed=11)
    try:
        losses = gk.gkb_unet_train(u, x_all, t_all, x_all.shape[0], 32, 32, 8, 150, 2e-3, seed=5)
    finally:
        gk.gkb_unet_destroy(u)
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-20:]) < 0.7 * np.mean(losses[:5])


def test_learned_form_argument_errors(lib):
    gk = lib
    u = _net(gk)
    try:
        # no level with 24 cells per side in a 64 x 64 hierarchy
        with pytest.raises(gk.GkbError):
            make_handle(gk, (64, 64), (D,) * 4, 1.0, 10.0, inner=gk.GKB_INNER_FCG_UNET, unet_side=24, net=u)
        # 3D grids have no learned form
        with pytest.raises(gk.GkbError):
            make_handle(gk, (8, 8, 8), (D,) * 6, 1.0, 10.0, inner=gk.GKB_INNER_FCG_UNET)
        # harvesting needs the FP64 GMG-PCG inner solver
        import torch
        h = make_handle(gk, (16, 16), (D,) * 4, 1.0, 10.0, precision=1)
        try:
            x = torch.zeros((4, 16, 16, 3), dtype=torch.float32, device="cuda")
            t = torch.zeros((4, 16, 16, 2), dtype=torch.float32, device="cuda")
            with pytest.raises(gk.GkbError):
                gk.gkb_harvest_pairs(h, np.ones(gk.gkb_layout(h)[0]), 4, x, t)
        finally:
            gk.gkb_destroy(h)
    finally:
        gk.gkb_unet_destroy(u)


def test_fcg_without_network_is_the_gmg_fallback(lib):
    """GKB_INNER_FCG_UNET with no network attached runs flexible CG on the
    plain V-cycle and still meets the bound."""
    gk = lib
    n = (48, 48)
    mu, gvec = _varvisc(48)
    grid, ops = oracle_problem(n, (D,) * 4, mu, 100.0)
    rvec = np.zeros(grid.n_cells)
    ref = oracle_truth(grid, ops, gvec, rvec)
    h = make_handle(gk, n, (D,) * 4, mu, 100.0, precision=1, inner=gk.GKB_INNER_FCG_UNET, tol_inner=1e-11,
                    maxit=200, maxit_inner=600)
    try:
        rc, w, p = gpu_solve(gk, h, gvec, rvec, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
    finally:
        gk.gkb_destroy(h)
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8
