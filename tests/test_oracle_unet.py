"""Pins of the oracle U-Net against library routines (torch CPU convolution,
interpolation, pooling, bfloat16 conversion, Adam), against a direct
definition of the convolution, and against central finite differences of the
loss."""
import numpy as np
import torch
import torch.nn.functional as F

from oracle import mac, unet


def _nchw(a):
    return torch.tensor(a).permute(0, 3, 1, 2)


def _nhwc(t):
    return t.permute(0, 2, 3, 1).numpy()


def test_conv_matches_direct_definition():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 4, 5, 2))
    w = rng.standard_normal((3, 3, 2, 3))
    b = rng.standard_normal(3)
    y = unet.conv(x, w, b)
    for i in range(4):
        for j in range(5):
            for o in range(3):
                s = b[o]
                for ky in range(3):
                    for kx in range(3):
                        ii, jj = i + ky - 1, j + kx - 1
                        if 0 <= ii < 4 and 0 <= jj < 5:
                            s += x[0, ii, jj, :] @ w[ky, kx, :, o]
                assert abs(y[0, i, j, o] - s) < 1e-12


def test_conv_and_its_gradients_match_torch():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 6, 9, 5))
    w = rng.standard_normal((3, 3, 5, 4))
    b = rng.standard_normal(4)
    dy = rng.standard_normal((2, 6, 9, 4))
    xt = _nchw(x).requires_grad_(True)
    wt = torch.tensor(w).permute(3, 2, 0, 1).contiguous().requires_grad_(True)
    bt = torch.tensor(b).requires_grad_(True)
    yt = F.conv2d(xt, wt, bt, padding=1)
    yt.backward(_nchw(dy))
    assert np.abs(unet.conv(x, w, b) - _nhwc(yt.detach())).max() < 1e-12
    dx, dw, db = unet.conv_backward(x, w, dy)
    assert np.abs(dx - _nhwc(xt.grad)).max() < 1e-11
    assert np.abs(dw - wt.grad.permute(2, 3, 1, 0).numpy()).max() < 1e-11
    assert np.abs(db - bt.grad.numpy()).max() < 1e-11


def test_pool_and_bilinear_up_match_torch():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 6, 8, 3))
    assert np.abs(unet.pool(x) - _nhwc(F.avg_pool2d(_nchw(x), 2))).max() < 1e-15
    for shape in [(1, 1, 1, 2), (2, 3, 5, 3), (1, 4, 2, 1)]:
        c = rng.standard_normal(shape)
        ref = F.interpolate(_nchw(c), scale_factor=2, mode="bilinear", align_corners=False)
        assert np.abs(unet.up(c) - _nhwc(ref)).max() < 1e-14


def test_bilinear_up_reproduces_linear_functions_inside():
    # bilinear interpolation is exact for affine data away from the clamped edge
    h, w = 5, 6
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    c = (0.3 + 2.0 * yy - 1.5 * xx)[None, :, :, None].astype(float)
    f = unet.up(c)[0, :, :, 0]
    fy, fx = np.meshgrid((np.arange(2 * h) + 0.5) / 2 - 0.5, (np.arange(2 * w) + 0.5) / 2 - 0.5, indexing="ij")
    exact = 0.3 + 2.0 * fy - 1.5 * fx
    assert np.abs(f[1:-1, 1:-1] - exact[1:-1, 1:-1]).max() < 1e-13


def test_pool_up_adjoints():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((1, 6, 4, 3))
    b = rng.standard_normal((1, 3, 2, 3))
    assert abs(np.sum(unet.pool(a) * b) - np.sum(a * unet.pool_backward(b))) < 1e-12
    assert abs(np.sum(unet.up(b) * a) - np.sum(b * unet.up_backward(a))) < 1e-12


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    shapes = unet.layer_shapes(c_in=3, c1=4, c2=6, c_out=2)
    n = unet.num_params(shapes)
    params = 0.3 * rng.standard_normal(n)
    x = rng.standard_normal((2, 8, 8, 3))
    t = rng.standard_normal((2, 8, 8, 2))
    loss, g = unet.loss_and_grad(params, x, t, shapes)
    assert abs(loss - np.sum((unet.forward(params, x, shapes) - t) ** 2) / 2) < 1e-12 * loss
    idx = rng.choice(n, size=60, replace=False)
    eps = 1e-6
    for k in idx:
        e = np.zeros(n)
        e[k] = eps
        fd = (unet.loss_and_grad(params + e, x, t, shapes)[0] - unet.loss_and_grad(params - e, x, t, shapes)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(5)
    a = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 65504.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(unet.bf16_round(a), ref)


def test_adam_matches_torch_and_first_step_closed_form():
    rng = np.random.default_rng(6)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(4)]
    # first step: bias correction makes the step lr * g / (|g| + eps)
    p1, _, _ = unet.adam_step(p0, grads[0], np.zeros(50), np.zeros(50), 1, 0.01, eps=0.0)
    assert np.abs(p1 - (p0 - 0.01 * np.sign(grads[0]))).max() < 1e-15
    pt = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=0.003, betas=(0.8, 0.95), eps=1e-6)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        pt.grad = torch.tensor(g)
        opt.step()
        p, m, v = unet.adam_step(p, g, m, v, t, 0.003, 0.8, 0.95, 1e-6)
    assert np.abs(p - pt.detach().numpy()).max() < 1e-14


def test_mac_image_maps():
    grid = mac.MacGrid((6, 4), 1.0 / 6)
    rng = np.random.default_rng(7)
    v = rng.standard_normal(grid.m)
    logmu = rng.standard_normal((6, 4))
    img = unet.mac_to_image(grid, v, logmu)
    # the west u face of cell (i, j) and the south v face
    assert img[2, 3, 0] == v[grid.face_index[0][3, 2]]
    assert img[1, 4, 1] == v[grid.face_index[1][4, 1]]
    assert img[2, 5, 2] == logmu[5, 2]
    # wall faces read zero (u at x = 0, v at y = 0)
    assert np.all(img[:, 0, 0] == 0) and np.all(img[0, :, 1] == 0)
    # the read-back is the transpose of the extraction
    im2 = rng.standard_normal((4, 6, 2))
    lhs = np.sum(unet.mac_to_image(grid, v, logmu)[:, :, :2] * im2)
    assert abs(lhs - v @ unet.image_to_mac(grid, im2)) < 1e-12
    # every unknown but the east / north boundary faces round-trips
    back = unet.image_to_mac(grid, img)
    covered = np.zeros(grid.m, bool)
    for c in range(2):
        idx = grid.face_index[c][:6, :4]
        covered[idx[idx >= 0]] = True
    assert np.array_equal(back[covered], v[covered]) and np.all(back[~covered] == 0)


def test_preconditioner_is_scale_equivariant():
    shapes = unet.layer_shapes()
    rng = np.random.default_rng(8)
    params = 0.1 * rng.standard_normal(unet.num_params(shapes))
    grid = mac.MacGrid((8, 12), 1.0 / 8)
    r = rng.standard_normal(grid.m)
    logmu = rng.standard_normal((8, 12))
    z = unet.apply_preconditioner(params, shapes, grid, r, logmu)
    zmax = np.abs(z).max()
    # z(a r) = a z(r) for a > 0, the target scale divides, z(0) = 0
    assert np.abs(unet.apply_preconditioner(params, shapes, grid, 7.5 * r, logmu) - 7.5 * z).max() < 1e-12 * zmax
    assert np.abs(unet.apply_preconditioner(params, shapes, grid, r, logmu, target_scale=4.0) - z / 4.0).max() < 1e-15 * zmax
    assert not np.any(unet.apply_preconditioner(params, shapes, grid, 0 * r, logmu))
    # on an all-Dirichlet box every unknown is a west or south face of a
    # cell, so the residual channels hold all of r: at unit RMS their squares
    # sum to the number of cells
    img = unet.mac_to_image(grid, r / (np.linalg.norm(r) / np.sqrt(96)), logmu)
    assert abs(np.sum(img[:, :, :2] ** 2) - 96) < 1e-9 * 96


def test_energy_optimal_step_of_the_correction():
    """With M given, the returned multiple of the network's direction is the
    best one in the M-norm: ||e - x||_M <= ||e - t z||_M for every t, and
    never above ||e||_M (e = M^-1 r); it stays scale equivariant."""
    shapes = unet.layer_shapes()
    rng = np.random.default_rng(9)
    params = 0.1 * rng.standard_normal(unet.num_params(shapes))
    grid = mac.MacGrid((8, 8), 1.0 / 8)
    logmu = 0.5 * rng.standard_normal((8, 8))
    M = mac.assemble(grid, np.exp(logmu), 100.0)["M"].toarray()
    r = rng.standard_normal(grid.m)
    e = np.linalg.solve(M, r)
    z = unet.apply_preconditioner(params, shapes, grid, r, logmu)
    x = unet.apply_preconditioner(params, shapes, grid, r, logmu, M=M)
    en = lambda v: float(v @ (M @ v))
    assert en(e - x) <= en(e) * (1 + 1e-12)
    for t in np.linspace(-2, 2, 41) * (np.abs(x).max() / np.abs(z).max()):
        assert en(e - x) <= en(e - t * z) * (1 + 1e-12)
    assert np.abs(unet.apply_preconditioner(params, shapes, grid, 3.0 * r, logmu, M=M) - 3.0 * x).max() \
        < 1e-12 * np.abs(x).max()
