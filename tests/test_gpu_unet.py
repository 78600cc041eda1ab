"""U-Net kernels against the FP64 oracle U-Net: FP32 forward, BF16
tensor-core forward (against the oracle with BF16-rounded operands), loss and
gradients, Adam, and a short training run."""
import numpy as np
import pytest

from oracle import unet as ou

pytestmark = pytest.mark.gpu

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


def _net(gk, params=None, seed=11):
    u = gk.gkb_unet_create(3, 16, 32, 2, seed, _stream())
    if params is not None:
        gk.gkb_unet_set_params(u, params)
    return u


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def test_parameter_count_and_seeded_init(lib):
    gk = lib
    u1, u2, u3 = _net(gk, seed=5), _net(gk, seed=5), _net(gk, seed=6)
    try:
        n = gk.gkb_unet_num_params(u1)
        assert n == ou.num_params(SHAPES)
        ps = []
        for u in (u1, u2, u3):
            p = np.empty(n, np.float32)
            gk.gkb_unet_get_params(u, p)
            ps.append(p)
        assert np.array_equal(ps[0], ps[1]) and not np.array_equal(ps[0], ps[2])
        for (w, b), (ci, co) in zip(ou.unpack(ps[0].astype(np.float64), SHAPES), SHAPES):
            assert np.all(b == 0)
            if w.size >= 2000:  # He-normal scale
                assert abs(w.std() / np.sqrt(2.0 / (9 * ci)) - 1) < 0.1
    finally:
        for u in (u1, u2, u3):
            gk.gkb_unet_destroy(u)


@pytest.mark.parametrize("nb,h,w", [(2, 24, 36), (1, 4, 4), (3, 20, 8)])
def test_forward_fp32_matches_oracle(lib, nb, h, w):
    import torch
    gk = lib
    p = _random_params(1)
    u = _net(gk, p)
    try:
        x = np.random.default_rng(2).standard_normal((nb, h, w, 3))
        y = torch.empty((nb, h, w, 2), dtype=torch.float32, device="cuda")
        gk.gkb_unet_forward(u, _dev(x), nb, h, w, y, 0)
        ref = ou.forward(p.astype(np.float64), x, SHAPES)
        err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 1e-5, err
    finally:
        gk.gkb_unet_destroy(u)


@pytest.mark.parametrize("nb,h,w", [(2, 24, 36), (1, 64, 48)])
def test_forward_tensor_cores_matches_bf16_oracle(lib, nb, h, w):
    import torch
    gk = lib
    p = _random_params(3)
    u = _net(gk, p)
    try:
        x = np.random.default_rng(4).standard_normal((nb, h, w, 3))
        y = torch.empty((nb, h, w, 2), dtype=torch.float32, device="cuda")
        gk.gkb_unet_forward(u, _dev(x), nb, h, w, y, 1)
        yt = y.cpu().numpy()
        ref_q = ou.forward(p.astype(np.float64), x, SHAPES, quant=ou.bf16_round)
        ref = ou.forward(p.astype(np.float64), x, SHAPES)
        scale = np.abs(ref).max()
        # BF16 operands with FP32 accumulation: close to the oracle evaluated
        # with BF16-rounded operands (rare one-ulp rounding flips where the FP32
        # and FP64 activations straddle a rounding boundary) ...
        assert np.abs(yt - ref_q).max() / scale < 3e-3
        # ... and within the BF16 error of the exact network
        assert np.abs(yt - ref).max() / scale < 3e-2
    finally:
        gk.gkb_unet_destroy(u)


def test_loss_and_gradient_match_oracle(lib):
    import torch
    gk = lib
    p = _random_params(5)
    u = _net(gk, p)
    try:
        rng = np.random.default_rng(6)
        nb, h, w = 2, 16, 20
        x = rng.standard_normal((nb, h, w, 3))
        t = rng.standard_normal((nb, h, w, 2))
        g = torch.empty(len(p), dtype=torch.float32, device="cuda")
        loss = gk.gkb_unet_loss_grad(u, _dev(x), _dev(t), nb, h, w, g)
        ref_loss, ref_g = ou.loss_and_grad(p.astype(np.float64), x, t, SHAPES)
        assert abs(loss - ref_loss) <= 1e-5 * ref_loss
        gg = g.cpu().numpy().astype(np.float64)
        off = 0
        for ci, co in SHAPES:
            k = 9 * ci * co + co
            a, b = gg[off:off + k], ref_g[off:off + k]
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b), (ci, co)
            off += k
        # the reductions are deterministic
        g2 = torch.empty_like(g)
        loss2 = gk.gkb_unet_loss_grad(u, _dev(x), _dev(t), nb, h, w, g2)
        assert loss2 == loss and torch.equal(g, g2)
    finally:
        gk.gkb_unet_destroy(u)


def test_adam_matches_oracle(lib):
    gk = lib
    p = _random_params(7)
    u = _net(gk, p)
    try:
        rng = np.random.default_rng(8)
        nb, h, w = 1, 8, 12
        x, t = rng.standard_normal((nb, h, w, 3)), rng.standard_normal((nb, h, w, 2))
        q, m, v = p.astype(np.float64), np.zeros(len(p)), np.zeros(len(p))
        for step in (1, 2, 3):
            g = np.empty(len(p), np.float32)
            cur = np.empty(len(p), np.float32)
            gk.gkb_unet_get_params(u, cur)
            gk.gkb_unet_loss_grad(u, _dev(x), _dev(t), nb, h, w, g)
            gk.gkb_unet_adam_step(u, 1e-3, 0.9, 0.999, 1e-8)
            q, m, v = ou.adam_step(cur.astype(np.float64), g.astype(np.float64), m, v, step, 1e-3)
            new = np.empty(len(p), np.float32)
            gk.gkb_unet_get_params(u, new)
            assert np.abs(new - q).max() < 2e-6
    finally:
        gk.gkb_unet_destroy(u)


def test_training_reduces_loss(lib):
    gk = lib
    u = _net(gk, seed=9)
    try:
        rng = np.random.default_rng(10)
        x = rng.standard_normal((4, 16, 16, 3))
        xd, td = _dev(x), _dev(0.5 * x[..., :2])
        losses = []
        for _ in range(60):
            losses.append(gk.gkb_unet_loss_grad(u, xd, td, 4, 16, 16))
            gk.gkb_unet_adam_step(u, 3e-3)
        assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    finally:
        gk.gkb_unet_destroy(u)


def test_unet_argument_errors(lib):
    import torch
    gk = lib
    with pytest.raises(gk.GkbError):
        gk.gkb_unet_create(3, 8, 32, 2, 0, _stream())
    u = _net(gk)
    try:
        x = torch.zeros((1, 6, 8, 3), dtype=torch.float32, device="cuda")
        y = torch.zeros((1, 6, 8, 2), dtype=torch.float32, device="cuda")
        with pytest.raises(gk.GkbError):  # sides must be divisible by 4
            gk.gkb_unet_forward(u, x, 1, 6, 8, y, 0)
        with pytest.raises(gk.GkbError):  # host arrays are rejected
            gk.gkb_unet_forward(u, np.zeros((1, 8, 8, 3), np.float32), 1, 8, 8, y, 0)
        assert "device" in gk.gkb_unet_last_error(u)
    finally:
        gk.gkb_unet_destroy(u)
