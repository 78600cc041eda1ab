"""U-Net forward and backward in FP64 (NumPy), the reference for the GPU kernels.

TEST INFRASTRUCTURE. Part of the oracle: only ``tests/`` and the baseline
legs of ``bench.py`` may import it; the GPU library shares no code with it.

The network (the learned preconditioner of the variable-viscosity form; the
paper has no learned component, the architecture follows the workload
definition: 3 levels, 16/32/32 channels, 3x3 convolutions):

    a1 = relu(conv(x, 3 -> c1));   s1 = relu(conv(a1, c1 -> c1))        full resolution
    b1 = relu(conv(pool(s1), c1 -> c2)); s2 = relu(conv(b1, c2 -> c2))  1/2
    c1_ = relu(conv(pool(s2), c2 -> c2)); c2_ = relu(conv(c1_, c2 -> c2))  1/4
    d1 = relu(conv([up(c2_), s2], 2 c2 -> c2))                         1/2
    e1 = relu(conv([up(d1), s1], c2 + c1 -> c1))                       full
    y  = conv(e1, c1 -> c_out)                                          full

conv: 3x3, zero padding, weights w[ky][kx][ci][co] plus a bias per output
channel; pool: 2x2 mean; up: bilinear doubling with pixel-centre alignment
(fine pixel 2k sits a quarter coarse pixel before coarse pixel k, 2k + 1 a
quarter after; edge neighbours clamped); [a, b]: channel concatenation.
Images are NHWC (batch, rows, columns, channels). The flat parameter vector
stores each layer's weights then its bias, layers in the order above (the
GPU library uses the same layout). Training loss: the batch mean of
||N(x) - target||^2.
"""
import numpy as np

LAYERS = ("a1", "a2", "b1", "b2", "c1", "c2", "d1", "e1", "out")


def layer_shapes(c_in=3, c1=16, c2=32, c_out=2):
    """(c_in, c_out) of each convolution in parameter order."""
    return [(c_in, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c2), (c2, c2), (2 * c2, c2), (c2 + c1, c1), (c1, c_out)]


def num_params(shapes):
    return sum(9 * ci * co + co for ci, co in shapes)


def unpack(params, shapes):
    out, off = [], 0
    for ci, co in shapes:
        w = params[off:off + 9 * ci * co].reshape(3, 3, ci, co)
        off += 9 * ci * co
        b = params[off:off + co]
        off += co
        out.append((w, b))
    return out


def conv(x, w, b):
    """3x3 convolution, zero padding: y[n,i,j,o] = b[o] + sum x[n,i+ky-1,j+kx-1,c] w[ky,kx,c,o]."""
    n, h, wd, c = x.shape
    xp = np.zeros((n, h + 2, wd + 2, c))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.broadcast_to(b, (n, h, wd, w.shape[3])).copy()
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("nijc,co->nijo", xp[:, ky:ky + h, kx:kx + wd, :], w[ky, kx])
    return y


def conv_backward(x, w, dy):
    """Gradients of conv w.r.t. its input, weights and bias."""
    n, h, wd, c = x.shape
    xp = np.zeros((n, h + 2, wd + 2, c))
    xp[:, 1:-1, 1:-1, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            dw[ky, kx] = np.einsum("nijc,nijo->co", xp[:, ky:ky + h, kx:kx + wd, :], dy)
            dxp[:, ky:ky + h, kx:kx + wd, :] += np.einsum("nijo,co->nijc", dy, w[ky, kx])
    return dxp[:, 1:-1, 1:-1, :], dw, dy.sum(axis=(0, 1, 2))


def pool(x):
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def _up1(x, axis):
    """Bilinear doubling along one axis: fine 2k = 3/4 c[k] + 1/4 c[k-1],
    fine 2k+1 = 3/4 c[k] + 1/4 c[k+1], neighbours clamped to the edge."""
    x = np.moveaxis(x, axis, 0)
    m = x.shape[0]
    k = np.arange(m)
    lo, hi = np.maximum(k - 1, 0), np.minimum(k + 1, m - 1)
    out = np.empty((2 * m,) + x.shape[1:])
    out[0::2] = 0.75 * x[k] + 0.25 * x[lo]
    out[1::2] = 0.75 * x[k] + 0.25 * x[hi]
    return np.moveaxis(out, 0, axis)


def _up1_adjoint(d, axis):
    """Transpose of _up1: every fine value sends its two weights back."""
    d = np.moveaxis(d, axis, 0)
    m = d.shape[0] // 2
    k = np.arange(m)
    lo, hi = np.maximum(k - 1, 0), np.minimum(k + 1, m - 1)
    out = np.zeros((m,) + d.shape[1:])
    np.add.at(out, k, 0.75 * d[0::2])
    np.add.at(out, lo, 0.25 * d[0::2])
    np.add.at(out, k, 0.75 * d[1::2])
    np.add.at(out, hi, 0.25 * d[1::2])
    return np.moveaxis(out, 0, axis)


def up(x):
    return _up1(_up1(x, 1), 2)


def up_backward(dy):
    return _up1_adjoint(_up1_adjoint(dy, 2), 1)


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even) after rounding to float32:
    the 16 low bits of the float32 pattern are rounded away."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, shapes, keep=False, quant=None):
    """Network output (and the activations when keep). ``quant``, when given,
    is applied to every convolution's input image and weights (not the bias):
    the reading of a convolution evaluated with rounded operands and exact
    accumulation."""
    L = unpack(params, shapes)
    q = quant if quant is not None else (lambda a: a)

    def cv(inp, k):
        return conv(q(inp), q(L[k][0]), L[k][1])

    act = {}
    act["x"] = x
    act["a1"] = relu(cv(x, 0))
    act["s1"] = relu(cv(act["a1"], 1))
    act["p1"] = pool(act["s1"])
    act["b1"] = relu(cv(act["p1"], 2))
    act["s2"] = relu(cv(act["b1"], 3))
    act["p2"] = pool(act["s2"])
    act["c1"] = relu(cv(act["p2"], 4))
    act["c2"] = relu(cv(act["c1"], 5))
    act["u2"] = np.concatenate([up(act["c2"]), act["s2"]], axis=3)
    act["d1"] = relu(cv(act["u2"], 6))
    act["u1"] = np.concatenate([up(act["d1"]), act["s1"]], axis=3)
    act["e1"] = relu(cv(act["u1"], 7))
    y = cv(act["e1"], 8)
    return (y, act) if keep else y


def loss_and_grad(params, x, target, shapes):
    """L = (1/B) sum over the B samples of ||y - target||^2, and dL/dparams."""
    L = unpack(params, shapes)
    y, act = forward(params, x, shapes, keep=True)
    diff = y - target
    nb = x.shape[0]
    loss = float(np.sum(diff * diff)) / nb
    grads = [None] * len(L)

    def back(idx, inp, out_act, dy, has_relu=True):
        if has_relu:
            dy = dy * (out_act > 0)
        dx, dw, db = conv_backward(inp, L[idx][0], dy)
        grads[idx] = (dw, db)
        return dx

    c2, c1 = shapes[3][1], shapes[0][1]
    de1 = back(8, act["e1"], None, (2.0 / nb) * diff, has_relu=False)
    du1 = back(7, act["u1"], act["e1"], de1)
    dd1 = up_backward(du1[..., :c2])
    ds1 = du1[..., c2:]
    du2 = back(6, act["u2"], act["d1"], dd1)
    dc2 = up_backward(du2[..., :c2])
    ds2 = du2[..., c2:]
    dc1 = back(5, act["c1"], act["c2"], dc2)
    dp2 = back(4, act["p2"], act["c1"], dc1)
    ds2 = ds2 + pool_backward(dp2)
    db1 = back(3, act["b1"], act["s2"], ds2)
    dp1 = back(2, act["p1"], act["b1"], db1)
    ds1 = ds1 + pool_backward(dp1)
    da1 = back(1, act["a1"], act["s1"], ds1)
    back(0, act["x"], act["a1"], da1)
    flat = np.concatenate([np.concatenate([dw.ravel(), db]) for dw, db in grads])
    return loss, flat


def adam_step(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) at step t >= 1:
    moment averages, bias correction by 1 - beta^t, step lr m^ / (sqrt(v^) + eps).
    Returns the new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


# ---- the network as a preconditioner on the MAC grid (2D) -----------------
# Cell (i, j) of the image (row j, column i) carries the velocity residual on
# its west u face and its south v face, and log viscosity; the network's two
# output channels are read back onto the same faces. Faces that are not
# unknowns (Dirichlet walls) read and write zero; east / north boundary faces
# belong to no cell and get zero.

def mac_to_image(grid, vel, logmu):
    """(ny, nx, 3) image of a velocity vector and the cell log-viscosity
    (array indexed [x, y])."""
    nx, ny = grid.n
    img = np.zeros((ny, nx, 3))
    for c in range(2):
        idx = grid.face_index[c][:nx, :ny]
        val = np.where(idx >= 0, vel[np.maximum(idx, 0)], 0.0)
        img[:, :, c] = val.T
    img[:, :, 2] = np.asarray(logmu).reshape(nx, ny).T
    return img


def image_to_mac(grid, img):
    """Velocity vector from the first two channels of an (ny, nx, >=2) image."""
    nx, ny = grid.n
    vel = np.zeros(grid.m)
    for c in range(2):
        idx = grid.face_index[c][:nx, :ny]
        act = idx >= 0
        vel[idx[act]] = img[:, :, c].T[act]
    return vel


def apply_preconditioner(params, shapes, grid, r, logmu, target_scale=1.0, quant=None, M=None):
    """The scale-equivariant use of the network as an approximate inverse of
    M: with c = ||r|| / sqrt(nx ny) (the RMS of r over the cells),
    z = c / target_scale * N(r / c, log mu) on the faces (z = 0 for r = 0).
    With the matrix M given, z is then scaled by the energy-optimal step
    omega = (r, z) / (z, M z) (0 unless (z, M z) > 0): the minimiser of
    ||M^-1 r - omega z||_M."""
    nr = float(np.linalg.norm(r))
    if nr == 0.0:
        return np.zeros_like(r)
    c = nr / np.sqrt(grid.n[0] * grid.n[1])
    img = mac_to_image(grid, r / c, logmu)[None]
    y = forward(params, img, shapes, quant=quant)[0]
    z = (c / target_scale) * image_to_mac(grid, y)
    if M is None:
        return z
    zmz = float(z @ (M @ z))
    return (float(r @ z) / zmz) * z if zmz > 0 else np.zeros_like(z)
