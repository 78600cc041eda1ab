"""gkb_apply_noalloc against gkb_apply.

Callers whose device memory belongs to another allocator (or a fixed arena),
or whose loops cannot afford the device synchronisation of cudaMalloc and
cudaFree, use gkb_apply_noalloc: it works without a handle and keeps its
padded work arrays in a static device array. These tests check that its
products equal those of the handle-based gkb_apply (same tolerance as the
operator tests: 1e-12 of the largest entry) on two calls in a row, so that
the contents left in the shared array by one call cannot leak into the next,
and that grids above the array's limit are refused.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

from gpu_helpers import make_handle

pytestmark = pytest.mark.gpu

D, N = 0, 1


@pytest.mark.parametrize("n,bc,mu0,gamma", [
    ((40, 37), (D, N, D, D), 1.7, 5.0),
    ((64, 64), (D,) * 4, 1.0, 1000.0),
    ((12, 10, 9), (D,) * 6, 0.6, 3.0),
])
def test_noalloc_matches_handle_apply(lib, n, bc, mu0, gamma):
    import torch
    gk = lib
    h = make_handle(gk, n, bc, mu0, gamma, inner=0)
    try:
        m, nc = gk.gkb_layout(h)
        grid = gk.make_grid(n, 1.0 / n[0], bc)
        rng = np.random.default_rng(17)
        for call in range(2):                     # two calls in a row
            for op in (gk.GKB_OP_W, gk.GKB_OP_M, gk.GKB_OP_A, gk.GKB_OP_AT):
                nin = nc if op == gk.GKB_OP_A else m
                nout = nc if op == gk.GKB_OP_AT else m
                x = torch.tensor(rng.standard_normal(nin), device="cuda")
                y_ref = torch.empty(nout, dtype=torch.float64, device="cuda")
                y = torch.full((nout,), float("nan"), dtype=torch.float64, device="cuda")
                gk.gkb_apply(h, op, x, y_ref)
                rc = gk.gkb_apply_noalloc(grid, mu0, gamma, 0.0, op, x, y,
                                          torch.cuda.current_stream().cuda_stream)
                assert rc == gk.GKB_OK
                a, b = y.cpu().numpy(), y_ref.cpu().numpy()
                assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (call, op)
    finally:
        gk.gkb_destroy(h)


def test_noalloc_calls_allocate_no_device_memory(lib):
    """The property the entry point exists for: after a first call (which
    looks up the static array's address), further calls leave the device's
    free memory unchanged."""
    import torch
    gk = lib
    n = (96, 80)
    grid = gk.make_grid(n, 1.0 / n[0])
    m = 95 * 80 + 96 * 79
    s = torch.cuda.current_stream().cuda_stream
    x = torch.randn(m, dtype=torch.float64, device="cuda")
    y = torch.empty(m, dtype=torch.float64, device="cuda")
    assert gk.gkb_apply_noalloc(grid, 1.0, 10.0, 0.0, gk.GKB_OP_M, x, y, s) == gk.GKB_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        for op in (gk.GKB_OP_W, gk.GKB_OP_M):
            assert gk.gkb_apply_noalloc(grid, 1.0, 10.0, 0.0, op, x, y, s) == gk.GKB_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


@pytest.mark.parametrize("n,ok", [((711, 711), True), ((712, 712), False), ((63, 63, 63), True),
                                  ((64, 64, 64), False)])
def test_noalloc_size_limit_at_the_boundary(lib, n, ok):
    """The largest square and cube the static array holds (its padded rows
    round n + 1 faces up to a multiple of 32) and the next size, refused."""
    import torch
    gk = lib
    d = len(n)
    m = d * (n[0] - 1) * n[0] ** (d - 1)
    grid = gk.make_grid(n, 1.0 / n[0])
    x = torch.randn(m, dtype=torch.float64, device="cuda")
    y = torch.zeros(m, dtype=torch.float64, device="cuda")
    rc = gk.gkb_apply_noalloc(grid, 1.0, 10.0, 0.0, gk.GKB_OP_M, x, y, torch.cuda.current_stream().cuda_stream)
    if ok:
        assert rc == gk.GKB_OK
        assert torch.isfinite(y).all() and float(y.abs().max()) > 0
    else:
        assert rc == gk.GKB_ERR_INVALID_ARG


def test_noalloc_rejects_grids_above_the_limit(lib):
    import torch
    gk = lib
    n = (1024, 1024)
    grid = gk.make_grid(n, 1.0 / 1024)
    m = 1023 * 1024 * 2
    x = torch.zeros(m, dtype=torch.float64, device="cuda")
    y = torch.zeros(m, dtype=torch.float64, device="cuda")
    assert gk.gkb_apply_noalloc(grid, 1.0, 1.0, 0.0, gk.GKB_OP_M, x, y) == gk.GKB_ERR_INVALID_ARG
    # host arrays are refused too
    xs, ys = np.zeros(10), np.zeros(10)
    small = gk.make_grid((4, 4), 0.25)
    assert gk.gkb_apply_noalloc(small, 1.0, 1.0, 0.0, gk.GKB_OP_W, xs, ys) == gk.GKB_ERR_INVALID_ARG
