"""The autotuner: its choice lies in the searched set, the tuned handle still
meets the parity bound, and the choice is cached in the process and in the
GKB_TUNE_CACHE file."""
import os

import numpy as np
import pytest

from oracle import mac

from gpu_helpers import energy_rel, gpu_solve, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D = mac.DIRICHLET


def _handle(gk, n, mu, gamma, precision, autotune=1):
    import torch
    opt = gk.gkb_default_options()
    opt.precision = precision
    opt.tol_inner = 1e-11
    opt.autotune = autotune
    opt.stream = torch.cuda.current_stream().cuda_stream
    h = gk.gkb_create(opt)
    visc = None if np.isscalar(mu) else np.ascontiguousarray(np.asarray(mu, dtype=np.float64).ravel(order="F"))
    gk.gkb_set_problem(h, gk.make_grid(n, 1.0 / n[0], (D,) * (2 * len(n))), visc, 1.0 if visc is not None else mu,
                       gamma, 0.0)
    return h


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_handle_meets_the_bound(lib, precision):
    gk = lib
    n = (64, 48)
    mu = np.exp(0.5 * np.random.default_rng(3).standard_normal(n))
    grid, ops = oracle_problem(n, (D,) * 4, mu, 100.0)
    g = np.random.default_rng(4).standard_normal(grid.m)
    r = np.zeros(grid.n_cells)
    ref = oracle_truth(grid, ops, g, r)
    h = _handle(gk, n, mu, 100.0, precision)
    try:
        o = gk.gkb_get_options(h)
        assert o.smoother_degree in (1, 2, 3) and o.kernel_variant in (0, 1, 2) and o.coarse_max in (8, 16, 32)
        assert o.cheb_lo in (0.05, 0.1, 0.2, 0.3) and o.cheb_hi == 1.1
        assert gk.gkb_stats(h)["tuned_inner_ms"] > 0
        rc, w, p = gpu_solve(gk, h, g, r, 1e-8, 5)
        assert rc == gk.GKB_OK, gk.gkb_last_error(h)
    finally:
        gk.gkb_destroy(h)
    assert energy_rel(ops["M"], w, ref["w"]) <= 1e-8


def test_tuning_is_cached_in_process_and_file(lib, tmp_path):
    gk = lib
    path = tmp_path / "tune.txt"
    os.environ["GKB_TUNE_CACHE"] = str(path)
    try:
        n = (40, 40)
        h1 = _handle(gk, n, 1.0, 10.0, 1)
        o1, s1 = gk.gkb_get_options(h1), gk.gkb_stats(h1)
        h2 = _handle(gk, n, 1.0, 10.0, 1)
        o2, s2 = gk.gkb_get_options(h2), gk.gkb_stats(h2)
        gk.gkb_destroy(h1)
        gk.gkb_destroy(h2)
    finally:
        del os.environ["GKB_TUNE_CACHE"]
    assert (o1.smoother_degree, o1.kernel_variant, o1.coarse_max) == (o2.smoother_degree, o2.kernel_variant, o2.coarse_max)
    assert s2["tuned_inner_ms"] == s1["tuned_inner_ms"]       # the cached entry, not a new search
    assert s2["setup_seconds"] < s1["setup_seconds"]
    lines = [ln.split() for ln in path.read_text().splitlines()]
    mine = [ln for ln in lines if "|40x40x1|" in ln[0]]
    assert len(mine) == 1
    assert [int(v) for v in mine[0][1:4]] == [o1.smoother_degree, o1.kernel_variant, o1.coarse_max]
    assert abs(float(mine[0][4]) - o1.cheb_lo) < 1e-12 and o1.cheb_lo in (0.05, 0.1, 0.2, 0.3)


def test_autotune_without_multigrid_is_a_no_op(lib):
    import torch
    gk = lib
    opt = gk.gkb_default_options()
    opt.inner = gk.GKB_INNER_CG
    opt.autotune = 1
    opt.stream = torch.cuda.current_stream().cuda_stream
    h = gk.gkb_create(opt)
    try:
        gk.gkb_set_problem(h, gk.make_grid((16, 16), 1.0 / 16, (D,) * 4), None, 1.0, 10.0, 0.0)
        assert gk.gkb_stats(h)["tuned_inner_ms"] == 0
    finally:
        gk.gkb_destroy(h)
