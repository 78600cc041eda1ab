"""The coarse end of the V-cycle fused into one thread-block-cluster kernel
(tail_side): the levels from the first one whose longer side is at most
tail_side down to the coarsest run inside one launch, every step over the
virtual blocks of the launch it replaces, with cluster barriers between the
steps. The same device bodies compute every value, so a V-cycle and a whole
solve must equal those of the separate launches bit for bit."""
import numpy as np
import pytest

from gpu_helpers import gpu_solve, make_handle, oracle_problem

pytestmark = pytest.mark.gpu

D = 0
FP64, MIXED = 0, 1


@pytest.mark.parametrize("prec", [FP64, MIXED])
# 256^2: tail 64, 32, 16, 8; 160 x 96: tail 40 x 24, 20 x 12, 10 x 6 and an
# odd 5 x 3 coarsest level
@pytest.mark.parametrize("n,bc", [((256, 256), (D, D, D, D)), ((160, 96), (D, D, D, D))])
def test_fused_tail_equals_separate_launches(lib, prec, n, bc):
    gk = lib
    outs = []
    for tail in (0, 64):
        h = make_handle(gk, n, bc, 1.0, 100.0, precision=prec, coarse_max=8, degree=2, kernel_variant=2,
                        tail_side=tail)
        try:
            assert gk.gkb_get_options(h).tail_side == tail
            m, _ = gk.gkb_layout(h)
            r = np.random.default_rng(3).standard_normal(m)
            z = np.empty(m)
            gk.gkb_precond(h, r, z)
            z2 = np.empty(m)
            gk.gkb_precond(h, r, z2)   # the plan is reused: the same again
            assert np.array_equal(z, z2)
            outs.append(z)
        finally:
            gk.gkb_destroy(h)
    assert np.any(outs[0])
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_solve_with_fused_tail_equals_separate_launches(lib, prec):
    gk = lib
    n, bc = (256, 192), (D,) * 4
    grid, _ = oracle_problem(n, bc, 1.0, 1000.0)
    g = np.random.default_rng(8).standard_normal(grid.m)
    res = []
    for tail in (0, 64):
        h = make_handle(gk, n, bc, 1.0, 1000.0, precision=prec, coarse_max=8, degree=2, tail_side=tail)
        try:
            rc, w, p = gpu_solve(gk, h, g, np.zeros(grid.n_cells))
            assert rc == gk.GKB_OK
            st = gk.gkb_stats(h)
            res.append((w, p, st["outer_iterations"], st["inner_iterations"]))
        finally:
            gk.gkb_destroy(h)
    (w0, p0, o0, i0), (w1, p1, o1, i1) = res
    assert (o0, i0) == (o1, i1)
    assert np.array_equal(w0, w1) and np.array_equal(p0, p1)


def test_tail_option_is_validated(lib):
    gk = lib
    opt = gk.gkb_default_options()
    assert opt.tail_side == 0
    opt.tail_side = -1
    with pytest.raises(gk.GkbError):
        gk.gkb_create(opt)
