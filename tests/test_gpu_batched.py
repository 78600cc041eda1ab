"""Batched form: many independent cavities solved in one graph launch.

Every problem's whole solve is one branch of a single CUDA graph; the
branches use per-problem reductions and states, so each problem must match
its own individual solve bit for bit, and the oracle within the FP64 bound.
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import energy_rel, make_handle, oracle_problem, oracle_truth

pytestmark = pytest.mark.gpu

D = 0


def _batch(count, seed_offset=6):
    sides = [64, 96, 48, 128, 80, 64][:count]
    return workloads.batched2d(count=len(sides), seed_offset=seed_offset, sides=sides)


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_equals_individual_and_oracle(lib, prec):
    import torch
    gk = lib
    probs = _batch(6)
    hs = [make_handle(gk, pr["n"], pr["bc"], pr["mu"], 100.0, precision=prec, tol_inner=1e-11) for pr in probs]
    try:
        g = [torch.tensor(pr["g"], device="cuda") for pr in probs]
        r = [torch.tensor(pr["r"], device="cuda") for pr in probs]
        w = [torch.empty(pr["m"], dtype=torch.float64, device="cuda") for pr in probs]
        p = [torch.empty(pr["ncells"], dtype=torch.float64, device="cuda") for pr in probs]
        for rep in range(2):  # second call reuses the captured graph
            rc = gk.gkb_solve_batched(hs, g, r, 1e-8, 5, w, p)
            assert rc == gk.GKB_OK, gk.gkb_last_error(hs[0])
        stats_b = [gk.gkb_stats(h) for h in hs]
        wb = [x.cpu().numpy() for x in w]
        pb = [x.cpu().numpy() for x in p]
        for i, (h, pr) in enumerate(zip(hs, probs)):
            wi = torch.empty_like(w[i])
            pi = torch.empty_like(p[i])
            assert gk.gkb_solve(h, g[i], r[i], 1e-8, 5, wi, pi) == gk.GKB_OK
            st = gk.gkb_stats(h)
            assert st["outer_iterations"] == stats_b[i]["outer_iterations"]
            assert st["inner_iterations"] == stats_b[i]["inner_iterations"]
            assert np.array_equal(wi.cpu().numpy(), wb[i]) and np.array_equal(pi.cpu().numpy(), pb[i])
        # one problem against the oracle
        pr = probs[2]
        grid, ops = oracle_problem(pr["n"], pr["bc"], pr["mu"], 100.0)
        ref = oracle_truth(grid, ops, pr["g"], pr["r"])
        assert energy_rel(ops["M"], wb[2], ref["w"]) <= 1e-8
        # re-setting one handle invalidates the cached graph
        gk.gkb_set_problem(hs[1], gk.make_grid(probs[1]["n"], probs[1]["h"], probs[1]["bc"]), None,
                           probs[1]["mu"], 10.0, 0.0)
        assert gk.gkb_solve_batched(hs, g, r, 1e-8, 5, w, p) == gk.GKB_OK
        grid, ops = oracle_problem(probs[1]["n"], probs[1]["bc"], probs[1]["mu"], 10.0)
        ref = oracle_truth(grid, ops, probs[1]["g"], probs[1]["r"])
        assert energy_rel(ops["M"], w[1].cpu().numpy(), ref["w"]) <= 1e-8
    finally:
        for h in hs:
            gk.gkb_destroy(h)


def test_batched_argument_errors(lib):
    import torch
    gk = lib
    pr = _batch(1)[0]
    h = make_handle(gk, pr["n"], pr["bc"], pr["mu"], 100.0)
    h2 = make_handle(gk, pr["n"], pr["bc"], pr["mu"], 100.0, use_graph=0)
    try:
        g = torch.tensor(pr["g"], device="cuda")
        r = torch.tensor(pr["r"], device="cuda")
        w = torch.empty(pr["m"], dtype=torch.float64, device="cuda")
        p = torch.empty(pr["ncells"], dtype=torch.float64, device="cuda")
        with pytest.raises(gk.GkbError):
            gk.gkb_solve_batched([h, h], [g, g], [r, r], 1e-8, 5, [w, w], [p, p])
        with pytest.raises(gk.GkbError):
            gk.gkb_solve_batched([h, h2], [g, g], [r, r], 1e-8, 5, [w, w], [p, p])
    finally:
        gk.gkb_destroy(h)
        gk.gkb_destroy(h2)
