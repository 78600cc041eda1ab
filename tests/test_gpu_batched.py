"""Batched form: many independent cavities solved in one graph launch.

By default every problem's whole solve is one branch of the graph. With the
batch_lockstep option, batches that qualify (2D, constant viscosity per
problem, GMG-PCG) run in lock step instead: every step of the solve is one
launch over all problems, with each problem's blocks running the body of its
own launch (same grid, same reduction buffers) and per-problem snapshot flags
deciding which problems take part in each loop iteration. Either way each
problem must match its own individual solve bit for bit, and the oracle
within the FP64 bound.
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


@pytest.mark.parametrize("prec", [0, 1])
def test_lockstep_batch_with_uneven_problems(lib, prec):
    """Problems that stop at very different points in one lock-step batch: a
    zero right-hand side (Algorithm 1 stops at beta_1 = 0), gammas from 1 to
    1e4 (outer iteration counts from many to few), sides whose hierarchies
    have 3 to 6 levels; every problem equals its individual solve bit for
    bit and the launches of the batch are counted."""
    import torch
    gk = lib
    sides = [64, 32, 96, 160, 48, 64, 128]
    gammas = [100.0, 1.0, 1e4, 10.0, 100.0, 1000.0, 100.0]
    probs = workloads.batched2d(count=len(sides), seed_offset=61, sides=sides)
    probs[5]["g"] = np.zeros_like(probs[5]["g"])
    hs = [make_handle(gk, pr["n"], pr["bc"], pr["mu"], gm, precision=prec, tol_inner=1e-11, batch_lockstep=1)
          for pr, gm in zip(probs, gammas)]
    try:
        g = [torch.tensor(pr["g"], device="cuda") for pr in probs]
        r = [torch.tensor(pr["r"], device="cuda") for pr in probs]
        w = [torch.empty(pr["m"], dtype=torch.float64, device="cuda") for pr in probs]
        p = [torch.empty(pr["ncells"], dtype=torch.float64, device="cuda") for pr in probs]
        rc = gk.gkb_solve_batched(hs, g, r, 1e-8, 5, w, p)
        assert rc == gk.GKB_OK, gk.gkb_last_error(hs[0])
        stats_b = [gk.gkb_stats(h) for h in hs]
        launches_b = sum(sum(st["kernel_launches"].values()) for st in stats_b)
        assert launches_b > 0
        wb = [x.cpu().numpy() for x in w]
        pb = [x.cpu().numpy() for x in p]
        assert not np.any(wb[5]) and not np.any(pb[5])
        outer = []
        launches_i = 0
        for i, h in enumerate(hs):
            wi = torch.empty_like(w[i])
            pi = torch.empty_like(p[i])
            assert gk.gkb_solve(h, g[i], r[i], 1e-8, 5, wi, pi) == gk.GKB_OK
            st = gk.gkb_stats(h)
            outer.append(st["outer_iterations"])
            assert st["outer_iterations"] == stats_b[i]["outer_iterations"], i
            assert st["inner_iterations"] == stats_b[i]["inner_iterations"], i
            assert np.array_equal(wi.cpu().numpy(), wb[i]) and np.array_equal(pi.cpu().numpy(), pb[i]), i
            launches_i += sum(st["kernel_launches"].values())
        assert max(outer) >= 2 * min(o for o in outer if o > 0)
        # lock step: one launch per step for all problems, far fewer than
        # the individual solves' launches together
        assert launches_b < launches_i / 2, (launches_b, launches_i)
        pr = probs[3]
        grid, ops = oracle_problem(pr["n"], pr["bc"], pr["mu"], gammas[3])
        ref = oracle_truth(grid, ops, pr["g"], pr["r"])
        assert energy_rel(ops["M"], wb[3], ref["w"]) <= 1e-8
    finally:
        for h in hs:
            gk.gkb_destroy(h)


def test_variable_viscosity_batch_uses_graph_branches(lib):
    """A batch the lock-step form does not take (per-cell viscosity) still
    solves every problem exactly as its individual solve."""
    import torch
    gk = lib
    probs = [workloads.varvisc2d(32, seed_offset=70 + 2 * i) for i in range(3)]
    hs = [make_handle(gk, pr["n"], pr["bc"], pr["mu"], 100.0, precision=1, tol_inner=1e-11) for pr in probs]
    try:
        g = [torch.tensor(pr["g"], device="cuda") for pr in probs]
        r = [torch.tensor(pr["r"], device="cuda") for pr in probs]
        w = [torch.empty(pr["m"], dtype=torch.float64, device="cuda") for pr in probs]
        p = [torch.empty(pr["ncells"], dtype=torch.float64, device="cuda") for pr in probs]
        assert gk.gkb_solve_batched(hs, g, r, 1e-8, 5, w, p) == gk.GKB_OK
        for i, h in enumerate(hs):
            wi = torch.empty_like(w[i])
            pi = torch.empty_like(p[i])
            assert gk.gkb_solve(h, g[i], r[i], 1e-8, 5, wi, pi) == gk.GKB_OK
            assert torch.equal(wi, w[i]) and torch.equal(pi, p[i])
    finally:
        for h in hs:
            gk.gkb_destroy(h)
