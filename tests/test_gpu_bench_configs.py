"""The benchmark configurations against the oracle at their own tolerance.

The timed metric is the time to a velocity within relative energy-norm
(M-norm) error 1e-8 of the exact saddle-point solution (Algorithm 1 with the
stopping rule of Eq. (5), Sec. 2.2). These tests run the forms `bench.py`
times, with the options it times them with (its own handle construction),
and compare the velocity with a tightly converged oracle solution:

* the default benchmark itself: the 1024 x 1024 enclosed cavity, plain FP64,
  GMG-PCG inner solves to 1e-10, tau = 1e-8, d = 5, autotuned handles, for
  gamma = 10 and 1000; the oracle runs Eq. (3), Algorithm 1 and Eq. (5) to
  tau = 1e-13 with sparse-LU inner solves (Sec. 4.1.2) at the same size;
* the 3D precision form (FP32 inner solves with FP64 residual replacement,
  FP64 GKB) on a 64^3 member of its family, against the stored oracle
  solution written by ``tests/golden/make_oracle_solutions.py``;
* the learned form (flexible CG with the U-Net correction two levels below
  the finest, mixed precision) on a 512 x 512 member of the log-normal
  viscosity family, with a network trained in the test on pairs harvested
  from 128 x 128 instances of the same family.

Bound: relative M-norm error of the velocity <= 1e-8 (the bound stated for
FP64 and for the forms whose inner solves are judged on the FP64 residual);
pressures within 1e-6 of their largest entry, the tolerance of the other
solve tests (the pressure is the Craig iterate's p_k, whose error the
stopping rule does not bound directly).
"""
import argparse
import os

import numpy as np
import pytest

import bench
from oracle import gkb as ogkb
from oracle import mac

from gpu_helpers import energy_rel

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def bench_args(**kw):
    """bench.py's defaults (its argument parser's), overridden by kw."""
    a = dict(gpus=1, steps=1, warmup=0, impl="ours", workload="stokes2d", unet_side=512, train_pairs=10000,
             harvest_seconds=120.0, train_steps=800, train_batch=8, train_lr=1e-3, learned_form="replace",
             kernel_variant=None, form=None, n=1024, batch=256, gammas=[10.0, 1000.0], tol=1e-8, tol_inner=1e-10,
             delay=5, autotune=-1, rank=0)
    a.update(kw)
    args = argparse.Namespace(**a)
    args.form_default = args.form is None
    if args.form is None:
        args.form = "fp64"
    return args


def run_bench_form(gk, args, autotune=1, learned="default", mixed_rtol=None, maxit=1000):
    """One step of the workload as bench.py times it; returns the solutions,
    statuses and statistics of its problems."""
    import torch
    wk = bench.Workload(args)
    if wk.learned:
        wk.net, _ = bench.train_network(gk, torch, wk, args)
    try:
        B = bench.Bound(gk, torch, wk, wk.form, autotune=autotune, learned=learned, mixed_rtol=mixed_rtol,
                        maxit=maxit)
        try:
            B.step(args)
            torch.cuda.synchronize()
            ws = [x.cpu().numpy() for x in B.w]
            ps = [x.cpu().numpy() for x in B.p]
            stats = B.stats()
            status = [st["status"] for st in stats]   # per problem (one batched call may cover several)
        finally:
            B.destroy()
    finally:
        if wk.net is not None:
            gk.gkb_unet_destroy(wk.net)
    return wk, ws, ps, status, stats


def check_against(ops, w, p, ref_w, ref_p, label):
    err = energy_rel(ops["M"], w, ref_w)
    perr = np.abs(p - ref_p).max() / np.abs(ref_p).max()
    print("%s: relative M-norm velocity error %.3e, pressure %.3e" % (label, err, perr))
    assert err <= 1e-8, (label, err)
    assert perr <= 1e-6, (label, perr)
    assert abs(p.mean()) <= 1e-12 * np.abs(p).max()


@pytest.fixture(scope="module")
def stokes2d_1024(lib):
    return run_bench_form(lib, bench_args())


@pytest.mark.parametrize("i", [0, 1], ids=["gamma10", "gamma1000"])
def test_default_benchmark_within_1e8_of_the_oracle(stokes2d_1024, i):
    wk, ws, ps, status, stats = stokes2d_1024
    pr = wk.problems[i]
    assert status[i] == 0
    assert stats[i]["estimate"] <= 1e-8
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    ops = mac.assemble(grid, 1.0, pr["gamma"])
    ref = ogkb.solve(grid, ops, pr["g"], pr["r"], tol=1e-13, delay=5, inner="direct")
    assert ref["converged"]
    check_against(ops, ws[i], ps[i], ref["w"], ref["p"], "1024^2 gamma %g" % pr["gamma"])


def test_precision_form_3d_64_within_1e8_of_the_oracle(lib):
    path = os.path.join(GOLDEN, "stokes3d_64_gamma100.npz")
    ref = np.load(path)
    args = bench_args(workload="stokes3d", n=64)
    wk, ws, ps, status, stats = run_bench_form(lib, args)
    pr = wk.problems[0]
    assert tuple(ref["n"]) == tuple(pr["n"]) and float(ref["gamma"]) == pr["gamma"]
    assert wk.form == "mixed" and status[0] == 0
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    ops = mac.assemble(grid, 1.0, pr["gamma"])
    check_against(ops, ws[0], ps[0], ref["w"], ref["p"], "64^3 mixed")
    # the same form without the FP64 residual replacement misses the bound
    wk2, ws2, ps2, status2, stats2 = run_bench_form(lib, args, autotune=0, mixed_rtol=0.0, maxit=100)
    e_abl = energy_rel(ops["M"], ws2[0], ref["w"])
    print("64^3 mixed without replacement: %.3e (%d outer, status %d)" % (e_abl, stats2[0]["outer_iterations"],
                                                                         status2[0]))
    assert e_abl > 1e-8


def test_fp32_inner_without_replacement_has_an_error_floor(lib):
    """The ablation of the precision form's FP64 residual replacement: the
    same mixed form with FP32 inner solves that end on the FP32 recursion's
    own convergence claim. Without the replacement the velocity misses the
    1e-8 bound (FP32 rounding of the inner solutions, unit roundoff 6e-8,
    is not corrected); with it the bound holds on the same problem."""
    args = bench_args(n=256, gammas=[100.0], form="mixed")
    wk, ws, ps, status, stats = run_bench_form(lib, args, autotune=0)
    wk2, ws2, ps2, status2, stats2 = run_bench_form(lib, args, autotune=0, mixed_rtol=0.0, maxit=100)
    pr = wk.problems[0]
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    ops = mac.assemble(grid, 1.0, pr["gamma"])
    ref = ogkb.solve(grid, ops, pr["g"], pr["r"], tol=1e-13, delay=5, inner="direct")
    e_rep = energy_rel(ops["M"], ws[0], ref["w"])
    e_abl = energy_rel(ops["M"], ws2[0], ref["w"])
    print("256^2 mixed: with replacement %.3e (%d outer), without %.3e (%d outer, status %d)"
          % (e_rep, stats[0]["outer_iterations"], e_abl, stats2[0]["outer_iterations"], status2[0]))
    assert status[0] == 0 and e_rep <= 1e-8
    assert e_abl > 1e-8 and e_abl > 10 * e_rep


@pytest.mark.parametrize("form", ["replace", "composite"])
def test_learned_form_512_within_1e8_of_the_oracle(lib, form):
    args = bench_args(workload="varvisc2d", n=512, unet_side=128, learned_form=form, train_pairs=600,
                      harvest_seconds=30.0, train_steps=150)
    wk, ws, ps, status, stats = run_bench_form(lib, args, autotune=1)
    pr = wk.problems[0]
    assert wk.learned == form and wk.form == "mixed" and status[0] == 0
    print("learned %s: %d outer, %d inner, %d fallbacks" % (form, stats[0]["outer_iterations"],
                                                             stats[0]["inner_iterations"],
                                                             stats[0]["inner_fallbacks"]))
    grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
    ops = mac.assemble(grid, pr["mu"], pr["gamma"])
    ref = ogkb.solve(grid, ops, pr["g"], pr["r"], tol=1e-13, delay=5, inner="direct")
    check_against(ops, ws[0], ps[0], ref["w"], ref["p"], "512^2 learned " + form)
