"""The seeded synthetic inputs against their stated recipe: the log-normal
viscosity's Gaussian field has unit variance and the squared-exponential
correlation of length 0.05; forcing is N(0, 1) per velocity unknown;
batched sides are 32 * U{2..16} with one log-normal viscosity per problem;
the Poiseuille inflow is the parabola 4y(1-y) (+ h^2 when shifted); every
generator is reproducible from its seed and distinct across offsets."""
import numpy as np

import workloads
from oracle import mac


def test_gaussian_field_variance_and_correlation():
    n, ell = 256, 0.05
    vals, cov = [], {0: [], 13: [], 26: []}
    for s in range(6):
        f = workloads.gaussian_random_field(n, 1.0, ell, workloads.rng(500 + s))
        vals.append(f.var())
        for lag in cov:
            cov[lag].append(np.mean(f * np.roll(f, lag, axis=0)) / 2 + np.mean(f * np.roll(f, lag, axis=1)) / 2)
    assert abs(np.mean(vals) - 1.0) < 0.1
    for lag, c in cov.items():
        dist = lag / n
        expect = np.exp(-dist ** 2 / (2 * ell ** 2))
        assert abs(np.mean(c) - expect) < 0.1, (lag, np.mean(c), expect)


def test_forcing_is_standard_normal_and_seeded():
    a = workloads.stokes2d(128)
    b = workloads.stokes2d(128)
    c = workloads.stokes2d(128, seed_offset=7)
    grid = mac.MacGrid(a["n"], a["h"], a["bc"])
    assert a["g"].shape == (grid.m,) and a["r"].shape == (grid.n_cells,) and not a["r"].any()
    assert np.array_equal(a["g"], b["g"]) and not np.array_equal(a["g"], c["g"])
    assert abs(a["g"].mean()) < 0.02 and abs(a["g"].std() - 1.0) < 0.02


def test_batched_sides_and_viscosities():
    probs = workloads.batched2d()
    assert len(probs) == 256
    sides = np.array([p["n"][0] for p in probs])
    assert np.all(sides % 32 == 0) and sides.min() >= 64 and sides.max() <= 512
    assert len(set(sides.tolist())) >= 12          # most of the 15 sizes occur
    mus = np.array([p["mu"] for p in probs])
    assert all(np.isscalar(p["mu"]) for p in probs)
    assert abs(np.log(mus).std() - 0.5) < 0.08 and abs(np.log(mus).mean()) < 0.1
    for p in probs[:5]:
        grid = mac.MacGrid(p["n"], p["h"], p["bc"])
        assert p["g"].shape == (grid.m,)


def test_poiseuille_inflow_profile():
    for shifted in (False, True):
        wl = workloads.poiseuille(16, shifted=shifted, guess=False)
        y = (np.arange(16) + 0.5) / 16
        expect = 4 * y * (1 - y) + ((1 / 16) ** 2 if shifted else 0.0)
        assert np.allclose(wl["inflow"], expect, rtol=0, atol=1e-15)
        assert wl["bc"] == (mac.DIRICHLET, mac.NATURAL, mac.DIRICHLET, mac.DIRICHLET)


def test_varvisc_instance_is_log_normal():
    pr = workloads.varvisc2d(128)
    logmu = np.log(pr["mu"])
    assert pr["mu"].shape == (128, 128) and np.all(pr["mu"] > 0)
    assert abs(logmu.std() - 1.0) < 0.35        # one field realisation at l = 0.05
