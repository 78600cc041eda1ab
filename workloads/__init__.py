"""Seeded synthetic inputs for the GKB saddle-point workloads.

This module holds no arithmetic of the method: it only draws the inputs that
the oracle and the GPU library both consume (grid sizes and boundary types,
forcing vectors, viscosity fields, inflow profiles, initial guesses), so that
the two sides see identical arrays. Everything is FP64 NumPy drawn from PCG64
with a fixed base seed plus a per-workload offset.

Workloads (all on the unit square / cube, uniform spacing h = 1/n):

* ``poiseuille``  2D channel, inflow ``u = 4y(1-y)`` on x = 0, no-slip walls at
  y = 0 and y = 1, natural outflow at x = 1; optional N(0,1) initial guess.
* ``stokes2d``    enclosed cavity (all sides Dirichlet, zero wall velocity),
  forcing ``g ~ N(0,1)`` on every velocity unknown, ``r = 0``, viscosity 1.
* ``stokes3d``    the same in 3D.
* ``varvisc2d``   enclosed 2D cavity with ``mu = exp(G)``, G a stationary
  Gaussian random field (squared-exponential covariance, sigma = 1,
  correlation length 0.05) sampled by FFT spectral synthesis on the periodic
  cell-centre grid, forcing ``g ~ N(0,1)``.
* ``batched2d``   many enclosed 2D cavities with side ``32 * U{2..16}`` and a
  per-problem constant viscosity ``exp(0.5 xi)``, ``xi ~ N(0,1)``.
"""
import numpy as np

BASE_SEED = 20010424
DIRICHLET = 0
NATURAL = 1


def rng(offset):
    return np.random.Generator(np.random.PCG64(BASE_SEED + int(offset)))


def active_counts(n, bc):
    """Number of active faces per velocity component for ``n`` cells per axis
    and side types ``bc`` (x-low, x-high, y-low, y-high[, z-low, z-high]).
    A face on a Dirichlet side normal to its component is not an unknown."""
    d = len(n)
    counts = []
    for c in range(d):
        k = n[c] + 1 - (bc[2 * c] == DIRICHLET) - (bc[2 * c + 1] == DIRICHLET)
        others = int(np.prod([n[a] for a in range(d) if a != c]))
        counts.append(k * others)
    return counts


def velocity_size(n, bc):
    return int(sum(active_counts(n, bc)))


def poiseuille(n=32, shifted=False, guess=True, seed_offset=1):
    """2D Poiseuille channel on the unit square with n x n cells.

    Returns a dict with the grid description, the inflow normal velocity on
    the x-low side (one value per cell row) and an optional N(0,1) initial
    guess. ``shifted`` adds h^2 to the inflow profile (the profile for which
    the MAC scheme with mirror walls is exact).
    """
    h = 1.0 / n
    bc = (DIRICHLET, NATURAL, DIRICHLET, DIRICHLET)
    y = (np.arange(n) + 0.5) * h
    inflow = 4.0 * y * (1.0 - y) + (h * h if shifted else 0.0)
    m = velocity_size((n, n), bc)
    out = {"n": (n, n), "h": h, "bc": bc, "mu": 1.0, "inflow": inflow,
           "m": m, "ncells": n * n}
    if guess:
        g = rng(seed_offset)
        out["w0"] = g.standard_normal(m)
        out["p0"] = g.standard_normal(n * n)
    return out


def stokes2d(n=1024, seed_offset=2):
    bc = (DIRICHLET,) * 4
    m = velocity_size((n, n), bc)
    g = rng(seed_offset).standard_normal(m)
    return {"n": (n, n), "h": 1.0 / n, "bc": bc, "mu": 1.0, "g": g,
            "r": np.zeros(n * n), "m": m, "ncells": n * n}


def stokes3d(n=256, seed_offset=3):
    bc = (DIRICHLET,) * 6
    m = velocity_size((n, n, n), bc)
    g = rng(seed_offset).standard_normal(m)
    return {"n": (n, n, n), "h": 1.0 / n, "bc": bc, "mu": 1.0, "g": g,
            "r": np.zeros(n ** 3), "m": m, "ncells": n ** 3}


def gaussian_random_field(n, sigma=1.0, corr_len=0.05, gen=None):
    """Periodic stationary Gaussian field on the n x n cell-centre grid of the
    unit square with covariance sigma^2 exp(-|x|^2 / (2 l^2)), by spectral
    synthesis: white noise filtered by the square root of the covariance's
    spectral density, normalised to unit variance in expectation.
    Indexed [x, y]."""
    if gen is None:
        gen = rng(4)
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    kx, ky = np.meshgrid(k, k, indexing="ij")
    spec = np.exp(-0.5 * corr_len ** 2 * (kx ** 2 + ky ** 2))  # density up to a constant
    amp = np.sqrt(spec)
    noise = gen.standard_normal((n, n))
    field = np.real(np.fft.ifft2(np.fft.fft2(noise) * amp))
    # E[field^2] = mean(amp^2) for unit white noise
    field *= sigma / np.sqrt(np.mean(amp ** 2))
    return field


def varvisc2d(n=2048, seed_offset=4, sigma=1.0, corr_len=0.05):
    bc = (DIRICHLET,) * 4
    gen = rng(seed_offset)
    logmu = gaussian_random_field(n, sigma, corr_len, gen)
    m = velocity_size((n, n), bc)
    g = rng(seed_offset + 1).standard_normal(m)
    return {"n": (n, n), "h": 1.0 / n, "bc": bc, "mu": np.exp(logmu), "g": g,
            "r": np.zeros(n * n), "m": m, "ncells": n * n}


def batched2d(count=256, seed_offset=6, sides=None, visc_sigma=0.5):
    """``count`` independent enclosed cavities; side lengths 32 * U{2..16}."""
    gen = rng(seed_offset)
    if sides is None:
        sides = 32 * gen.integers(2, 17, size=count)
    problems = []
    for i, s in enumerate(sides):
        s = int(s)
        mu = float(np.exp(visc_sigma * gen.standard_normal()))
        bc = (DIRICHLET,) * 4
        m = velocity_size((s, s), bc)
        g = gen.standard_normal(m)
        problems.append({"n": (s, s), "h": 1.0 / s, "bc": bc, "mu": mu, "g": g,
                         "r": np.zeros(s * s), "m": m, "ncells": s * s})
    return problems
