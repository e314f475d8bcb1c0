"""Seeded synthetic particle sets (host-side numpy), shared by the tests and the benchmark.

This module holds no part of the octree method: it only draws coordinates and masses. The same
arrays feed the CUDA library and the CPU oracle. Distributions:

* ``uniform``  - i.i.d. U[0,1)^3, the unit cube is the box.
* ``plummer``  - Plummer sphere of scale radius a: r = a / sqrt(U^(-2/3) - 1), redrawn while
  r > r_max, isotropic direction (the 3D analogue of the paper's Gaussian / 1/r test sets).
* ``clumps``   - 1,000 Gaussian clumps with centres U[0,1)^3 and sigma = 10^U(-4,-2), 80% of the
  particles pick a clump uniformly at random, 20% are a U[0,1)^3 background.
* ``gaussian`` - one isotropic 3D Gaussian, sigma 0.1 around (0.5, 0.5, 0.5) (the density profile
  of the paper's Table 1, whose width the paper does not state).
* ``lognormal_masses`` - float32 masses, lognormal(0, 1).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20230626


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, seed: int):
    g = _rng(seed)
    return g.random(n), g.random(n), g.random(n)


def _unit_vectors(g: np.random.Generator, n: int):
    cos_t = 2.0 * g.random(n) - 1.0
    phi = 2.0 * np.pi * g.random(n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t


def plummer(n: int, seed: int, a: float = 1.0, r_max: float = 20.0):
    g = _rng(seed)
    r = np.empty(n, np.float64)
    todo = np.arange(n)
    while todo.size:
        u = g.random(todo.size)
        u = np.where(u <= 0.0, np.finfo(np.float64).tiny, u)
        rr = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        ok = rr <= r_max
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    ux, uy, uz = _unit_vectors(g, n)
    return r * ux, r * uy, r * uz


def clumps(n: int, seed: int, n_clumps: int = 1000, clump_fraction: float = 0.8):
    g = _rng(seed)
    centres = g.random((n_clumps, 3))
    sigma = 10.0 ** g.uniform(-4.0, -2.0, n_clumps)
    in_clump = g.random(n) < clump_fraction
    which = g.integers(0, n_clumps, n)
    out = []
    for d in range(3):
        c = np.empty(n, np.float64)
        k = np.nonzero(in_clump)[0]
        w = which[k]
        c[k] = centres[w, d] + sigma[w] * g.standard_normal(k.size)
        b = np.nonzero(~in_clump)[0]
        c[b] = g.random(b.size)
        out.append(c)
    return out[0], out[1], out[2]


def gaussian(n: int, seed: int, sigma: float = 0.1):
    g = _rng(seed)
    return (0.5 + sigma * g.standard_normal(n), 0.5 + sigma * g.standard_normal(n),
            0.5 + sigma * g.standard_normal(n))


def lognormal_masses(n: int, seed: int) -> np.ndarray:
    return _rng(seed).lognormal(0.0, 1.0, n).astype(np.float32)


def batched_sets(n_sets: int, seed: int, lo_exp: float = 10.0, hi_exp: float = 20.0):
    """Independent sets of log-uniform size in [2^lo_exp, 2^hi_exp), each uniform (unit cube) or
    Plummer (bounding cube) by a fair coin. Returns a list of (x, y, z, kind)."""
    g = _rng(seed)
    sizes = np.floor(2.0 ** g.uniform(lo_exp, hi_exp, n_sets)).astype(np.int64)
    kinds = g.random(n_sets) < 0.5
    sets = []
    for s in range(n_sets):
        if kinds[s]:
            x, y, z = uniform(int(sizes[s]), seed + 1000 + s)
            sets.append((x, y, z, "uniform"))
        else:
            x, y, z = plummer(int(sizes[s]), seed + 1000 + s)
            sets.append((x, y, z, "plummer"))
    return sets


def displacement(n: int, seed: int, sigma: float):
    """Per-step Gaussian displacement of every particle (time-step sequence)."""
    g = _rng(seed)
    return sigma * g.standard_normal(n), sigma * g.standard_normal(n), sigma * g.standard_normal(n)


def plummer_device(n: int, seed: int, device, a: float = 1.0, r_max: float = 20.0):
    """Plummer sphere drawn on the device with torch's generator (same recipe as ``plummer``), for
    workloads too large to draw on the host quickly."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    r = torch.empty(n, dtype=torch.float64, device=device)
    todo = torch.arange(n, device=device)
    while todo.numel():
        u = torch.rand(todo.numel(), dtype=torch.float64, device=device, generator=g).clamp_min(1e-300)
        rr = a / torch.sqrt(u ** (-2.0 / 3.0) - 1.0)
        ok = rr <= r_max
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    cos_t = 2.0 * torch.rand(n, dtype=torch.float64, device=device, generator=g) - 1.0
    phi = 2.0 * torch.pi * torch.rand(n, dtype=torch.float64, device=device, generator=g)
    sin_t = torch.sqrt(torch.clamp(1.0 - cos_t * cos_t, min=0.0))
    return r * sin_t * torch.cos(phi), r * sin_t * torch.sin(phi), r * cos_t


def gaussian_device(n: int, seed: int, device, sigma: float = 0.1):
    """One isotropic 3D Gaussian drawn on the device with torch's generator (same recipe as
    ``gaussian``), for the largest sizes of the Table 1 replay."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return tuple(0.5 + sigma * torch.randn(n, dtype=torch.float64, device=device, generator=g) for _ in range(3))
