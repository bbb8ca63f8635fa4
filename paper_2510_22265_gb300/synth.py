"""Seeded synthetic lat-lon fields shaped like the paper's ERA5 workloads.

No ERA5 data is available, so these generators stand in for the paper's
benchmark inputs (Benchmarks: ERA5 at 0.25 degree, 721x1440, 37 pressure
levels; temperature, geopotential and wind components).  The fields reproduce
the shapes and the kind of structure -- smooth large-scale modes, fronts,
cyclones, noise, heavy-tailed spikes -- not any ERA5 record.

This module holds no part of the compression method: it only draws inputs, and
both the CUDA path and the oracle consume what it returns.
"""
from __future__ import annotations

import numpy as np

GRIDS = [(91, 180), (181, 360), (361, 720), (721, 1440), (1441, 2880)]


def _axes(ny: int, nx: int):
    lam = np.linspace(0.0, 2 * np.pi, nx, endpoint=False)
    theta = np.linspace(-np.pi / 2, np.pi / 2, ny)
    return lam, theta


def _modes(rng, ny, nx, nmodes=40, kmax=8, kscale=1.0):
    """Sum of nmodes separable modes a cos(ky theta + psi) sin(kx lambda + phi),
    a = 1 / (kx^2 + ky^2), as one (ny x nmodes) by (nmodes x nx) product."""
    lam, theta = _axes(ny, nx)
    col = np.empty((ny, nmodes), np.float64)
    row = np.empty((nmodes, nx), np.float64)
    amax = 0.0
    for m in range(nmodes):
        kx = int(rng.integers(1, kmax + 1))
        ky = int(rng.integers(1, kmax + 1))
        a = 1.0 / (kx * kx + ky * ky)
        amax = max(amax, a)
        phi, psi = rng.uniform(0, 2 * np.pi, 2)
        col[:, m] = a * np.cos(ky * kscale * theta + psi)
        row[m] = np.sin(kx * kscale * lam + phi)
    return col @ row, amax


def _vortex(out, rng, sigma, amp):
    ny, nx = out.shape
    cy, cx = rng.uniform(0, ny), rng.uniform(0, nx)
    r = int(np.ceil(4 * sigma))
    y0, y1 = max(0, int(cy) - r), min(ny, int(cy) + r + 1)
    yy = np.arange(y0, y1)[:, None]
    xx = (np.arange(int(cx) - r, int(cx) + r + 1) % nx)[None, :]
    dx = (np.arange(int(cx) - r, int(cx) + r + 1) - cx)[None, :]
    g = amp * np.exp(-((yy - cy) ** 2 + dx ** 2) / (2 * sigma * sigma))
    np.add.at(out, (np.broadcast_to(yy, g.shape), np.broadcast_to(xx, g.shape)), g)


def smooth_field(ny: int = 181, nx: int = 360, seed: int = 0, kscale: float = 1.0,
                 noise: float = 1e-3, spikes: float = 0.0) -> np.ndarray:
    """40 random low-order modes (amplitude 1/k^2) + 3 Gaussian vortices of
    width 3 cells + N(0, noise) noise; optionally a fraction `spikes` of cells
    replaced by Student-t (nu = 2) spikes scaled by the field's std."""
    rng = np.random.default_rng(seed)
    f, amax = _modes(rng, ny, nx, kscale=kscale)
    for _ in range(3):
        _vortex(f, rng, 3.0, rng.choice([-1, 1]) * rng.uniform(0.5, 1.0) * amax)
    f += rng.normal(0.0, noise, size=(ny, nx))
    if spikes > 0:
        n = int(round(spikes * ny * nx))
        idx = rng.choice(ny * nx, size=n, replace=False)
        f.flat[idx] = f.flat[idx] + f.std() * rng.standard_t(2.0, size=n)
    return f.astype(np.float32)


def era5_like(var: int, level: int, ny: int = 721, nx: int = 1440) -> np.ndarray:
    """One pressure level of one of four ERA5-like variables, seed 1000*var+level:
    0 temperature-like (k<=4 modes + meridional gradient, 200-310 K),
    1 geopotential-like (very smooth, offset growing with level),
    2/3 wind components (modes + tanh fronts of 1-cell width + 10 cyclones)."""
    rng = np.random.default_rng(1000 * var + level)
    lam, theta = _axes(ny, nx)
    if var == 0:
        f, _ = _modes(rng, ny, nx, nmodes=40, kmax=4)
        f = 255.0 + 45.0 * np.cos(theta)[:, None] ** 2 - 0.8 * level + 12.0 * f / max(1e-9, np.abs(f).max())
        f += rng.normal(0, 0.05, size=(ny, nx))
        return f.astype(np.float32)
    if var == 1:
        f, _ = _modes(rng, ny, nx, nmodes=20, kmax=3)
        f = 1000.0 * (37 - level) + 600.0 * np.cos(theta)[:, None] + 300.0 * f / max(1e-9, np.abs(f).max())
        return f.astype(np.float32)
    f, _ = _modes(rng, ny, nx, nmodes=40, kmax=8)
    f = 15.0 * f / max(1e-9, np.abs(f).max())
    for _ in range(3):  # fronts
        y0 = rng.uniform(0.2, 0.8) * ny
        slope = rng.uniform(-0.3, 0.3)
        yy = np.arange(ny)[:, None] - (y0 + slope * (np.arange(nx)[None, :] - nx / 2))
        f += rng.uniform(5, 15) * np.tanh(yy / 1.0)
    for _ in range(10):  # cyclones
        _vortex(f, rng, rng.uniform(2, 6), rng.choice([-1, 1]) * rng.uniform(10, 30))
    f += rng.normal(0, 0.1, size=(ny, nx))
    return f.astype(np.float32)


def batch_spec(n: int = 512, seed: int = 3):
    """Uneven grids drawn uniformly from GRIDS, bounds log-uniform in [0.1%, 10%]."""
    rng = np.random.default_rng(seed)
    g = rng.integers(0, len(GRIDS), size=n)
    b = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), size=n))
    return [(GRIDS[int(k)], float(bb), seed * 100000 + i) for i, (k, bb) in enumerate(zip(g, b))]


def batch_field(grid, seed):
    ny, nx = grid
    return smooth_field(ny, nx, seed=seed, kscale=max(1.0, nx / 360.0) ** 0.5)


def poisson_arrivals(rate: float = 2000.0, duration: float = 10.0, seed: int = 5,
                     frac_compress: float = 0.7):
    """Arrival times (s) and request kinds (True = compress) of a Poisson stream."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        out.append((t, bool(rng.uniform() < frac_compress), float(rng.choice([1e-3, 1e-2, 1e-1]))))
    return out
